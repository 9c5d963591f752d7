"""GPU parity of the fused sparse gradient kernel against the FP64 oracle.

Integer work (sample coordinates, rejection attempts) must be bit-exact;
gradients are compared by per-array relative Frobenius error <= 1e-5 (FP32
path) and the sampled loss within 1e-4 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synthetic as S
from oracle import gcp

TOL_G = 1e-5
TOL_F = 1e-4


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2110_14514_gb300 as sg
    return sg


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def row_err(G, Go):
    """Worst per-row error of a gradient matrix: max_i ||G_i - Go_i|| / max(||Go_i||, ||Go|| / sqrt(I)).
    A Zipf head row dominates ||Go||, so the per-array Frobenius error alone would let a cold row be
    wrong by 100 %; the floor ||Go|| / sqrt(I) (the RMS row norm) keeps rows that are zero or nearly
    so from dividing by nothing."""
    G = np.asarray(G, np.float64)
    Go = np.asarray(Go, np.float64)
    floor = np.linalg.norm(Go) / np.sqrt(Go.shape[0])
    den = np.maximum(np.linalg.norm(Go, axis=1), floor)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.linalg.norm(G - Go, axis=1) / den))


def zipf_case(dims, nnz, R, seed=0, scale=0.5):
    cfg = S.workload("sparse_binary_zipf")
    idx, val = S.sparse_slice(cfg, 1 + seed, nnz=nnz, dims=dims)
    rng = np.random.default_rng(100 + seed)
    A = [(scale * rng.standard_normal((n, R))).astype(np.float32) for n in dims]
    s = (rng.random(R) + 0.5).astype(np.float32)
    return idx, val, A, s


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def make_ctx(sg, dims, R, loss, A, **kw):
    p = sg.params(dims, R, loss, **kw)
    return sg.Context(p, [dev(a) for a in A])


@pytest.mark.parametrize("set_", [0, 1, 2, 3])
def test_sample_coordinates_are_bit_exact(sg, set_):
    dims, R = (300, 200, 100), 8
    idx, val, A, s = zipf_case(dims, 20000, R)
    seed, t, draw = 0x1234_5678_9ABC, 7, 13
    with make_ctx(sg, dims, R, "bernoulli_logit", A, p=3000, q=2500, p_obj=4000, q_obj=1500, seed=seed) as ctx:
        obj = set_ in (1, 3)
        n = (4000 + 1500) if obj else (3000 + 2500)
        coords, att = ctx.sample_coords(dev(idx), dev(val), set_, t, draw, n)
        ctx.check()
    names = {0: ("grad_nz", "grad_z"), 1: ("obj_nz", "obj_z"), 2: ("tgrad_nz", "tgrad_z"), 3: ("tobj_nz", "tobj_z")}[set_]
    p, q = (4000, 1500) if obj else (3000, 2500)
    c, x, w = gcp.stratified_samples(idx, val, dims, p, q, seed, t, draw, gcp.PURPOSE[names[0]], gcp.PURPOSE[names[1]])
    assert np.array_equal(coords.cpu().numpy().astype(np.int64), c)
    keys = np.sort(gcp.linear_keys(idx, dims))
    _, att_o = gcp.zero_sample_coords(dims, q, seed, t, draw, gcp.PURPOSE[names[1]], keys, 64)
    assert np.array_equal(att.cpu().numpy()[p:], att_o)
    assert np.all(att.cpu().numpy()[:p] == -1)


@pytest.mark.parametrize("loss", ["bernoulli_logit", "poisson", "gaussian", "bernoulli_odds"])
@pytest.mark.parametrize("R", [4, 8, 16, 32, 64, 128])
def test_sampled_gradient_matches_oracle(sg, loss, R):
    dims = (257, 130, 61)                       # ragged: no dimension is a tile multiple
    idx, val, A, s = zipf_case(dims, 9000, R, seed=R)
    if loss in ("poisson", "bernoulli_odds"):
        A = [np.abs(a) + 0.05 for a in A]
        if loss == "poisson":
            val = (1 + (np.arange(len(val)) % 3)).astype(np.float32)
    p, q, seed, t, draw = 5001, 4003, 42, 5, 3
    with make_ctx(sg, dims, R, loss, A, p=p, q=q, seed=seed) as ctx:
        G, gs, f = ctx.gradient(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), t=t, draw=draw)
        ctx.check()
        Go, gso, Fo = gcp.sampled_gradient(idx, val, dims, s, A, loss, p, q, seed, t, draw)
        for k in range(3):
            assert rel(G[k].cpu().numpy(), Go[k]) < TOL_G, (k, rel(G[k].cpu().numpy(), Go[k]))
            assert row_err(G[k].cpu().numpy(), Go[k]) < TOL_G, (k, row_err(G[k].cpu().numpy(), Go[k]))
        assert rel(gs.cpu().numpy(), gso) < TOL_G
        assert abs(f.item() - Fo) <= TOL_F * max(abs(Fo), 1.0)
        # temporal sample set, accumulate and y_scale
        scale = torch.tensor([0.25], dtype=torch.float32, device="cuda")
        G2, gs2, f2 = ctx.gradient(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), t=t, draw=draw,
                                   sample_set=sg.SAMPLES_TEMPORAL_GRAD, y_scale=scale,
                                   G=[g.clone() for g in G], gs=gs.clone(), f=f.clone(), accumulate=True)
        Gt, gst, Ft = gcp.sampled_gradient(idx, val, dims, s, A, loss, p, q, seed, t, draw, temporal=True)
        for k in range(3):
            assert rel(G2[k].cpu().numpy(), Go[k] + 0.25 * Gt[k]) < TOL_G
        assert rel(gs2.cpu().numpy(), gso + 0.25 * gst) < TOL_G
        assert abs(f2.item() - (Fo + 0.25 * Ft)) <= TOL_F * max(abs(Fo), 1.0)


@pytest.mark.parametrize("dims", [(40, 50), (12, 9, 7, 11)])
def test_two_and_four_way_slices(sg, dims):
    R = 16
    rng = np.random.default_rng(3)
    omega = int(np.prod(dims))
    lin = rng.choice(omega, size=omega // 5, replace=False)
    idx = np.stack(np.unravel_index(lin, dims), axis=1).astype(np.int32)
    val = np.ones(len(lin), np.float32)
    A = [(0.5 * rng.standard_normal((n, R))).astype(np.float32) for n in dims]
    s = (rng.random(R) + 0.5).astype(np.float32)
    with make_ctx(sg, dims, R, "bernoulli_logit", A, p=700, q=900, seed=9) as ctx:
        G, gs, f = ctx.gradient(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), t=2, draw=1)
        ctx.check()
    Go, gso, Fo = gcp.sampled_gradient(idx, val, dims, s, A, "bernoulli_logit", 700, 900, 9, 2, 1)
    for k in range(len(dims)):
        assert rel(G[k].cpu().numpy(), Go[k]) < TOL_G
        assert row_err(G[k].cpu().numpy(), Go[k]) < TOL_G
    assert rel(gs.cpu().numpy(), gso) < TOL_G
    assert abs(f.item() - Fo) <= TOL_F * max(abs(Fo), 1.0)


def test_empty_and_full_slices(sg):
    dims, R = (6, 5, 4), 8
    rng = np.random.default_rng(4)
    A = [(0.5 * rng.standard_normal((n, R))).astype(np.float32) for n in dims]
    s = (rng.random(R) + 0.5).astype(np.float32)
    # empty slice: only zero samples, weight omega / q
    idx = np.zeros((0, 3), np.int32)
    val = np.zeros(0, np.float32)
    with make_ctx(sg, dims, R, "bernoulli_logit", A, p=50, q=64, seed=5) as ctx:
        G, gs, f = ctx.gradient(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), t=1)
        ctx.check()
    Go, gso, Fo = gcp.sampled_gradient(idx, val, dims, s, A, "bernoulli_logit", 50, 64, 5, 1, 0)
    for k in range(3):
        assert rel(G[k].cpu().numpy(), Go[k]) < TOL_G
    # full slice: no zeros, the zero stratum is dropped
    idx = np.array(list(np.ndindex(*dims)), np.int32)
    val = np.ones(len(idx), np.float32)
    with make_ctx(sg, dims, R, "bernoulli_logit", A, p=50, q=64, seed=5) as ctx:
        G, gs, f = ctx.gradient(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), t=1)
        ctx.check()
    Go, gso, Fo = gcp.sampled_gradient(idx, val, dims, s, A, "bernoulli_logit", 50, 64, 5, 1, 0)
    for k in range(3):
        assert rel(G[k].cpu().numpy(), Go[k]) < TOL_G
    assert abs(f.item() - Fo) <= TOL_F * max(abs(Fo), 1.0)


def test_sampling_limit_and_bad_coordinates_are_reported(sg):
    dims, R = (4, 4, 4), 4
    A = [np.ones((n, R), np.float32) for n in dims]
    s = np.ones(R, np.float32)
    # 63 of 64 entries are nonzero and only one attempt is allowed: most slots fail
    lin = np.arange(63)
    idx = np.stack(np.unravel_index(lin, dims), axis=1).astype(np.int32)
    val = np.ones(63, np.float32)
    with make_ctx(sg, dims, R, "bernoulli_logit", A, p=8, q=64, seed=1, zero_attempt_cap=1) as ctx:
        ctx.gradient(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val))
        with pytest.raises(sg.SgcpError) as e:
            ctx.check()
        assert e.value.status == sg.ERR_SAMPLING_LIMIT
        with pytest.raises(sg.SgcpError) as e:          # the context stays latched
            ctx.check()
        assert e.value.status == sg.ERR_STATE
    bad = idx.copy()
    bad[5, 1] = 4                                     # out of range
    with make_ctx(sg, dims, R, "bernoulli_logit", A, p=8, q=8, seed=1) as ctx:
        ctx.ingest(idx=dev(bad), vals=dev(val))
        with pytest.raises(sg.SgcpError) as e:
            ctx.check()
        assert e.value.status == sg.ERR_DATA
    dup = idx.copy()
    dup[7] = dup[3]
    with make_ctx(sg, dims, R, "bernoulli_logit", A, p=8, q=8, seed=1) as ctx:
        ctx.ingest(idx=dev(dup), vals=dev(val))
        with pytest.raises(sg.SgcpError) as e:
            ctx.check()
        assert e.value.status == sg.ERR_DATA


def bad_coordinate_case(dims, R, pad, nnz=60, seed=8):
    """A small COO slice whose entry 17 has i_1 = I_1 (one past the last row), and factor matrices
    with `pad` extra rows past I_k so that even an unguarded row access would stay inside them."""
    rng = np.random.default_rng(seed)
    lin = rng.choice(int(np.prod(dims)), nnz, replace=False)
    idx = np.stack(np.unravel_index(lin, dims), axis=1).astype(np.int32)
    idx[17, 0] = dims[0]
    val = np.ones(nnz, np.float32)
    A = [(0.5 * rng.standard_normal((n + pad, R))).astype(np.float32) for n in dims]
    s = (rng.random(R) + 0.5).astype(np.float32)
    return idx, val, A, s


def oracle_without_bad_samples(idx, val, dims, s, A, loss, p, q, seed, t, draw):
    """The oracle's draw on the same slice with every sample that lands on an out-of-range entry
    removed (the zero stratum is unaffected: the bad entry's linear key is >= prod I_k, so no zero
    candidate can equal it)."""
    A = [a[:n].astype(np.float64) for a, n in zip(A, dims)]
    coords, x, w = gcp.stratified_samples(idx, val, dims, p, q, seed, t, draw, gcp.PURPOSE["grad_nz"],
                                          gcp.PURPOSE["grad_z"])
    keep = np.all(coords < np.asarray(dims)[None, :], axis=1)
    assert (~keep).sum() > 0, "the draw never sampled the bad entry"
    uc, yt = gcp.strat_grad_tensor(coords[keep], x[keep], w[keep], s, A, loss)
    G = [gcp.sparse_mttkrp(uc, yt, s, A, k) for k in range(len(A))]
    return G, gcp.sparse_temporal(uc, yt, A), gcp.sampled_loss(coords[keep], x[keep], w[keep], s, A, loss)


def test_out_of_range_coordinates_are_never_dereferenced(sg):
    """sgcp_gradient on a slice with a coordinate equal to I_1: the call reports SGCP_ERR_DATA, the
    samples that hit the bad entry are dropped (the rest equals the oracle's draw without them), and
    the gradient rows past I_k, which the kernel could only reach through the bad coordinate, keep
    the value they had."""
    dims, R, pad, p, q = (40, 30, 20), 8, 4, 4000, 100
    idx, val, A, s = bad_coordinate_case(dims, R, pad)
    with make_ctx(sg, dims, R, "bernoulli_logit", [a[:n] for a, n in zip(A, dims)], p=p, q=q, seed=3) as ctx:
        G = [torch.full((n + pad, R), 7.0, device="cuda") for n in dims]
        _, gs, f = ctx.gradient(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), t=2, draw=1, G=G)
        with pytest.raises(sg.SgcpError) as e:
            ctx.check()
        assert e.value.status == sg.ERR_DATA
    Go, gso, Fo = oracle_without_bad_samples(idx, val, dims, s, A, "bernoulli_logit", p, q, 3, 2, 1)
    for k, n in enumerate(dims):
        Gk = G[k].cpu().numpy()
        assert np.all(Gk[n:] == 7.0), k
        assert rel(Gk[:n], Go[k]) < TOL_G, k
    assert rel(gs.cpu().numpy(), gso) < TOL_G
    assert abs(f.item() - Fo) <= TOL_F * max(abs(Fo), 1.0)


def test_host_slice_matches_device_slice(sg):
    dims, R = (300, 200, 100), 32
    idx, val, A, s = zipf_case(dims, 5000, R, seed=3)
    with make_ctx(sg, dims, R, "bernoulli_logit", A, p=2000, q=2000, seed=8) as ctx:
        Gd, gsd, fd = ctx.gradient(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), t=4)
        Gh, gsh, fh = ctx.gradient(dev(s), [dev(a) for a in A], idx=torch.from_numpy(idx).pin_memory(),
                                   vals=torch.from_numpy(val).pin_memory(), t=4)
        ctx.check()
        for k in range(3):
            assert rel(Gh[k].cpu().numpy(), Gd[k].cpu().numpy()) < 1e-6


@pytest.fixture(scope="module")
def full_size_case():
    cfg = S.workload("sparse_binary_zipf")
    idx, val = S.sparse_slice(cfg, 1)
    A = S.init_factors(cfg)
    rng = np.random.default_rng(5)
    s = (rng.random(cfg["rank"]) + 0.5).astype(np.float32)
    Go, gso, Fo = gcp.sampled_gradient(idx, val, cfg["dims"], s, A, cfg["loss"], cfg["p"], cfg["q"], 2024, 1, 0)
    return cfg, idx, val, A, s, (Go, gso, Fo)


@pytest.mark.parametrize("hot_rows", [-1, 0, 64])
def test_full_size_sparse_binary_zipf_gradient(sg, full_size_case, hot_rows):
    """The benchmark workload itself: 10000 x 5000 x 2000, 1e6 Zipf nonzeros, R = 32,
    Bernoulli-logit, 1e5 + 1e5 samples, in the launch configuration the bench times; with the
    default number of shared-memory hot rows per mode, none, and the most."""
    cfg, idx, val, A, s, (Go, gso, Fo) = full_size_case
    dims, R = cfg["dims"], cfg["rank"]
    with make_ctx(sg, dims, R, cfg["loss"], A, p=cfg["p"], q=cfg["q"], p_obj=cfg["p_obj"], q_obj=cfg["q_obj"],
                  seed=2024, hot_rows=hot_rows) as ctx:
        # factor gradient alone (the launch the factor solver makes), then temporal gradient + loss
        G, _, _ = ctx.gradient(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), t=1, draw=0,
                               want=sg.WANT_FACTORS)
        _, gs, f = ctx.gradient(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), t=1, draw=0,
                                want=sg.WANT_TEMPORAL | sg.WANT_LOSS)
        ctx.check()
    for k in range(3):
        assert rel(G[k].cpu().numpy(), Go[k]) < TOL_G, (k, rel(G[k].cpu().numpy(), Go[k]))
        # every row, cold rows included (the hot-row shared-memory flush and the direct scatters)
        assert row_err(G[k].cpu().numpy(), Go[k]) < TOL_G, (k, row_err(G[k].cpu().numpy(), Go[k]))
    assert rel(gs.cpu().numpy(), gso) < TOL_G
    assert abs(f.item() - Fo) <= TOL_F * max(abs(Fo), 1.0)
