"""The no-allocation sparse gradient entry point, against the FP64 oracle and the context-based one.

sgcp_gradient_sparse_noalloc serves callers that must not let the library
allocate device memory (a process that reserves its whole GPU memory budget
up front, or a loop where a synchronising cudaMalloc is not acceptable); it
keeps its hash table in a fixed array inside the library.  Two calls in a
row, on slices of different sizes, must each give the oracle's gradient for
the same draw (and what sgcp_gradient gives), the second must not see the
first call's table, and once the entry point has run on a device, further
calls leave the device's free memory unchanged.
"""
import ctypes

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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def outputs(dims, R, rows=None):
    """Output buffers pre-filled with 7 (a call that does not overwrite them shows up)."""
    rows = rows or dims
    G = [torch.full((n, R), 7.0, device="cuda") for n in rows]
    gs = torch.full((R,), 7.0, device="cuda")
    f = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    return G, gs, f, err


def noalloc_call(sg, p, idx, val, s, A, want, t, draw, sample_set, out, with_err=True):
    G, gs, f, err = out
    opts = sg.sgcp_grad_opts(want=want, sample_set=sample_set, t=t, draw=draw, accumulate=0, y_scale=None)
    st = sg.sgcp_gradient_sparse_noalloc(ctypes.byref(p), idx.shape[0], ctypes.c_void_p(idx.data_ptr()),
                                         ctypes.c_void_p(val.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                         sg._ptr_array(A), ctypes.byref(opts), sg._ptr_array(G),
                                         ctypes.c_void_p(gs.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                         ctypes.c_void_p(err.data_ptr() if with_err else 0),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == sg.OK, sg.sgcp_status_string(st)


def test_no_alloc_gradient_matches_the_oracle_twice(sg):
    dims, R = (3000, 2000, 700), 32
    cfg = S.workload("sparse_binary_zipf")
    rng = np.random.default_rng(21)
    A_np = [(0.5 * rng.standard_normal((n, R))).astype(np.float32) for n in dims]
    s_np = (rng.random(R) + 0.5).astype(np.float32)
    A = [dev(a) for a in A_np]
    s = dev(s_np)
    p = sg.params(dims, R, "bernoulli_logit", p=30000, q=30000, p_obj=20000, q_obj=20000, seed=314)
    want = sg.WANT_FACTORS | sg.WANT_TEMPORAL | sg.WANT_LOSS
    # a larger slice, then a smaller one: the second call uses a smaller part of the shared table
    calls = [(200000, 3, 11, sg.SAMPLES_FACTOR_GRAD), (30000, 4, 2, sg.SAMPLES_TEMPORAL_GRAD)]
    slices = [S.sparse_slice(cfg, 40 + c, nnz=nnz, dims=dims) for c, (nnz, _, _, _) in enumerate(calls)]
    dslices = [(dev(i), dev(v)) for i, v in slices]
    outs = [outputs(dims, R) for _ in calls]
    expected = []
    for (idx_np, val_np), (nnz, t, draw, sset) in zip(slices, calls):
        Go, gso, Fo = gcp.sampled_gradient(idx_np, val_np, dims, s_np, A_np, "bernoulli_logit", p.p, p.q, p.seed,
                                           t, draw, temporal=sset == sg.SAMPLES_TEMPORAL_GRAD)
        expected.append((Go, gso, Fo))

    def run_both(check):
        for c, ((idx, val), (nnz, t, draw, sset)) in enumerate(zip(dslices, calls)):
            noalloc_call(sg, p, idx, val, s, A, want, t, draw, sset, outs[c])
        torch.cuda.synchronize()
        for c, (G, gs, f, err) in enumerate(outs):
            Go, gso, Fo = expected[c]
            assert err.item() == 0, c
            for k in range(3):
                assert rel(G[k].cpu().numpy(), Go[k]) < TOL_G, (check, c, k)
            assert rel(gs.cpu().numpy(), gso) < TOL_G, (check, c)
            assert abs(f.item() - Fo) <= TOL_F * max(abs(Fo), 1.0), (check, c)

    run_both("first pass")     # also the set-up of this device (address of the scratch array)
    for o in outs:             # poison the outputs so that the second pass must write them again
        for g in o[0]:
            g.fill_(7.0)
        o[1].fill_(7.0)
        o[2].fill_(7.0)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    run_both("second pass")
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, (free_before, free_after)

    # and the context-based entry point on the same draws
    for c, ((idx, val), (nnz, t, draw, sset)) in enumerate(zip(dslices, calls)):
        with sg.Context(p, A) as ctx:
            Gr, gsr, fr = ctx.gradient(s, A, idx=idx, vals=val, want=want, t=t, draw=draw, sample_set=sset)
            ctx.check()
        G, gs, f, _ = outs[c]
        for k in range(3):
            assert rel(G[k].cpu().numpy(), Gr[k].cpu().numpy()) < TOL_G, (c, k)
        assert rel(gs.cpu().numpy(), gsr.cpu().numpy()) < TOL_G
        assert abs(f.item() - fr.item()) <= TOL_F * max(abs(fr.item()), 1.0)


@pytest.mark.parametrize("with_err", [True, False])
def test_no_alloc_out_of_range_coordinate(sg, with_err):
    """A coordinate equal to I_1 is reported in err_out (bit 1) when err_out is given, and with or
    without err_out no row past I_k is touched: the factor and gradient buffers carry padding rows,
    so even an unguarded access would stay inside them, and the padding keeps its value.  The
    samples that hit the bad entry are dropped; the rest equals the oracle's draw without them."""
    dims, R, pad, pq = (40, 30, 20), 8, 4, (4000, 100)
    rng = np.random.default_rng(8)
    lin = rng.choice(int(np.prod(dims)), 60, replace=False)
    idx_np = np.stack(np.unravel_index(lin, dims), axis=1).astype(np.int32)
    idx_np[17, 0] = dims[0]
    val_np = np.ones(60, np.float32)
    A_np = [(0.5 * rng.standard_normal((n + pad, R))).astype(np.float32) for n in dims]
    s_np = (rng.random(R) + 0.5).astype(np.float32)
    p = sg.params(dims, R, "bernoulli_logit", p=pq[0], q=pq[1], seed=5)
    out = outputs(dims, R, rows=[n + pad for n in dims])
    noalloc_call(sg, p, dev(idx_np), dev(val_np), dev(s_np), [dev(a) for a in A_np],
                 sg.WANT_FACTORS | sg.WANT_TEMPORAL | sg.WANT_LOSS, 2, 1, sg.SAMPLES_FACTOR_GRAD, out,
                 with_err=with_err)
    torch.cuda.synchronize()
    G, gs, f, err = out
    if with_err:
        assert err.item() & 1
    else:
        assert err.item() == -1
    A64 = [a[:n].astype(np.float64) for a, n in zip(A_np, dims)]
    coords, x, w = gcp.stratified_samples(idx_np, val_np, dims, pq[0], pq[1], 5, 2, 1, gcp.PURPOSE["grad_nz"],
                                          gcp.PURPOSE["grad_z"])
    keep = np.all(coords < np.asarray(dims)[None, :], axis=1)
    assert (~keep).sum() > 0
    uc, yt = gcp.strat_grad_tensor(coords[keep], x[keep], w[keep], s_np, A64, "bernoulli_logit")
    for k, n in enumerate(dims):
        Gk = G[k].cpu().numpy()
        assert np.all(Gk[n:] == 7.0), k
        assert rel(Gk[:n], gcp.sparse_mttkrp(uc, yt, s_np, A64, k)) < TOL_G, k
    assert rel(gs.cpu().numpy(), gcp.sparse_temporal(uc, yt, A64)) < TOL_G
    Fo = gcp.sampled_loss(coords[keep], x[keep], w[keep], s_np, A64, "bernoulli_logit")
    assert abs(f.item() - Fo) <= TOL_F * max(abs(Fo), 1.0)


def test_no_alloc_rejects_slices_beyond_its_scratch(sg):
    dims, R = (3000, 2000, 700), 8
    p = sg.params(dims, R, "bernoulli_logit", p=100, q=100, seed=1)
    A = [torch.zeros((n, R), device="cuda") for n in dims]
    s = torch.zeros(R, device="cuda")
    G = [torch.zeros_like(a) for a in A]
    idx = torch.zeros((262145, 3), dtype=torch.int32, device="cuda")
    val = torch.ones(262145, device="cuda")
    opts = sg.sgcp_grad_opts(want=sg.WANT_FACTORS, sample_set=0, t=1, draw=0, accumulate=0, y_scale=None)
    st = sg.sgcp_gradient_sparse_noalloc(ctypes.byref(p), 262145, ctypes.c_void_p(idx.data_ptr()),
                                         ctypes.c_void_p(val.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                         sg._ptr_array(A), ctypes.byref(opts), sg._ptr_array(G), None, None, None,
                                         None)
    assert st == sg.ERR_UNSUPPORTED
