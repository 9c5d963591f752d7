"""GPU parity of the batched-streams mode: every stream of a batch, advanced by
one persistent kernel per time step, against its own FP64 oracle stream
(Alg. 1 body), teacher-forced on the accept / reject decisions the GPU took."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import solver


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


def bits(mask, n):
    return [bool((mask >> e) & 1) for e in range(n)]


# uneven streams: ragged tiles, several units, Gram and update chunks, ranks 4..32, three losses
SHAPES = [((37, 45, 70), 8, "gaussian"), ((20, 33, 31), 4, "poisson"), ((70, 12, 40), 16, "gaussian"),
          ((9, 64, 65), 12, "poisson"), ((33, 40, 34), 32, "bernoulli_logit")]
KW = dict(H=2, w=1.5, theta=0.9, kappa_w=2, tau_w=6, alpha_w=0.05, kappa_f=2, tau_f=6, alpha_f=0.01, lam=0.01,
          mu=0.02)


def make_streams(n_steps, seed=3, shapes=SHAPES):
    rng = np.random.default_rng(seed)
    streams = []
    for s, (dims, R, loss) in enumerate(shapes):
        At = [rng.random((n, R)) for n in dims]
        A0 = [(a + 0.1 * rng.random(a.shape)).astype(np.float32) for a in At]
        Xs = []
        for t in range(n_steps):
            st = rng.random(R) + 0.2
            M = np.einsum("ir,jr,kr,r->ijk", *At, st) / R
            if loss == "gaussian":
                X = M + 0.05 * rng.standard_normal(dims)
            elif loss == "poisson":
                X = rng.poisson(M)
            else:
                X = (rng.random(dims) < M / (1.0 + M)).astype(np.float64)
            Xs.append(X.astype(np.float32))
        streams.append(dict(dims=dims, R=R, loss=loss, A0=A0, X=Xs, seed=100 + s))
    return streams


def run_and_compare(sg, streams, n_steps, tol, batch_kw=None, host=False, ftol=1e-5):
    """Every stream against its own oracle stream after every step: s and the factor matrices within
    `tol` (per-array relative Frobenius error), the objective estimates within `ftol`."""
    plist = [sg.params(st["dims"], st["R"], st["loss"], seed=st["seed"], **KW) for st in streams]
    init = [[torch.from_numpy(a).cuda() for a in st["A0"]] for st in streams]
    oracles = [solver.OnlineGCP(solver.Params(dims=st["dims"], rank=st["R"], loss=st["loss"], seed=st["seed"], **KW),
                                [a.astype(np.float64) for a in st["A0"]]) for st in streams]
    with sg.Batch(plist, init, **(batch_kw or {})) as b:
        for t in range(n_steps):
            X = [torch.from_numpy(st["X"][t]) for st in streams]
            b.step(X if host else [x.cuda() for x in X])
            for s, st in enumerate(streams):
                ss = b.stats(s)
                assert ss["error_bits"] == 0 and ss["t"] == t + 1
                dw = bits(ss["accept_w"], ss["epochs_w"])
                df = bits(ss["accept_f"], ss["epochs_f"])
                og = oracles[s]
                out = og.step(solver.Slice(dims=st["dims"], X=st["X"][t].astype(np.float64)),
                              decisions_w=iter(dw), decisions_f=iter(df))
                A, sv, tt = b.factors(s)
                assert tt == t + 1
                assert rel(sv.cpu().numpy(), out["s"]) < tol, (s, t, "s", rel(sv.cpu().numpy(), out["s"]))
                for k in range(3):
                    e = rel(A[k].cpu().numpy(), og.Abar[k])
                    assert e < tol, (s, t, "A", k, e)
                assert abs(ss["F_f"] - out["F_f"]) <= ftol * max(abs(out["F_f"]), 1.0), (s, t, ss["F_f"], out["F_f"])
                assert abs(ss["F_w"] - out["F_w"]) <= ftol * max(abs(out["F_w"]), 1.0), (s, t, ss["F_w"], out["F_w"])
                assert ss["iter"] == og.i and ss["hist_len"] == len(og.hist_t)
        return b.tune_table(), [b.unit_config(s) for s in range(len(streams))]


def test_batched_streams_match_their_oracles(sg):
    streams = make_streams(3)
    run_and_compare(sg, streams, 3, tol=2e-5)


# the large end of the batched workload: ranks 48 and 64 (the 64-column register tiles), modes of
# 128 to 160 rows (several Gram / update chunks per mode and many tile boxes per stream)
SHAPES_LARGE = [((130, 40, 36), 48, "gaussian"), ((33, 150, 47), 64, "poisson"), ((160, 32, 70), 64, "gaussian"),
                ((41, 37, 128), 24, "poisson")]


def test_batched_streams_at_ranks_48_and_64_with_long_modes(sg):
    """(Every gradient element of these slices sums up to 2e5 FP32 terms -- 130 x 40 x 36 -- whose
    rounding errors add up to ~sqrt(n) 2^-24 ~ 3e-5 relative, hence 1e-4 for the state.)"""
    streams = make_streams(2, seed=13, shapes=SHAPES_LARGE)
    run_and_compare(sg, streams, 2, tol=1e-4)


def test_batched_streams_host_slices(sg):
    """x_on_host = 1: the call copies the host slices itself."""
    streams = make_streams(2, seed=5)
    run_and_compare(sg, streams, 2, tol=2e-5, host=True)


def test_batched_host_slices_queued_without_waiting(sg):
    """Pinned host slices, three steps queued with no host wait (the staging buffers alternate and
    the third step refills the first while the second runs), every stream's (F_w, F_f) read back
    behind each step with sgcp_batch_objectives_async: the values agree with a batch that waits
    after every step (FP32 sums: 1e-5) and, after the last step, equal sgcp_batch_stats exactly."""
    n_steps = 3
    streams = make_streams(n_steps, seed=9)
    plist = [sg.params(st["dims"], st["R"], st["loss"], seed=st["seed"], **KW) for st in streams]
    n = len(streams)
    pinned = [[torch.from_numpy(st["X"][t]).pin_memory() for st in streams] for t in range(n_steps)]
    ref = []
    with sg.Batch(plist, [[torch.from_numpy(a).cuda() for a in st["A0"]] for st in streams]) as b:
        for t in range(n_steps):
            b.step(pinned[t])
            ref.append([(b.stats(s)["F_w"], b.stats(s)["F_f"]) for s in range(n)])
    out = torch.full((n_steps, 2 * n), float("nan"), dtype=torch.float64).pin_memory()
    with sg.Batch(plist, [[torch.from_numpy(a).cuda() for a in st["A0"]] for st in streams]) as b:
        for t in range(n_steps):
            b.step(pinned[t])
            b.objectives_async(out[t])
        b.stream.synchronize()
        b.check()
        last = [(b.stats(s)["F_w"], b.stats(s)["F_f"]) for s in range(n)]
    got = out.numpy()
    assert np.isfinite(got).all()
    for s in range(n):
        assert (got[-1, 2 * s], got[-1, 2 * s + 1]) == last[s], s
        for t in range(n_steps):
            for c in range(2):
                r = ref[t][s][c]
                assert abs(got[t, 2 * s + c] - r) <= 1e-5 * max(abs(r), 1.0), (t, s, c, got[t, 2 * s + c], r)


def test_autotuned_unit_shapes_keep_parity(sg):
    streams = make_streams(2, seed=7, shapes=SHAPES[:3])
    table, cfg = run_and_compare(sg, streams, 2, tol=2e-5, batch_kw=dict(autotune=True, tune_reps=2))
    assert len(table) == 3 and all(e["us"] > 0 for e in table)
    for e in cfg:
        assert 2 <= e["b1log"] <= 4 and (1 << e["b1log"]) * e["n1"] <= 32 and (64 >> e["b1log"]) * e["n2"] <= 32
    # a later batch reuses the table without timing again
    streams2 = make_streams(1, seed=8, shapes=SHAPES[:3])
    table2, cfg2 = run_and_compare(sg, streams2, 1, tol=2e-5, batch_kw=dict(table=table))
    assert cfg2 == cfg and len(table2) == 3


def test_single_shape_choice_across_tiles(sg):
    """The same stream under every valid tile shape gives the same result (the unit shape is a
    schedule, not arithmetic): compare each against the oracle."""
    streams = make_streams(1, seed=9, shapes=[((45, 37, 40), 8, "gaussian")])
    key = dict(bucket=(2, 2, 2), rank=8, loss=0, us=0.0)
    for b1log, n1, n2 in [(2, 1, 1), (2, 8, 2), (3, 2, 1), (4, 2, 8)]:
        run_and_compare(sg, streams, 1, tol=2e-5, batch_kw=dict(table=[dict(key, b1log=b1log, n1=n1, n2=n2)]))


def test_spin_limit_reports_timeout_without_hanging(sg):
    """A spin limit of one empty poll makes idle blocks give up at once: the step still completes
    (the block that publishes a phase always finds it), and the batch reports SGCP_ERR_TIMEOUT."""
    streams = make_streams(1, seed=11, shapes=SHAPES[:2])
    plist = [sg.params(st["dims"], st["R"], st["loss"], **KW) for st in streams]
    init = [[torch.from_numpy(a).cuda() for a in st["A0"]] for st in streams]
    with sg.Batch(plist, init, spin_limit=1) as b:
        b.step([torch.from_numpy(st["X"][0]).cuda() for st in streams])
        with pytest.raises(sg.SgcpError) as ei:
            b.check()
        assert ei.value.status == sg.ERR_TIMEOUT
        with pytest.raises(sg.SgcpError) as ei:
            b.step([torch.from_numpy(st["X"][0]).cuda() for st in streams])
        assert ei.value.status == sg.ERR_STATE
