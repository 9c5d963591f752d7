"""GPU parity of the warm start (static GCP-SGD on the first slices stacked as a (d+1)-way tensor,
Sec. 4.4 / Sec. 6) against the oracle, of the stream that continues from it, and of the
OnlineSGD special case of OnlineGCP (Sec. 5)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synthetic as S
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def bits(mask, n):
    return [bool((mask >> e) & 1) for e in range(n)]


def check_warm(sg, ctx, og, S_gpu, S_o, st, F_o, tol, ftol):
    A, s, t = ctx.factors()
    assert t == og.t
    for k in range(len(A)):
        assert rel(A[k].cpu().numpy(), og.Abar[k]) < tol, ("A", k, rel(A[k].cpu().numpy(), og.Abar[k]))
    assert rel(S_gpu.cpu().numpy(), S_o) < tol, ("S", rel(S_gpu.cpu().numpy(), S_o))
    assert rel(s.cpu().numpy(), og.s) < tol
    assert abs(st["F"] - F_o) <= ftol * max(abs(F_o), 1.0), (st["F"], F_o)
    h, sh = ctx.history()
    assert h == og.hist_t
    assert rel(sh.cpu().numpy(), np.array(og.hist_s)) < tol


def continue_stream(ctx, og, slices, tol, ftol, check_own=False):
    for X in slices:
        if "X" in X:
            ctx.step(X=dev(X["X"]))
            Xo = solver.Slice(dims=og.P.dims, X=X["X"])
        else:
            ctx.step(idx=dev(X["idx"]), vals=dev(X["val"]))
            Xo = solver.Slice(dims=og.P.dims, idx=X["idx"], val=X["val"])
        st = ctx.stats()
        assert st["error_bits"] == 0
        dw = bits(st["accept_w"], st["epochs_w"]) if og.P.temporal == "adam" else []
        df = bits(st["accept_f"], st["epochs_f"])
        lw, lf = len(og.log_w), len(og.log_f)
        out = og.step(Xo, decisions_w=iter(dw), decisions_f=iter(df))
        if check_own:
            assert [e["own"] for e in og.log_w[lw:]] == dw and [e["own"] for e in og.log_f[lf:]] == df
        A, s, t = ctx.factors()
        assert t == og.t
        assert rel(s.cpu().numpy(), out["s"]) < tol
        for k in range(len(A)):
            assert rel(A[k].cpu().numpy(), og.Abar[k]) < tol
        assert abs(st["F_f"] - out["F_f"]) <= ftol * max(abs(out["F_f"]), 1.0)
        assert ctx.history()[0] == og.hist_t


def test_warm_start_dense_2way_fp64_and_the_stream_after_it(sg):
    """The 20 x 30, R = 4 Gaussian stream: warm start on its first 5 slices (history window 3, so
    the reservoir rule already replaces entries), then 3 streamed steps; FP64 on both sides, so
    every accept / reject decision is the GPU's own and must equal the oracle's."""
    cfg = S.workload("dense_gaussian_2way")
    A0 = S.init_factors(cfg)
    Xs = [S.dense_slice(cfg, t)[0] for t in range(1, 9)]
    kw = dict(H=3, w=1.0, theta=0.9, lam=0.01, kappa_w=2, tau_w=6, alpha_w=0.05, kappa_f=3, tau_f=8,
              alpha_f=0.02, seed=41)
    p = sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=sg.PREC_F64, **kw)
    P = solver.Params(dims=cfg["dims"], rank=cfg["rank"], loss="gaussian", **kw)
    with sg.Context(p, [dev(a) for a in A0]) as ctx:
        S_gpu, st = ctx.warm_start([dev(x) for x in Xs[:5]])
        log = []
        og, S_o, F_o = solver.warm_start([solver.Slice(dims=cfg["dims"], X=x) for x in Xs[:5]],
                                         [a.astype(np.float64) for a in A0], np.ones((5, cfg["rank"])), P, log=log)
        assert [e["own"] for e in log] == bits(st["accept"], st["epochs"])
        check_warm(sg, ctx, og, S_gpu, S_o, st, F_o, 1e-9, 1e-9)
        continue_stream(ctx, og, [{"X": x} for x in Xs[5:]], 1e-9, 1e-9, check_own=True)


def test_warm_start_dense_3way_fp32_poisson_from_given_weights(sg):
    dims, R, n = (30, 25, 20), 8, 4
    rng = np.random.default_rng(2)
    At = [rng.random((k, R)) for k in dims]
    A0 = [(a + 0.1 * rng.random(a.shape)).astype(np.float32) for a in At]
    Xs = [rng.poisson(np.einsum("ir,jr,kr,r->ijk", *At, rng.random(R))).astype(np.float32) for _ in range(n)]
    S0 = (rng.random((n, R)) + 0.5).astype(np.float32)
    kw = dict(H=5, kappa_f=3, tau_f=10, alpha_f=0.01, seed=3)
    p = sg.params(dims, R, "poisson", **kw)
    with sg.Context(p, [dev(a) for a in A0]) as ctx:
        S_gpu, st = ctx.warm_start([dev(x) for x in Xs], S_init=dev(S0))
        og, S_o, F_o = solver.warm_start([solver.Slice(dims=dims, X=x) for x in Xs], A0, S0,
                                         solver.Params(dims=dims, rank=R, loss="poisson", **kw),
                                         decisions=iter(bits(st["accept"], st["epochs"])))
        check_warm(sg, ctx, og, S_gpu, S_o, st, F_o, 2e-5, 1e-5)


def test_warm_start_sparse_fp32_with_host_slices_then_the_stream(sg):
    """Sparse Zipf slices (host COO, staged by the call) sampled per slice, teacher-forced; then two
    streamed steps from the warm-started state."""
    dims, R, n = (120, 90, 60), 8, 3
    cfg = S.workload("sparse_binary_zipf")
    rng = np.random.default_rng(4)
    A0 = [(0.3 * rng.random((k, R)) + 0.05).astype(np.float32) for k in dims]
    sl = [S.sparse_slice(cfg, t, nnz=4000, dims=dims) for t in range(1, n + 3)]
    kw = dict(H=2, kappa_w=2, tau_w=5, alpha_w=0.05, kappa_f=2, tau_f=6, alpha_f=0.01, p=800, q=800, p_obj=1500,
              q_obj=1500, seed=77)
    p = sg.params(dims, R, "bernoulli_logit", **kw)
    P = solver.Params(dims=dims, rank=R, loss="bernoulli_logit", **kw)
    with sg.Context(p, [dev(a) for a in A0]) as ctx:
        S_gpu, st = ctx.warm_start([(torch.from_numpy(i), torch.from_numpy(v)) for i, v in sl[:n]])
        og, S_o, F_o = solver.warm_start([solver.Slice(dims=dims, idx=i, val=v) for i, v in sl[:n]], A0,
                                         np.ones((n, R)), P, decisions=iter(bits(st["accept"], st["epochs"])))
        check_warm(sg, ctx, og, S_gpu, S_o, st, F_o, 2e-5, 1e-5)
        continue_stream(ctx, og, [{"idx": i, "val": v} for i, v in sl[n:]], 2e-5, 1e-5)


def test_warm_start_needs_a_fresh_context(sg):
    cfg = S.workload("dense_gaussian_2way")
    A0 = S.init_factors(cfg)
    X = S.dense_slice(cfg, 1)[0]
    p = sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=sg.PREC_F64, kappa_f=1, tau_f=2, kappa_w=1,
                  tau_w=2)
    with sg.Context(p, [dev(a) for a in A0]) as ctx:
        ctx.step(X=dev(X))
        with pytest.raises(sg.SgcpError) as e:
            ctx.warm_start([dev(X)])
        assert e.value.status == sg.ERR_ARG


def test_online_sgd_special_case_stream(sg):
    """Sec. 5: OnlineGCP with the Gaussian loss, the least-squares temporal solve, the dense
    gradient, no history window and one factor iteration per slice is OnlineSGD.  That setting
    through sgcp_step, FP64, against the oracle (whose first step is pinned to the closed form on
    the CPU), the GPU's own accept / reject decisions equal to the oracle's."""
    cfg = S.workload("dense_gaussian_2way")
    A0 = S.init_factors(cfg)
    Xs = [S.dense_slice(cfg, t)[0] for t in range(1, 11)]
    kw = dict(H=0, kappa_f=1, tau_f=1, alpha_f=0.05, seed=6)
    p = sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=sg.PREC_F64, temporal=sg.TEMPORAL_LSQ, **kw)
    og = solver.OnlineGCP(solver.Params(dims=cfg["dims"], rank=cfg["rank"], loss="gaussian", temporal="lsq", **kw),
                          [a.astype(np.float64) for a in A0])
    with sg.Context(p, [dev(a) for a in A0]) as ctx:
        continue_stream(ctx, og, [{"X": x} for x in Xs], 1e-9, 1e-9, check_own=True)
        st = ctx.stats()
        assert st["epochs_f"] == 1 and st["hist_len"] == 0
