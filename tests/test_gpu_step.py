"""GPU parity of the whole OnlineGCP step (Alg. 1 body: temporal solve, factor
solve with history, reservoir update) against the oracle, teacher-forced on
the per-epoch accept/reject decisions the GPU took."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synthetic as S
from oracle import gcp, solver


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


def oracle_params(P, **kw):
    return solver.Params(**kw)


def run_stream(sg, p, A0, slices, okw, tol, check_own=False, ftol=None):
    """Step the library and the oracle through the same slices (teacher-forced on the GPU's
    accept / reject bits) and compare the state after every step: s, the factor matrices and the
    history weights within `tol` (per-array relative Frobenius error), the objective estimates
    F_w, F_f within `ftol` (relative to max(|F|, 1); default `tol`)."""
    ftol = tol if ftol is None else ftol
    ctx = sg.Context(p, [dev(a) for a in A0])
    og = solver.OnlineGCP(solver.Params(**okw), [a.astype(np.float64) for a in A0])
    try:
        for t, X in enumerate(slices, start=1):
            if "X" in X:
                ctx.step(X=dev(X["X"]))
                Xo = solver.Slice(dims=okw["dims"], X=X["X"])
            else:
                ctx.step(idx=dev(X["idx"]), vals=dev(X["val"]))
                Xo = solver.Slice(dims=okw["dims"], idx=X["idx"], val=X["val"])
            st = ctx.stats()
            ctx.last_stats = st
            assert st["error_bits"] == 0 and st["t"] == t
            dw = bits(st["accept_w"], st["epochs_w"]) if okw.get("temporal", "adam") == "adam" else []
            df = bits(st["accept_f"], st["epochs_f"])
            lw, lf = len(og.log_w), len(og.log_f)
            out = og.step(Xo, decisions_w=iter(dw), decisions_f=iter(df))
            if check_own:
                assert [e["own"] for e in og.log_w[lw:]] == dw
                assert [e["own"] for e in og.log_f[lf:]] == df
            A, s, tt = ctx.factors()
            assert tt == t
            assert rel(s.cpu().numpy(), out["s"]) < tol, ("s", t, rel(s.cpu().numpy(), out["s"]))
            for k in range(len(A0)):
                assert rel(A[k].cpu().numpy(), og.Abar[k]) < tol, ("A", t, k, rel(A[k].cpu().numpy(), og.Abar[k]))
            assert abs(st["F_f"] - out["F_f"]) <= ftol * max(abs(out["F_f"]), 1.0), (st["F_f"], out["F_f"])
            if out["F_w"] is not None:
                assert abs(st["F_w"] - out["F_w"]) <= ftol * max(abs(out["F_w"]), 1.0), (st["F_w"], out["F_w"])
            assert st["iter"] == og.i
            h, sh = ctx.history()
            assert h == og.hist_t
            if h:
                assert rel(sh.cpu().numpy(), np.array(og.hist_s)) < tol
    finally:
        ctx.close()
    return ctx


def test_dense_2way_fp64_stream_matches_oracle(sg):
    """The 20 x 30, R = 4, Gaussian FP64 stream with a history window of 3 over 6 slices:
    FP64 on both sides, so the GPU's own accept/reject decisions must equal the oracle's."""
    cfg = S.workload("dense_gaussian_2way")
    A0 = S.init_factors(cfg)
    slices = [{"X": S.dense_slice(cfg, t)[0]} for t in range(1, 7)]
    kw = dict(H=3, w=1.0, theta=0.9, kappa_w=3, tau_w=8, alpha_w=0.05, kappa_f=3, tau_f=8, alpha_f=0.01, seed=77)
    p = sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=sg.PREC_F64, **kw)
    okw = dict(dims=cfg["dims"], rank=cfg["rank"], loss="gaussian", **kw)
    run_stream(sg, p, A0, slices, okw, tol=1e-9, check_own=True)


def test_dense_2way_lsq_temporal_fp64(sg):
    cfg = S.workload("dense_gaussian_2way")
    A0 = S.init_factors(cfg)
    slices = [{"X": S.dense_slice(cfg, t)[0]} for t in range(1, 5)]
    kw = dict(H=2, kappa_f=2, tau_f=6, alpha_f=0.01, lam=0.1, mu=0.2, seed=3)
    p = sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=sg.PREC_F64, temporal=sg.TEMPORAL_LSQ, **kw)
    okw = dict(dims=cfg["dims"], rank=cfg["rank"], loss="gaussian", temporal="lsq", **kw)
    run_stream(sg, p, A0, slices, okw, tol=1e-9, check_own=True)


def test_dense_3way_fp32_poisson_stream(sg):
    dims, R = (30, 25, 20), 8
    rng = np.random.default_rng(1)
    At = [rng.random((n, R)) for n in dims]
    A0 = [(a + 0.1 * rng.random(a.shape)).astype(np.float32) for a in At]
    slices = []
    for t in range(4):
        st = rng.random(R)
        M = np.einsum("ir,jr,kr,r->ijk", *At, st)
        slices.append({"X": rng.poisson(M).astype(np.float32)})
    kw = dict(H=2, w=2.0, kappa_w=2, tau_w=10, alpha_w=0.05, kappa_f=2, tau_f=10, alpha_f=0.005, seed=5)
    p = sg.params(dims, R, "poisson", **kw)
    okw = dict(dims=dims, rank=R, loss="poisson", **kw)
    run_stream(sg, p, A0, slices, okw, tol=2e-5, ftol=1e-5)


@pytest.mark.parametrize("loss", ["bernoulli_logit", "poisson"])
def test_sparse_stream_matches_oracle(sg, loss):
    dims, R = (120, 90, 60), 8
    cfg = S.workload("sparse_binary_zipf")
    rng = np.random.default_rng(2)
    A0 = [(0.3 * rng.random((n, R)) + 0.05).astype(np.float32) for n in dims]
    slices = []
    for t in range(1, 5):
        # growing slices: the second one needs a larger nonzero hash (2^14 slots instead of 2^13),
        # which the step graph, captured at the first step, must then use
        idx, val = S.sparse_slice(cfg, t, nnz=3000 + 800 * t, dims=dims)
        slices.append({"idx": idx, "val": val})
    kw = dict(H=2, w=1.0, kappa_w=2, tau_w=6, alpha_w=0.05, kappa_f=2, tau_f=6, alpha_f=0.01,
              p=800, q=800, p_obj=1500, q_obj=1500, seed=99)
    p = sg.params(dims, R, loss, **kw)
    okw = dict(dims=dims, rank=R, loss=loss, **kw)
    run_stream(sg, p, A0, slices, okw, tol=2e-5, ftol=1e-5)


@pytest.mark.parametrize("R,alpha_f", [(12, 0.01), (32, 0.01), (32, 3.0)])
def test_sparse_fp32_history_factor_update_ranks_and_rollbacks(sg, R, alpha_f):
    """FP32 factor solve with history at R = 12 and 32 on modes whose row counts are not multiples of
    the update's 64-row blocks: the update forms the next iteration's history coefficients itself,
    and with alpha_f = 3 epochs are rejected, so an epoch restarts from rolled-back factors (the Gram
    chain runs again there)."""
    dims = (300, 170, 90)
    cfg = S.workload("sparse_binary_zipf")
    rng = np.random.default_rng(R)
    A0 = [(0.3 * rng.random((n, R)) + 0.05).astype(np.float32) for n in dims]
    slices = []
    for t in range(1, 4):
        idx, val = S.sparse_slice(cfg, t, nnz=6000, dims=dims)
        slices.append({"idx": idx, "val": val})
    kw = dict(H=3, w=1.0, kappa_w=2, tau_w=5, alpha_w=0.05, kappa_f=3, tau_f=5, alpha_f=alpha_f,
              p=900, q=900, p_obj=1500, q_obj=1500, seed=31)
    p = sg.params(dims, R, "bernoulli_logit", **kw)
    okw = dict(dims=dims, rank=R, loss="bernoulli_logit", **kw)
    ctx = run_stream(sg, p, A0, slices, okw, tol=2e-5, ftol=1e-5)
    if alpha_f > 1.0:
        st = ctx.last_stats
        assert st["epochs_f"] > 0 and st["accept_f"] != (1 << st["epochs_f"]) - 1, "no epoch was rejected"


@pytest.mark.parametrize("dims,nnz,pq", [((60, 50), 600, 200), ((30, 20, 15, 12), 3000, 600)])
def test_sparse_fp32_history_two_and_four_way(sg, dims, nnz, pq):
    """The FP32 factor update with history on 2-way and 4-way slices (its blocks hold one mode each
    and form B_k, C_k over the other d - 1 modes)."""
    R = 8
    cfg = S.workload("sparse_binary_zipf")
    rng = np.random.default_rng(len(dims))
    A0 = [(0.3 * rng.random((n, R)) + 0.05).astype(np.float32) for n in dims]
    slices = []
    for t in range(1, 4):
        idx, val = S.sparse_slice(cfg, t, nnz=nnz, dims=dims)
        slices.append({"idx": idx, "val": val})
    kw = dict(H=2, w=1.0, kappa_w=2, tau_w=5, alpha_w=0.05, kappa_f=2, tau_f=5, alpha_f=0.01,
              p=pq, q=pq, p_obj=pq, q_obj=pq, seed=17)
    p = sg.params(dims, R, "bernoulli_logit", **kw)
    okw = dict(dims=dims, rank=R, loss="bernoulli_logit", **kw)
    run_stream(sg, p, A0, slices, okw, tol=2e-5, ftol=1e-5)


def test_full_size_sparse_step_with_history(sg):
    """Two steps of the 10000 x 5000 x 2000 stream itself (1e6 Zipf nonzeros per slice, R = 32,
    Bernoulli-logit, p = q = p' = q' = 1e5) with a history window, so the second step's factor
    solve runs the history terms: the factor update at full size (17000 rows), its FP32 Gram sums
    over every block, and the hot-row tables inside the solve.  Short solves (kappa = 1,
    tau = 3) keep the oracle at a few seconds; teacher-forced."""
    cfg = S.workload("sparse_binary_zipf")
    dims, R = cfg["dims"], cfg["rank"]
    A0 = S.init_factors(cfg)
    slices = []
    for t in range(1, 3):
        idx, val = S.sparse_slice(cfg, t)
        slices.append({"idx": idx, "val": val})
    kw = dict(H=2, w=1.0, theta=0.9, lam=1e-3, kappa_w=1, tau_w=3, alpha_w=0.1, kappa_f=1, tau_f=3, alpha_f=1e-3,
              p=cfg["p"], q=cfg["q"], p_obj=cfg["p_obj"], q_obj=cfg["q_obj"], seed=2025)
    p = sg.params(dims, R, cfg["loss"], **kw)
    okw = dict(dims=dims, rank=R, loss=cfg["loss"], **kw)
    ctx = run_stream(sg, p, A0, slices, okw, tol=2e-5, ftol=1e-5)
    assert ctx.last_stats["hist_len"] == 2   # step 2 solved against the window {1}, then added itself


def test_checkpoint_resume_continues_the_trajectory(sg):
    cfg = S.workload("dense_gaussian_2way")
    A0 = S.init_factors(cfg)
    slices = [S.dense_slice(cfg, t)[0] for t in range(1, 6)]
    kw = dict(H=2, kappa_w=2, tau_w=5, alpha_w=0.05, kappa_f=2, tau_f=5, alpha_f=0.01, seed=12)
    p = sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=sg.PREC_F64, **kw)
    with sg.Context(p, [dev(a) for a in A0]) as full:
        for X in slices:
            full.step(X=dev(X))
        Af, sf, tf = full.factors()
        stf = full.stats()
    with sg.Context(p, [dev(a) for a in A0]) as first:
        for X in slices[:3]:
            first.step(X=dev(X))
        blob = first.state_export()
    with sg.Context(p, [dev(a) for a in A0]) as resumed:
        resumed.state_import(blob)
        for X in slices[3:]:
            resumed.step(X=dev(X))
        Ar, sr, tr = resumed.factors()
        st = resumed.stats()
    assert tr == tf == 5 and st["iter"] == stf["iter"]
    for a, b in zip(Ar, Af):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-12
    assert rel(sr.cpu().numpy(), sf.cpu().numpy()) < 1e-12


def test_dense_2way_lbfgs_fp64_stream_matches_oracle(sg):
    """Projected L-BFGS factor solver (two-loop recursion, Armijo backtracking) with the LSQ
    temporal solve and a history window: FP64 on both sides."""
    cfg = S.workload("dense_gaussian_2way")
    A0 = S.init_factors(cfg)
    slices = [{"X": S.dense_slice(cfg, t)[0]} for t in range(1, 5)]
    kw = dict(H=2, lam=0.05, lbfgs_iters=8, lbfgs_mem=3, seed=4)
    p = sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=sg.PREC_F64, temporal=sg.TEMPORAL_LSQ,
                  optimizer=sg.OPT_LBFGS, **kw)
    okw = dict(dims=cfg["dims"], rank=cfg["rank"], loss="gaussian", temporal="lsq", optimizer="lbfgs", **kw)
    run_stream(sg, p, A0, slices, okw, tol=1e-8)


def test_dense_3way_fp32_lbfgs_decreases_the_objective(sg):
    dims, R = (30, 25, 20), 8
    rng = np.random.default_rng(11)
    At = [rng.random((n, R)) for n in dims]
    A0 = [(a + 0.2 * rng.random(a.shape)).astype(np.float32) for a in At]
    X = rng.poisson(np.einsum("ir,jr,kr,r->ijk", *At, rng.random(R) + 0.5)).astype(np.float32)
    p = sg.params(dims, R, "poisson", optimizer=sg.OPT_LBFGS, lbfgs_iters=15, H=0, kappa_w=2, tau_w=10, alpha_w=0.05)
    with sg.Context(p, [dev(a) for a in A0]) as ctx:
        ctx.step(X=dev(X))
        st = ctx.stats()
        A1, s1, _ = ctx.factors()
    Xo = solver.Slice(dims=dims, X=X.astype(np.float64))
    P = solver.Params(dims=dims, rank=R, loss="poisson")
    F0 = solver.full_objective(Xo, [a.astype(np.float64) for a in A0], s1.cpu().numpy(), A0, [], [], P)
    F1 = solver.full_objective(Xo, [a.cpu().numpy().astype(np.float64) for a in A1], s1.cpu().numpy(), A0, [], [], P)
    assert st["epochs_f"] >= 1 and F1 < F0
    assert abs(st["F_f"] - F1) <= 1e-4 * abs(F1)


def test_lbfgs_step_is_one_asynchronous_graph(sg):
    """The L-BFGS factor solve runs inside the step's graph (line searches as device-side WHILE
    loops): with a 0.2 s sleep kernel queued ahead of it on the context stream, sgcp_step returns
    while the stream is still busy, i.e. without waiting for any result on the host; the step
    then gives the same factors as a step taken on an idle stream."""
    import time
    cfg = S.workload("dense_gaussian_2way")
    A0 = S.init_factors(cfg)
    X1, X2 = S.dense_slice(cfg, 1)[0], S.dense_slice(cfg, 2)[0]
    kw = dict(H=2, lam=0.05, lbfgs_iters=6, lbfgs_mem=3, seed=4)
    p = sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=sg.PREC_F64, temporal=sg.TEMPORAL_LSQ,
                  optimizer=sg.OPT_LBFGS, **kw)
    with sg.Context(p, [dev(a) for a in A0]) as ref:
        ref.step(X=dev(X1))
        ref.step(X=dev(X2))
        Ar, sr, _ = ref.factors()
        st_r = ref.stats()
    with sg.Context(p, [dev(a) for a in A0]) as ctx:
        ctx.step(X=dev(X1))                 # builds the graph
        ctx.check()
        x2 = dev(X2)
        with torch.cuda.stream(ctx.stream):
            torch.cuda._sleep(int(0.2 * 2.0e9))
        t0 = time.perf_counter()
        ctx.step(X=x2)
        host_s = time.perf_counter() - t0
        busy = not ctx.stream.query()
        A, s, _ = ctx.factors()
        st = ctx.stats()
    assert busy and host_s < 0.1, host_s
    assert st["epochs_f"] == st_r["epochs_f"] >= 1
    for a, b in zip(A, Ar):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-12
    assert rel(s.cpu().numpy(), sr.cpu().numpy()) < 1e-12


@pytest.mark.parametrize("kind", ["dense_fp64", "dense_fp32", "sparse"])
def test_stored_slice_history_stream_matches_oracle(sg, kind):
    """The stored-slice history of eq. gcp_stream_problem_1: the window keeps the slices, and the
    factor solve adds sum_h w_h sum_i f(x_ih, m_ih) at (A, s_h) (sampled per stored slice for
    sparse slices).  H = 2 over 5 slices so the reservoir replaces stored slices; FP64 with the
    GPU's own decisions, FP32 teacher-forced."""
    if kind == "sparse":
        dims, R = (120, 90, 60), 8
        cfg = S.workload("sparse_binary_zipf")
        rng = np.random.default_rng(8)
        A0 = [(0.3 * rng.random((n, R)) + 0.05).astype(np.float32) for n in dims]
        slices = [dict(zip(("idx", "val"), S.sparse_slice(cfg, t, nnz=3000 + 500 * t, dims=dims)))
                  for t in range(1, 6)]
        kw = dict(H=2, w=1.5, theta=0.8, kappa_w=2, tau_w=5, alpha_w=0.05, kappa_f=2, tau_f=5, alpha_f=0.01,
                  p=700, q=700, p_obj=1200, q_obj=1200, seed=19)
        loss, prec, tol, ftol = "bernoulli_logit", sg.PREC_F32, 2e-5, 1e-5
    elif kind == "dense_fp32":
        dims, R = (30, 25, 20), 8
        rng = np.random.default_rng(9)
        At = [rng.random((n, R)) for n in dims]
        A0 = [(a + 0.1 * rng.random(a.shape)).astype(np.float32) for a in At]
        slices = [{"X": rng.poisson(np.einsum("ir,jr,kr,r->ijk", *At, rng.random(R))).astype(np.float32)}
                  for _ in range(5)]
        kw = dict(H=2, w=2.0, theta=0.9, kappa_w=2, tau_w=8, alpha_w=0.05, kappa_f=2, tau_f=8, alpha_f=0.005, seed=5)
        loss, prec, tol, ftol = "poisson", sg.PREC_F32, 2e-5, 1e-5
    else:
        cfg = S.workload("dense_gaussian_2way")
        dims, R = cfg["dims"], cfg["rank"]
        A0 = S.init_factors(cfg)
        slices = [{"X": S.dense_slice(cfg, t)[0]} for t in range(1, 6)]
        kw = dict(H=2, w=1.0, theta=0.9, lam=0.01, kappa_w=2, tau_w=6, alpha_w=0.05, kappa_f=3, tau_f=6,
                  alpha_f=0.02, seed=23)
        loss, prec, tol, ftol = "gaussian", sg.PREC_F64, 1e-9, 1e-9
    p = sg.params(dims, R, loss, precision=prec, history_kind=sg.HISTORY_SLICES, **kw)
    okw = dict(dims=dims, rank=R, loss=loss, history="slices", **kw)
    run_stream(sg, p, A0, slices, okw, tol=tol, ftol=ftol, check_own=(kind == "dense_fp64"))


def test_stored_slice_history_rejects_lbfgs_mixed_slices_and_checkpoints(sg):
    cfg = S.workload("dense_gaussian_2way")
    A0 = [dev(a) for a in S.init_factors(cfg)]
    with pytest.raises(sg.SgcpError) as e:
        sg.Context(sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=sg.PREC_F64, H=2,
                             history_kind=sg.HISTORY_SLICES, optimizer=sg.OPT_LBFGS), A0)
    assert e.value.status == sg.ERR_UNSUPPORTED
    p = sg.params(cfg["dims"], cfg["rank"], "gaussian", H=2, history_kind=sg.HISTORY_SLICES, kappa_w=1, tau_w=2,
                  kappa_f=1, tau_f=2, p=10, q=10, p_obj=10, q_obj=10)
    A32 = [a.float() for a in A0]
    with sg.Context(p, A32) as ctx:
        ctx.step(X=dev(S.dense_slice(cfg, 1)[0].astype(np.float32)))
        idx = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(sg.SgcpError) as e:
            ctx.step(idx=idx, vals=torch.ones(1, device="cuda"))
        assert e.value.status == sg.ERR_ARG
        with pytest.raises(sg.SgcpError) as e:
            ctx.state_export()
        assert e.value.status == sg.ERR_UNSUPPORTED


def test_objective_read_back_without_draining_the_stream(sg):
    """sgcp_objectives_async queues each step's (F_w, F_f) copy behind that step: four steps from
    pinned host slices with no host wait in between give, after one wait, the last values that
    sgcp_stats reports, and every step's values agree with a context stepped with a wait after each
    step (FP32 atomic sums: relative 1e-5)."""
    dims, R = (300, 170, 90), 16
    cfg = S.workload("sparse_binary_zipf")
    rng = np.random.default_rng(5)
    A0 = [(0.3 * rng.random((n, R)) + 0.05).astype(np.float32) for n in dims]
    host = []
    for t in range(1, 5):
        idx, val = S.sparse_slice(cfg, t, nnz=6000, dims=dims)
        host.append((torch.from_numpy(np.ascontiguousarray(idx)).pin_memory(),
                     torch.from_numpy(np.ascontiguousarray(val)).pin_memory()))
    kw = dict(H=2, w=1.0, kappa_w=2, tau_w=5, alpha_w=0.05, kappa_f=2, tau_f=5, alpha_f=0.01,
              p=900, q=900, p_obj=1500, q_obj=1500, seed=23)
    p = sg.params(dims, R, "bernoulli_logit", **kw)
    ref = []
    with sg.Context(p, [dev(a) for a in A0]) as ctx:
        for i, v in host:
            ctx.step(idx=i, vals=v)
            st = ctx.stats()
            ref.append((st["F_w"], st["F_f"]))
    out = torch.full((len(host), 2), float("nan"), dtype=torch.float64).pin_memory()
    with sg.Context(p, [dev(a) for a in A0]) as ctx:
        for k, (i, v) in enumerate(host):
            ctx.step(idx=i, vals=v)
            ctx.objectives_async(out[k])
        ctx.stream.synchronize()
        ctx.check()
        st = ctx.stats()
        assert out[-1, 0].item() == st["F_w"] and out[-1, 1].item() == st["F_f"]
    got = out.numpy()
    assert np.isfinite(got).all()
    for k, (fw, ff) in enumerate(ref):
        assert abs(got[k, 0] - fw) <= 1e-5 * max(abs(fw), 1.0), (k, got[k, 0], fw)
        assert abs(got[k, 1] - ff) <= 1e-5 * max(abs(ff), 1.0), (k, got[k, 1], ff)
    assert len({float(x) for x in got[:, 1]}) == len(host)   # one value per step, not one repeated
