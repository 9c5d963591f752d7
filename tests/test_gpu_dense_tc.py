"""GPU parity of the tensor-core (tcgen05 / TMEM) dense gradient kernel.

MTTKRP operands are BF16 or FP16 with FP32 accumulation, so gradients must be
within 2e-2 relative (Frobenius, per array) of the FP64 oracle; the model m
is formed from split-BF16 products, so the loss stays close to FP32 accuracy.
The full-size 256^3, R = 64 test prints the error of every result for the
precision report (FP32 CUDA-core kernel, BF16 and FP16 tensor-core kernel).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synthetic as S
from oracle import gcp


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


def run(sg, X, A, s, loss, precision):
    dims, R = X.shape, A[0].shape[1]
    p = sg.params(dims, R, loss, precision=precision)
    with sg.Context(p, [dev(a) for a in A]) as ctx:
        G, gs, f = ctx.gradient(dev(s), [dev(a) for a in A], X=dev(X))
        ctx.check()
        return [g.cpu().numpy() for g in G], gs.cpu().numpy(), f.item()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("loss", ["gaussian", "poisson"])
@pytest.mark.parametrize("dims,R", [((20, 37, 300), 64), ((33, 40, 150), 32), ((9, 17, 130), 16), ((16, 30, 128), 48)])
def test_tensor_core_gradient_matches_oracle(sg, prec, loss, dims, R):
    rng = np.random.default_rng(R + len(loss))
    if loss == "poisson":
        A = [(0.2 + rng.random((n, R))).astype(np.float32) for n in dims]
        s = (0.2 + rng.random(R)).astype(np.float32)
        X = rng.poisson(1.5, dims).astype(np.float32)
    else:
        A = [(rng.standard_normal((n, R)) / R ** (1 / 6)).astype(np.float32) for n in dims]
        s = (0.5 + rng.random(R)).astype(np.float32)
        X = rng.standard_normal(dims).astype(np.float32)
    G, gs, f = run(sg, X, A, s, loss, sg.PREC_BF16_MTTKRP if prec == "bf16" else sg.PREC_F16_MTTKRP)
    Go, gso, Fo = gcp.dense_gradient(X, s, A, loss)
    for k in range(3):
        assert rel(G[k], Go[k]) < 2e-2, (k, rel(G[k], Go[k]))
    assert rel(gs, gso) < 2e-2
    assert abs(f - Fo) <= 1e-4 * abs(Fo), (f, Fo)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_blocks_spanning_i3_blocks_and_partial_wants(sg, prec):
    """234 tiles of 8 x 16 x 128 over 152 SMs: one block runs two tiles of different i3 blocks
    (the A3 panel is rebuilt and G3 flushed mid-run); each requested output alone and all three
    together."""
    rng = np.random.default_rng(17)
    dims, R = (97, 82, 260), 32
    A = [(rng.standard_normal((n, R)) / R ** (1 / 6)).astype(np.float32) for n in dims]
    s = (0.5 + rng.random(R)).astype(np.float32)
    X = rng.standard_normal(dims).astype(np.float32)
    Go, gso, Fo = gcp.dense_gradient(X, s, A, "gaussian")
    p = sg.params(dims, R, "gaussian", precision=sg.PREC_BF16_MTTKRP if prec == "bf16" else sg.PREC_F16_MTTKRP)
    with sg.Context(p, [dev(a) for a in A]) as ctx:
        Ad, sd, Xd = [dev(a) for a in A], dev(s), dev(X)
        for want in (sg.WANT_FACTORS, sg.WANT_TEMPORAL, sg.WANT_LOSS, sg.WANT_FACTORS | sg.WANT_TEMPORAL | sg.WANT_LOSS):
            G, gs, f = ctx.gradient(sd, Ad, X=Xd, want=want)
            ctx.check()
            if want & sg.WANT_FACTORS:
                for k in range(3):
                    assert rel(G[k].cpu().numpy(), Go[k]) < 2e-2, (want, k)
            else:
                assert G is None
            if want & sg.WANT_TEMPORAL:
                assert rel(gs.cpu().numpy(), gso) < 2e-2, want
            if want & sg.WANT_LOSS:
                assert abs(f.item() - Fo) <= 1e-4 * abs(Fo), (want, f.item(), Fo)


def test_precision_report_dense_gaussian_256(sg):
    """256^3, R = 64, Gaussian loss with noise at 1% of the planted RMS: error of every result
    against the FP64 oracle for the FP32 CUDA-core path and the BF16 / FP16 tensor-core paths."""
    cfg = S.workload("dense_gaussian_3way")
    X, s_true = S.dense_slice(cfg, 1)
    A_true = S.truth(cfg)
    rng = np.random.default_rng(9)
    # a point near the planted factors (where a solver spends its time)
    A = [(a + 0.05 * rng.standard_normal(a.shape)).astype(np.float32) for a in A_true]
    s = s_true.astype(np.float32)
    Go, gso, Fo = gcp.dense_gradient(X, s, A, "gaussian")
    report = {}
    for name, prec in [("fp32", sg.PREC_F32), ("bf16", sg.PREC_BF16_MTTKRP), ("fp16", sg.PREC_F16_MTTKRP)]:
        G, gs, f = run(sg, X, A, s, "gaussian", prec)
        report[name] = [rel(G[k], Go[k]) for k in range(3)] + [rel(gs, gso), abs(f - Fo) / abs(Fo)]
    for name, errs in report.items():
        print(f"precision {name}: rel err G1 {errs[0]:.3e} G2 {errs[1]:.3e} G3 {errs[2]:.3e} gs {errs[3]:.3e} F {errs[4]:.3e}")
    assert max(report["fp32"][:4]) < 1e-5 and report["fp32"][4] < 1e-4
    for name in ("bf16", "fp16"):
        assert max(report[name][:4]) < 2e-2
        assert report[name][4] < 1e-4
