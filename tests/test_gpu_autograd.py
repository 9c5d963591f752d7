"""The GCPLoss autograd Function: forward = GCP loss, backward = the fused
gradient kernel (m recomputed), checked against the oracle's gradient and
against central finite differences of the forward."""
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


def test_dense_poisson_backward_matches_oracle_and_finite_differences(sg):
    from paper_2110_14514_gb300.autograd import gcp_loss
    cfg = S.workload("dense_poisson_3way")
    X_np, _ = S.dense_slice(cfg, 3)
    A_np = S.init_factors(cfg)
    s_np = np.full(cfg["rank"], 0.5, np.float32)
    X = torch.from_numpy(X_np).cuda()
    A = [torch.from_numpy(a).cuda().requires_grad_(True) for a in A_np]
    s = torch.from_numpy(s_np).cuda().requires_grad_(True)
    p = sg.params(cfg["dims"], cfg["rank"], "poisson")
    with sg.Context(p, [a.detach() for a in A]) as ctx:
        F = gcp_loss(ctx, s, A, X=X)
        (3.0 * F).backward()                    # grad_out = 3 reaches the kernel as y_scale
        Go, gso, Fo = gcp.dense_gradient(X_np, s_np, A_np, "poisson")
        assert abs(F.item() - Fo) <= 1e-4 * abs(Fo)
        for k in range(3):
            assert rel(A[k].grad.cpu().numpy(), 3.0 * Go[k]) < 1e-5
        assert rel(s.grad.cpu().numpy(), 3.0 * gso) < 1e-5


def test_backward_matches_central_differences_of_the_forward(sg):
    """Directional central difference of the forward (FP32 entries, double sum) on a small
    Poisson slice whose model values stay well away from zero."""
    from paper_2110_14514_gb300.autograd import gcp_loss
    dims, R = (30, 25, 20), 8
    rng = np.random.default_rng(0)
    A_np = [(0.3 + 0.7 * rng.random((n, R))).astype(np.float32) for n in dims]
    s_np = (0.5 + rng.random(R)).astype(np.float32)
    X = torch.from_numpy(rng.poisson(2.0, dims).astype(np.float32)).cuda()
    A = [torch.from_numpy(a).cuda().requires_grad_(True) for a in A_np]
    s = torch.from_numpy(s_np).cuda().requires_grad_(True)
    p = sg.params(dims, R, "poisson")
    with sg.Context(p, [a.detach() for a in A]) as ctx:
        gcp_loss(ctx, s, A, X=X).backward()
        V = [torch.from_numpy(rng.standard_normal(a.shape).astype(np.float32)).cuda() for a in A_np]
        vs = torch.from_numpy(rng.standard_normal(R).astype(np.float32)).cuda()
        an = sum(float((a.grad.double() * v.double()).sum()) for a, v in zip(A, V)) + \
            float((s.grad.double() * vs.double()).sum())
        h = 1e-2
        with torch.no_grad():
            Fp = gcp_loss(ctx, s + h * vs, [a + h * v for a, v in zip(A, V)], X=X).item()
            Fm = gcp_loss(ctx, s - h * vs, [a - h * v for a, v in zip(A, V)], X=X).item()
    fd = (Fp - Fm) / (2 * h)
    assert abs(fd - an) <= 1e-3 * abs(an), (fd, an)


def test_sparse_backward_is_the_sampled_gradient(sg):
    from paper_2110_14514_gb300.autograd import gcp_loss
    dims, R = (300, 200, 100), 16
    cfg = S.workload("sparse_binary_zipf")
    idx_np, val_np = S.sparse_slice(cfg, 5, nnz=8000, dims=dims)
    rng = np.random.default_rng(1)
    A_np = [(0.5 * rng.standard_normal((n, R))).astype(np.float32) for n in dims]
    s_np = (rng.random(R) + 0.5).astype(np.float32)
    A = [torch.from_numpy(a).cuda().requires_grad_(True) for a in A_np]
    s = torch.from_numpy(s_np).cuda().requires_grad_(True)
    p = sg.params(dims, R, "bernoulli_logit", p=3000, q=3000, seed=8)
    with sg.Context(p, [a.detach() for a in A]) as ctx:
        F = gcp_loss(ctx, s, A, idx=torch.from_numpy(idx_np).cuda(), vals=torch.from_numpy(val_np).cuda(), t=2, draw=4)
        F.backward()
    Go, gso, Fo = gcp.sampled_gradient(idx_np, val_np, dims, s_np, A_np, "bernoulli_logit", 3000, 3000, 8, 2, 4)
    assert abs(F.item() - Fo) <= 1e-4 * abs(Fo)
    for k in range(3):
        assert rel(A[k].grad.cpu().numpy(), Go[k]) < 1e-5
    assert rel(s.grad.cpu().numpy(), gso) < 1e-5


def test_graph_captured_step_matches_oracle_after_new_inputs(sg):
    """GraphedGCPLoss: forward + backward captured once; after new values are written into the
    static slice and factors, a replay gives the oracle's loss and gradients at the new point."""
    from paper_2110_14514_gb300.autograd import GraphedGCPLoss
    cfg = S.workload("dense_poisson_3way")
    A_np = S.init_factors(cfg)
    s_np = np.full(cfg["rank"], 0.5, np.float32)
    X = torch.from_numpy(S.dense_slice(cfg, 3)[0]).cuda()
    A = [torch.from_numpy(a).cuda().requires_grad_(True) for a in A_np]
    s = torch.from_numpy(s_np).cuda().requires_grad_(True)
    p = sg.params(cfg["dims"], cfg["rank"], "poisson")
    with sg.Context(p, [a.detach() for a in A]) as ctx:
        step = GraphedGCPLoss(ctx, s, A, X=X)
        rng = np.random.default_rng(11)
        for t in (4, 5):
            X2 = S.dense_slice(cfg, t)[0]
            A2 = [(a * (0.9 + 0.2 * rng.random(a.shape))).astype(np.float32) for a in A_np]
            s2 = (s_np * (0.8 + 0.4 * rng.random(s_np.shape))).astype(np.float32)
            with torch.no_grad():
                X.copy_(torch.from_numpy(X2))
                s.copy_(torch.from_numpy(s2))
                for a, a2 in zip(A, A2):
                    a.copy_(torch.from_numpy(a2))
            F = step.replay().item()
            Go, gso, Fo = gcp.dense_gradient(X2, s2, A2, "poisson")
            assert abs(F - Fo) <= 1e-4 * abs(Fo)
            for k in range(3):
                assert rel(A[k].grad.cpu().numpy(), Go[k]) < 1e-5
            assert rel(s.grad.cpu().numpy(), gso) < 1e-5
        ctx.check()
