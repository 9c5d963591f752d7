"""GPU parity of the dense fused gradient kernel (exact gradient over every entry)."""
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


def case(dims, R, loss, dtype, seed=0):
    rng = np.random.default_rng(seed)
    if loss in ("poisson", "bernoulli_odds"):
        A = [rng.random((n, R)).astype(dtype) + 0.05 for n in dims]
        s = (rng.random(R) + 0.2).astype(dtype)
    else:
        A = [(rng.standard_normal((n, R)) / np.sqrt(R) ** (1 / len(dims))).astype(dtype) for n in dims]
        s = (rng.random(R) + 0.5).astype(dtype)
    if loss == "gaussian":
        X = rng.standard_normal(dims).astype(dtype)
    elif loss == "poisson":
        X = rng.poisson(1.0, dims).astype(dtype)
    else:
        X = (rng.random(dims) < 0.3).astype(dtype)
    return X, A, s


def run(sg, X, A, s, loss, precision, want=7):
    dims, R = X.shape, A[0].shape[1]
    p = sg.params(dims, R, loss, precision=precision)
    with sg.Context(p, [dev(a) for a in A]) as ctx:
        G, gs, f = ctx.gradient(dev(s), [dev(a) for a in A], X=dev(X), want=want)
        ctx.check()
        return ([g.cpu().numpy() for g in G] if G is not None else None,
                gs.cpu().numpy() if gs is not None else None, f.item() if f is not None else None)


@pytest.mark.parametrize("loss", ["gaussian", "poisson", "bernoulli_logit", "bernoulli_odds"])
@pytest.mark.parametrize("dims,R", [((37, 45, 70), 16), ((33, 31, 29), 32), ((20, 70, 40), 64),
                                    ((8, 9, 40), 4), ((50, 3, 33), 12), ((41, 29, 67), 40), ((36, 50, 33), 48)])
def test_dense3_fp32_matches_oracle(sg, loss, dims, R):
    X, A, s = case(dims, R, loss, np.float32)
    G, gs, f = run(sg, X, A, s, loss, sg.PREC_F32)
    Go, gso, Fo = gcp.dense_gradient(X, s, A, loss)
    for k in range(3):
        assert rel(G[k], Go[k]) < 1e-5, (k, rel(G[k], Go[k]))
    assert rel(gs, gso) < 1e-5
    assert abs(f - Fo) <= 1e-4 * max(abs(Fo), 1.0)


@pytest.mark.parametrize("dims,R", [((20, 30), 4), ((70, 45), 16), ((33, 100), 64)])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_dense2(sg, dims, R, precision):
    dt = np.float64 if precision == "f64" else np.float32
    X, A, s = case(dims, R, "gaussian", dt, seed=1)
    G, gs, f = run(sg, X, A, s, "gaussian", sg.PREC_F64 if precision == "f64" else sg.PREC_F32)
    Go, gso, Fo = gcp.dense_gradient(X, s, A, "gaussian")
    tol = 1e-12 if precision == "f64" else 1e-5
    for k in range(2):
        assert rel(G[k], Go[k]) < tol, (k, rel(G[k], Go[k]))
    assert rel(gs, gso) < tol
    assert abs(f - Fo) <= (1e-12 if precision == "f64" else 1e-4) * max(abs(Fo), 1.0)


def test_dense3_fp64(sg):
    X, A, s = case((21, 34, 45), 16, "poisson", np.float64, seed=2)
    G, gs, f = run(sg, X, A, s, "poisson", sg.PREC_F64)
    Go, gso, Fo = gcp.dense_gradient(X, s, A, "poisson")
    for k in range(3):
        assert rel(G[k], Go[k]) < 1e-12
    assert rel(gs, gso) < 1e-12


def test_dense_loss_only_and_partial_wants(sg):
    X, A, s = case((30, 40, 50), 16, "poisson", np.float32, seed=3)
    Go, gso, Fo = gcp.dense_gradient(X, s, A, "poisson")
    G, gs, f = run(sg, X, A, s, "poisson", sg.PREC_F32, want=sg.WANT_LOSS)
    assert G is None and gs is None
    assert abs(f - Fo) <= 1e-4 * max(abs(Fo), 1.0)
    G, gs, f = run(sg, X, A, s, "poisson", sg.PREC_F32, want=sg.WANT_TEMPORAL)
    assert rel(gs, gso) < 1e-5


def test_misaligned_factor_or_gradient_pointer_is_an_argument_error(sg):
    """s, A[k], G_out[k] 4 bytes off a 16-byte boundary: rejected on the host, nothing launched."""
    X, A, s = case((20, 24, 28), 16, "gaussian", np.float32, seed=4)
    p = sg.params(X.shape, 16, "gaussian")
    with sg.Context(p, [dev(a) for a in A]) as ctx:
        Ad = [dev(a) for a in A]
        base = torch.zeros(A[1].size + 4, dtype=torch.float32, device="cuda")
        off = base[1:1 + A[1].size].view(A[1].shape)
        off.copy_(Ad[1])
        with pytest.raises(sg.SgcpError) as ei:
            ctx.gradient(dev(s), [Ad[0], off, Ad[2]], X=dev(X), want=sg.WANT_LOSS)
        assert ei.value.status == sg.ERR_ARG
        G = [torch.zeros_like(a) for a in Ad]
        gbase = torch.zeros(G[2].numel() + 4, dtype=torch.float32, device="cuda")
        G[2] = gbase[2:2 + G[2].numel()].view(G[2].shape)
        with pytest.raises(sg.SgcpError) as ei:
            ctx.gradient(dev(s), Ad, X=dev(X), want=sg.WANT_FACTORS, G=G)
        assert ei.value.status == sg.ERR_ARG
        sbase = torch.zeros(s.size + 1, dtype=torch.float32, device="cuda")
        s_off = sbase[1:]
        s_off.copy_(dev(s))
        with pytest.raises(sg.SgcpError) as ei:
            ctx.gradient(s_off, Ad, X=dev(X), want=sg.WANT_LOSS)
        assert ei.value.status == sg.ERR_ARG
        ctx.gradient(dev(s), Ad, X=dev(X), want=sg.WANT_FACTORS)   # the context is still usable
        ctx.check()


def test_full_size_dense_poisson_3way(sg):
    cfg = S.workload("dense_poisson_3way")
    X, _ = S.dense_slice(cfg, 1)
    A = S.init_factors(cfg)
    s = np.full(cfg["rank"], 0.5, np.float32)
    G, gs, f = run(sg, X, A, s, "poisson", sg.PREC_F32)
    Go, gso, Fo = gcp.dense_gradient(X, s, A, "poisson")
    for k in range(3):
        assert rel(G[k], Go[k]) < 1e-5
    assert rel(gs, gso) < 1e-5
    assert abs(f - Fo) <= 1e-4 * abs(Fo)


def test_full_size_dense_gaussian_3way_fp32(sg):
    cfg = S.workload("dense_gaussian_3way")
    X, s_true = S.dense_slice(cfg, 1)
    A = S.init_factors(cfg)
    s = s_true.astype(np.float32)
    G, gs, f = run(sg, X, A, s, "gaussian", sg.PREC_F32)
    Go, gso, Fo = gcp.dense_gradient(X, s, A, "gaussian")
    for k in range(3):
        assert rel(G[k], Go[k]) < 1e-5
    assert rel(gs, gso) < 1e-5
    assert abs(f - Fo) <= 1e-4 * abs(Fo)
