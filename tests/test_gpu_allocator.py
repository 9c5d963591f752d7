"""The sgcp_allocator hook: a caller's memory manager owns every device buffer of a context or a
batch.  With torch's caching allocator the state appears in torch's own accounting and goes back
to it on destroy, and the results equal those of a context that allocates by itself; an
allocator that fails makes the call return SGCP_ERR_OOM and leaves nothing allocated."""
import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synthetic as S


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


def allocated():
    """torch's count of allocated device bytes once unreachable objects (left by earlier tests)
    have been collected and the device is idle."""
    gc.collect()
    torch.cuda.synchronize()
    return torch.cuda.memory_allocated()


class Counting:
    """torch's caching allocator behind a counter: the allocation numbered fail_at (0-based) and
    every later one fail; live holds the addresses handed out and not yet freed."""

    def __init__(self, sg, stream, fail_at=None):
        self.calls = 0
        self.fail_at = fail_at
        self.live = set()

        def alloc(n):
            k = self.calls
            self.calls += 1
            if self.fail_at is not None and k >= self.fail_at:
                return 0
            ptr = torch.cuda.caching_allocator_alloc(n, stream=stream)
            self.live.add(ptr)
            return ptr

        def free(ptr):
            self.live.remove(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self.a = sg.Allocator(alloc, free)


def sparse_case():
    dims, R = (300, 200, 100), 16
    cfg = S.workload("sparse_binary_zipf")
    idx, val = S.sparse_slice(cfg, 1, nnz=6000, dims=dims)
    rng = np.random.default_rng(3)
    A0 = [(0.3 * rng.random((n, R)) + 0.05).astype(np.float32) for n in dims]
    kw = dict(H=2, kappa_w=1, tau_w=4, kappa_f=2, tau_f=4, p=1000, q=1000, p_obj=1000, q_obj=1000, seed=8)
    return dims, R, idx, val, A0, kw


def test_torch_caching_allocator_owns_the_context_state(sg):
    dims, R, idx, val, A0, kw = sparse_case()
    p = sg.params(dims, R, "bernoulli_logit", **kw)
    Ad = [dev(a) for a in A0]
    base = allocated()
    ref = sg.Context(p, Ad)
    ctx = sg.Context(p, Ad, allocator="torch")
    try:
        state = 8 * sum(dims) * R * 4               # A, Abar, G, u, v and three checkpoints
        assert torch.cuda.memory_allocated() - base >= state
        for t in range(2):                           # the first step allocates the hash lazily
            for c in (ref, ctx):
                c.step(idx=dev(idx), vals=dev(val))
        Ar, sr, _ = ref.factors()
        Aa, sa, _ = ctx.factors()
        ctx.check()
        ref.check()
        for k in range(3):
            assert rel(Aa[k].cpu().numpy(), Ar[k].cpu().numpy()) < 1e-5
        assert rel(sa.cpu().numpy(), sr.cpu().numpy()) < 1e-5
        assert abs(ctx.stats()["F_f"] - ref.stats()["F_f"]) <= 1e-5 * abs(ref.stats()["F_f"])
    finally:
        ref.close()
        ctx.close()
        del Aa, sa, Ar, sr
    assert allocated() == base


def test_failing_allocator_reports_oom_and_leaks_nothing(sg):
    dims, R, idx, val, A0, kw = sparse_case()
    p = sg.params(dims, R, "bernoulli_logit", **kw)
    Ad = [dev(a) for a in A0]
    stream = torch.cuda.Stream()
    ok = Counting(sg, stream)
    with sg.Context(p, Ad, stream=stream, allocator=ok.a):
        n_create = ok.calls
    assert n_create > 10 and not ok.live
    for k in sorted({0, 1, n_create // 2, n_create - 1}):
        bad = Counting(sg, stream, fail_at=k)
        with pytest.raises(sg.SgcpError) as e:
            sg.Context(p, Ad, stream=stream, allocator=bad.a)
        assert e.value.status == sg.ERR_OOM, k
        assert not bad.live, (k, len(bad.live))
    # a lazy allocation (the hash of the first sparse slice) that fails: the step reports OOM,
    # destroy frees everything that was obtained
    lazy = Counting(sg, stream, fail_at=n_create)
    ctx = sg.Context(p, Ad, stream=stream, allocator=lazy.a)
    with pytest.raises(sg.SgcpError) as e:
        ctx.step(idx=dev(idx), vals=dev(val))
    assert e.value.status == sg.ERR_OOM
    assert lazy.live
    ctx.close()
    assert not lazy.live


def test_batch_with_torch_allocator_and_failing_allocator(sg):
    rng = np.random.default_rng(4)
    shapes = [((37, 45, 70), 8, "gaussian"), ((20, 33, 31), 16, "poisson")]
    plist, init, X = [], [], []
    for s_, (dims, R, loss) in enumerate(shapes):
        plist.append(sg.params(dims, R, loss, H=2, kappa_w=2, tau_w=4, kappa_f=2, tau_f=4, seed=s_))
        init.append([dev((rng.random((n, R)) + 0.1).astype(np.float32)) for n in dims])
        X.append(dev(rng.poisson(1.0, dims).astype(np.float32)))
    base = allocated()
    with sg.Batch(plist, init) as ref, sg.Batch(plist, init, allocator="torch") as b:
        assert torch.cuda.memory_allocated() > base
        ref.step(X)
        b.step(X)
        b.check()
        ref.check()
        for s_ in range(len(shapes)):
            Ar, sr, _ = ref.factors(s_)
            Ab, sb, _ = b.factors(s_)
            for k in range(3):
                assert rel(Ab[k].cpu().numpy(), Ar[k].cpu().numpy()) < 1e-5
            assert rel(sb.cpu().numpy(), sr.cpu().numpy()) < 1e-5
        del Ar, sr, Ab, sb
    assert allocated() == base
    stream = torch.cuda.Stream()
    for k in (0, 3):
        bad = Counting(sg, stream, fail_at=k)
        with pytest.raises(sg.SgcpError) as e:
            sg.Batch(plist, init, stream=stream, allocator=bad.a)
        assert e.value.status == sg.ERR_OOM
        assert not bad.live
