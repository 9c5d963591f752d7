"""The no-allocation sparse gradient entry point against the context-based one.

sgcp_gradient_sparse_noalloc serves callers that must not let the library
allocate device memory (a process that reserves its whole GPU memory budget
up front, or a loop where a synchronising cudaMalloc is not acceptable); it
keeps its hash table in a fixed array inside the library.  Two calls in a
row, on slices of different sizes, must each give what sgcp_gradient gives
for the same draw, and the second must not see the first call's table.
"""
import ctypes

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


def noalloc_call(sg, p, idx, val, s, A, want, t, draw, sample_set=0):
    R = p.rank
    dims = [p.dims[k] for k in range(p.ndim)]
    G = [torch.full((n, R), 7.0, device="cuda") for n in dims]       # overwritten by the call
    gs = torch.full((R,), 7.0, device="cuda")
    f = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    opts = sg.sgcp_grad_opts(want=want, sample_set=sample_set, t=t, draw=draw, accumulate=0, y_scale=None)
    st = sg.sgcp_gradient_sparse_noalloc(ctypes.byref(p), idx.shape[0], ctypes.c_void_p(idx.data_ptr()),
                                         ctypes.c_void_p(val.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                         sg._ptr_array(A), ctypes.byref(opts), sg._ptr_array(G),
                                         ctypes.c_void_p(gs.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                         ctypes.c_void_p(err.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == sg.OK, sg.sgcp_status_string(st)
    torch.cuda.synchronize()
    assert err.item() == 0
    return G, gs, f


def test_no_alloc_gradient_matches_the_context_entry_point_twice(sg):
    dims, R = (3000, 2000, 700), 32
    cfg = S.workload("sparse_binary_zipf")
    rng = np.random.default_rng(21)
    A = [dev((0.5 * rng.standard_normal((n, R))).astype(np.float32)) for n in dims]
    s = dev((rng.random(R) + 0.5).astype(np.float32))
    p = sg.params(dims, R, "bernoulli_logit", p=30000, q=30000, p_obj=20000, q_obj=20000, seed=314)
    want = sg.WANT_FACTORS | sg.WANT_TEMPORAL | sg.WANT_LOSS
    # a larger slice, then a smaller one: the second call uses a smaller part of the shared table
    for call, (nnz, t, draw, sset) in enumerate([(200000, 3, 11, 0), (30000, 4, 2, 2)]):
        idx_np, val_np = S.sparse_slice(cfg, 40 + call, nnz=nnz, dims=dims)
        idx, val = dev(idx_np), dev(val_np)
        G, gs, f = noalloc_call(sg, p, idx, val, s, A, want, t, draw, sset)
        with sg.Context(p, A) as ctx:
            Gr, gsr, fr = ctx.gradient(s, A, idx=idx, vals=val, want=want, t=t, draw=draw, sample_set=sset)
            ctx.check()
        for k in range(3):
            assert rel(G[k].cpu().numpy(), Gr[k].cpu().numpy()) < 1e-5, (call, k)
        assert rel(gs.cpu().numpy(), gsr.cpu().numpy()) < 1e-5
        assert abs(f.item() - fr.item()) <= 1e-4 * max(abs(fr.item()), 1.0)


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
