"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, and the ctypes structs have the C layout (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sgcp.h")


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2110_14514_gb300 as sg
    return sg


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sgcp_[a-z_0-9]+)\s*\(", src)))


def test_header_functions_are_exported(sg):
    names = declared_functions()
    assert "sgcp_gradient" in names and "sgcp_step" in names and len(names) >= 17
    lib = ctypes.CDLL(sg.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    bound = {n for n, _, _ in sg.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_struct_layout_matches_c(sg, tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sgcp.h"\n'
        "int main(void){\n"
        'printf("%zu %zu %zu %zu\\n", sizeof(sgcp_params), sizeof(sgcp_slice), sizeof(sgcp_grad_opts), sizeof(sgcp_stats_t));\n'
        'printf("%zu %zu %zu %zu %zu\\n", offsetof(sgcp_params, lambda), offsetof(sgcp_params, p_obj), '
        "offsetof(sgcp_params, zero_attempt_cap), offsetof(sgcp_params, seed), offsetof(sgcp_stats_t, kernels_launched));\n"
        'printf("%zu %zu %zu %zu\\n", sizeof(sgcp_tune_entry), sizeof(sgcp_batch_opts), offsetof(sgcp_tune_entry, us), '
        "offsetof(sgcp_batch_opts, spin_limit));\n"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    assert sizes[:4] == [ctypes.sizeof(sg.sgcp_params), ctypes.sizeof(sg.sgcp_slice),
                         ctypes.sizeof(sg.sgcp_grad_opts), ctypes.sizeof(sg.sgcp_stats_t)]
    assert sizes[4:9] == [sg.sgcp_params.lambda_.offset, sg.sgcp_params.p_obj.offset,
                          sg.sgcp_params.zero_attempt_cap.offset, sg.sgcp_params.seed.offset,
                          sg.sgcp_stats_t.kernels_launched.offset]
    assert sizes[9:] == [ctypes.sizeof(sg.sgcp_tune_entry), ctypes.sizeof(sg.sgcp_batch_opts),
                         sg.sgcp_tune_entry.us.offset, sg.sgcp_batch_opts.spin_limit.offset]


def test_defaults_follow_table_2(sg):
    p = sg.params((10, 20, 30), 8)
    assert (p.beta1, p.beta2, p.adam_eps, p.tau_w, p.tau_f, p.theta, p.lambda_, p.mu) == \
        (0.9, 0.999, 1e-8, 100, 100, 1.0, 0.0, 0.0)
    assert p.tol_w == float("-inf") and p.zero_attempt_cap == 64


def test_argument_errors_are_synchronous_without_a_gpu(sg):
    out = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 3)()
    bad = sg.params((10, 20, 30), 6)           # rank not a multiple of 4
    assert sg.sgcp_create(ctypes.byref(bad), arr, 0, None, None, 0, None, None, ctypes.byref(out)) == sg.ERR_UNSUPPORTED
    bad = sg.params((10, 20, 30, 4, 5)[:4], 8, precision=sg.PREC_BF16_MTTKRP)
    bad.ndim = 5
    assert sg.sgcp_create(ctypes.byref(bad), arr, 0, None, None, 0, None, None, ctypes.byref(out)) == sg.ERR_UNSUPPORTED
    bad = sg.params((10, 20, 30), 8, "poisson", temporal=sg.TEMPORAL_LSQ)
    assert sg.sgcp_create(ctypes.byref(bad), arr, 0, None, None, 0, None, None, ctypes.byref(out)) in (sg.ERR_ARG, sg.ERR_CUDA)
    assert sg.sgcp_create(None, arr, 0, None, None, 0, None, None, ctypes.byref(out)) == sg.ERR_ARG
    half = sg.sgcp_allocator()                 # an allocator without a free callback
    half.alloc = sg.ALLOC_FN(lambda n, u: None)
    good = sg.params((10, 20, 30), 8)
    assert sg.sgcp_create(ctypes.byref(good), arr, 0, None, None, 0, ctypes.byref(half), None,
                          ctypes.byref(out)) == sg.ERR_ARG
    assert sg.sgcp_status_string(sg.ERR_SAMPLING_LIMIT) == b"SGCP_ERR_SAMPLING_LIMIT"
    assert sg.sgcp_params_default(None) == sg.ERR_ARG


def test_noalloc_alignment_errors_are_synchronous_without_a_gpu(sg):
    """s, A[k], G_out[k] off a 16-byte boundary are refused before any device work (the pointer
    values below are never dereferenced)."""
    p = sg.params((100, 80, 60), 8, "bernoulli_logit", p=64, q=64)
    opts = sg.sgcp_grad_opts(want=sg.WANT_FACTORS)
    A_ok = (ctypes.c_void_p * 3)(0x10000, 0x20000, 0x30000)
    G_ok = (ctypes.c_void_p * 3)(0x40000, 0x50000, 0x60000)
    A_bad = (ctypes.c_void_p * 3)(0x10000, 0x20004, 0x30000)
    G_bad = (ctypes.c_void_p * 3)(0x40000, 0x50000, 0x60008)
    def call(s, A, G):
        return sg.sgcp_gradient_sparse_noalloc(ctypes.byref(p), 10, 0x70000, 0x80000, s, A, ctypes.byref(opts), G,
                                               None, None, None, None)
    assert call(0x90004, A_ok, G_ok) == sg.ERR_ARG
    assert call(0x90000, A_bad, G_ok) == sg.ERR_ARG
    assert call(0x90000, A_ok, G_bad) == sg.ERR_ARG


def test_no_cpu_fallback_when_cuda_is_missing(sg):
    """Without a device the library refuses to create a context (it never computes on the host)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    out = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 3)()
    p = sg.params((10, 20, 30), 8)
    assert sg.sgcp_create(ctypes.byref(p), arr, 0, None, None, 0, None, None, ctypes.byref(out)) == sg.ERR_CUDA


def test_batch_argument_errors_are_synchronous_without_a_gpu(sg):
    """sgcp_batch_create validates every stream before touching the device."""
    out = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 6)(*([1] * 6))   # non-NULL placeholders: never dereferenced on these paths
    def create(plist, opts=None):
        pa = (sg.sgcp_params * len(plist))(*plist)
        return sg.sgcp_batch_create(len(plist), pa, arr, ctypes.byref(opts) if opts else None, None, None,
                                    ctypes.byref(out))
    good = sg.params((40, 50, 60), 16)
    assert create([good, sg.params((40, 50), 16)]) == sg.ERR_UNSUPPORTED           # 2-way slice
    assert create([good, sg.params((40, 50, 60), 80)]) == sg.ERR_UNSUPPORTED       # rank above 64
    assert create([good, sg.params((40, 50, 60), 16, precision=sg.PREC_F64)]) == sg.ERR_UNSUPPORTED
    assert create([good, sg.params((40, 50, 60), 16, optimizer=sg.OPT_LBFGS)]) == sg.ERR_UNSUPPORTED
    assert create([good, sg.params((40, 50, 60), 16, kappa_f=33)]) == sg.ERR_ARG
    opts = sg.sgcp_batch_opts()
    assert sg.sgcp_batch_opts_default(ctypes.byref(opts)) == sg.OK
    assert (opts.autotune, opts.tune_reps, opts.grid_blocks, opts.spin_limit) == (0, 3, 0, 0)
    bad_entry = (sg.sgcp_tune_entry * 1)()
    bad_entry[0].b1log, bad_entry[0].n1, bad_entry[0].n2 = 1, 1, 1             # tile row split out of range
    opts.table, opts.n_table = bad_entry, 1
    assert create([good], opts) == sg.ERR_ARG
    assert sg.sgcp_batch_create(0, None, arr, None, None, None, ctypes.byref(out)) == sg.ERR_ARG
    assert sg.sgcp_batch_check(None) == sg.ERR_ARG
    # an allocator needs both callbacks (checked before any device work)
    half = sg.sgcp_allocator()
    half.alloc = sg.ALLOC_FN(lambda n, u: None)
    pa = (sg.sgcp_params * 1)(good)
    assert sg.sgcp_batch_create(1, pa, arr, None, ctypes.byref(half), None, ctypes.byref(out)) == sg.ERR_ARG


def test_objective_read_back_argument_errors_without_a_gpu(sg):
    """The asynchronous objective read-backs check their handles and output pointer before any
    CUDA call."""
    buf = (ctypes.c_double * 4)()
    assert sg.sgcp_objectives_async(None, buf) == sg.ERR_ARG
    assert sg.sgcp_objectives_async(None, None) == sg.ERR_ARG
    assert sg.sgcp_batch_objectives_async(None, buf) == sg.ERR_ARG
    assert sg.sgcp_batch_objectives_async(None, None) == sg.ERR_ARG


def test_every_entry_point_cites_its_passage():
    """Each function the header declares sits under a comment (shared by a run of declarations
    with no blank line between) that cites the passage of the paper defining its operation
    (Alg., eq., Sec. or Table) or says it is library plumbing with no such passage."""
    src = open(HEADER).read()
    tokens = re.finditer(r"/\*.*?\*/|\b(sgcp_[a-z_0-9]+)\s*\(", src, flags=re.S)
    last_comment, last_end, seen = None, 0, {}
    for m in tokens:
        if m.group(0).startswith("/*"):
            last_comment = re.sub(r"\s*\n\s*\*?\s*", " ", m.group(0))   # one line, no leading '*'
            last_end = m.end()
            continue
        between = src[last_end:m.start()]
        if last_comment is None or re.search(r"\n[ \t]*\n", between):
            seen.setdefault(m.group(1), None)
            continue
        seen.setdefault(m.group(1), last_comment)
    names = declared_functions()
    assert set(names) <= set(seen), set(names) - set(seen)
    cite = re.compile(r"Alg\. \d|eqs?\. |Sec\. \d|Table \d|library plumbing")
    missing = [n for n in names if not (seen[n] and cite.search(seen[n]))]
    assert not missing, missing
