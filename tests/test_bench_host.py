"""Host-side parts of bench.py that need no GPU: the reference arm's JSON line (the FP64 oracle
timed on host cores) and the multi-rank timing reduction, on two gloo ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "samples/s"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    sys.path.insert(0, ROOT)
    import bench
    import synthetic as S
    assert bench.run_reference(None, S.workload(bench.WORKLOAD), 2, 1) is None


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], torch.device("cpu"))
        q.put((rank, t, bench.whole_job_rate(world, 5, 1000.0, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_on_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [1.5, 2.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, rate in got:
        assert t == 2.5                                # every rank reports the slowest rank's time
        assert rate == pytest.approx(2 * 5 * 1000.0 / 2.5)


def test_single_process_max_is_the_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None) == 3.25
    assert bench.whole_job_rate(1, 4, 10.0, 2.0) == 20.0


# functions that make up bench.py's CPU-baseline legs (the oracle timed on host cores) and the
# helpers that only they reach
_BASELINE_LEGS = {"cpu_baseline", "batched_cpu_baseline", "dense_oracle_errors", "run_reference"}
_LEG_HELPERS = {"_oracle_init", "_oracle_sparse_worker", "OraclePool"}


def _guarded(node, parents):
    """True where `node` sits in a baseline leg, a leg helper, or the body of an `if` that tests
    --no-cpu-baseline or --impl."""
    import ast
    child = node
    while child in parents:
        p = parents[child]
        if isinstance(p, (ast.FunctionDef, ast.ClassDef)) and p.name in _BASELINE_LEGS | _LEG_HELPERS:
            return True
        if isinstance(p, ast.If) and child in p.body:
            names = {a.attr for a in ast.walk(p.test) if isinstance(a, ast.Attribute)}
            if names & {"no_cpu_baseline", "impl"}:
                return True
        child = p
    return False


def test_bench_reaches_the_oracle_only_from_its_baseline_legs():
    """bench.py imports the oracle only inside its CPU-baseline legs or behind their flags, and
    calls those legs only behind the same flags: the timed device path never runs oracle code."""
    import ast
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    parents = {c: p for p in ast.walk(tree) for c in ast.iter_child_nodes(p)}
    imports = [n for n in ast.walk(tree)
               if (isinstance(n, ast.ImportFrom) and (n.module or "").split(".")[0] == "oracle")
               or (isinstance(n, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in n.names))]
    assert len(imports) >= 3
    for n in imports:
        assert _guarded(n, parents), f"oracle imported outside a baseline leg at bench.py:{n.lineno}"
    uses = [n for n in ast.walk(tree) if isinstance(n, ast.Name) and n.id in _BASELINE_LEGS | _LEG_HELPERS]
    assert uses
    for n in uses:
        assert _guarded(n, parents), f"{n.id} used outside a baseline leg at bench.py:{n.lineno}"


def test_dense_record_errors_vanish_at_the_oracle_gradient():
    """dense_oracle_errors compares each precision's results with the oracle's FP64 gradient at
    the record's point: the oracle's own gradient scores zero, a perturbed one its perturbation."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from oracle import gcp
    _, X, _, s_pt, A_pt = bench.dense_record_point()
    Go, gso, Fo = gcp.dense_gradient(X, s_pt, A_pt, "gaussian")
    G2 = [g.copy() for g in Go]
    G2[1] *= 1.001
    err, timing = bench.dense_oracle_errors({"exact": (Go, gso, Fo), "g2": (G2, gso, Fo * (1 + 1e-6))})
    assert all(v == 0.0 for v in err["exact"].values()), err["exact"]
    assert err["g2"]["G1"] == 0.0 and err["g2"]["G3"] == 0.0 and err["g2"]["gs"] == 0.0
    assert abs(err["g2"]["G2"] - 1e-3) < 1e-9 and abs(err["g2"]["F"] - 1e-6) < 1e-9
    assert timing["kind"] == "oracle" and timing["cores"] == 1 and timing["value"] > 0
    assert np.isfinite(timing["value"])
