"""Benchmark of the GB300 streaming-GCP library on the sparse sampled workload.

Workload: slices of 10000 x 5000 x 2000 with 1e6 Zipf(1.2) nonzeros (binary),
rank 32, Bernoulli-logit loss, stratified sampling of 1e5 nonzeros + 1e5
zeros per gradient and per objective estimate, history window 10 -- a step is
one OnlineGCP slice update (Alg. 1 body: 5 x 100 temporal-gradient
iterations, 5 x 100 factor-gradient iterations with history terms and ADAM,
12 objective estimates, reservoir update), run as one CUDA graph.

metric: fused-gradient sampled entries (nonzero + zero samples) processed per
second over whole slice updates; ms_per_step is the per-slice update time.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl native|reference]

--impl reference times the FP64 CPU oracle (arXiv 2110.14514 restated in
numpy) on the same metric, on a bounded sample of each step.
Under torchrun (N > 1) every rank runs its own independent stream (no data
exchange); the value is the total over ranks divided by the slowest rank's time.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

# The oracle baselines run on one host core: keep numpy's BLAS pools at one thread.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

WORKLOAD = "sparse_binary_zipf"
SOLVER = dict(H=10, w=1.0, theta=1.0, kappa_w=5, kappa_f=5, tau_w=100, tau_f=100, alpha_w=0.1, alpha_f=1e-3)
BYTES_PER_SAMPLE = 784      # 12 B coords + 4 B value + 3 x 128 B row gathers + 3 x 128 B row scatters (R = 32)
BYTES_PER_SAMPLE_TEMPORAL = 400   # 12 B coords + 4 B value + 3 x 128 B row gathers (no scatters)
N_SLICES = 4                # distinct slices cycled through (every step re-ingests its slice)
METRIC = "fused GCP gradient nnz/s"


def recorded_counters(summary="sparse_grad_factor_R32_zipf1e6.md"):
    """Counters of a dominant kernel from the machine-readable line of its committed ncu summary
    (key=value pairs: dram_bytes_per_launch, and where captured lts_bytes_per_launch,
    lts_throughput_pct), or {} when the kernel's source changed since that capture."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        line = re.search(r"machine-readable: (.*)", text).group(1)
        kv = dict(re.findall(r"(\w+)=(\S+)", line))
        src = open(os.path.join(ROOT, kv["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != kv["source_sha256_16"]:
            return {}
        return {k: float(v) if "." in v else int(v) for k, v in kv.items()
                if k not in ("kernel", "source", "source_sha256_16")}
    except Exception:
        return {}


def recorded_traffic(summary="sparse_grad_factor_R32_zipf1e6.md"):
    """DRAM bytes per launch of a dominant kernel from its committed ncu summary, or None when
    the kernel's source changed since that capture."""
    v = recorded_counters(summary).get("dram_bytes_per_launch")
    return int(v) if v is not None else None


def host_cores():
    """Host cores this process may run on (the oracle baselines' worker count)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


_ORACLE_SLICE = {}


def _oracle_init(idx, val, A):
    """Worker set-up: the slice and the factors, sent once per process."""
    _ORACLE_SLICE.update(idx=idx, val=val, A=A)


def _oracle_sparse_worker(job):
    """FP64 oracle sampled gradients of the worker's slice for `budget` seconds (at least one),
    each with its own draw index.  Returns (evaluations, seconds)."""
    from oracle import gcp
    dims, s, loss, p, q, draw0, budget, n_max = job
    d = _ORACLE_SLICE
    t0 = time.perf_counter()
    n = 0
    while n < n_max and (n == 0 or time.perf_counter() - t0 < budget):
        gcp.sampled_gradient(d["idx"], d["val"], dims, s, d["A"], loss, p, q, 7, 1, draw0 + n)
        n += 1
    return n, time.perf_counter() - t0


class OraclePool:
    """`workers` host processes running the oracle (spawned, so that no process is forked from one
    that holds a CUDA context), each holding the same slice; workers = 1 runs in this process."""

    def __init__(self, cfg, slice0, workers):
        self.cfg, self.workers = cfg, workers
        A = S.init_factors(cfg)
        if workers == 1:
            _oracle_init(slice0[0], slice0[1], A)
            self.pool = None
        else:
            import multiprocessing as mp
            self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_init,
                                                     initargs=(slice0[0], slice0[1], A))

    def rate(self, budget_s, n_max=10**9, draw0=0):
        """Samples/s over all workers: each runs independent draws of the slice for budget_s (at
        most n_max evaluations); all evaluations over the slowest worker's time."""
        c = self.cfg
        s = np.full(c["rank"], 0.5, np.float32)
        jobs = [(c["dims"], s, c["loss"], c["p"], c["q"], draw0 + 100000 * w, budget_s, n_max)
                for w in range(self.workers)]
        res = [_oracle_sparse_worker(jobs[0])] if self.pool is None else self.pool.map(_oracle_sparse_worker, jobs)
        n = sum(r[0] for r in res)
        return n * (c["p"] + c["q"]) / max(r[1] for r in res), n

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for n, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, device):
    """The largest of every rank's x (the slowest rank's time); x itself on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, units_per_step_per_rank, total_s):
    """Units processed by all ranks (weak scaling: each rank its own replica) per second of the
    slowest rank's timed region."""
    return world * steps * units_per_step_per_rank / total_s


def make_slices(cfg, n):
    return [S.sparse_slice(cfg, t) for t in range(1, n + 1)]


# ----------------------------------------------------------------------------- reference arm (oracle)
def run_reference(args, cfg, world, rank):
    """The FP64 oracle on the same metric: each step is a bounded sample of oracle sampled-gradient
    evaluations of the same slice, one per host core (one process per core)."""
    if rank != 0:
        return None
    cores = host_cores()
    pool = OraclePool(cfg, S.sparse_slice(cfg, 1), cores)
    try:
        for w in range(args.warmup):
            pool.rate(0.0, n_max=1, draw0=w)
        t0 = time.perf_counter()
        n_all = 0
        for k in range(args.steps):
            n_all += pool.rate(0.0, n_max=1, draw0=1000 + k)[1]
        t_all = time.perf_counter() - t0
    finally:
        pool.close()
    value = n_all * (cfg["p"] + cfg["q"]) / t_all
    sample = (f"{cores} FP64 numpy sampled-gradient evaluations per step (p + q = {cfg['p'] + cfg['q']} each; "
              f"one per host core, one process per core), same slice")
    return {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": workload_name(cfg), "step": sample},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def workload_name(cfg):
    return (f"{WORKLOAD}: slices {cfg['dims'][0]}x{cfg['dims'][1]}x{cfg['dims'][2]}, nnz={cfg['nnz']} Zipf(1.2), "
            f"R={cfg['rank']}, {cfg['loss']}, p=q={cfg['p']}, p'=q'={cfg['p_obj']}")


# ----------------------------------------------------------------------------- native arm
def run_native(args, cfg, world, rank, local):
    import torch
    import paper_2110_14514_gb300 as sg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    p = sg.params(cfg["dims"], cfg["rank"], cfg["loss"], p=cfg["p"], q=cfg["q"], p_obj=cfg["p_obj"],
                  q_obj=cfg["q_obj"], seed=1000 + rank, **SOLVER)
    A0 = [torch.from_numpy(a).to(dev) for a in S.init_factors(cfg, stream=rank)]
    host = make_slices(cfg, N_SLICES)
    dslices = [(torch.from_numpy(i).to(dev), torch.from_numpy(v).to(dev)) for i, v in host]
    pinned = [(torch.from_numpy(i).pin_memory(), torch.from_numpy(v).pin_memory()) for i, v in host]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    ctx = sg.Context(p, A0)
    stream = ctx.stream
    n_tmp = SOLVER["kappa_w"] * SOLVER["tau_w"]
    n_fac = SOLVER["kappa_f"] * SOLVER["tau_f"]
    n_obj = 2 + SOLVER["kappa_w"] + SOLVER["kappa_f"]
    grads_per_step = n_tmp + n_fac
    samples_per_step = grads_per_step * (cfg["p"] + cfg["q"])
    counters = recorded_counters()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for w in range(args.warmup):
        i, v = dslices[w % N_SLICES]
        ctx.step(idx=i, vals=v)
    ctx.check()
    k0 = ctx.stats()["kernels_launched"]
    clocks = Clocks(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(float(k))                     # L2 flush, outside the timed events
        i, v = dslices[(args.warmup + k) % N_SLICES]
        with torch.cuda.stream(stream):
            stream.wait_stream(torch.cuda.default_stream(dev))
            ev[k][0].record(stream)
            ctx.step(idx=i, vals=v)
            ev[k][1].record(stream)
    barrier()
    clk = clocks.stop()
    ctx.check()
    st = ctx.stats()
    launches = st["kernels_launched"] - k0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dev)
    value = whole_job_rate(world, args.steps, samples_per_step, total_s)

    # dominant kernel: the fused sampled factor gradient, timed alone back to back on the context stream
    i, v = dslices[0]
    s0 = torch.full((cfg["rank"],), 0.5, device=dev)
    A, _, _ = ctx.factors()
    G = [torch.zeros_like(a) for a in A]
    nrep = 200
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ctx.gradient(s0, A, idx=i, vals=v, want=sg.WANT_FACTORS, t=1, draw=0, G=G, accumulate=True)
        torch.cuda._sleep(50_000_000)             # keep the GPU busy while the launches queue up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for r in range(nrep):
            ctx.gradient(s0, A, idx=i, vals=v, want=sg.WANT_FACTORS, t=1, draw=r, G=G, accumulate=True)
        e1.record(stream)
    torch.cuda.synchronize()
    kern_s = e0.elapsed_time(e1) / 1e3 / nrep
    peak, peak_kind = peaks()
    achieved = BYTES_PER_SAMPLE * (cfg["p"] + cfg["q"]) / kern_s / 1e9

    # end to end through the C ABI with host buffers: H2D of the slice, D2H of the step's objective values
    # (every step's slice copied from pinned host memory inside sgcp_step; every step's F_w, F_f
    # copied back into its own pinned row behind that step, without draining the GPU in between)
    e2e_steps = max(2, min(args.steps, 5))
    f_host = torch.zeros((e2e_steps, 2), dtype=torch.float64).pin_memory()
    for w in range(2):                            # untimed: the two staging buffers are allocated here
        i, v = pinned[w % N_SLICES]
        ctx.step(idx=i, vals=v)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        i, v = pinned[k % N_SLICES]
        ctx.step(idx=i, vals=v)
        ctx.objectives_async(f_host[k])
    ctx.stream.synchronize()
    e2e_s = time.perf_counter() - t0
    ctx.check()
    if not bool(torch.isfinite(f_host).all()):
        raise RuntimeError("end-to-end steps returned a non-finite objective")
    h2d = int(host[0][0].nbytes + host[0][1].nbytes)
    d2h = 2 * 8
    e2e_value = world * e2e_steps * samples_per_step / e2e_s
    ctx.close()

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(cfg), "step": "one OnlineGCP slice update (graph)",
                       "factor_grads_per_step": n_fac, "temporal_grads_per_step": n_tmp,
                       "bytes_per_sample": {"factor_gradient": BYTES_PER_SAMPLE,
                                            "temporal_gradient": BYTES_PER_SAMPLE_TEMPORAL},
                       "objective_estimates_per_step": n_obj,
                       "value_counts": "samples of the factor and temporal gradients (p + q each); the "
                                       "objective estimates' samples are not counted",
                       "H": SOLVER["H"],
                       "l2": "flushed between steps by a 256 MB write (outside the per-step events)",
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": int(launches),
            "roofline": {"bound": "l2-latency (effective vs HBM)", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": recorded_traffic(), "peak_kind": peak_kind,
                         "traffic_note": "ncu dram read+write bytes per launch, cold caches (working set is L2-resident)",
                         "lts_bytes_per_launch": counters.get("lts_bytes_per_launch"),
                         "lts_throughput_pct": counters.get("lts_throughput_pct"),
                         "note": "achieved = 784 B x (p + q) per launch / CUDA-event launch time: the effective "
                                 "bandwidth of the algorithmic gathers and scatters, most of which L2 serves",
                         "kernel": "k_sparse_grad<3,32> (factor gradient, 2e5 samples)",
                         "kernel_us": kern_s * 1e6},
            "e2e": {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "note": "wall clock of steps queued back to back from pinned host slices, each step's F_w, "
                            "F_f read back; no L2 flush between these steps (the device-timed value flushes)"},
            "clocks": clk,
            "step_ms": {"min": min(step_ms), "max": max(step_ms)},
        }
        if not args.no_dense_record:
            out["dense_256_r64"], dense_results = dense_precision_record(dev)
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(cfg, host[0])
            if not args.no_dense_record:
                err, timing = dense_oracle_errors(dense_results)
                out["dense_256_r64"]["err_vs_fp64"] = err
                out["cpu_baseline"]["dense_256_r64"] = timing
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return out


def cpu_baseline(cfg, slice0, budget_s=10.0):
    """The oracle as it stands: FP64 numpy sampled gradients of the same slice, ~10 s on one core,
    then ~10 s on every host core (one process per core, independent draws)."""
    pool = OraclePool(cfg, slice0, 1)
    one, n1 = pool.rate(budget_s)
    cores = host_cores()
    allc, na = one, n1
    if cores > 1:
        pool = OraclePool(cfg, slice0, cores)
        try:
            pool.rate(0.0, n_max=1)                      # worker start-up outside the timing
            allc, na = pool.rate(budget_s, draw0=1)
        finally:
            pool.close()
    pq = cfg["p"] + cfg["q"]
    return {"value": allc, "unit": "samples/s", "cores": cores, "nproc": cores, "kind": "oracle",
            "sample": f"{na} FP64 oracle sampled-gradient evaluations (p + q = {pq}) of one slice on {cores} cores "
                      f"(one process per core, ~{budget_s:.0f} s each)",
            "one_core": {"value": one, "unit": "samples/s", "cores": 1,
                         "sample": f"{n1} evaluations on one core (~{budget_s:.0f} s)"}}


# ----------------------------------------------------------------------------- dense workload (precision study)
DENSE_SOLVER = dict(H=10, w=1.0, theta=1.0, kappa_w=20, kappa_f=5, tau_w=100, tau_f=100, alpha_w=10.0, alpha_f=1e-4)


def dense_record_point():
    """The 256^3, R = 64 Gaussian slices 1 and 2 and the point of the precision record: planted
    factors + 0.05 N(0,1) (seed 9) and the planted s_1 (inputs only; no gradient arithmetic)."""
    cfg = S.workload("dense_gaussian_3way")
    X, s_true = S.dense_slice(cfg, 1)
    X2, _ = S.dense_slice(cfg, 2)
    rng = np.random.default_rng(9)
    A_pt = [(a + 0.05 * rng.standard_normal(a.shape)).astype(np.float32) for a in S.truth(cfg)]
    return cfg, X, X2, s_true.astype(np.float32), A_pt


def dense_precision_record(dev, n_time=2):
    """The second half of the metric on the 256^3, R = 64 Gaussian slices: per-slice update time
    (sgcp_step with the Table 2 Gaussian-row solvers, kappa_w = 20, kappa_f = 5, tau = 100) and the
    dense factor-gradient kernel time for the plain FP32 path and the BF16 / FP16 tensor-core MTTKRP
    paths. Also returns every gradient result (G1, G2, G3, g_s, F) of each path at one point near
    the planted factors; the cpu_baseline leg compares them with the FP64 oracle
    (dense_oracle_errors)."""
    import torch
    import paper_2110_14514_gb300 as sg
    cfg, X, X2, s_pt, A_pt = dense_record_point()
    Xd = [torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(dev) for x in (X, X2)]
    A0 = [torch.from_numpy(a).to(dev) for a in S.init_factors(cfg)]
    Apd = [torch.from_numpy(a).to(dev) for a in A_pt]
    spd = torch.from_numpy(s_pt).to(dev)

    out = {"solver": DENSE_SOLVER, "point": "planted factors + 0.05 N(0,1), planted s_1"}
    results = {}
    for name, prec in (("fp32", sg.PREC_F32), ("bf16", sg.PREC_BF16_MTTKRP), ("fp16", sg.PREC_F16_MTTKRP)):
        p = sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=prec, seed=77, **DENSE_SOLVER)
        with sg.Context(p, A0) as ctx:
            G, gs, f = ctx.gradient(spd, Apd, X=Xd[0])
            ctx.check()
            results[name] = ([g.cpu().numpy() for g in G], gs.cpu().numpy(), f.item())
            ctx.step(X=Xd[0])                          # graph build and warm-up
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n_time)]
            with torch.cuda.stream(ctx.stream):
                for k in range(n_time):
                    ev[2 * k].record(ctx.stream)
                    ctx.step(X=Xd[(k + 1) % 2])
                    ev[2 * k + 1].record(ctx.stream)
            torch.cuda.synchronize()
            ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(n_time)) / n_time
            Gk = [torch.zeros_like(a) for a in Apd]
            nrep = 20
            with torch.cuda.stream(ctx.stream):
                ctx.gradient(spd, Apd, X=Xd[0], want=sg.WANT_FACTORS, G=Gk, accumulate=True)
                torch.cuda._sleep(20_000_000)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(ctx.stream)
                for r in range(nrep):
                    ctx.gradient(spd, Apd, X=Xd[r % 2], want=sg.WANT_FACTORS, G=Gk, accumulate=True)
                e1.record(ctx.stream)
            torch.cuda.synchronize()
            ctx.check()
        out[f"{name}_ms_per_slice"] = ms
        out[f"{name}_kernel_us"] = e0.elapsed_time(e1) * 1e3 / nrep
    out["bf16_speedup_vs_fp32_per_slice"] = out["fp32_ms_per_slice"] / out["bf16_ms_per_slice"]
    return out, results


def dense_oracle_errors(results):
    """cpu_baseline leg of the dense record: the FP64 oracle's gradient (loss + all gradients) of the
    record's slice at the record's point, timed on one host core, and the relative error of every
    result of each precision against it."""
    from oracle import gcp
    _, X, _, s_pt, A_pt = dense_record_point()
    t0 = time.perf_counter()
    Go, gso, Fo = gcp.dense_gradient(X, s_pt, A_pt, "gaussian")
    dt = time.perf_counter() - t0

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))
    err = {}
    for name, (G, gs, f) in results.items():
        err[name] = {f"G{k + 1}": rel(G[k], Go[k]) for k in range(3)}
        err[name]["gs"] = rel(gs, gso)
        err[name]["F"] = abs(f - Fo) / abs(Fo)
    timing = {"value": X.size / dt, "unit": "entries/s", "cores": 1, "kind": "oracle",
              "sample": "one FP64 oracle dense gradient (loss + all gradients) of one 256^3 slice, R = 64"}
    return err, timing


def run_native_dense(args, cfg, world, rank, local):
    """256^3, R = 64 Gaussian slices (Table 2 Gaussian row): per-slice update time and the dense
    gradient kernel's roofline for the FP32 CUDA-core or the BF16 / FP16 tensor-core path."""
    import torch
    import paper_2110_14514_gb300 as sg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = {"fp32": sg.PREC_F32, "bf16": sg.PREC_BF16_MTTKRP, "fp16": sg.PREC_F16_MTTKRP}[args.precision]
    lsq_lbfgs = args.solver == "lsq_lbfgs"
    extra = dict(temporal=sg.TEMPORAL_LSQ, optimizer=sg.OPT_LBFGS) if lsq_lbfgs else {}
    p = sg.params(cfg["dims"], cfg["rank"], cfg["loss"], precision=prec, seed=2000 + rank, **DENSE_SOLVER, **extra)
    A0 = [torch.from_numpy(a).to(dev) for a in S.init_factors(cfg, stream=rank)]
    n_sl = 2
    host = [S.dense_slice(cfg, t + 1, stream=rank)[0] for t in range(n_sl)]
    dsl = [torch.from_numpy(x).to(dev) for x in host]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx = sg.Context(p, A0)
    stream = ctx.stream
    omega = int(np.prod(cfg["dims"]))
    grads_per_step = DENSE_SOLVER["kappa_w"] * DENSE_SOLVER["tau_w"] + DENSE_SOLVER["kappa_f"] * DENSE_SOLVER["tau_f"]
    for w in range(args.warmup):
        ctx.step(X=dsl[w % n_sl])
    ctx.check()
    k0 = ctx.stats()["kernels_launched"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(float(k))
        with torch.cuda.stream(stream):
            stream.wait_stream(torch.cuda.default_stream(dev))
            ev[k][0].record(stream)
            ctx.step(X=dsl[(args.warmup + k) % n_sl])
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ctx.check()
    st_last = ctx.stats()
    launches = ctx.stats()["kernels_launched"] - k0
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    value = world * args.steps * grads_per_step * omega / total_s
    if lsq_lbfgs:   # L-BFGS: gradient evaluations per step vary; report slice updates / s
        value = world * args.steps / total_s
    # dominant kernel: one factor gradient over the slice, back to back behind a sleep kernel
    A, _, _ = ctx.factors()
    s0 = torch.full((cfg["rank"],), 1.0, device=dev)
    G = [torch.zeros_like(a) for a in A]
    nrep = 50
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ctx.gradient(s0, A, X=dsl[0], want=sg.WANT_FACTORS, G=G, accumulate=True)
        torch.cuda._sleep(50_000_000)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for r in range(nrep):
            ctx.gradient(s0, A, X=dsl[r % n_sl], want=sg.WANT_FACTORS, G=G, accumulate=True)
        e1.record(stream)
    torch.cuda.synchronize()
    kern_s = e0.elapsed_time(e1) / 1e3 / nrep
    # end to end through the C ABI: every step's slice from pinned host memory (staged by the
    # library, overlapping the step before), every step's F_w, F_f read back without a host wait;
    # two untimed host steps allocate the staging buffers
    pinned = [torch.from_numpy(x).pin_memory() for x in host]
    e2e_steps = max(2, min(args.steps, 4))
    f_host = torch.zeros((e2e_steps, 2), dtype=torch.float64).pin_memory()
    for w in range(2):
        ctx.step(X=pinned[w % n_sl])
    torch.cuda.synchronize()
    te = time.perf_counter()
    for k in range(e2e_steps):
        ctx.step(X=pinned[k % n_sl])
        ctx.objectives_async(f_host[k])
    stream.synchronize()
    e2e_s = time.perf_counter() - te
    ctx.check()
    if not bool(torch.isfinite(f_host).all()):
        raise RuntimeError("dense end-to-end steps returned a non-finite objective")
    e2e_value = world * e2e_steps * (1 if lsq_lbfgs else grads_per_step * omega) / e2e_s
    ctx.close()
    peak, peak_kind = peaks()
    R = cfg["rank"]
    bytes_alg = 4 * omega                        # X read once; factors and G are < 0.2 MB
    flops_alg = 6 * R * omega                    # m (2R) + T = Y A3 (2R) + G3 = Y' KR (2R)
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        tflops_peak = float(d["bf16_tflops"])
    except Exception:
        tflops_peak = 1900.0
    if args.precision == "fp32":   # CUDA-core path: bound by FP32 FMA throughput
        sm_clock = clk.get("sm_max_mhz") or 2070.0
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        fp32_peak = n_sm * 128 * 2 * sm_clock * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops_alg / kern_s / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": flops_alg / kern_s / 1e12 / fp32_peak, "traffic": None,
                "peak_kind": f"FP32 FMA: {n_sm} SMs x 128 lanes x 2 flop x {sm_clock:.0f} MHz",
                "kernel_us": kern_s * 1e6, "hbm_gbs": bytes_alg / kern_s / 1e9}
    else:
        roof = {"bound": "hbm", "achieved": bytes_alg / kern_s / 1e9, "peak": peak, "unit": "GB/s",
                "frac": bytes_alg / kern_s / 1e9 / peak, "traffic": recorded_traffic("dense_grad_tc_bf16_R64_256cubed.md")
                if args.precision == "bf16" else None, "peak_kind": peak_kind,
                "kernel_us": kern_s * 1e6,
                "tensor_tflops": flops_alg / kern_s / 1e12,
                "tensor_frac_of_bf16_peak": flops_alg / kern_s / 1e12 / tflops_peak}
    return {
        "metric": "slice updates/s" if lsq_lbfgs else "dense GCP gradient entries/s", "value": value,
        "unit": "slices/s" if lsq_lbfgs else "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16 MTTKRP / split-bf16 model, f32 accumulate",
                  "fp16": "f16 MTTKRP / split-bf16 model, f32 accumulate"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"dense_gaussian_3way: 256^3 slices, R=64, gaussian, noise 1% RMS",
                   "grads_per_step": None if lsq_lbfgs else grads_per_step,
                   "solver": "LSQ temporal solve + projected L-BFGS factor solve (defaults)" if lsq_lbfgs else DENSE_SOLVER,
                   "lbfgs_last_slice": {"iterations": st_last["epochs_f"], "evaluations": st_last["evals_f"]}
                   if lsq_lbfgs else None,
                   "l2": "flushed between steps (256 MB write)", "precision": args.precision},
        "gpu_launches": int(launches),
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "slices/s" if lsq_lbfgs else "entries/s",
                "h2d_bytes_per_step": int(host[0].nbytes), "d2h_bytes_per_step": 16},
        "clocks": clk,
    }


# ----------------------------------------------------------------------------- autograd form
def run_native_autograd(args, cfg, world, rank, local):
    """100^3, R = 16 Poisson slices (the autograd configuration): one step is the GCP loss forward
    and its hand-written backward through torch.autograd (GCPLoss; m recomputed in the backward
    launch), set beside the same loss and gradients from one fused FP32 call; the cpu_baseline leg
    compares both with the FP64 oracle gradient of the first slice."""
    import torch
    import paper_2110_14514_gb300 as sg
    from paper_2110_14514_gb300.autograd import GraphedGCPLoss, gcp_loss

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    R = cfg["rank"]
    p = sg.params(cfg["dims"], R, cfg["loss"], precision=sg.PREC_F32, seed=3000 + rank)
    A0 = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev) for a in S.init_factors(cfg, stream=rank)]
    n_sl = 2
    host = [np.ascontiguousarray(S.dense_slice(cfg, t + 1, stream=rank)[0], np.float32) for t in range(n_sl)]
    dsl = [torch.from_numpy(x).to(dev) for x in host]
    pinned = [torch.from_numpy(x).pin_memory() for x in host]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ctx = sg.Context(p, A0)
    A = [a.clone().requires_grad_(True) for a in A0]
    s = torch.full((R,), 0.5, dtype=torch.float32, device=dev, requires_grad=True)
    omega = int(np.prod(cfg["dims"]))

    def ag_step(X):
        for t in A + [s]:
            t.grad = None
        loss = gcp_loss(ctx, s, A, X=X)
        loss.backward()
        return loss

    def timed(fn, nsteps, off):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        torch.cuda.synchronize()
        for k in range(nsteps):
            flush.fill_(float(k))
            ev[k][0].record()
            fn((off + k) % n_sl)
            ev[k][1].record()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    for w in range(args.warmup):
        ag_step(dsl[w % n_sl])
    torch.cuda.synchronize()
    k0 = ctx.stats()["kernels_launched"]
    clocks = Clocks(local)
    clocks.start()
    total_s = timed(lambda i: ag_step(dsl[i]), args.steps, args.warmup)
    clk = clocks.stop()
    launches = ctx.stats()["kernels_launched"] - k0
    value = world * args.steps * omega / total_s
    # the same loss and gradients from one fused call per step
    sd, Ad = s.detach(), [a.detach() for a in A]
    plain_s = timed(lambda i: ctx.gradient(sd, Ad, X=dsl[i]), args.steps, 0)
    # the autograd step captured once in a CUDA graph (GraphedGCPLoss) and replayed; each step first
    # copies its slice into the graph's static slice buffer (device to device, inside the events)
    Xs = dsl[0].clone()
    gstep = GraphedGCPLoss(ctx, s, A, X=Xs)

    def graphed(i):
        Xs.copy_(dsl[i])
        return gstep.replay()
    graphed(0)
    graphed_s = timed(graphed, args.steps, 0)
    # end to end: the slice copied from pinned host memory each step, the loss read back
    def e2e(i):
        X = pinned[i].to(dev, non_blocking=True)
        return ag_step(X).item()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for k in range(args.steps):
        e2e(k % n_sl)
    t1.record()
    torch.cuda.synchronize()
    e2e_s = t0.elapsed_time(t1) / 1e3
    # both gradients of the first slice at the current point (the cpu_baseline leg compares them
    # with the FP64 oracle's)
    ag_step(dsl[0])
    G_ag = [a.grad.double().cpu().numpy() for a in A]
    gs_ag = s.grad.double().cpu().numpy()
    Gp, gsp, _ = ctx.gradient(sd, Ad, X=dsl[0])
    Gp = [g.double().cpu().numpy() for g in Gp]
    gsp = gsp.double().cpu().numpy()
    s_cur = sd.double().cpu().numpy()
    A_cur = [a.double().cpu().numpy() for a in Ad]
    # the kernels alone: the two launches of an autograd step (loss pass, then the factor and
    # temporal gradients) back to back behind a sleep kernel, outputs preallocated (the 4 MB
    # slice stays in L2 across these launches)
    G = [torch.zeros_like(a) for a in Ad]
    gs = torch.zeros(R, dtype=torch.float32, device=dev)
    f = torch.zeros(1, dtype=torch.float64, device=dev)
    nrep = 100
    torch.cuda.synchronize()
    with torch.cuda.stream(ctx.stream):
        ctx.gradient(sd, Ad, X=dsl[0], want=sg.WANT_LOSS, f=f, accumulate=True)
        torch.cuda._sleep(20_000_000)
        k_e0, k_e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k_e0.record(ctx.stream)
        for r in range(nrep):
            ctx.gradient(sd, Ad, X=dsl[r % n_sl], want=sg.WANT_LOSS, f=f, accumulate=True)
            ctx.gradient(sd, Ad, X=dsl[r % n_sl], want=sg.WANT_FACTORS | sg.WANT_TEMPORAL, G=G, gs=gs,
                         accumulate=True)
        k_e1.record(ctx.stream)
    torch.cuda.synchronize()
    kern_s = k_e0.elapsed_time(k_e1) / 1e3 / nrep
    ctx.close()
    sm_clock = clk.get("sm_max_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_clock * 1e6 / 1e12
    flops = 8 * R * omega           # forward model (2R) + backward model, T and G3 (6R) per entry
    achieved = flops / kern_s / 1e12
    out = {
        "metric": "GCP loss forward + backward entries/s", "value": value, "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "dense_poisson_3way: 100^3 slices, R=16, poisson, autograd forward + backward",
                   "bound_by": "host: torch.autograd and the two library calls per step take longer than the kernels",
                   "l2": "flushed between steps (256 MB write)", "plain_fused_ms_per_step": 1e3 * plain_s / args.steps,
                   "graphed_ms_per_step": 1e3 * graphed_s / args.steps,
                   "graphed_value": world * args.steps * omega / graphed_s,
                   "graphed_note": "GraphedGCPLoss: the same forward + backward captured in a CUDA graph and "
                                   "replayed after a device copy of the step's slice into its static buffer",
},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": None,
                     "peak_kind": f"FP32 FMA: {n_sm} SMs x 128 lanes x 2 flop x {sm_clock:.0f} MHz",
                     "kernel_us": kern_s * 1e6,
                     "note": "the loss and gradient launches of one step, back to back: 8R flops per entry"},
        "e2e": {"value": world * args.steps * omega / e2e_s, "unit": "entries/s",
                "h2d_bytes_per_step": 4 * omega, "d2h_bytes_per_step": 8},
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's gradients of the first slice at the current point, ~10 s on one host core; the
        # first also gives the accuracy of both device gradients
        from oracle import gcp
        Xh = host[0].astype(np.float64)
        t0c = time.perf_counter()
        n = 0
        while n == 0 or time.perf_counter() - t0c < 10.0:
            Go, gso, _ = gcp.dense_gradient(Xh, s_cur, A_cur, cfg["loss"])
            n += 1
        dt = time.perf_counter() - t0c
        out["cpu_baseline"] = {"value": n * omega / dt, "unit": "entries/s", "cores": 1, "kind": "oracle",
                               "sample": f"{n} FP64 oracle dense gradients (loss + all gradients) of one 100^3 slice"}

        def rel(a, b):
            return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
        out["config"]["accuracy_rel_max"] = {
            "autograd_vs_oracle": max([rel(G_ag[k], Go[k]) for k in range(3)] + [rel(gs_ag, gso)]),
            "plain_vs_oracle": max([rel(Gp[k], Go[k]) for k in range(3)] + [rel(gsp, gso)])}
    return out


# ----------------------------------------------------------------------------- batched streams
BATCH_SOLVER = dict(H=10, w=1.0, theta=0.9, kappa_w=5, tau_w=20, kappa_f=5, tau_f=20, alpha_w=0.05, alpha_f=1e-3)


def batched_flops_per_step(shapes, sol):
    """Algorithmic FP32 flops of one batched step: per slice entry 2R for a loss pass (model),
    4R for a gradient-of-s pass (model + T = Y A3), 6R for a factor-gradient pass (model + T + G3)."""
    loss_passes = 2 + sol["kappa_w"] + sol["kappa_f"]
    tgrad_passes = sol["kappa_w"] * sol["tau_w"]
    fgrad_passes = sol["kappa_f"] * sol["tau_f"]
    flops = entries = 0
    for dims, R, _ in shapes:
        om = int(np.prod(dims))
        flops += om * R * (2 * loss_passes + 4 * tgrad_passes + 6 * fgrad_passes)
        entries += om * (loss_passes + tgrad_passes + fgrad_passes)
    return flops, entries


def run_native_batched(args, cfg, world, rank, local):
    """64 independent dense streams of uneven shape (I_k ~ U{32..160}, R ~ U{8..64}, Gaussian / Poisson):
    one sgcp_batch_step per time step (one persistent kernel), against the same streams stepped one
    after another through single-stream contexts."""
    import torch
    import paper_2110_14514_gb300 as sg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    shapes = S.batched_stream_shapes(cfg)
    n = len(shapes)
    scfg = [S.batched_stream_cfg(cfg, s) for s in range(n)]
    plist = [sg.params(c["dims"], c["rank"], c["loss"], seed=3000 + 97 * rank + s, **BATCH_SOLVER)
             for s, c in enumerate(scfg)]
    A0 = [[torch.from_numpy(a).to(dev) for a in S.init_factors(c, stream=rank)] for c in scfg]
    n_sl = 2
    host = [[torch.from_numpy(S.dense_slice(c, t + 1, stream=rank)[0]).pin_memory() for c in scfg]
            for t in range(n_sl)]
    dsl = [[x.to(dev) for x in h] for h in host]
    t0 = time.time()
    b = sg.Batch(plist, A0, autotune=True, tune_reps=2)
    tune_s = time.time() - t0
    flops, entries = batched_flops_per_step(shapes, BATCH_SOLVER)
    for w in range(args.warmup):
        b.step(dsl[w % n_sl])
    b.check()
    k0 = b.stats(0)["kernels_launched"]
    stream = b.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            ev[k][0].record(stream)
        b.step(dsl[(args.warmup + k) % n_sl])
        with torch.cuda.stream(stream):
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    b.check()
    launches = b.stats(0)["kernels_launched"] - k0
    step_s = [a.elapsed_time(c) / 1e3 for a, c in ev]
    total_s = sum(step_s)
    value = world * args.steps * entries / total_s
    # end to end: host slices copied inside the call, per-stream objectives read back
    # (every stream's F_w, F_f gathered and copied back behind each step, without draining the GPU)
    e2e_steps = max(3, args.steps // 2)
    f_host = torch.zeros((e2e_steps, 2 * n), dtype=torch.float64).pin_memory()
    for w in range(2):                            # untimed: the two staging buffers are allocated here
        b.step(host[w % n_sl])
    torch.cuda.synchronize()
    te = time.perf_counter()
    d2h = 0
    for k in range(e2e_steps):
        b.step(host[k % n_sl])
        b.objectives_async(f_host[k])
        d2h += n * 16
    b.stream.synchronize()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - te
    b.check()
    if not bool(torch.isfinite(f_host).all()):
        raise RuntimeError("batched end-to-end steps returned a non-finite objective")
    h2d = sum(int(np.prod(d)) * 4 for d, _, _ in shapes)
    table = b.tune_table()
    b.close()
    # the same streams, one single-stream context after another (plain FP32 sgcp_step)
    ctxs = [sg.Context(p, A) for p, A in zip(plist, A0)]
    for c, x in zip(ctxs, dsl[0]):
        c.step(X=x)
    torch.cuda.synchronize()
    seq_steps = 2
    ts = time.perf_counter()
    for k in range(seq_steps):
        for c, x in zip(ctxs, dsl[(k + 1) % n_sl]):
            c.step(X=x)
        torch.cuda.synchronize()
    seq_s = (time.perf_counter() - ts) / seq_steps
    for c in ctxs:
        c.close()
    sm_clock = clk.get("sm_max_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tflops = n_sm * 128 * 2 * sm_clock * 1e6 / 1e12
    achieved = flops / (total_s / args.steps) / 1e12
    out = {
        "metric": "batched GCP gradient entries/s", "value": value, "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched_streams: 64 dense streams, I_k ~ U{32..160}, R ~ U{8..64}, "
                               "Gaussian (even) / Poisson (odd)",
                   "solver": BATCH_SOLVER, "entries_per_step": entries,
                   "l2": "inputs larger than L2 (sum of slices %.0f MB, re-read by every pass)" % (h2d / 1e6),
                   "sequential_ms_per_step": 1e3 * seq_s,
                   "speedup_vs_sequential": seq_s / (total_s / args.steps),
                   "autotune_s": tune_s, "tune_keys": len(table)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": None,
                     "peak_kind": f"FP32 FMA: {n_sm} SMs x 128 lanes x 2 flop x {sm_clock:.0f} MHz"},
        "e2e": {"value": e2e_steps * entries / e2e_s, "unit": "entries/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h // e2e_steps},
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = batched_cpu_baseline(scfg)
    return out


def batched_cpu_baseline(scfg, budget_s=12.0):
    """The oracle's dense gradient (FP64 numpy) on whole slices of the batch's streams, in stream
    order until the time budget is spent."""
    from oracle import gcp
    t0 = time.perf_counter()
    ent = 0
    done = 0
    for c in scfg:
        X, _ = S.dense_slice(c, 1)
        A = S.init_factors(c)
        sv = np.ones(c["rank"])
        gcp.dense_gradient(X.astype(np.float64), sv, [a.astype(np.float64) for a in A], c["loss"])
        ent += X.size
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": ent / el, "unit": "entries/s", "cores": 1, "kind": "oracle",
            "sample": f"full FP64 oracle gradients of {done} stream slices (one pass each)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dense-record", action="store_true",
                    help="sparse workload: skip the 256^3 R=64 per-precision slice-update record")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "dense_gaussian_3way", "dense_poisson_3way", "batched_streams"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--solver", default="adam", choices=["adam", "lsq_lbfgs"],
                    help="dense workload: ADAM solvers (Alg. 3 / 4) or the LSQ + L-BFGS options")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    cfg = S.workload(args.workload)
    if args.impl == "reference":
        out = run_reference(args, S.workload(WORKLOAD), world, rank)
    elif args.workload == "batched_streams":
        out = run_native_batched(args, cfg, world, rank, local)
    elif args.workload == "dense_poisson_3way":
        out = run_native_autograd(args, cfg, world, rank, local)
    elif args.workload != WORKLOAD:
        out = run_native_dense(args, cfg, world, rank, local)
    else:
        out = run_native(args, cfg, world, rank, local)
    if out is not None and rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
