#!/usr/bin/env python
"""Throughput of the forward + inverse SHT on GB300 (one JSON line on stdout, rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--L 1024] [--batch 64]

A step is one inverse SHT (coefficients -> samples) followed by one forward SHT (samples ->
coefficients) of a batch of synthetic signals: every stage of the path (ring DFTs, the order
chain with its solves and alias subtractions, the synthesis contraction, the fold and inverse
ring DFTs) runs once per step.  Default workload: 64 complex signals at L = 1024, f_l^m re/im iid
N(0,1) * (l+1)^-1, float64-accurate results with the contractions on the BF16 tensor cores from
exact slices (--dtype f64 for the float64 pipe).  Inputs (1 GiB per buffer) are larger than L2.

Under torchrun (N > 1) every rank transforms its own batch (weak scaling, no collective on the
data path); the time is the max over ranks.

--impl reference times the plain float64 CPU oracle on this host (rank 0 only): each step runs,
in one process per host core, a bounded sample of the same workload - 1/16 of the orders of
Procedure 2's and Procedure 1's loops, spread evenly over m - counted as 1/16 of a signal each.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+inv SHT signals/s at L=1024 vs FP64 oracle error; % tensor-pipe peak"
SAMPLE_FRACTION = 16  # the reference arm runs 1/16 of the order loop of each procedure


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


# float64 pipe of a GB300: 1.25 TFLOP/s at the 2070 MHz boost clock (NVIDIA's figure, which the
# FFMA64 microbenchmark recorded in profiles/fp64_peak.md reproduces); scaled by the measured clock.
FP64_TFLOPS_NOMINAL = 1.25
FP64_NOMINAL_MHZ = 2070.0


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    """(dist, rank, world size, local rank) from the torchrun environment; NCCL on GPUs, gloo
    without (the CPU tests of the multi-rank logic)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return dist, dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def _max_over_ranks(value, dist, device="cpu"):
    """The slowest rank's figure (a step is done when every rank is done)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def _whole_job_rate(world_size, batch_per_rank, ms_per_step):
    """Signals per second of the whole job: every rank transforms its own batch (weak scaling)."""
    return world_size * batch_per_rank / (ms_per_step * 1e-3)


def _oracle_order(L):
    """The oracle's greedy ring ordering: the stored file (written by
    tests/golden/make_ring_orders.py) when there is one, else computed."""
    from oracle import sampling
    path = os.path.join(ROOT, "tests", "golden", f"ring_order_L{L}.txt")
    if os.path.exists(path):
        return np.loadtxt(path, dtype=np.int64, comments="#")
    return sampling.greedy_order_secular(L)


def _oracle_sample(L, seed, frac, residue=0):
    """One bounded oracle sample: seconds for the iterations m = residue (mod frac) of each
    procedure's order loop, i.e. 1/frac of the orders spread evenly over 0..L-1 (so the sample
    has the cost profile of the whole loop)."""
    from oracle import sht as osht
    from oracle import sampling
    from paper_1403_4661_gb300 import synth

    theta = sampling.equiangular_set(L)[_oracle_order(L)]
    c = synth.decaying_coeffs(L, 1, seed)
    orders = range(residue % frac, L, frac)
    t0 = time.perf_counter()
    s = osht.inverse(c, L, theta, orders=orders)
    osht.forward(s, L, theta, orders=orders)
    return time.perf_counter() - t0


def _host_cores():
    """Cores this process may run on (at most 64 oracle processes: ~0.2 GB each at L = 1024)."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(n, 64))


def _cpu_baseline_parallel(L, frac, steps, procs):
    """Time the oracle on `procs` host cores at once: one fresh single-threaded process per core
    (spawned, never touching the GPU), each timing `steps` bounded samples of its own signals.
    Returns, per step, the slowest process's seconds (the processes run concurrently, so `procs`
    samples complete in that time)."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps([bench._oracle_sample(%d, 100 + i + 1000 * %d, %d, %d + i) for i in range(%d)]))")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    ps = [subprocess.Popen([sys.executable, "-c", code % (ROOT, L, p, frac, p, steps)], stdout=subprocess.PIPE,
                           stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT) for p in range(procs)]
    outs = [p.communicate() for p in ps]
    for p, (_, err) in zip(ps, outs):
        if p.returncode != 0:
            raise RuntimeError("oracle timing failed: " + err[-2000:])
    times = [json.loads(out.strip().splitlines()[-1]) for out, _ in outs]
    return [max(t[k] for t in times) for k in range(steps)]


def _sample_text(L, procs):
    return (f"{procs} signals at L={L}, one per host core in {procs} concurrent single-threaded "
            f"processes; each runs the iterations m = r (mod {SAMPLE_FRACTION}) of Procedure 2's and "
            f"Procedure 1's order loops (1/{SAMPLE_FRACTION} of the orders, spread evenly over 0..L-1; "
            f"r differs per process and step), counted as 1/{SAMPLE_FRACTION} of a signal")


def run_reference(args):
    dist, rank, ws, _ = _dist() if int(os.environ.get("WORLD_SIZE", "1")) > 1 else (None, 0, 1, 0)
    if rank != 0:
        return
    procs = _host_cores()
    times = _cpu_baseline_parallel(args.L, SAMPLE_FRACTION, args.warmup + args.steps, procs)[args.warmup:]
    # a step runs `procs` bounded samples at once, each 1/SAMPLE_FRACTION of one signal's work
    step_s = statistics.mean(times)
    value = procs / (SAMPLE_FRACTION * step_s)
    sample = _sample_text(args.L, procs)
    cfg = _config(args)
    cfg["arithmetic"] = "f64 (plain float64 numpy oracle on the host CPU)"
    cfg["workload"] = (f"{args.batch} complex signals at L={args.L}, f_lm re/im iid N(0,1)/(l+1); inverse SHT "
                       "then forward SHT by the oracle's Procedures 2 and 1 (plain float64, host CPU); "
                       "timed on a bounded sample, see cpu_baseline.sample")
    cfg["launch"] = "host processes, one per core"
    cfg["l2"] = "host memory; no GPU is used"
    cfg["e2e"] = "the oracle reads and writes host arrays: no copies, e2e equals the value"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "signals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * step_s, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": "signals/s", "cores": procs, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "signals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(args):
    arith = {"f64": "plain float64",
             "f64_tensor": "float64-accurate, contractions on the BF16 tensor cores from exact slices",
             "bf16_refined": "forward by iterative refinement with BF16 contractions, float64-accurate residual",
             "bf16x2_refined": "forward by iterative refinement with BF16x2 contractions, float64-accurate residual",
             "tf32_refined": "forward by iterative refinement with TF32 contractions, float64-accurate residual",
             "f32": "plain float32 (complex64 signals)"}
    return {"workload": f"{args.batch} complex signals at L={args.L}, f_lm re/im iid N(0,1)/(l+1); "
                        f"inverse SHT then forward SHT, {arith.get(getattr(args, 'dtype', 'f64'))}",
            "arithmetic": getattr(args, "dtype", "f64"),
            "L": args.L, "batch_per_gpu": args.batch, "ordering": "greedy (Sec. III-E)",
            "l2": "inputs larger than L2 (16 L^2 B bytes per buffer, 8 L^2 B for f32), no flush",
            "e2e": "pinned host -> device copy of each step's batch and device -> host copy of its result, "
                   "on a second stream with two device buffer sets (overlapping the neighbouring steps)",
            "launch": "one CUDA graph per step" if not getattr(args, "no_graph", False) else "eager"}


def _vs_stored_oracle(L, seed, s, c2):
    """Signal 0 of the batch against the oracle at the seeded indices stored for it in
    tests/golden/oracle_L{L}.txt (written from oracle/ only, for this same signal: decaying spectrum,
    seed 1000, the stored greedy rings): the GPU inverse against the oracle's inverse, and the GPU
    round trip forward(inverse(c)) against the oracle's.  None when there is no record for L."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_L{L}.txt")
    if seed != 1000 or not os.path.exists(path):
        return None
    hdr, ci, cv, si, sv = {}, [], [], [], []
    for line in open(path):
        if line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "c":
            ci.append(int(f[1])); cv.append(float(f[2]) + 1j * float(f[3]))
        elif f[0] == "s":
            si.append(int(f[1])); sv.append(float(f[2]) + 1j * float(f[3]))
        else:
            hdr[f[0]] = f[1]
    if int(hdr.get("seed", -1)) != seed:
        return None
    c_g = c2[0].cpu().numpy()[np.array(ci)]
    s_g = s[0].cpu().numpy()[np.array(si)]
    return {"coeff_max_abs_diff": float(np.abs(c_g - np.array(cv)).max()),
            "sample_max_rel_diff": float(np.abs(s_g - np.array(sv)).max() / max(1.0, float(hdr["max_abs_s"]))),
            "n_coeff": len(ci), "n_sample": len(si), "oracle_E1_max": float(hdr["oracle_E1_max"]),
            "source": f"tests/golden/oracle_L{L}.txt"}


def run_ours(args):
    import torch

    from paper_1403_4661_gb300 import build, synth
    from paper_1403_4661_gb300.sht import Plan

    dist, rank, ws, local = _dist()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    L, B = args.L, args.batch

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle in spawned single-threaded processes, one per host core, before the GPU work
        procs = _host_cores()
        t = _cpu_baseline_parallel(L, SAMPLE_FRACTION, 1, procs)
        cpu = {"value": procs / (t[0] * SAMPLE_FRACTION), "unit": "signals/s", "cores": procs,
               "kind": "oracle", "sample": _sample_text(L, procs)}

    t0 = time.time()
    plan = Plan(L, dtype=args.dtype)  # greedy ring ordering on the GPU, tables, per-order inverses
    plan_s = time.time() - t0
    if args.dtype.endswith("refined"):
        if args.refine_iters > 0:
            plan.set_refinement(args.refine_iters, 0.0)   # fixed count: capturable
        elif not args.no_graph:
            args.no_graph = True  # tolerance-driven refinement synchronises each iteration
    plan.reserve(B)
    cdtype = torch.complex64 if args.dtype == "f32" else torch.complex128
    c_host = torch.from_numpy(synth.decaying_coeffs(L, B, 1000 + rank)).to(cdtype).pin_memory()
    c = c_host.to(dev)
    s = torch.empty_like(c)
    c2 = torch.empty_like(c)
    stream = torch.cuda.current_stream()

    def eager_on(x, y):
        def run():
            plan.inverse(x, out=s)
            plan.forward(s, out=y)
        return run

    def capture(fn):
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g):
                fn()
        torch.cuda.current_stream().wait_stream(side)
        return g

    eager_step = eager_on(c, c2)
    for _ in range(args.warmup):
        eager_step()
    torch.cuda.synchronize()
    err = (c2 - c).abs().max().item()
    vs_oracle = _vs_stored_oracle(L, 1000 + rank, s, c2) if args.dtype != "f32" else None
    step = eager_step
    graph = None
    if not args.no_graph:
        # one CUDA graph per step: the library allocates nothing and makes no attribute or
        # synchronising call once its workspaces are reserved, so the whole step is capturable
        plan.set_timing(True)      # the stage event pairs are captured as graph nodes
        plan.stage_times()
        launches_after_capture0 = plan.info()["kernel_launches"]
        graph = capture(eager_step)
        plan.set_timing(False)
        captured_launches = plan.info()["kernel_launches"] - launches_after_capture0
        step = graph.replay
        for _ in range(2):
            step()
        torch.cuda.synchronize()

    # ---- device-resident timed region --------------------------------------------------------
    if graph is None:
        plan.set_timing(True)
        plan.stage_times()
    launches0 = plan.info()["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    if graph is None:
        launches = plan.info()["kernel_launches"] - launches0
        stages = plan.stage_times()
        plan.set_timing(False)
        stage_steps = args.steps
    else:
        # the graph's event pairs hold the spans of its last replay (the last timed step)
        launches = captured_launches * args.steps
        stages = plan.stage_times()
        stage_steps = 1
    ms = _max_over_ranks(ms, dist, dev)

    # ---- end to end: host buffers, copies inside the timed region ----------------------------
    # Every step copies its batch from pinned host memory and its result back.  The copies run on
    # a second stream into and out of two device buffer sets, so that step i's copies overlap the
    # compute of steps i - 1 and i + 1 (a serving pipeline); the timed region spans the first
    # copy in to the last copy out.
    out_host = torch.empty_like(c_host).pin_memory()
    c_b, c2_b = torch.empty_like(c), torch.empty_like(c2)
    step_b = eager_on(c_b, c2_b)
    if graph is not None:
        step_b = capture(step_b).replay
    sets = [(c, c2, step), (c_b, c2_b, step_b)]
    copy = torch.cuda.Stream()
    ev = {k: [torch.cuda.Event(), torch.cuda.Event()] for k in ("h2d", "comp", "d2h")}

    def run_e2e(k):
        copy.wait_stream(stream)
        with torch.cuda.stream(copy):
            c.copy_(c_host, non_blocking=True)
            ev["h2d"][0].record(copy)
        for i in range(k):
            b = i & 1
            if i + 1 < k:   # next batch into the other set, once step i - 1 has read it
                with torch.cuda.stream(copy):
                    if i >= 1:
                        copy.wait_event(ev["comp"][1 - b])
                    sets[1 - b][0].copy_(c_host, non_blocking=True)
                    ev["h2d"][1 - b].record(copy)
            stream.wait_event(ev["h2d"][b])
            if i >= 2:      # this set's previous result has been copied out
                stream.wait_event(ev["d2h"][b])
            sets[b][2]()
            ev["comp"][b].record(stream)
            with torch.cuda.stream(copy):
                copy.wait_event(ev["comp"][b])
                out_host.copy_(sets[b][1], non_blocking=True)
                ev["d2h"][b].record(copy)
        stream.wait_stream(copy)

    run_e2e(2)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run_e2e(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    ms_e2e = _max_over_ranks(ms_e2e, dist, dev)
    err_e2e = float(np.abs(out_host.numpy() - c_host.numpy()).max())

    if rank != 0:
        return
    # ---- roofline of the dominant kernel --------------------------------------------------------
    sm_mhz = (clk or {}).get("sm_mhz") or FP64_NOMINAL_MHZ
    peaks = _peaks()
    roof = _roofline(args.dtype, L, B, stages, stage_steps, peaks, sm_mhz)

    # ---- the other arithmetic forms on the same workload and rings (outside the timed region) ----
    forms = None
    if not args.no_forms and args.dtype == "f64_tensor":
        forms = {}
        del graph, step, step_b, sets
        for dt, iters in (("f64", 0), ("tf32_refined", args.forms_refine_iters)):
            forms[dt] = _time_form(dt, L, B, plan.theta, c, min(args.steps, 5), 2, iters, peaks, sm_mhz)

    value = _whole_job_rate(ws, B, ms)
    line = {
        "metric": METRIC, "value": value, "unit": "signals/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f64": "f64", "f64_tensor": "f64 (bf16 tensor-core slices)", "f32": "f32",
                  "tf32_refined": "tf32 contractions + f64 residual (refined)"}.get(
            args.dtype, "bf16 contractions + f64 residual (refined)"),
        "data": "synthetic",
        "config": dict(_config(args), parallelism=f"dp{ws}" if ws > 1 else "single GPU"),
        "accuracy": {"E1_max_round_trip": err, "E1_max_round_trip_e2e": err_e2e,
                     "definition": "max |forward(inverse(c)) - c| over the batch, both GPU transforms "
                                   "(Exp. 1 of Sec. IV-A); GPU-vs-oracle parity is checked by the tests",
                     "vs_oracle_sampled": vs_oracle},
        "roofline": roof,
        "forms": forms,
        "cpu_baseline": cpu,
        "e2e": {"value": _whole_job_rate(ws, B, ms_e2e), "unit": "signals/s",
                "h2d_bytes_per_step": c_host.element_size() * L * L * B,
                "d2h_bytes_per_step": c_host.element_size() * L * L * B},
        "clocks": clk,
        "gpu_launches": launches,
        "plan_seconds": plan_s,
    }
    print(json.dumps(line), flush=True)


def _chain_flops(L, B):
    """The method's own real flops of one forward's order chain (Eqs. (14)-(16)): the solves
    sum_n 2 n^2 4B and the alias products sum_m 2 m (L - m) 4B."""
    return 8.0 * B * (L * (L + 1) * (2 * L + 1) / 6.0 + (L ** 3 - L) / 6.0)


def _synthesis_flops(L, B):
    """Real flops of Eq. (11) for every order and ring: sum_m 2 L (L - m) 4B."""
    return 4.0 * B * L * L * (L + 1)


def _ring_dft_flops(L, B):
    """float64 flops of one direction's ring DFTs, by the ring classes of csrc/dft.cu: direct
    rings (N <= 63) 8 N^2; chirp-z rings two FFTs of the ring's convolution length M (the
    nominal 5 M log2 M each) plus the chirp and filter products (6 M + 12 N)."""
    tot = 0.0
    for k in range(L):
        N = 2 * k + 1
        if N <= 63:
            tot += 8.0 * N * N
            continue
        M = _bluestein_length(N)
        tot += 2 * 5.0 * M * math.log2(M) + 6.0 * M + 12.0 * N
    return tot * B


def _bluestein_length(N):
    """Convolution length of a chirp-z ring of length N, as csrc/dft.cu chooses it: the smallest
    2^a or 3 * 2^a that is at least 2N - 1."""
    best = None
    for a in range(4, 30):
        p2, p3 = 1 << a, 3 << (a - 1)
        if p3 >= 2 * N - 1 and p3 >= 16:
            best = p3 if best is None else min(best, p3)
        if p2 >= 2 * N - 1:
            return p2 if best is None else min(best, p2)
    return best


def _src_hash(name):
    import hashlib
    path = os.path.join(ROOT, "paper_1403_4661_gb300", "csrc", name)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16] if os.path.exists(path) else None


def _traffic(kernel, L, batch, src):
    """DRAM bytes of one launch from profiles/traffic.txt, valid only while the kernel's source
    file has the hash recorded with the capture (else the record is stale: None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None, "no capture recorded"
    for line in open(path):
        parts = dict(p.split("=", 1) for p in line.split() if "=" in p)
        if parts.get("kernel") == kernel and parts.get("L") == str(L) and parts.get("batch") == str(batch):
            if parts.get("src_sha") != _src_hash(src):
                return None, f"stale: {src} changed since the capture"
            return float(parts["dram_bytes_per_launch"]), parts.get("note", "ncu capture")
    return None, "no capture of this kernel at this workload"


def _roofline(dtype, L, B, stages, stage_steps, peaks, sm_mhz):
    """Roofline entries: the dominant kernel first, then the other stages (algorithmic work per
    launch divided by the stage's CUDA-event span, against the measured peaks)."""
    bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
    bf16_src = ("MEASURED_PEAKS.json bf16_tflops_sustained (of measured)" if peaks.get("bf16_tflops_sustained")
                else "fallback 1.7 PFLOP/s sustained bf16")
    hbm = peaks.get("hbm_gbs") or 6800.0
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s"
    fp64 = FP64_TFLOPS_NOMINAL
    fp64_src = ("GB300 float64 pipe: 152 SMs x 2 FP64 FMA per clock x 2 flops at 2070 MHz = 1.25 TFLOP/s "
                f"(clock-scaled at the measured median {sm_mhz:.0f} MHz: {fp64 * sm_mhz / FP64_NOMINAL_MHZ:.3f})")

    def span(stage):
        ms, n = stages[stage]
        return (ms / n * 1e-3, n) if n else (None, 0)

    chain_f, syn_f = _chain_flops(L, B), _synthesis_flops(L, B)
    entries = []
    syn_s, _ = span("synthesis")
    if dtype == "f32":
        fp32 = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        a = syn_f / syn_s / 1e12
        tr, note = _traffic("synthesis_f32", L, B, "gemm_f64.cu")
        main = {"bound": "alu", "kernel": "k_gemm<float,64,64,4,...,MODE_SYNTH> (float32 synthesis, Eq. (11))",
                "achieved": a, "peak": fp32, "unit": "TFLOP/s", "frac": a / fp32,
                "peak_source": f"GB300 FP32 pipe: 152 SMs x 128 lanes x 2 flops at {sm_mhz:.0f} MHz",
                "flops_per_launch": syn_f, "traffic": tr, "traffic_note": note}
    elif dtype == "f64":
        a = syn_f / syn_s / 1e12
        tr, note = _traffic("synthesis_f64", L, B, "gemm_f64.cu")
        main = {"bound": "alu", "kernel": "k_gemm<double,64,64,4,...,MODE_SYNTH> (float64 synthesis, Eq. (11))",
                "achieved": a, "peak": fp64, "unit": "TFLOP/s", "frac": a / fp64, "peak_source": fp64_src,
                "flops_per_launch": syn_f, "traffic": tr, "traffic_note": note}
    else:
        ch_s, ch_n = span("solve")
        tf32 = dtype == "tf32_refined"
        peak = bf16 * 1.1 / 2.25 if tf32 else bf16
        a = chain_f / ch_s / 1e12
        pairs = {"f64_tensor": 36.0, "bf16x2_refined": 3.0, "bf16_refined": 1.0, "tf32_refined": 1.0}[dtype]
        tr, note = _traffic("chain_tf32" if tf32 else "chain_tc", L, B, "chain.cu")
        main = {"bound": "tensor",
                "kernel": "k_chain (forward order chain, Eqs. (14)-(16), one persistent cooperative launch; "
                          + ("tcgen05 kind::tf32)" if tf32 else "tcgen05 on BF16 slices)"),
                "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                "peak_source": bf16_src + (" x 1.1/2.25 (nominal dense TF32 / BF16)" if tf32 else ""),
                "flops_per_launch": chain_f,
                "flops_definition": "the method's own real flops: solves sum_n 2 n^2 4B + alias products "
                                    "sum_m 2 m (L-m) 4B = 8B[L(L+1)(2L+1)/6 + (L^3-L)/6]",
                "launches_per_step": ch_n / stage_steps,
                "mma_issue": {"products_per_method_product": pairs, "achieved": pairs * a, "unit": "TFLOP/s",
                              "frac": pairs * a / peak,
                              "note": "rate of the tensor-core products actually issued (slice pairs)"},
                "vs_fp64_pipe": a / fp64,
                "traffic": tr, "traffic_note": note}
        if syn_s:
            sa = syn_f / syn_s / 1e12
            entries.append({"stage": "synthesis", "kernel": "k_synthesis (Eq. (11), TMA + tcgen05 on BF16 slices)",
                            "bound": "tensor", "achieved": sa, "peak": bf16, "unit": "TFLOP/s", "frac": sa / bf16,
                            "flops_per_launch": syn_f, "mma_issue_tflops": 36.0 * sa,
                            "vs_fp64_pipe": sa / fp64})
    eb = 8 if dtype == "f32" else 16
    dft_f = _ring_dft_flops(L, B)
    for stage, kern, byts in (("ring_dft", "k_ring_dft (forward ring DFTs into order-major bins)",
                               2.0 * eb * L * L * B),
                              ("ring_idft", "k_ring_idft (fold of the orders into ring bins + inverse ring DFTs)",
                               eb * (2 * L * L - L) * B + eb * L * L * B)):
        t, n = span(stage)
        if not t:
            continue
        per = n / stage_steps
        gbs = byts / (t * per) / 1e9
        fl = dft_f / (t * per) / 1e12
        entries.append({"stage": stage, "kernel": kern, "bound": "hbm", "achieved": gbs, "peak": hbm,
                        "unit": "GB/s", "frac": gbs / hbm, "peak_source": hbm_src, "bytes_per_step": byts,
                        "fp64_alu": {"achieved": fl, "peak": fp64, "unit": "TFLOP/s", "frac": fl / fp64,
                                     "flops_per_step": dft_f,
                                     "note": "the DFTs are float64-pipe bound: chirp-z FFT flops per step"}
                        if dtype != "f32" else None})
    main["secondary"] = entries
    main["stage_ms_per_step"] = {k: v[0] / stage_steps for k, v in stages.items()}
    main["stage_launch_spans_per_step"] = {k: v[1] / stage_steps for k, v in stages.items()}
    return main


def _time_form(dtype, L, B, theta, c, steps, warmup, refine_iters, peaks, sm_mhz):
    """Step rate of another arithmetic on the same workload and rings: one CUDA graph per step
    (inverse then forward), CUDA events on the launching stream, stage spans of the last replay."""
    import torch
    from paper_1403_4661_gb300.sht import Plan

    t0 = time.time()
    plan = Plan(L, theta=theta, dtype=dtype)
    plan_s = time.time() - t0
    if dtype.endswith("refined"):
        plan.set_refinement(refine_iters, 0.0)   # fixed iteration count: capturable
    plan.reserve(B)
    s = torch.empty_like(c)
    c2 = torch.empty_like(c)

    def run():
        plan.inverse(c, out=s)
        plan.forward(s, out=c2)

    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    err = (c2 - c).abs().max().item()
    plan.set_timing(True)
    plan.stage_times()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            run()
    torch.cuda.current_stream().wait_stream(side)
    plan.set_timing(False)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    stages = plan.stage_times()
    roof = _roofline(dtype, L, B, stages, 1, peaks, sm_mhz)
    out = {"value": B / (ms * 1e-3), "unit": "signals/s", "ms_per_step": ms, "steps": steps,
           "E1_max_round_trip": err, "plan_seconds": plan_s, "roofline": roof}
    if dtype.endswith("refined"):
        out["refine_iterations"] = refine_iters
    del g
    plan.close()
    torch.cuda.synchronize()
    return out


def run_uneven(args):
    """The uneven-batch workload on a bounded draw: nsig signals with L log-uniform in [lo, hi]
    (seeded), f_lm re/im uniform[-1, 1]; one plan per distinct L (greedy rings, plan time
    reported apart); inverse then forward of the whole batch as one persistent launch per
    direction (sht_uneven_*), captured in a CUDA graph, beside the per-plan grouped calls."""
    import torch

    from paper_1403_4661_gb300 import build, synth
    from paper_1403_4661_gb300.sht import Plan, UnevenBatch, forward_uneven, inverse_uneven

    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    Ls = [int(L) for L in synth.loguniform_bandlimits(args.uneven_n, args.uneven_lo, args.uneven_hi, 4)]
    distinct = sorted(set(Ls))
    t0 = time.time()
    plans, cached = [], 0
    for L in distinct:
        # --plan-cache: the greedy co-latitudes of an earlier run (the ordering is deterministic),
        # so that only the tables are rebuilt
        path = os.path.join(args.plan_cache, f"thetas_L{L}.npy") if args.plan_cache else None
        theta = np.load(path) if path and os.path.exists(path) else None
        cached += theta is not None
        if args.table_free:   # float64 plans without their P~ tables; the launches regenerate P~
            pl = Plan(L, theta=theta, dtype="f64", keep_ptilde=False)
        else:
            pl = Plan(L, theta=theta, dtype=args.dtype)
        if path and theta is None:
            os.makedirs(args.plan_cache, exist_ok=True)
            np.save(path, pl.theta)
        plans.append(pl)
    plan_s = time.time() - t0
    table_bytes = sum(p.info()["table_bytes"] for p in plans)
    index = [distinct.index(L) for L in Ls]
    offsets, pos = [], 0
    for L in Ls:
        offsets.append(pos)
        pos += L * L
    packed = np.concatenate([synth.uniform_coeffs(L, 1, 5000 + i)[0] for i, L in enumerate(Ls)])
    c = torch.from_numpy(packed).to(dev)
    s, c2 = torch.zeros_like(c), torch.zeros_like(c)
    ub = UnevenBatch(plans, index, offsets)
    ub.set_wait_limit(30.0)   # one phase of a large batch can take over a second
    stream = torch.cuda.current_stream()

    def step():
        ub.inverse(c, out=s)
        ub.forward(s, out=c2)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ub.check()
    err = float((c2 - c).abs().max())
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            step()
    stream.wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the two launches apart (eager, one step): where the step's time goes
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    ub.inverse(c, out=s)
    ev[1].record(stream)
    ub.forward(s, out=c2)
    ev[2].record(stream)
    torch.cuda.synchronize()
    ub.check()
    ms_dir = {"inverse_ms": ev[0].elapsed_time(ev[1]), "forward_ms": ev[1].elapsed_time(ev[2])}
    # the same batch through the grouped per-plan calls (eager; not offered by table-free plans)
    ms_grouped = None
    for _ in range(0 if args.table_free else 2):
        forward_uneven(plans, index, offsets, inverse_uneven(plans, index, offsets, c))
    if not args.table_free:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(max(1, args.steps // 2)):
            forward_uneven(plans, index, offsets, inverse_uneven(plans, index, offsets, c))
        e1.record(stream)
        torch.cuda.synchronize()
        ms_grouped = e0.elapsed_time(e1) / max(1, args.steps // 2)
    flops = sum(8.0 * L ** 3 for L in Ls)   # inverse 4 L^3 + forward 4 L^3 per signal (Sec. IV-C counts)
    line = {
        "metric": "uneven batch fwd+inv signals/s (one persistent launch per direction)",
        "value": len(Ls) / (ms * 1e-3), "unit": "signals/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{len(Ls)} complex signals, L log-uniform in [{args.uneven_lo}, {args.uneven_hi}] "
                               f"(seed 4), f_lm re/im iid U[-1,1]; inverse then forward",
                   "distinct_L": len(distinct), "L_max": max(Ls),
                   "plan_arithmetic": "f64, no P~ tables (regenerated by the recursion)" if args.table_free else args.dtype,
                   "plan_table_bytes": table_bytes, "plans_from_cache": cached,
                   "launch": "one CUDA graph per step: two cooperative launches"},
        "directions": ms_dir,
        "grouped_calls": ({"ms_per_step": ms_grouped, "value": len(Ls) / (ms_grouped * 1e-3)}
                          if ms_grouped else None),
        "roofline": {"bound": "alu", "kernel": "k_uneven_inverse + k_uneven_forward (float64 SIMT)",
                     "achieved": flops / (ms * 1e-3) / 1e12, "peak": FP64_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                     "frac": flops / (ms * 1e-3) / 1e12 / FP64_TFLOPS_NOMINAL,
                     "flops_per_step": flops, "flops_definition": "sum over signals of 8 L^3"},
        "accuracy": {"E1_max_round_trip": err},
        "plan_seconds": plan_s,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=1024)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dtype", default="f64_tensor",
                    choices=["f64", "f64_tensor", "bf16_refined", "bf16x2_refined", "tf32_refined", "f32"])
    ap.add_argument("--refine-iters", type=int, default=0,
                    help="refined forms: fixed iteration count (0: iterate to 1e-12)")
    ap.add_argument("--no-graph", action="store_true", help="launch eagerly instead of one CUDA graph per step")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip timing the f64 and tf32_refined forms of the same workload")
    ap.add_argument("--forms-refine-iters", type=int, default=5,
                    help="fixed iteration count of the tf32_refined form (5 reaches the float64 "
                         "path's round-trip error at L=1024)")
    ap.add_argument("--uneven", action="store_true",
                    help="time the uneven-batch workload (one persistent launch per direction) instead")
    ap.add_argument("--uneven-n", type=int, default=512)
    ap.add_argument("--uneven-lo", type=int, default=32)
    ap.add_argument("--uneven-hi", type=int, default=256)
    ap.add_argument("--plan-cache", default=None,
                    help="uneven workload: directory of ring co-latitudes per L, read when present "
                         "and written otherwise (skips the greedy ordering on later runs)")
    ap.add_argument("--table-free", action="store_true",
                    help="uneven workload with float64 plans that keep no P~ table (needed to fit "
                         "L up to 1024: the launches regenerate P~ by its recursion)")
    args = ap.parse_args()
    if args.uneven:
        run_uneven(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
