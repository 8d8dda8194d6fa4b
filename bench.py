#!/usr/bin/env python
"""Throughput of the cascade (states/s) against the plain FP64 cascade, at the
stated error, on one GB300.

Headline workload (seeded, synthetic): the large fused form, m = 1024,
p = q = 64, 8 sequences of L = 65536 steps, Abar = 0.9999 Q + rank-4 E (Q
Haar-orthogonal), N = 15 (16 stages), BF16 hi/lo split with FP32
accumulation, powers by FP64 squaring.  A step is one forward pass of the
whole cascade over the batch (first stage fused with Bbar u, stages 1..15 on
the tensor cores, y = C v + D u); the forward + backward, the work-efficient
(about 2L products) schedule, the FP64 plain cascade and the FP64 sequential
recursion on the same GPU are measured beside it.  The precision form (m =
256, p = q = 1, 64 sequences x 16384 steps, one trapezoidal step per
sequence, N = 13) is measured the same way and reported under
"precision_form".  The powers are prepared once outside the timed region;
set-up plus forward is reported separately (e2e_with_setup).

The error of the timed output against the CPU FP64 oracle comes from the
cpu_baseline leg: the oracle's outputs on its timed sample (whole sequences,
the last one of the batch first) are compared with the GPU's y, in norm and
element-wise, per sequence; the run fails above the bar.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run: every rank runs an independent
replica of the whole workload on its own GPU (no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cascade states/s (fwd, fwd+bwd) vs plain FP64 cascade on GB300 at stated error"
TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16_split": 2e-3}

# name -> (precision, one-line description, run backward?)
SPECS = {
    "large_form": ("bf16_split", "large_form: Abar=0.9999 Q + rank-4 E, m=1024 p=q=64, 8 seqs x "
                   "L=65536, N=15, BF16 hi/lo split, FP32 accumulate, FP64 squaring, fwd+bwd",
                   True),
    "precision_form": ("bf16_split", "precision_form: HiPPO-LegS m=256 p=q=1, 64 seqs x L=16384, "
                       "N=13, delta log-uniform [1e-4,1e-1] per sequence, BF16 hi/lo split, "
                       "FP32 accumulate", True),
    "plain_fp64": ("fp64", "plain_fp64: HiPPO-LegS m=64 p=q=1, 1 seq x L=4096, delta=1/4096, "
                   "N=11, FP64 (equals the recursion)", False),
    "batching_form": ("fp32", "batching_form: HiPPO-LegS m=128 p=q=4, 512 seqs, L_i log-uniform "
                      "[1024,65536] (8.85e6 rows), Abar*(1+1e-6), N_i from eps=1e-6, FP32 "
                      "(3xTF32)", False),
    "differentiation_form": ("bf16_split", "differentiation_form: HiPPO-LegS m=256 p=q=16, "
                             "32 seqs x L=8192, delta=1e-3, N=12, BF16 split, fwd+bwd", True),
}

# DRAM bytes (read + write) of one stage_tc_kernel launch, from ncu captures of
# the current kernel on a smaller case, scaled by the rows processed to the
# full launch (the traffic of these launches grows in proportion to the rows).
# workload -> (bytes per full launch, the stage captured, note); absent: null.
TRAFFIC = {
    "large_form": (8 * 500.9e6, 8,
                   "ncu dram__bytes_read.sum + dram__bytes_write.sum of stage_tc_kernel, stage 8, "
                   "1 of 8 sequences (274.2 + 226.7 MB), x8 to the full launch; about 40 MB of "
                   "writes still dirty in L2 at kernel end are not counted"),
    "precision_form": (4 * 506.2e6, 8,
                       "ncu dram__bytes_read.sum + dram__bytes_write.sum of stage_tc_kernel, "
                       "stage 8, 16 of 64 sequences (284.1 + 222.1 MB), x4 to the full launch; "
                       "about 43 MB of writes still dirty in L2 at kernel end are not counted"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_form", choices=sorted(SPECS),
                    help="headline workload (large_form is the benchmark)")
    ap.add_argument("--also", default="precision_form",
                    help="second workload measured the same way ('none' to skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle leg (and with it the error check)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparators")
    ap.add_argument("--no-bwd", action="store_true", help="skip the forward+backward measurement")
    ap.add_argument("--no-scan", action="store_true",
                    help="skip the work-efficient (about 2L products) schedule measurement")
    ap.add_argument("--seqs", type=int, default=0,
                    help="keep only the first SEQS sequences (profiler captures only)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, world, device):
    """The slowest rank's time: every replica must have finished its units."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units all replicas processed per second of the slowest rank's time."""
    return units_per_rank * world / (ms / 1000.0)


def load_workload(name, seqs=0):
    """The seeded workload, with u cast to float32 for the tensor-core
    precisions (the oracle then sees the same float32 values)."""
    import numpy as np
    import workloads as wl
    w = wl.WORKLOADS[name]()
    if seqs and seqs < w.nseq:
        w = w.subset(range(seqs))
    if SPECS[name][0] != "fp64":
        w.u = w.u.astype(np.float32).astype(np.float64)
    return w


def config_of(name, w, world):
    """The config object: the same keys on both arms."""
    return {"workload": SPECS[name][1], "global_batch": int(w.nseq) * world,
            "seq_len": int(w.lengths.max()),
            "parallelism": f"replicas{world}" if world > 1 else "single"}


# --------------------------------------------------------------------- oracle leg
def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads") for d in threadpool_info() if d.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_model():
    """The host CPU's model name (x86: 'model name'; Arm: implementer and part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return None
    for key in ("model name", "Model"):
        for line in info:
            if line.startswith(key) and ":" in line:
                return line.split(":", 1)[1].strip()
    impl = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")]
    part = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")]
    if impl and part:
        return f"Arm implementer {impl[0]} part {part[0]}"
    return None


def oracle_sample(w, budget_s=12.0, keep=False):
    """The oracle as it stands on whole sequences of the workload, the last one
    of the batch first (its rows sit at the highest offsets), then from the
    first on, until the time budget is used (at least one sequence).  Returns
    (states/s, sample description, seconds, {sequence: oracle y} if keep)."""
    import oracle
    t0 = time.perf_counter()
    states = 0
    outs = {}
    cache = {}
    order = [w.nseq - 1] + list(range(w.nseq - 1))
    done = []
    for i in order:
        sl = w.seq(i)
        L = sl.stop - sl.start
        if L == 0:
            continue
        s = int(w.sys_of_seq[i])
        if s not in cache:
            cache[s] = oracle.system_matrices(w, s)
        Abar, Bbar, C, D = cache[s]
        N = w.N if w.N >= 0 else oracle.choose_N(Abar, int(w.lengths.max()), w.eps)
        y = oracle.cascade_forward_seq(Abar, Bbar, C, D, w.u[sl], oracle.effective_N(N, L))
        if keep:
            outs[i] = y
        states += L
        done.append(i)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    desc = (f"{len(done)} of {w.nseq} whole sequences ({states} states; the last sequence, "
            f"then from the first), powers included")
    return states / dt, desc, dt, outs


ONE_THREAD = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle
import workloads as wl
w = wl.WORKLOADS[sys.argv[2]]()
i = w.nseq - 1
L = int(w.lengths[i])
Abar, Bbar, C, D = oracle.system_matrices(w, int(w.sys_of_seq[i]))
N = oracle.effective_N(w.N if w.N >= 0 else oracle.choose_N(Abar, L, w.eps), L)
powers = oracle.squaring_chain(Abar, N)
rows = int(min(L, max(512, 4e9 / (2.0 * w.m * w.m * (N + 1)))))
u = w.u[w.seq(i)][:rows].astype(np.float32).astype(np.float64)
t0 = time.perf_counter()
oracle.cascade_forward_seq(Abar, Bbar, C, D, u, N, powers=powers)
dt = time.perf_counter() - t0
print(json.dumps({"value": rows / dt, "rows": rows, "seconds": dt}))
"""


def oracle_one_thread(name):
    """The oracle on one host thread (BLAS limited to one thread in a child
    process): the first steps of the last sequence, powers formed beforehand
    and not timed.  None if it does not finish within a minute."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", ONE_THREAD, ROOT, name], env=env,
                           capture_output=True, text=True, timeout=60)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    return {"value": d["value"], "unit": "states/s", "cores": 1,
            "sample": f"the first {d['rows']} steps of the last sequence, powers not timed"}


def seq_errors(yg, yo, Du, out_eps, absDu):
    """Relative Frobenius and element-wise errors of one sequence on y and on
    Cx = y - Du, the latter beyond an allowance for the rounding of the
    delivered y: 2 out_eps ||y|| in norm, (p + 2) out_eps (|y| + |D| |u|) per
    element (y's last rounding and the p products of D u in the output type)."""
    import numpy as np
    d = yg - yo
    ny, my = np.linalg.norm(yo), np.max(np.abs(yo))
    nd, md = np.linalg.norm(d), np.max(np.abs(d))
    cx = yo - Du
    ncx, mcx = np.linalg.norm(cx), np.max(np.abs(cx))
    pw = absDu.shape[1]
    excess = np.max(np.maximum(np.abs(d) - (pw + 2) * out_eps * (np.abs(yo) + absDu), 0.0))
    return (nd / ny if ny > 0 else nd,
            max(nd - 2 * out_eps * ny, 0.0) / ncx if ncx > 0 else 0.0,
            md / my if my > 0 else md,
            excess / mcx if mcx > 0 else 0.0)


def error_of(w, y_gpu, outs, precision, sample):
    """The error object: worst per-sequence errors of the timed y against the
    oracle's outputs on the cpu_baseline sample."""
    import numpy as np
    out_eps = 2.0 ** -53 if precision == "fp64" else 2.0 ** -24
    worst = np.zeros(4)
    for i, yo in outs.items():
        sl = w.seq(i)
        D = w.D[min(int(w.sys_of_seq[i]), w.D.shape[0] - 1)]
        worst = np.maximum(worst, seq_errors(y_gpu[sl], yo, w.u[sl] @ D.T, out_eps,
                                             np.abs(w.u[sl]) @ np.abs(D).T))
    bar = TOL[precision]
    return {"frob_y": float(worst[0]), "frob_cx": float(worst[1]), "elem_y": float(worst[2]),
            "elem_cx": float(worst[3]), "bar": bar, "pass": bool(np.all(worst <= bar)),
            "sequences": sorted(int(i) for i in outs),
            "what": "per sequence, worst over the sample: ||y - y_o|| / ||y_o|| and on Cx = "
                    "y - Du; max|y - y_o| / max|y_o| and on Cx (beyond the rounding of the "
                    "delivered y and of its FP32 D u); oracle = CPU FP64 cascade",
            "sample": sample}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu=uuid,{self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "50"]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # sampling has begun once the first line is out (at most 3 s): the timed
            # region then starts with the sampler running
            t0 = time.time()
            while time.time() - t0 < 3.0 and self.proc.poll() is None:
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.01)
            self.n_before = sum(1 for _ in open(self.path))
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
        rows, before = [], []
        for i, line in enumerate(open(self.path)):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            # samples taken before the timed region are kept aside: a region shorter
            # than the sampling period falls back to the one just before it
            (before if i < getattr(self, "n_before", 0) else rows).append(parts)
        if not rows:
            rows = before[-1:]
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def peaks():
    """HBM GB/s, BF16 TFLOP/s burst and sustained, and where they come from."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        burst = float(d["bf16_tflops"])
        return (float(d["hbm_gbs"]), burst, float(d.get("bf16_tflops_sustained", burst)),
                "measured")
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


# --------------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle (CPU FP64) timed on the host cores on bounded samples of the
    same workload: each step runs whole sequences for a fixed time budget."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    w = load_workload(args.workload, args.seqs)
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(w, budget_s=min(per_step, 2.0))
    vals, samples, secs = [], [], 0.0
    for _ in range(args.steps):
        v, sample, dt, _ = oracle_sample(w, budget_s=per_step)
        vals.append(v)
        samples.append(sample)
        secs += dt
    value = statistics.median(vals)
    cores = blas_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "states/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * secs / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args.workload, w, 1),
            "cpu_baseline": {"value": value, "unit": "states/s", "cores": cores,
                             "kind": "oracle", "sample": samples[-1],
                             "host_cpus": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "states/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- our arm
def events(n):
    import torch
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(n)]


def timed_steps(fn, steps, flush, stream):
    """Per-step device milliseconds of fn, L2 flushed before each step."""
    import torch
    ev = events(steps)
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def stage_roofline(w, c, stage_ms, precision, args):
    """Roofline of the stage kernel from its per-launch durations (a separate
    pass with an event pair around every stage launch)."""
    import numpy as np
    hbm_peak, bf16_peak, bf16_sustained, peak_kind = peaks()
    m = w.m
    f64 = precision == "fp64"
    esize = 4 if precision == "bf16_split" else 8
    Ls = w.lengths.astype(np.int64)
    Ns = c.seq_N()
    # stage 1 forming v^(1) on chip is another kernel variant (more warps, bound by
    # instruction issue): reported on its own, with the bytes it moves
    # stages 1 .. J as one pass with the states on chip (timed as stage 1), or
    # stage 1 forming v^(1) on chip: other kernels, reported on their own
    J = 0 if f64 else c.fused_stages()
    first = (not f64) and (J > 0 or c.first_fused())
    first_ms = float(np.mean(stage_ms[1])) if first and 1 in stage_ms else 0.0
    plain = {k: v for k, v in stage_ms.items() if not (first and k == 1)}
    tot = {k: sum(v) for k, v in plain.items()}
    nl = sum(len(v) for v in plain.values())
    avg_ms = sum(tot.values()) / max(1, nl)
    fused = c.output_fused()
    bytes_l, flops_l = [], []
    for k in plain:
        s = 1 << k
        live = Ns >= k
        last = live & (Ns == k) if fused else np.zeros_like(live)
        mid = live & ~last
        upd = int(np.maximum(Ls[live] - s, 0).sum())
        upd_mid = int(np.maximum(Ls[mid] - s, 0).sum())
        rows_mid, rows_last = int(Ls[mid].sum()), int(Ls[last].sum())
        # before a sequence's last stage: read every row of v^(k) once and write the
        # updated rows of v^(k+1) (esize bytes per element); its last stage with the
        # output fused reads every row of v^(k) and u and writes y, not v (v as well
        # when the plan keeps its stage outputs); plus the power's operand planes
        bytes_l.append(esize * m * (rows_mid + upd_mid) + (esize * m + 4 * (w.p + w.q)) * rows_last
                       + w.nsys * m * m * esize)
        flops_l.append((1 if f64 else 3) * 2 * m * m * upd)
    alg_bytes = float(np.mean(bytes_l)) if bytes_l else 0.0
    alg_flops = float(np.mean(flops_l)) if flops_l else 0.0
    gbs = alg_bytes / (avg_ms / 1000.0) / 1e9 if avg_ms > 0 else 0.0
    tfs = alg_flops / (avg_ms / 1000.0) / 1e12 if avg_ms > 0 else 0.0
    stage_total = sum(tot.values()) / max(1, args.steps)
    if f64:
        return {"bound": "alu", "achieved": tfs, "peak": 1.25, "unit": "TFLOP/s",
                "frac": tfs / 1.25, "traffic": None, "kernel": "stage_f64_kernel",
                "peak_kind": "nominal FP64 (1.25 TFLOP/s)", "alg_flops_per_launch": alg_flops,
                "avg_launch_ms": avg_ms, "launches_per_step": len(plain)}
    # Tensor peak: the BF16 pair's measured rate (the TF32 pair's is half of it, the
    # nominal 1.1 vs 2.25 PFLOP/s); the sustained figure when the stage launches of one
    # step keep the tensor cores busy for 10 ms or more (the power cap then holds the
    # clock down), the burst figure otherwise.
    long_step = stage_total >= 10.0
    tpk = (bf16_sustained if long_step else bf16_peak) * (1.0 if esize == 4 else 0.5)
    tpk_kind = (f"{peak_kind} BF16 {'sustained' if long_step else 'burst'}"
                + ("" if esize == 4 else " x 0.5 (TF32)"))
    hbm_part = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "alg_bytes_per_launch": alg_bytes, "peak_kind": peak_kind}
    tensor_part = {"achieved": tfs, "peak": tpk, "unit": "TFLOP/s", "frac": tfs / tpk,
                   "alg_flops_per_launch": alg_flops, "peak_kind": tpk_kind}
    intensity = alg_flops / alg_bytes if alg_bytes > 0 else 0.0
    ridge = tpk * 1e12 / (hbm_peak * 1e9)
    tensor_bound = intensity > ridge
    main, other = (tensor_part, hbm_part) if tensor_bound else (hbm_part, tensor_part)
    kname = f"stage_tc_kernel<{'bf16' if esize == 4 else 'tf32'}>"
    traffic, traffic_note = None, None
    tr = TRAFFIC.get(args.cur_workload)
    traffic_alg = None
    if tr and not args.seqs and tr[1] in plain:
        traffic, traffic_note = tr[0], tr[2]
        traffic_alg = float(bytes_l[list(plain).index(tr[1])])
    roof = {"bound": "tensor" if tensor_bound else "hbm", "achieved": main["achieved"],
            "peak": main["peak"], "unit": main["unit"], "frac": main["frac"],
            "traffic": traffic, "traffic_note": traffic_note,
            "traffic_stage": tr[1] if traffic else None,
            "alg_bytes_traffic_stage": traffic_alg,
            "kernel": kname + (" (stages 2..N; stage 1 with v^(1) formed on chip under "
                               "stage1_on_chip)" if first else " (stages 1..N)"),
            "peak_kind": main["peak_kind"], "intensity_flop_per_byte": intensity,
            "ridge_flop_per_byte": ridge, "alg_bytes_per_launch": alg_bytes,
            "alg_flops_per_launch": alg_flops, "avg_launch_ms": avg_ms,
            "launches_per_step": len(plain), "stage_ms_per_step": stage_total,
            "hbm" if tensor_bound else "tensor": other}
    if J > 0 and first_ms > 0:
        # reads u, writes v^(J+1) (every row of the sequences); useful products
        # 6 m^2 per updated row per stage, and the windows' halo on top
        H = (2 << J) - 2
        rows = int(Ls.sum())
        bJ = (esize * m + 4 * w.p) * rows
        useful = sum(6.0 * m * m * float(np.maximum(Ls - (1 << k), 0).sum()) for k in range(1, J + 1))
        wins = int(sum((int(L) + (128 - H) - 1) // (128 - H) for L in Ls))
        executed = 6.0 * m * m * 128 * wins * J
        tf = useful / (first_ms / 1000.0) / 1e12
        roof["fused_first_stages"] = {
            "kernel": f"fused_stages_kernel<{m}>: stages 1..{J} in one pass from u, states on "
                      f"chip, windows of 128 steps with a {H}-row halo",
            "stages": J, "ms": first_ms, "alg_bytes": bJ,
            "achieved_gbs": bJ / (first_ms / 1000.0) / 1e9, "useful_flops": useful,
            "executed_flops": executed, "achieved": tf, "unit": "TFLOP/s",
            "frac_of_tensor": tf / (bf16_peak if esize == 4 else bf16_peak * 0.5),
            "executed_frac_of_tensor": executed / (first_ms / 1000.0) / 1e12 /
            (bf16_peak if esize == 4 else bf16_peak * 0.5)}
        roof["kernel"] = kname + f" (stages {J + 1}..N; stages 1..{J} under fused_first_stages)"
    elif first and first_ms > 0:
        rows1 = int(Ls[Ns >= 1].sum())
        b1 = (esize * m + 4 * w.p) * rows1 + w.nsys * m * m * esize
        roof["stage1_on_chip"] = {
            "kernel": kname + " with v^(1) = Bbar u + Abar Bbar u_(l-1) formed on chip",
            "ms": first_ms, "alg_bytes": b1, "achieved": b1 / (first_ms / 1000.0) / 1e9,
            "unit": "GB/s", "frac_of_hbm": b1 / (first_ms / 1000.0) / 1e9 / hbm_peak}
    # every stage of a forward together (§3 algorithmic products over the summed
    # stage launch times, the fused first pass included)
    all_flops = sum((1 if f64 else 3) * 2.0 * m * m * float(np.maximum(Ls[Ns >= k] - (1 << k), 0).sum())
                    for k in range(1, int(Ns.max(initial=0)) + 1))
    all_ms = stage_total + first_ms
    if all_ms > 0 and not f64:
        tf = all_flops / (all_ms / 1000.0) / 1e12
        roof["all_stages"] = {"flops_per_step": all_flops, "ms_per_step": all_ms,
                              "achieved": tf, "unit": "TFLOP/s", "frac_of_tensor": tf / tpk,
                              "peak_kind": tpk_kind}
    return roof


def measure(name, args, dev, world, rank):
    """Every figure of one workload: forward (timed without per-stage events),
    per-stage times (separate pass), end to end with host buffers and with
    set-up, the work-efficient schedule, forward + backward, the FP64
    comparators, and the oracle leg with the error of the timed y."""
    import ctypes
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2411_17729_gb300 import cascade
    from paper_2411_17729_gb300._abi import (CASCADE_FLAG_GRAPH, CASCADE_FLAG_RECOMPUTE,
                                             CASCADE_FLAG_SAVE_STATES, CASCADE_FLAG_SCAN)
    args.cur_workload = name
    precision, description, has_bwd = SPECS[name]
    w = load_workload(name, args.seqs)
    m = w.m
    f64 = precision == "fp64"
    dt = torch.float64 if f64 else torch.float32
    t_prep0 = time.perf_counter()
    c = cascade.from_workload(w, precision=precision, device=dev)
    torch.cuda.synchronize()
    prep_s = time.perf_counter() - t_prep0
    u = torch.as_tensor(w.u, dtype=dt).to(dev).contiguous()
    y = torch.empty((w.rows, w.q), dtype=dt, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    lib = c.lib

    def step():
        c.forward(u, y)

    Ns = c.seq_N()
    shape = c.autotune(u, y, reps=3) if not f64 else (0, 0, 0)   # kernel shape (untimed)
    stage_shapes = {} if f64 else {str(k): list(v) for k, v in c.stage_shapes().items()
                                   if tuple(v) != tuple(shape)}
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if c.device_error() != 0:
        raise RuntimeError("device wait timed out during warm-up")

    # ---- timed region: K forward passes, L2 flushed before each, no per-stage events
    ev = events(args.steps)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = lib.cascade_launch_count()
    torch.cuda.nvtx.range_push("timed")         # profiler filter (ncu --nvtx-include timed/)
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    launches = lib.cascade_launch_count() - launches0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_per_step = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)
    states_per_step = int(w.rows)
    value = whole_job_rate(states_per_step, world, ms_per_step)
    if c.device_error() != 0:
        raise RuntimeError("device wait timed out in the timed region")
    y_host = y.double().cpu().numpy()        # the timed output, for the error check

    # ---- per-stage durations: a separate pass with an event pair per stage launch
    c.enable_stage_timing(True)
    stage_ms = {}
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        step()
        for k, ms in c.stage_times():
            stage_ms.setdefault(k, []).append(ms)
    torch.cuda.synchronize()
    c.enable_stage_timing(False)
    roofline = stage_roofline(w, c, stage_ms, precision, args)
    roofline["share_of_step"] = roofline.get("stage_ms_per_step", 0.0) / ms_per_step

    # ---- end to end through the public API with host buffers: one
    # cascade_forward_host call per step (u copied in, forward, y copied out)
    u_pin = torch.as_tensor(w.u, dtype=dt).pin_memory()
    y_pin = torch.empty((w.rows, w.q), dtype=dt).pin_memory()

    def e2e_step():
        c.forward_host(u_pin, y_pin, u, y)

    e2e_ms = max_over_ranks(sum(timed_steps(e2e_step, args.steps, flush, stream)) / args.steps,
                            world, dev)
    shape_now = (shape, {int(k): tuple(v) for k, v in stage_shapes.items()})
    c.close()
    torch.cuda.empty_cache()

    # ---- set-up (discretisation, squaring chain, operand split) plus one forward,
    # host buffers in and out, the kernel shape saved from the tuning above
    def setup_and_forward():
        cc = cascade.from_workload(w, precision=precision, device=dev)
        if not f64:
            cc.set_kernel_shape(*shape_now[0])
            cc.set_stage_shapes(shape_now[1])
        cc.forward_host(u_pin, y_pin, u, y)
        return cc

    setup_and_forward().close()                     # warm (first-touch of the host arrays)
    ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        ta = time.perf_counter()
        cc = setup_and_forward()
        ts.append(time.perf_counter() - ta)
        cc.close()
    setup_fwd_ms = 1000.0 * statistics.median(ts)

    # ---- the work-efficient schedule (about 2L products per sequence), same workload
    scan = None
    if not f64 and not args.no_scan:
        torch.cuda.nvtx.range_push("scan")         # profiler filter (ncu --nvtx-include scan/)
        # the level launches are short: the timed steps replay a CUDA graph of the
        # whole schedule (captured once per buffer set), without per-level events
        cg = cascade.from_workload(w, precision=precision,
                                   flags=CASCADE_FLAG_SCAN | CASCADE_FLAG_GRAPH, device=dev)
        scan_shape = cg.autotune(u, y, reps=6)
        for _ in range(max(args.warmup, 3)):
            cg.forward(u, y)
        scan_ms = max_over_ranks(
            sum(timed_steps(lambda: cg.forward(u, y), args.steps, flush, stream)) / args.steps,
            world, dev)
        if cg.device_error() != 0:
            raise RuntimeError("device wait timed out in the scan region")
        scan_levels = cg.stage_shapes()
        cg.close()
        torch.cuda.empty_cache()
        # per-level durations: the same schedule launched directly, with events
        cs = cascade.from_workload(w, precision=precision, flags=CASCADE_FLAG_SCAN, device=dev)
        cs.set_kernel_shape(*scan_shape)      # the shapes the timed steps ran
        cs.set_stage_shapes(scan_levels)
        for _ in range(max(args.warmup, 3)):
            cs.forward(u, y)
        cs.enable_stage_timing(True)
        lev_ms = {}
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            cs.forward(u, y)
            for k, ms in cs.stage_times():
                lev_ms.setdefault(k, []).append(ms)
        torch.cuda.synchronize()
        cs.enable_stage_timing(False)
        if cs.device_error() != 0:
            raise RuntimeError("device wait timed out in the scan region")
        nmv = ctypes.c_int64()
        cs._check(cs.lib.cascade_get_matvec_count(cs.plan, ctypes.byref(nmv)))
        Ls = w.lengths.astype(np.int64)
        # algorithmic bytes of the level launches: per updated row, read the
        # destination and the source row and write the destination (esize bytes
        # per element), plus the power planes per system and launch
        esize = 4 if precision == "bf16_split" else 8
        upd = nmv.value - sum(int(L) // 2 for L in Ls)      # products made on the tensor cores
        stage_lev = {k: v for k, v in lev_ms.items() if k < 300}
        nlev = len(stage_lev)
        lev_tot = sum(sum(v) for v in stage_lev.values()) / args.steps
        top_ms = sum(sum(v) for k, v in lev_ms.items() if k >= 300) / args.steps
        upd0 = sum(max(int(L) - 1, 0) // 2 for L in Ls) if cs.first_fused() else 0
        lev_bytes = (3 * esize * m * (upd - upd0) + (esize * m + 4 * w.p) * upd0
                     + nlev * w.nsys * m * m * esize)
        lev_gbs = lev_bytes / (lev_tot / 1000.0) / 1e9 if lev_tot > 0 else 0.0
        hbm_peak, bf16_peak = peaks()[:2]
        # 3 BF16 products of 2 m^2 per level product (the first level's products are
        # the input projection's, not a level launch's)
        lev_flops = 6.0 * m * m * upd
        tpk = bf16_peak * (1.0 if esize == 4 else 0.5)
        lev_tfs = lev_flops / (lev_tot / 1000.0) / 1e12 if lev_tot > 0 else 0.0
        scan_tensor = lev_bytes > 0 and lev_flops / lev_bytes > tpk * 1e12 / (hbm_peak * 1e9)
        scan = {"value": whole_job_rate(states_per_step, world, scan_ms), "unit": "states/s",
                "ms_per_step": scan_ms, "matvecs_per_step": int(nmv.value),
                "levels": nlev, "level_ms_per_step": lev_tot, "top_of_tree_ms_per_step": top_ms,
                # per launch: up-sweep level k as "k", down-sweep level k as "100+k", the
                # top of the tree as "300+k0" (median ms)
                "level_ms": {str(k): round(statistics.median(v), 4) for k, v in sorted(lev_ms.items())},
                "roofline": ({"bound": "tensor", "achieved": lev_tfs, "peak": tpk,
                              "unit": "TFLOP/s", "frac": lev_tfs / tpk,
                              "hbm_frac": lev_gbs / hbm_peak}
                             if scan_tensor else
                             {"bound": "hbm", "achieved": lev_gbs, "peak": hbm_peak,
                              "unit": "GB/s", "frac": lev_gbs / hbm_peak,
                              "tensor_frac": lev_tfs / tpk})
                | {"kernel": "stage_tc_kernel, strided in-place levels",
                   "alg_bytes_per_step": lev_bytes, "alg_flops_per_step": lev_flops},
                "schedule": "up-sweep k=1..K-1, down-sweep k=K-2..0 (first level fused "
                            "with Bbar u), in place",
                "timing": "CUDA graph replay of the level launches; per-level durations "
                          "from separate direct launches with events",
                "kernel_shape": {"stages": scan_shape[0], "ring": scan_shape[1],
                                 "chunks_per_step": scan_shape[2],
                                 "per_level": {str(k): list(v) for k, v in scan_levels.items()
                                               if tuple(v) != tuple(scan_shape)}}}
        cs.close()
        torch.cuda.empty_cache()
        torch.cuda.nvtx.range_pop()

    # ---- forward + backward, same workload
    fb = None
    if has_bwd and not args.no_bwd:
        torch.cuda.nvtx.range_push("fwd_bwd")
        # the differentiation workload recomputes stage outputs from checkpoints
        recompute = name == "differentiation_form"
        cb = cascade.from_workload(w, precision=precision,
                                   flags=CASCADE_FLAG_RECOMPUTE if recompute
                                   else CASCADE_FLAG_SAVE_STATES, device=dev)
        cb.autotune(u, y, reps=1)
        dy = torch.randn((w.rows, w.q), dtype=dt, device=dev,
                         generator=torch.Generator(device=dev).manual_seed(0))
        for _ in range(2):
            cb.forward(u, y)
            cb.backward(u, dy)
        fb_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                  torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            fb_ev[i][0].record(stream)
            cb.forward(u, y)
            fb_ev[i][1].record(stream)
            cb.backward(u, dy)
            fb_ev[i][2].record(stream)
        torch.cuda.synchronize()
        if cb.device_error() != 0:
            raise RuntimeError("device wait timed out in the fwd+bwd region")
        fb_ms = sum(a.elapsed_time(cc) for a, _, cc in fb_ev) / args.steps
        bwd_ms = sum(b.elapsed_time(cc) for _, b, cc in fb_ev) / args.steps
        fb_ms = max_over_ranks(fb_ms, world, dev)
        fb = {"value": whole_job_rate(states_per_step, world, fb_ms), "unit": "states/s",
              "ms_per_step": fb_ms, "backward_ms": bwd_ms,
              "gradients": "u, A (or Abar), B (or Bbar), C, D",
              "stage_outputs": "recomputed from checkpoints" if recompute else "kept",
              "workspace_bytes": int(cb.workspace_size())}
        cb.close()
        torch.cuda.empty_cache()
        torch.cuda.nvtx.range_pop()

    # ---- FP64 plain cascade and FP64 recursion on the same GPU (comparators)
    fp64 = None
    rec = None
    nsub = min(8 if m <= 256 else 1, w.nseq)   # FP64 runs near 1.25 TFLOP/s: bound the sample
    if not args.no_fp64 and not f64:
        sub = w.subset(range(nsub))
        c64 = cascade.from_workload(sub, precision="fp64", device=dev)
        u64 = torch.as_tensor(sub.u, dtype=torch.float64).to(dev)
        c64.forward(u64)
        ms = timed_steps(lambda: c64.forward(u64), 1, flush, stream)[0]
        fp64 = {"value": sub.rows / (ms / 1000.0), "unit": "states/s",
                "sample": f"{sub.nseq} of {w.nseq} sequences, one pass", "error_bar": TOL["fp64"]}
        c64.close()
    if not args.no_fp64:
        # one block per sequence, one step after the other: its rate does not depend
        # on the length, so a prefix of the first sequence bounds the time
        nrec = min(int(w.lengths[0]), 4096 if m >= 512 else 65536)
        sub = w.subset([0])
        sub.offsets = np.array([0, nrec], np.int64)
        sub.u = sub.u[:nrec]
        cr = cascade.from_workload(sub, precision="fp64", device=dev, max_len=nrec)
        u64 = torch.as_tensor(sub.u, dtype=torch.float64).to(dev)
        ms = timed_steps(lambda: cr.recursion(u64), 1, flush, stream)[0]
        rec = {"value": nrec / (ms / 1000.0), "unit": "states/s",
               "sample": f"the first {nrec} steps of one sequence, one block"}
        cr.close()

    # ---- oracle on the host cores (rank 0, N = 1 only), and the error of the timed y
    cpu, error = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, sample, _, outs = oracle_sample(w, budget_s=12.0, keep=True)
        cpu = {"value": v, "unit": "states/s", "cores": blas_threads(), "kind": "oracle",
               "sample": sample, "host_cpus": os.cpu_count(), "cpu_model": cpu_model(),
               "one_thread": oracle_one_thread(name)}
        error = error_of(w, y_host, outs, precision, sample)

    Ls = w.lengths.astype(np.int64)
    res = {
        "value": value, "ms_per_step": ms_per_step,
        "dtype": {"bf16_split": "bf16", "fp32": "tf32", "fp64": "f64"}[precision],
        "config": config_of(name, w, world),
        "roofline": roofline,
        "error": error,
        "cpu_baseline": cpu,
        "e2e": {"value": whole_job_rate(states_per_step, world, e2e_ms), "unit": "states/s",
                "call": "cascade_forward_host (page-locked host u and y)",
                "h2d_bytes_per_step": int(u.numel() * u.element_size()),
                "d2h_bytes_per_step": int(y.numel() * y.element_size())},
        "e2e_with_setup": {"value": states_per_step / (setup_fwd_ms / 1000.0), "unit": "states/s",
                           "ms": setup_fwd_ms,
                           "what": "plan creation, discretisation, FP64 squaring chain and "
                                   "operand split, host-to-device u, forward, device-to-host y "
                                   "(host clock, median of 3)"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "fwd_bwd": fb,
        "scan_fwd": scan,
        "fp64_cascade": fp64,
        "fp64_recursion": rec,
        # products by powers per step: executed by the stage schedule of §3, the 2L
        # bound of the abstract and §6, and the L of the recursion (Eq. 1.2)
        "op_count": {
            "stage_schedule": int(sum(sum(max(int(L) - (1 << k), 0) for k in range(int(Nk) + 1))
                                      for L, Nk in zip(Ls, Ns))),
            "work_efficient_schedule": scan["matvecs_per_step"] if scan else None,
            "paper_bound_2L": int(2 * Ls.sum()), "recursion_L": int(Ls.sum())},
        "precompute_s": prep_s,
        "kernel_shape": {"stages": shape[0], "ring": shape[1], "chunks_per_step": shape[2],
                         "per_stage": stage_shapes},
        "stage_ms": {str(k): statistics.median(v) for k, v in sorted(stage_ms.items())},
        "wall_s": wall,
    }
    return res


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    from paper_2411_17729_gb300 import build
    build()

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    head = measure(args.workload, args, dev, world, rank)
    also = None
    if args.also and args.also != "none" and args.also != args.workload:
        also = measure(args.also, args, dev, world, rank)

    failed = [r for r in (head, also) if r and r["error"] and not r["error"]["pass"]]
    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": "states/s", "n_gpus": world,
                "steps": args.steps, "warmup": max(args.warmup, 3),
                "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": head["dtype"], "data": "synthetic",
                "config": head["config"],
                "timing": "CUDA events on the launching stream around each step, L2 flushed "
                          "(256 MiB write) before each timed step, no per-stage events in the "
                          "timed steps",
                **{k: v for k, v in head.items()
                   if k not in ("value", "ms_per_step", "dtype", "config")}}
        if also:
            line[args.also] = also
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    if failed:
        print("error above the bar: " + "; ".join(json.dumps(r["error"]) for r in failed),
              file=sys.stderr, flush=True)
        sys.exit(3)


if __name__ == "__main__":
    main()
