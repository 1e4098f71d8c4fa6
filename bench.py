"""Benchmark of the SALT hot path on GB300.

One step = one pass of the BLAS-1 sweep's top size through the library:
for FP32 and FP64, n = 2^28 elements,
  e = alpha*a + beta*b - c o d   (fused 4-operand expression, salt_eval)
  y = alpha*x + beta*y           (salt_axpby)
  dot(x, y)                      (salt_dot)
  nrm2(x)                        (salt_nrm2)
with alpha = 1.5, beta = -0.25 and inputs uniform[-1, 1) from the
counter-based generator.  value = algorithmic bytes moved by the step (each
operand element read once, each result written once) / device time, summed
over ranks (each rank is an independent replica).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead (the reference arm of this repository: there is no other
implementation of the paper's method to run).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused vector-expr HBM GB/s (% of peak), batched vs plain; served p50/p99 µs"
ALPHA, BETA = 1.5, -0.25
DTYPES = ("f32", "f64")
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal (~8 TB/s); the measured copy rate is the roofline peak
# (op, bytes moved per element in units of the element size, flops per element)
OPS = {"e": (5, 5), "axpby": (3, 3), "dot": (2, 2), "nrm2": (1, 2)}


def is_pow2(s: float) -> bool:
    """s = +-2^e with 2^e a normal FP64 number."""
    m, e = math.frexp(s)
    return abs(m) == 0.5 and -1022 <= e - 1 <= 1023


# FP64 instructions per element of each op's kernel (ALU roofline of FP64).
# e = alpha*a + beta*b - c o d and y = alpha*x + beta*y issue beta*b + (...)
# as one FMA when beta is a power of two (the product is then exact for the
# operands' ranges): 4 and 2 instructions instead of 5 and 3.
F64_INSTR = {"e": 5 - is_pow2(BETA), "axpby": 3 - is_pow2(BETA), "dot": 1, "nrm2": 1}
ES = {"f32": 4, "f64": 8}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured", float(p.get("sm_max_mhz", 2070.0))
    except Exception:
        return 6800.0, "fallback", 2070.0


# FP64 ALU peak from unit counts and clocks: 2 FP64 instructions per clock per
# SM (GB300), 152 SMs, at the maximum SM clock.
def f64_alu_peak_gops(sm_mhz: float) -> float:
    return 2 * 152 * sm_mhz * 1e6 / 1e9


# The sources that define each profiled kernel (its template, the headers it
# instantiates and the file that instantiates it); a traffic figure is used
# only while these are unchanged since the capture.
KERNEL_SOURCES = {
    "e_f64": ["prog.cuh", "common.cuh", "fused.cuh", "reduce.cuh", "shapes.h", "registry.h", "inst.cuh",
              "inst_f64_vb16.cu", "inst_f64_vb32.cu"],
    "axpby_f64": ["prog.cuh", "common.cuh", "fused.cuh", "reduce.cuh", "shapes.h", "registry.h", "inst.cuh",
                  "inst_f64_vb16.cu", "inst_f64_vb32.cu"],
    "e_f64_staged": ["prog.cuh", "common.cuh", "fused.cuh", "staged.cuh", "shapes.h", "registry.h",
                     "inst_staged.cu"],
    "axpby_f64_staged": ["prog.cuh", "common.cuh", "fused.cuh", "staged.cuh", "shapes.h", "registry.h",
                         "inst_staged.cu"],
    "dot_f64_staged": ["prog.cuh", "common.cuh", "fused.cuh", "staged.cuh", "shapes.h", "registry.h",
                       "inst_staged.cu"],
}


def source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1109_1264_gb300", "csrc")
    for name in sorted(KERNEL_SOURCES.get(kernel, [])):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for_smi(torch) -> str:
    try:
        u = str(torch.cuda.get_device_properties(0).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
    return vis or "0"


# ---------------------------------------------------------------- workload --
class Workload:
    """Device buffers of one dtype: a, b, c, d inputs, out for e, y for axpby."""

    def __init__(self, torch, salt, dt: str, n: int, seed: int = 0):
        tdt = torch.float32 if dt == "f32" else torch.float64
        self.dt, self.n = dt, n
        self.a, self.b, self.c, self.d = (torch.empty(n, dtype=tdt, device="cuda") for _ in range(4))
        self.out = torch.empty(n, dtype=tdt, device="cuda")
        self.y = torch.empty(n, dtype=tdt, device="cuda")
        self.red = torch.zeros(2, dtype=torch.float64, device="cuda")
        for k, t in enumerate((self.a, self.b, self.c, self.d, self.y)):
            salt.salt_fill_uniform(t, key=seed * 16 + k + 1)

    def tune(self, salt) -> dict:
        """Autotunes the launch shape of each op of the step (setup, untimed)."""
        from paper_1109_1264_gb300.programs import PROG_AXPBY, PROG_DOT, PROG_E
        got = {}
        r = 4  # timed calls per candidate: the schedules differ by a few percent at this size
        got["e"], _ = salt.salt_autotune(salt.KERNEL_PROGRAM, PROG_E, [self.a, self.b, self.c, self.d, self.out],
                                         [ALPHA, BETA], reps=r)
        got["axpby"], _ = salt.salt_autotune(salt.KERNEL_PROGRAM, PROG_AXPBY, [self.a, self.y], [ALPHA, BETA], reps=r)
        got["dot"], _ = salt.salt_autotune(salt.KERNEL_PROGRAM, PROG_DOT, [self.a, self.b], red_out=self.red[0:1],
                                           reps=r)
        got["nrm2"], _ = salt.salt_autotune(salt.KERNEL_NRM2, None, [self.c], red_out=self.red[1:2], reps=r)
        return got

    def ops(self, salt):
        """(name, callable) of the step, in order."""
        from paper_1109_1264_gb300.programs import PROG_E
        return [
            ("e", lambda: salt.salt_eval(PROG_E, [self.a, self.b, self.c, self.d, self.out], [ALPHA, BETA])),
            ("axpby", lambda: salt.salt_axpby(ALPHA, self.a, BETA, self.y)),
            ("dot", lambda: salt.salt_dot(self.a, self.b, self.red[0:1])),
            ("nrm2", lambda: salt.salt_nrm2(self.c, self.red[1:2])),
        ]


def refine_in_step(torch, salt, steps, n: int, tuned: dict, reps: int = 3) -> dict:
    """The library's autotuner times each call on its own, back to back; in
    the step every kernel follows a different one (and the write-back of its
    dirty L2 lines), and between the two loop schedules, which often come
    within a few percent of each other alone, the faster alone was at times
    the slower in the step.  So for each op with a compiled shape the
    autotuned configuration is compared, inside the running step (the other
    ops as tuned), with a few register-tiled and staged alternatives, and the
    fastest there is kept (median of `reps` steps of that op's own events).
    Setup only, before the warm-up and the timed steps."""
    import numpy as np

    from paper_1109_1264_gb300.programs import PROG_AXPBY, PROG_DOT, PROG_E
    progs = {"e": PROG_E, "axpby": PROG_AXPBY, "dot": PROG_DOT}
    alternatives = [(2, 32, 256, 0, 0), (4, 32, 128, 0, 0), (1, 32, 256, 0, 0), (2, 32, 256, 4, 0),
                    (1, 16, 128, 0, 16384), (1, 16, 256, 0, 16384), (1, 16, 128, 0, 8192)]
    stream = torch.cuda.current_stream()

    def op_ms(idx):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(steps) + 1)]
        ts = []
        for _ in range(reps):
            ev[0].record(stream)
            for i, (_, _, fn) in enumerate(steps):
                fn()
                ev[i + 1].record(stream)
            torch.cuda.synchronize()
            ts.append(ev[idx].elapsed_time(ev[idx + 1]))
        return float(np.median(ts))

    chosen = {}
    for idx, (dt, op, _) in enumerate(steps):
        if op not in progs:
            continue
        code = salt.F32 if dt == "f32" else salt.F64
        first = salt.salt_tune_get(progs[op], code, n)
        cands = [tuple(first.values())] + [c for c in alternatives if c != tuple(first.values())]
        best, best_ms = None, None
        for c in cands:
            salt.salt_tune_set(progs[op], code, n, *c)
            ms = op_ms(idx)
            if best_ms is None or ms < best_ms:
                best, best_ms = c, ms
        salt.salt_tune_set(progs[op], code, n, *best)
        chosen[f"{op}_{dt}"] = dict(zip(("unroll", "vec_bytes", "block", "blocks_per_sm", "stage_bytes"), best))
    return chosen


def algorithmic_bytes(n: int) -> dict:
    return {(dt, op): OPS[op][0] * ES[dt] * n for dt in DTYPES for op in OPS}


# ---------------------------------------------------------------- CPU leg --
def oracle_pass(n: int, seed: int = 0):
    """Run the step's ops on the CPU oracle once at size n; returns (seconds,
    algorithmic bytes)."""
    import numpy as np

    import oracle
    from paper_1109_1264_gb300 import inputs
    total_t, total_b = 0.0, 0
    for dt in DTYPES:
        npdt = np.float32 if dt == "f32" else np.float64
        a, b, c, d, y = (inputs.hash_uniform(seed * 16 + k + 1, n, npdt) for k in range(5))
        out = np.empty_like(a)
        t0 = time.perf_counter()
        oracle.eval_program(oracle.PROG_E, [a, b, c, d, out], [ALPHA, BETA])
        oracle.eval_program(oracle.PROG_AXPBY, [a, y], [ALPHA, BETA])
        oracle.dot(a, b)
        oracle.nrm2(c)
        total_t += time.perf_counter() - t0
        total_b += sum(OPS[op][0] for op in OPS) * ES[dt] * n
    return total_t, total_b


def cpu_baseline(n_sample: int, budget_s: float = 12.0) -> dict:
    import oracle
    oracle.build()
    t, b, passes = 0.0, 0, 0
    while passes < 1 or (t < budget_s and passes < 50):
        dt, db = oracle_pass(n_sample)
        t += dt
        b += db
        passes += 1
    return {"value": round(b / t / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"e, axpby, dot, nrm2 x FP32/FP64 at n=2^{n_sample.bit_length() - 1}, {passes} pass(es), "
                      f"single-threaded C oracle (unfused, one loop per node)"}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    n_sample = 1 << args.cpu_log2
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle_pass(n_sample)
    t, b = 0.0, 0
    for _ in range(args.steps):
        dt, db = oracle_pass(n_sample)
        t += dt
        b += db
    value = b / t / 1e9
    sample = (f"e, axpby, dot, nrm2 x FP32/FP64 at n=2^{args.cpu_log2} per step (1/{1 << (args.log2n - args.cpu_log2)} "
              f"of the workload), single-threaded C oracle")
    line = {"metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(args.log2n, world),
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm --
def workload_config(log2n: int, world: int) -> dict:
    return {"workload": "BLAS-1 sweep top size: e=alpha*a+beta*b-c*d, y=alpha*x+beta*y, dot, nrm2; "
                        "FP32 and FP64; n=2^%d" % log2n,
            "n": 1 << log2n, "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (no flush needed)"}


def max_over_ranks(torch, dist, ms: float, world: int, device: str) -> float:
    """The slowest rank's time: every rank is an independent replica of the
    step, so the whole job ends when the slowest one does."""
    if world <= 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(step_bytes: int, steps: int, world: int, max_ms: float) -> float:
    """Algorithmic bytes all ranks moved / the max-over-ranks time (weak scaling)."""
    return world * step_bytes * steps / (max_ms * 1e-3) / 1e9


def traffic_for(kernel: str, n: int):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on
    the current kernel sources (scaled from the captured size to n)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    ent = t.get(kernel)
    if not ent or kernel not in KERNEL_SOURCES or ent.get("source_hash") != source_hash(kernel):
        return None
    return int(ent["dram_bytes_per_launch"] * n / ent["n"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="salt", choices=["salt", "reference"])
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--cpu-log2", type=int, default=22)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--batched-items", type=int, default=4096)
    ap.add_argument("--batched-fixed", action="store_true", help="skip the batch autotuner (profiling runs)")
    ap.add_argument("--only-batched", action="store_true", help="run only the batched leg (profiling runs)")
    ap.add_argument("--sweep", action="store_true", help="the paper's four-op size sweep instead of the step")
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=16, help="chunks per vector in the end-to-end pipeline")
    ap.add_argument("--tune-save", default=None, help="write the autotuned launch table to this file")
    ap.add_argument("--tune-load", default=None,
                    help="profiling runs: load a saved launch table instead of autotuning")
    ap.add_argument("--only-cg", action="store_true", help="run only the CG leg (profiling runs)")
    ap.add_argument("--only-served", action="store_true", help="run only the served leg (profiling runs)")
    ap.add_argument("--schedules", action="store_true",
                    help="register-tiled versus staged loop for the compiled shapes (n = 2^24, 2^28); one JSON line")
    ap.add_argument("--fixed-cfg", action="append", default=None,
                    help="profiling runs: skip the autotuner and pin OP[_f32|_f64]=U,VB,BLOCK,BLOCKS_PER_SM[,STAGE_BYTES]"
                         " for OP in e, axpby, dot (repeatable)")
    ap.add_argument("--fixed-e-cfg", default=None,
                    help="profiling runs: skip the autotuner and launch e with U,VB,BLOCK,BLOCKS_PER_SM[,STAGE_BYTES]")
    ap.add_argument("--cg-log2", type=int, default=28)
    ap.add_argument("--no-generic", action="store_true")
    ap.add_argument("--trace-reductions", action="store_true",
                    help="per-block timelines of dot and nrm2 from n = 2^4 to 2^26 (launch ramp, tail, combine)")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.impl == "reference", "at least 3 warm-up steps"

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_1109_1264_gb300 import salt

    if args.sweep:
        if rank == 0:
            print(json.dumps(sweep_measure(torch, salt)), flush=True)
        return

    if args.schedules:
        if rank == 0:
            print(json.dumps(schedules_measure(torch, salt)), flush=True)
        return

    if args.trace_reductions:
        if rank == 0:
            print(json.dumps(reduction_trace_measure(torch, salt)), flush=True)
        return

    if args.only_served:
        if rank == 0:
            print(json.dumps({"served": served_measure(salt)}), flush=True)
        return

    if args.only_cg:
        if rank == 0:
            cg = cg_measure(torch, salt, log2n=args.cg_log2)
            cg["per_iteration_latency"] = cg_latency_measure(torch, salt)
            print(json.dumps({"cg": cg}), flush=True)
        return

    if args.only_batched:
        if rank == 0:
            print(json.dumps({"batched": batched_measure(torch, salt, nitems=args.batched_items,
                                                         fixed=args.batched_fixed)}), flush=True)
        return

    n = 1 << args.log2n
    loads = {dt: Workload(torch, salt, dt, n, seed=rank) for dt in DTYPES}
    fixed = list(args.fixed_cfg or []) + ([f"e={args.fixed_e_cfg}"] if args.fixed_e_cfg else [])
    if fixed:
        from paper_1109_1264_gb300.programs import PROG_AXPBY, PROG_DOT, PROG_E
        progs = {"e": PROG_E, "axpby": PROG_AXPBY, "dot": PROG_DOT}
        tuned = {"others": "defaults"}
        for spec in fixed:
            key, _, cfg = spec.partition("=")
            op, _, dtn = key.partition("_")
            vals = [int(v) for v in cfg.split(",")]
            if op not in progs or dtn not in ("", "f32", "f64") or len(vals) not in (4, 5):
                raise SystemExit(f"--fixed-cfg: cannot parse {spec!r}")
            u, vb, blk, bps = vals[:4]
            sb = vals[4] if len(vals) > 4 else 0
            codes = {"f32": [salt.F32], "f64": [salt.F64], "": [salt.F32, salt.F64]}[dtn]
            for code in codes:
                salt.salt_tune_set(progs[op], code, n, u, vb, blk, bps, sb)
            tuned[key] = {"unroll": u, "vec_bytes": vb, "block": blk, "blocks_per_sm": bps, "stage_bytes": sb}
    elif args.tune_load:
        salt.salt_tune_load(args.tune_load)
        tuned = {"loaded": os.path.basename(args.tune_load)}
    elif not args.no_tune:
        tuned = {dt: loads[dt].tune(salt) for dt in DTYPES}
    else:
        tuned = None
    steps = []
    for dt in DTYPES:
        for name, fn in loads[dt].ops(salt):
            steps.append((dt, name, fn))
    if tuned is not None and not args.tune_load and not fixed:
        tuned["in_step"] = refine_in_step(torch, salt, steps, n, tuned)
        if args.tune_save:
            salt.salt_tune_save(args.tune_save)
    abytes = algorithmic_bytes(n)
    step_bytes = sum(abytes[(dt, op)] for dt, op, _ in steps)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        for _, _, fn in steps:
            fn()
    barrier()

    clocks = ClockSampler(gpu_id_for_smi(torch))
    time.sleep(0.3)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(steps) + 1)] for _ in range(args.steps)]
    launches0 = salt.salt_launch_count()
    # for ncu launch lists: library launches before the timed steps (-s)
    print(f"library launches before the timed steps: {launches0}", file=sys.stderr, flush=True)
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        for i, (_, _, fn) in enumerate(steps):
            fn()
            ev[k][i + 1].record(stream)
    t_end.record(stream)
    barrier()
    launches = salt.salt_launch_count() - launches0
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    total_ms = max_over_ranks(torch, dist, total_ms, world, "cuda")

    per_kernel = {}
    for i, (dt, name, _) in enumerate(steps):
        per_kernel[(dt, name)] = sum(ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(args.steps)) / args.steps
    # the step's reduction results (judged in the CPU leg), and the same dot
    # over the first 2^26 elements (after the timed region)
    step_red = {}
    for dt in DTYPES:
        dot, nrm = loads[dt].red.cpu().tolist()
        step_red[dt] = {"dot": dot, "nrm2": nrm}
        if n > (1 << 26):
            r26 = torch.zeros(1, dtype=torch.float64, device="cuda")
            salt.salt_dot(loads[dt].a[:1 << 26], loads[dt].b[:1 << 26], r26)
            step_red[dt]["dot_2e26"] = r26.item()

    ms_per_step = total_ms / args.steps
    value = whole_job_gbs(step_bytes, args.steps, world, total_ms)
    hbm_peak, peak_kind, sm_max = load_peaks()
    alu_peak = f64_alu_peak_gops(sm_max)

    # dominant kernel and its roofline
    (ddt, dop), dms = max(per_kernel.items(), key=lambda kv: kv[1])
    achieved_gbs = abytes[(ddt, dop)] / (dms * 1e-3) / 1e9
    roof = {"kernel": f"{dop}_{ddt}", "ms": round(dms, 4)}
    hbm_frac = achieved_gbs / hbm_peak
    if ddt == "f64":
        achieved_gops = F64_INSTR[dop] * n / (dms * 1e-3) / 1e9
        alu_frac = achieved_gops / alu_peak
        # the binding roof is the one whose lower bound on time is larger
        t_hbm = abytes[(ddt, dop)] / (hbm_peak * 1e9)
        t_alu = F64_INSTR[dop] * n / (alu_peak * 1e9)
        if t_alu > t_hbm:
            roof.update({"bound": "alu", "achieved": round(achieved_gops / 1e3, 4), "peak": round(alu_peak / 1e3, 4),
                         "unit": "T FP64 instr/s", "frac": round(alu_frac, 4),
                         "instr_per_elem": F64_INSTR[dop],
                         "peak_note": "FP64 pipe: 2 instr/clk/SM x 152 SMs x max SM clock (an FMA issues once)",
                         "hbm_achieved_gbs": round(achieved_gbs, 1), "hbm_frac": round(hbm_frac, 4)})
        else:
            roof.update({"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(hbm_frac, 4), "alu_frac": round(alu_frac, 4)})
    else:
        roof.update({"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(hbm_frac, 4)})
    # the HBM peak is the measured copy rate; the FP64 peak is derived from
    # unit counts and the clock (the live probe below gives a measured rate)
    roof["peak_kind"] = "derived" if roof["bound"] == "alu" else peak_kind
    # the traffic figure belongs to the schedule (register-tiled or staged) the op ran
    tkey = f"{dop}_{ddt}"
    if dop in ("e", "axpby", "dot"):
        from paper_1109_1264_gb300.programs import PROG_AXPBY, PROG_DOT, PROG_E
        prog = {"e": PROG_E, "axpby": PROG_AXPBY, "dot": PROG_DOT}[dop]
        if salt.salt_tune_get(prog, salt.F32 if ddt == "f32" else salt.F64, n)["stage_bytes"]:
            tkey += "_staged"
    roof["schedule"] = "staged" if tkey.endswith("_staged") else "register-tiled"
    roof["traffic"] = traffic_for(tkey, n)
    roof["algorithmic_bytes"] = abytes[(ddt, dop)]

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic: counter-based uniform[-1,1) (SplitMix64) operands, alpha=1.5, beta=-0.25",
        "config": dict(workload_config(args.log2n, world), tuned=tuned),
        "frac_of_measured_hbm": round(value / world / hbm_peak, 4),
        "frac_of_nominal_hbm": round(value / world / NOMINAL_HBM_GBS, 4),
        "roofline": roof,
        "per_kernel_ms": {f"{op}_{dt}": round(ms, 4) for (dt, op), ms in per_kernel.items()},
        "per_kernel_gbs": {f"{op}_{dt}": round(abytes[(dt, op)] / (ms * 1e-3) / 1e9, 1)
                           for (dt, op), ms in per_kernel.items()},
        "per_kernel_frac_of_measured_hbm": {f"{op}_{dt}": round(abytes[(dt, op)] / (ms * 1e-3) / 1e9 / hbm_peak, 3)
                                            for (dt, op), ms in per_kernel.items()},
        "gpu_launches": int(launches),
        "clocks": clk,
    }

    if not args.no_e2e:
        result["e2e"] = e2e_measure(torch, salt, loads, args, world, steps, abytes)
    del loads
    steps = None
    torch.cuda.empty_cache()
    samples = {"batched": [], "served": []}
    if not args.no_cg:
        torch.cuda.empty_cache()
        result["cg"] = cg_measure(torch, salt, log2n=args.cg_log2)
        result["cg"]["per_iteration_latency"] = cg_latency_measure(torch, salt)
    if not args.no_batched:
        torch.cuda.empty_cache()
        result["batched"] = batched_measure(torch, salt, nitems=args.batched_items, fixed=args.batched_fixed,
                                            collect=samples["batched"])
    if not args.no_served:
        torch.cuda.empty_cache()
        result["served"] = served_measure(salt, collect=samples["served"])
    result["config1_figure1"] = config1_measure(torch, salt)
    if not args.no_generic:
        torch.cuda.empty_cache()
        result["generic"] = generic_measure(torch, salt)
    probe = fp64_probe(torch, salt)
    sampler = ClockSampler(gpu_id_for_smi(torch))
    time.sleep(0.3)  # the sampler's first reading
    try:
        # the FP64 pipe's rate from registers, per instruction kind (the SM
        # clock during these loops beside it: under the power cap it can sit
        # below the maximum after the legs before)
        probe["register_gops"] = {k: round(salt.salt_fp64_rate(op), 1) for k, op in
                                  (("dfma", salt.FP64_FMA), ("dadd", salt.FP64_ADD), ("dmul", salt.FP64_MUL))}
    except salt.SaltError as e:
        probe["register_gops"] = {"error": e.message[:200]}
    probe["register_clocks"] = sampler.stop()
    result["fp64_probe"] = probe
    if roof["bound"] == "alu" and probe.get("gops"):
        roof["probe_gops"] = probe["gops"]
        roof["frac_vs_probe"] = round(roof["achieved"] * 1e3 / probe["gops"], 4)
        reg = probe["register_gops"].get("dfma")
        if reg:
            # every FP64 node issues as a DFMA: the register-only DFMA rate is
            # the measured ceiling beside the derived peak
            roof["register_dfma_gops"] = reg
            roof["frac_vs_register_dfma"] = round(roof["achieved"] * 1e3 / reg, 4)

    if rank == 0 and world == 1 and not args.no_cpu:
        # The CPU-oracle leg: the oracle timed on the host, and the oracle's
        # exact references judging the GPU reductions' precision.
        result["cpu_baseline"] = cpu_baseline(1 << args.cpu_log2)
        torch.cuda.empty_cache()
        prec = {"measure": "rel_value = |got - exact| / |exact| (the tolerance's measure); "
                           "rel_scale = |got - exact| / sum|x_i y_i|",
                "step_n2e28": step_precision(step_red, n, seed=rank)}
        if samples["batched"]:
            prec["batched_rho"] = batched_precision(samples["batched"])
        if samples["served"]:
            prec["served"] = served_precision(samples["served"])
        prec["config3"] = precision_measure(torch, salt)
        result["cpu_baseline"]["precision_vs_exact"] = prec
    if rank == 0:
        result["summary"] = summary_of(result)
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def summary_of(r: dict) -> dict:
    """The headline numbers of every leg in a compact object that the line
    ends with: the step, batched vs plain, served saturation and p50 / p99
    per load, Figure 1, the CG forms and the precision of every reduction."""
    out = {"step_gbs": r["value"], "frac_of_measured_hbm": r.get("frac_of_measured_hbm"),
           "roofline": {k: r["roofline"].get(k) for k in ("kernel", "bound", "frac", "hbm_frac", "frac_vs_probe",
                                                           "frac_vs_register_dfma")}}
    if "e2e" in r:
        out["e2e_gbs"] = r["e2e"]["value"]
    b = r.get("batched")
    if b:
        out["batched"] = {dt: {"gbs": b[dt]["batched_gbs"], "plain_gbs": b[dt]["plain_gbs"],
                               "ratio": b[dt]["ratio"]} for dt in DTYPES if dt in b}
    sv = r.get("served")
    if sv:
        out["served"] = {"saturation_gbs": sv["saturation_gbs"], "vs_unbatched": sv["batched_vs_unbatched"],
                         "p50_p99_us": {str(pt["load"]): [pt["p50_us"], pt["p99_us"]] for pt in sv["points"]}}
        if "one_at_a_time" in sv:
            out["served"]["one_at_a_time_p50_p99_us"] = [sv["one_at_a_time"]["p50_us"], sv["one_at_a_time"]["p99_us"]]
        pz = sv.get("persistent")
        if pz:
            out["served_persistent"] = {
                "saturation_gbs": pz["saturation_gbs"],
                "p50_p99_us": {str(pt["load"]): [pt["p50_us"], pt["p99_us"]] for pt in pz["points"]},
                "one_at_a_time_p50_p99_us": [pz["one_at_a_time"]["p50_us"], pz["one_at_a_time"]["p99_us"]]}
    if "config1_figure1" in r:
        c = r["config1_figure1"]
        out["figure1_us"] = {k: c[k] for k in ("l2_warm_us", "l2_flushed_us") if k in c}
    cg = r.get("cg")
    if cg:
        out["cg_gbs"] = {dt: {"two_pass": cg[dt]["gbs_fused"], "one_reduction": cg[dt]["one_reduction"]["gbs"],
                              "auto": cg[dt]["auto"]["form"], "auto_vs_best": cg[dt]["auto"]["vs_best"]}
                         for dt in DTYPES if dt in cg}
        lat = cg.get("per_iteration_latency", {}).get("rows", {})
        out["cg_auto_vs_best_per_iteration"] = {dt: [r.get("auto_vs_best") for r in rows] for dt, rows in lat.items()}
    g = r.get("generic")
    if g:
        out["generic_gbs"] = {k: [v["interpreter"]["gbs"], v["jit"]["gbs"]] for k, v in g["rows"].items()}
    pv = r.get("cpu_baseline", {}).get("precision_vs_exact")
    if pv:
        worst = {}
        for dt, row in pv.get("step_n2e28", {}).items():
            worst[f"step_dot_{dt}"] = row["dot"]["rel_value"]
            worst[f"step_nrm2_{dt}"] = row["nrm2"]["rel_value"]
        for dt, row in pv.get("batched_rho", {}).items():
            worst[f"batched_rho_{dt}"] = row["max_rel_value"]
        for k, row in pv.get("served", {}).items():
            worst[f"served_{k}"] = row["max_rel_value"]
        out["precision_rel_value"] = {k: float(f"{v:.3g}") for k, v in worst.items()}
    return out


def generic_measure(torch, salt, log2ns=(24, 28), reps: int = 5) -> dict:
    """The generic path: a program with no compiled instantiation (6
    operands: f = (a - b) o (c + d) - 2.5 e, and sum f^2), FP32 and FP64, run
    on the interpreter kernel (SALT_JIT_OFF) and as a run-time compiled fused
    kernel (SALT_JIT_ON).  GB/s of algorithmic bytes (5 reads + 1 write per
    element), fraction of the measured copy rate, and the first call's
    compile time."""
    import numpy as np

    prog = [("VEC", 0), ("VEC", 1), ("SUB", 0), ("VEC", 2), ("VEC", 3), ("ADD", 0), ("MUL", 0),
            ("SCAL", 0), ("VEC", 4), ("SMUL", 0), ("SUB", 0), ("STORE", 5), ("VEC", 5), ("SUMSQ", 0)]
    hbm_peak, _, _ = load_peaks()
    stream = torch.cuda.current_stream()
    prev = salt.salt_jit_stats()["mode"]
    out = {}
    try:
        for dt, tdt, es in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
            nmax = 1 << max(log2ns)
            vb = [torch.empty(nmax, dtype=tdt, device="cuda") for _ in range(6)]
            for k, t in enumerate(vb):
                salt.salt_fill_uniform(t, 700 + k)
            red = torch.zeros(1, dtype=torch.float64, device="cuda")
            for lg in log2ns:
                n = 1 << lg
                v = [t[:n] for t in vb]
                row = {}
                for label, mode in (("interpreter", salt.JIT_OFF), ("jit", salt.JIT_ON)):
                    salt.salt_set_jit(mode)
                    st0 = salt.salt_jit_stats()
                    t0 = time.perf_counter()
                    salt.salt_eval(prog, v, [2.5], red_out=red)  # first call: compile (JIT)
                    torch.cuda.synchronize()
                    first_ms = (time.perf_counter() - t0) * 1e3
                    st1 = salt.salt_jit_stats()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(reps):
                        salt.salt_eval(prog, v, [2.5], red_out=red)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / reps
                    gbs = 6 * es * n / (ms * 1e-3) / 1e9
                    row[label] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac_measured": round(gbs / hbm_peak, 3),
                                  "first_call_ms": round(first_ms, 1),
                                  "compiled": st1["kernels"] - st0["kernels"],
                                  "from_disk": st1["disk_hits"] - st0["disk_hits"]}
                row["jit_speedup"] = round(row["interpreter"]["ms"] / row["jit"]["ms"], 2)
                out[f"{dt}_2^{lg}"] = row
            del vb
            torch.cuda.empty_cache()
    finally:
        salt.salt_set_jit(prev)
    return {"program": "f = (a - b) o (c + d) - 2.5 e; sum f^2 (6 operands, no compiled shape)", "rows": out}


def fp64_probe(torch, salt, log2n: int = 26, reps: int = 5) -> dict:
    """FP64 instruction rate through the library's own fused kernel: a
    program of 14 FP64 nodes per element (t <- t o x + x, seven times from
    t = x: 7 multiplies and 7 adds), compiled at run time, on n = 2^26
    elements -- 16 bytes per element against 14 FP64 instructions, so the
    FP64 pipe, not HBM, bounds it.  The measured denominator beside the
    derived one."""
    n = 1 << log2n
    prog = [("VEC", 0)]
    for _ in range(7):
        prog += [("VEC", 0), ("MUL", 0), ("VEC", 0), ("ADD", 0)]
    prog += [("STORE", 1)]
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    salt.salt_fill_uniform(x, key=977)
    prev = salt.salt_jit_stats()["mode"]
    try:
        salt.salt_set_jit(salt.JIT_ON)
        for _ in range(3):
            salt.salt_eval(prog, [x, y])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            salt.salt_eval(prog, [x, y])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
    except salt.SaltError as e:
        return {"gops": None, "error": e.message[:200]}
    finally:
        salt.salt_set_jit(prev)
    return {"gops": round(14 * n / (ms * 1e-3) / 1e9, 1), "ms": round(ms, 4), "n": n,
            "program": "14 FP64 nodes per element (7 x (t*x + x)), 16 B per element, run-time compiled"}


def batched_measure(torch, salt, reps: int = 20, nitems: int = 4096, fixed: bool = False,
                    collect: list | None = None) -> dict:
    """4096 CG-style updates (r <- r - alpha q; rho = r.r; p <- r + beta p),
    lengths log-uniform in [64, 2^20], in one persistent graph-replayed launch
    (autotuned) versus 4096 plain per-call launches on one stream.  With
    `collect`, a sample of items (their operands before one more launch and
    the rho it returns) is appended for the CPU leg to judge."""
    import numpy as np

    from paper_1109_1264_gb300 import inputs
    from paper_1109_1264_gb300.programs import PROG_CG
    lens = inputs.loguniform_lengths(0, nitems, 64, 1 << 20)
    ab = inputs.cg_scalars(0, nitems)
    out = {}
    stream = torch.cuda.current_stream()
    for dt, tdt, es in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
        align = 32 // es  # items start on 32-byte boundaries (256-bit accesses)
        offs, o = [], 0
        for n in lens:
            offs.append(o)
            o += -(-int(n) // align) * align
        bufs = [torch.empty(o, dtype=tdt, device="cuda") for _ in range(3)]
        for k, buf in enumerate(bufs):
            salt.salt_fill_uniform(buf, inputs.vector_key(0, 0, k))
        b = salt.Batch(nitems)
        slots = []
        for i in range(nitems):
            n = int(lens[i])
            slots.append(b.add(PROG_CG, [buf[offs[i]:offs[i] + n] for buf in bufs], list(ab[i])))
        red = torch.zeros(nitems, dtype=torch.float64, device="cuda")
        nbytes = b.info()["bytes"]
        if fixed:  # the shape the autotuner picks on GB300 (for profiling runs)
            b.set_config(4, 128, 0, 32768 if dt == "f32" else 131072)
            best_ms = float("nan")
        else:
            best_ms = b.autotune(red, reps=3)
        cfg = b.get_config()

        def timed(fn, k):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / k

        ms_b = timed(lambda: b.launch(red), reps)
        ms_p = timed(lambda: b.launch_plain(red), max(3, reps // 4))
        if collect is not None:
            # the 4 longest items and 12 more spread over the table
            pick = sorted(set(np.argsort(lens)[-4:].tolist()) | set(range(0, nitems, nitems // 12)))
            before = {i: [buf[offs[i]:offs[i] + int(lens[i])].cpu().numpy() for buf in bufs] for i in pick}
            b.launch(red)
            redh = red.cpu().numpy()
            for i in pick:
                collect.append({"dt": dt, "item": i, "ab": list(ab[i]), "operands": before[i],
                                "got": float(redh[slots[i]])})
        out[dt] = {"batched_gbs": round(nbytes / (ms_b * 1e-3) / 1e9, 1),
                   "plain_gbs": round(nbytes / (ms_p * 1e-3) / 1e9, 1),
                   "ratio": round(ms_p / ms_b, 2), "batched_ms": round(ms_b, 4), "plain_ms": round(ms_p, 4),
                   "bytes_per_launch": nbytes, "autotune_best_ms": round(best_ms, 4), "config": cfg}
        b.close()
        del bufs
        torch.cuda.empty_cache()
    out["workload"] = ("%d CG updates per launch, n log-uniform in [64, 2^20] (sum %d), one graph-replayed "
                       "persistent launch vs %d plain salt_eval calls" % (nitems, int(lens.sum()), nitems))
    return out


def sweep_measure(torch, salt, reps: int = 21, max_log2: int = 28) -> dict:
    """The BLAS-1 size sweep: every n = 2^k and 2^k + 7, k = 10 .. 28, FP32
    and FP64, for y = a x + y (axpy), dot, nrm2 and the fused e = a a + b b -
    c o d -- and the paper's own benchmark set (Section 5): xSCAL (x = a x)
    and the out-of-place scaling y = a x that BLAS must express as xCOPY +
    xSCAL, fused (one pass, 2 x es bytes per element) against the two calls
    (4 x es).  Launch shapes autotuned per size bucket (untimed setup); L2
    flushed (a 256 MiB read, leaving clean lines) before every timed call;
    median of reps.  Per cell: GB/s of algorithmic bytes, its fraction of
    the measured copy rate and of the nominal 8 TB/s, for FP64 the FP64-pipe
    fraction (instructions per element x n / time against 2 / clock / SM x
    152 SMs at the maximum clock), and whether it meets the 85%-of-HBM gate
    (n >= 2^24).  torch's own kernels (torch.dot = cuBLAS dot, add_,
    copy_ + mul_) are timed the same way as context."""
    import numpy as np

    from paper_1109_1264_gb300.programs import PROG_DOT, PROG_E, PROG_SCALE
    scal = [("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 0)]
    axpy = [("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1), ("ADD", 0), ("STORE", 1)]
    copy = [("VEC", 0), ("STORE", 1)]
    hbm_peak, _, sm_max = load_peaks()
    alu_peak = f64_alu_peak_gops(sm_max)
    # FP64 instructions per element (one per node; the reductions' FMA; e as
    # in the step, with beta a power of two; axpy's alpha = 1e-3 is not one)
    f64_instr = {"axpy": 2 - is_pow2(1e-3), "dot": 1, "nrm2": 1, "e": F64_INSTR["e"], "scal": 1,
                 "copy_scal_fused": 1}
    # L2 flush: READ a 256 MiB buffer before each timed call, so that L2 holds
    # clean lines of another buffer (a write-based flush would leave up to
    # the whole L2 dirty, and the timed kernel would pay its write-back).
    flush = torch.zeros(64 << 20, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sizes = sorted({1 << k for k in range(10, max_log2 + 1)} | {(1 << k) + 7 for k in range(10, max_log2 + 1)})
    out = {}

    def timed(fn):
        ts = []
        for _ in range(reps):
            flush.sum()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for dt, tdt, es in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
        rows = []
        nmax = (1 << max_log2) + 7
        a, b, c, d, x, y = (torch.empty(nmax, dtype=tdt, device="cuda") for _ in range(6))
        for k, t in enumerate((a, b, c, d, x, y)):
            salt.salt_fill_uniform(t, 11 + k)
        red = torch.zeros(1, dtype=torch.float64, device="cuda")
        salt.salt_tune_clear()
        for n in sizes:
            if n > nmax:
                continue
            va, vb, vc, vd, vx, vy = (t[:n] for t in (a, b, c, d, x, y))
            r = {"n": n}
            if n & (n - 1) == 0:
                # the library's autotuner, once per size bucket (untimed setup);
                # for operands that fit in L2 it flushes L2 before each timed
                # call, like the calls timed here
                salt.salt_autotune(salt.KERNEL_PROGRAM, axpy, [vx, vy], [1e-3], reps=5)
                salt.salt_autotune(salt.KERNEL_PROGRAM, PROG_DOT, [vx, vy], red_out=red, reps=5)
                salt.salt_autotune(salt.KERNEL_NRM2, None, [vx], red_out=red, reps=5)
                salt.salt_autotune(salt.KERNEL_PROGRAM, PROG_E, [va, vb, vc, vd, vy], [ALPHA, BETA], reps=5)
                salt.salt_autotune(salt.KERNEL_PROGRAM, scal, [vx], [1.0], reps=5)
                salt.salt_autotune(salt.KERNEL_PROGRAM, PROG_SCALE, [vx, vy], [1.0], reps=5)
                salt.salt_autotune(salt.KERNEL_PROGRAM, copy, [vx, vy], reps=5)
            cells = {
                "axpy": (3, lambda: salt.salt_eval(axpy, [vx, vy], [1e-3])),
                "dot": (2, lambda: salt.salt_eval(PROG_DOT, [vx, vy], red_out=red)),
                "nrm2": (1, lambda: salt.salt_nrm2(vx, red)),
                "e": (5, lambda: salt.salt_eval(PROG_E, [va, vb, vc, vd, vy], [ALPHA, BETA])),
                "scal": (2, lambda: salt.salt_eval(scal, [vx], [0.999])),
                "copy_scal_fused": (2, lambda: salt.salt_eval(PROG_SCALE, [vx, vy], [1.5])),
                # GB/s of the operation itself (2 x es bytes per element), two calls
                "copy_scal_two_calls": (2, lambda: (salt.salt_eval(copy, [vx, vy]),
                                                    salt.salt_eval(scal, [vy], [1.5]))),
            }
            for op, (units, fn) in cells.items():
                ms = timed(fn)
                gbs = units * es * n / (ms * 1e-3) / 1e9
                cell = {"gbs": round(gbs, 1), "frac_measured": round(gbs / hbm_peak, 3),
                        "frac_nominal": round(gbs / NOMINAL_HBM_GBS, 3)}
                if dt == "f64" and op in f64_instr:
                    cell["frac_fp64_pipe"] = round(f64_instr[op] * n / (ms * 1e-3) / 1e9 / alu_peak, 3)
                if n >= (1 << 24) and op != "copy_scal_two_calls":
                    cell["gate_85"] = bool(gbs >= 0.85 * NOMINAL_HBM_GBS)
                r[op] = cell
            r["torch_dot_gbs"] = round(2 * es * n / (timed(lambda: torch.dot(vx, vy)) * 1e-3) / 1e9, 1)
            r["torch_axpy_gbs"] = round(3 * es * n / (timed(lambda: vy.add_(vx, alpha=1e-3)) * 1e-3) / 1e9, 1)
            r["torch_copy_scal_gbs"] = round(2 * es * n / (timed(lambda: vy.copy_(vx).mul_(1.5)) * 1e-3) / 1e9, 1)
            rows.append(r)
        out[dt] = rows
        salt.salt_tune_clear()
        del a, b, c, d, x, y
        torch.cuda.empty_cache()
    return {"sweep": out, "hbm_peak_measured_gbs": hbm_peak, "nominal_gbs": NOMINAL_HBM_GBS,
            "fp64_peak_derived_gops": round(alu_peak, 1),
            "note": "GB/s of algorithmic bytes; launch shapes autotuned per size bucket; L2 flushed before each "
                    "timed call; median of %d; CUDA events on this GPU advance in 2.048 us steps" % reps}


def reduction_trace_measure(torch, salt, log2ns=(4, 12, 16, 20, 22, 24, 26), reps: int = 7) -> dict:
    """Where a reduction's time goes: dot and nrm2, FP32 and FP64, autotuned
    as in the sweep, each call timed with CUDA events after an L2 flush while
    every block records its timeline (salt_trace_set).  Per call (the median
    by event time of `reps`):
      event_us        CUDA-event time of the call
      span_us         first block start to last block end (global timer)
      outside_us      event_us - span_us: launch latency outside the blocks
      start_spread_us last block start - first block start (dispatch ramp)
      tiles_us        median over blocks of (whole tiles done - block start)
      tail_us         last block's deposit - median block's deposit
      combine_us      end of the final combine - last deposit
      hbm_us          algorithmic bytes / the measured copy rate"""
    import numpy as np

    from paper_1109_1264_gb300.programs import PROG_DOT
    hbm_peak, _, _ = load_peaks()
    flush = torch.zeros(64 << 20, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    cap = 152 * 32
    trace = torch.zeros(cap * salt.TRACE_WORDS, dtype=torch.int64, device="cuda")
    out = {}
    for dt, tdt, es in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
        nmax = 1 << max(log2ns)
        xb = torch.empty(nmax, dtype=tdt, device="cuda")
        yb = torch.empty(nmax, dtype=tdt, device="cuda")
        salt.salt_fill_uniform(xb, 11)
        salt.salt_fill_uniform(yb, 12)
        red = torch.zeros(1, dtype=torch.float64, device="cuda")
        for lg in log2ns:
            n = 1 << lg
            x, y = xb[:n], yb[:n]
            salt.salt_tune_clear()
            cfg_dot, _ = salt.salt_autotune(salt.KERNEL_PROGRAM, PROG_DOT, [x, y], red_out=red, reps=5)
            cfg_nrm, _ = salt.salt_autotune(salt.KERNEL_NRM2, None, [x], red_out=red, reps=5)
            for op, fn, nbytes, cfg in (("dot", lambda: salt.salt_dot(x, y, red), 2 * es * n, cfg_dot),
                                        ("nrm2", lambda: salt.salt_nrm2(x, red), es * n, cfg_nrm)):
                runs = []
                salt.salt_trace_set(trace, cap)
                try:
                    for _ in range(reps):
                        trace.zero_()
                        flush.sum()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        fn()
                        e1.record(stream)
                        torch.cuda.synchronize()
                        w = trace.view(-1, salt.TRACE_WORDS).cpu().numpy()
                        w = w[w[:, 0] != 0]
                        runs.append((e0.elapsed_time(e1) * 1e3, w))
                finally:
                    salt.salt_trace_set(None)
                runs.sort(key=lambda r: r[0])
                ev_us, w = runs[len(runs) // 2]
                start, tiles, pre, end = (w[:, k].astype(np.float64) for k in range(4))
                last = w[:, 5] == 1
                t0 = start.min()
                row = {"blocks": int(w.shape[0]), "config": cfg,
                       "event_us": round(ev_us, 2), "span_us": round((end.max() - t0) / 1e3, 2),
                       "outside_us": round(ev_us - (end.max() - t0) / 1e3, 2),
                       "start_spread_us": round((start.max() - t0) / 1e3, 2),
                       "tiles_us": round(float(np.median(tiles - start)) / 1e3, 2),
                       "tail_us": round((pre.max() - np.median(pre)) / 1e3, 2),
                       "combine_us": round(((end[last].max() if last.any() else end.max()) - pre.max()) / 1e3, 2),
                       "hbm_us": round(nbytes / (hbm_peak * 1e9) * 1e6, 2),
                       "gbs": round(nbytes / (ev_us * 1e-6) / 1e9, 1)}
                out[f"{op}_{dt}_2^{lg}"] = row
        salt.salt_tune_clear()
        del xb, yb
    return {"reduction_trace": out, "note": "median call of %d by CUDA-event time, L2 flushed before each; "
                                            "global-timer stamps per block (salt_trace_set)" % reps}


def schedules_measure(torch, salt, log2ns=(24, 28), reps: int = 15) -> dict:
    """Register-tiled loop versus staged loop (operand tiles copied into shared
    memory by bulk asynchronous copies) for the compiled shapes, through the
    library's own calls: each configuration pinned with salt_tune_set, timed
    as the median of `reps` calls (L2 flushed by a 256 MiB read before each),
    the best of each schedule reported with its configuration."""
    import numpy as np

    from paper_1109_1264_gb300.programs import PROG_AXPBY, PROG_CG, PROG_D, PROG_DOT, PROG_E, PROG_SUMSQ
    axpy = [("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("VEC", 1), ("ADD", 0), ("STORE", 1)]
    scal = [("SCAL", 0), ("VEC", 0), ("SMUL", 0), ("STORE", 0)]
    copy = [("VEC", 0), ("STORE", 1)]
    cgxr = [("VEC", 0), ("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 0), ("VEC", 2), ("SCAL", 0),
            ("VEC", 3), ("SMUL", 0), ("SUB", 0), ("STORE", 2), ("VEC", 2), ("SUMSQ", 0)]
    # name: (program, operands, scalars (bounded under repetition), bytes per element / element size)
    shapes = {"e": (PROG_E, 5, [1.5, -0.25], 5), "axpby": (PROG_AXPBY, 2, [1.5, -0.25], 3),
              "axpy": (axpy, 2, [1e-3], 3), "d": (PROG_D, 4, [], 4), "scal": (scal, 1, [0.999], 2),
              "copy": (copy, 2, [], 2), "dot": (PROG_DOT, 2, [], 2), "sumsq": (PROG_SUMSQ, 1, [], 1),
              "cg": (PROG_CG, 3, [1e-3, 0.5], 5), "cgxr": (cgxr, 4, [1e-3], 6)}
    register = [(1, 32, 256, 0, 0), (2, 32, 256, 0, 0), (2, 32, 128, 0, 0), (4, 32, 128, 0, 0),
                (4, 16, 256, 0, 0), (2, 32, 256, 4, 0)]
    staged = [(1, 16, 128, 0, 4096), (1, 16, 128, 0, 8192), (1, 16, 128, 0, 16384), (1, 16, 256, 0, 8192),
              (1, 16, 256, 0, 16384)]
    flush = torch.zeros(64 << 20, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    red = torch.zeros(1, dtype=torch.float64, device="cuda")

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.sum()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    out = {}
    for lg in log2ns:
        n = 1 << lg
        rows = {}
        for dt, tdt, es, code in (("f32", torch.float32, 4, salt.F32), ("f64", torch.float64, 8, salt.F64)):
            bufs = [torch.empty(n, dtype=tdt, device="cuda") for _ in range(5)]
            for k, t in enumerate(bufs):
                salt.salt_fill_uniform(t, 40 + k)
            for name, (prog, nv, sc, bpe) in shapes.items():
                vecs = bufs[:nv]
                nred = sum(1 for o, _ in prog if o in ("DOT", "SUMSQ"))
                best = {}
                for kind, cands in (("register", register), ("staged", staged)):
                    top = None
                    for cfg in cands:
                        salt.salt_tune_set(prog, code, n, *cfg)
                        ms = timed(lambda: salt.salt_eval(prog, vecs, sc, red_out=red if nred else None))
                        gbs = bpe * es * n / (ms * 1e-3) / 1e9
                        if top is None or gbs > top["gbs"]:
                            top = {"gbs": round(gbs, 1), "ms": round(ms, 4),
                                   "cfg": dict(zip(("unroll", "vec_bytes", "block", "blocks_per_sm",
                                                    "stage_bytes"), cfg))}
                    best[kind] = top
                best["staged_over_register"] = round(best["staged"]["gbs"] / best["register"]["gbs"], 3)
                rows[f"{name}_{dt}"] = best
            salt.salt_tune_clear()
            del bufs
        out[f"2^{lg}"] = rows
    return {"schedules": out, "note": "GB/s of algorithmic bytes, best configuration of each schedule, "
                                      "L2 flushed before each timed call, median of %d" % reps}


def cg_measure(torch, salt, log2n: int = 28, iters: int = 16, reps: int = 3) -> dict:
    """Conjugate gradients for diag(d) x = b with every scalar on the device
    (alpha = rho / p.q and beta = rho' / rho as DSCAL quotients), d in [1, 8):
    salt_cg_diag (two fused passes per iteration: 11 vector passes) against
    the same iteration as six single-operation calls of this library (run-time
    compiled where no compiled shape exists: 15 vector passes, 6 launches).
    Operands (>= 1 GiB each) exceed L2.  GB/s counts the fused schedule's
    algorithmic bytes for both, so the ratio is the speed-up."""
    import numpy as np

    n = 1 << log2n
    stream = torch.cuda.current_stream()
    out = {}
    for dt, tdt, es in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
        d, b, x, r, p, q = (torch.empty(n, dtype=tdt, device="cuda") for _ in range(6))
        salt.salt_fill_uniform(d, 21)
        d.add_(1.0).mul_(3.5).add_(1.0)
        salt.salt_fill_uniform(b, 22)
        rho = torch.zeros(2 * iters + 1, dtype=torch.float64, device="cuda")
        rho_u = torch.zeros(2 * iters + 1, dtype=torch.float64, device="cuda")
        vecs = [d, p, q, x, r, b]
        # The autotuner on the two passes' shapes (by-value scalars: the same
        # compiled shapes and launch-shape table entries as the device-scalar
        # form); setup, untimed.
        p.copy_(b)
        r.copy_(b)
        tune = torch.zeros(2, dtype=torch.float64, device="cuda")
        cgpq = [("VEC", 4), ("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 1), ("VEC", 0), ("VEC", 1),
                ("MUL", 0), ("STORE", 2), ("VEC", 1), ("VEC", 2), ("DOT", 0)]
        cgxr = [("VEC", 3), ("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 3), ("VEC", 4), ("SCAL", 0),
                ("VEC", 2), ("SMUL", 0), ("SUB", 0), ("STORE", 4), ("VEC", 4), ("SUMSQ", 0)]
        tuned = {"pq": salt.salt_autotune(salt.KERNEL_PROGRAM, cgpq, vecs, [0.0], red_out=tune[0:1], reps=2)[0],
                 "xr": salt.salt_autotune(salt.KERNEL_PROGRAM, cgxr, vecs, [0.0], red_out=tune[1:2], reps=2)[0]}
        # ... and on the compiled shapes the six-call form uses (AXPBY, DOT,
        # AXPY, SUMSQ, COPY), so that both schedules run tuned launch shapes
        for prog, sc, red in (([("SCAL", 0), ("VEC", 4), ("SMUL", 0), ("SCAL", 1), ("VEC", 1), ("SMUL", 0),
                                ("ADD", 0), ("STORE", 1)], [1.0, 0.0], None),
                               ([("VEC", 1), ("VEC", 2), ("DOT", 0)], [], tune[0:1]),
                               ([("SCAL", 0), ("VEC", 1), ("SMUL", 0), ("VEC", 3), ("ADD", 0), ("STORE", 3)], [0.0],
                                None),
                               ([("VEC", 4), ("SUMSQ", 0)], [], tune[1:2]),
                               ([("VEC", 4), ("STORE", 1)], [], None)):
            salt.salt_autotune(salt.KERNEL_PROGRAM, prog, vecs, sc, red_out=red, reps=2)
        r0 = [("VEC", 5), ("VEC", 0), ("VEC", 3), ("MUL", 0), ("SUB", 0), ("STORE", 4), ("VEC", 4), ("SUMSQ", 0)]
        quot = [("DSCAL", 0), ("DSCAL", 1), ("DIV", 0)]
        p_upd = [("SCAL", 0), ("VEC", 4), ("SMUL", 0)] + quot + [("VEC", 1), ("SMUL", 0), ("ADD", 0), ("STORE", 1)]
        q_mul = [("VEC", 0), ("VEC", 1), ("MUL", 0), ("STORE", 2)]
        pq_dot = [("VEC", 1), ("VEC", 2), ("DOT", 0)]
        x_upd = quot + [("VEC", 1), ("SMUL", 0), ("VEC", 3), ("ADD", 0), ("STORE", 3)]
        r_upd = quot + [("NEG", 0), ("VEC", 2), ("SMUL", 0), ("VEC", 4), ("ADD", 0), ("STORE", 4)]
        rr = [("VEC", 4), ("SUMSQ", 0)]

        def fused():
            salt.salt_cg_diag(d, b, x, r, p, q, iters, rho)

        def unfused():
            salt.salt_eval(r0, vecs, red_out=rho_u[0:1])
            for k in range(iters):
                pq = rho_u[2 * k + 1:2 * k + 2]
                if k == 0:
                    salt.salt_eval([("VEC", 4), ("STORE", 1)], vecs)
                else:
                    salt.salt_eval(p_upd, vecs, [1.0], dscalars=[rho_u[2 * k:2 * k + 1], rho_u[2 * k - 2:2 * k - 1]])
                salt.salt_eval(q_mul, vecs)
                salt.salt_eval(pq_dot, vecs, red_out=pq)
                ds = [rho_u[2 * k:2 * k + 1], pq]
                salt.salt_eval(x_upd, vecs, dscalars=ds)
                salt.salt_eval(r_upd, vecs, dscalars=ds)
                salt.salt_eval(rr, vecs, red_out=rho_u[2 * k + 2:2 * k + 3])

        def timed(fn):
            ts = []
            for _ in range(reps + 1):
                x.zero_()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return float(np.median(ts[1:]))  # first run: warm-up (and JIT compilation)

        prev = salt.salt_jit_stats()["mode"]
        salt.salt_set_jit(salt.JIT_ON)
        try:
            ms_u = timed(unfused)
        finally:
            salt.salt_set_jit(prev)
        ms_f = timed(fused)
        passes = 4 + 4 + 6 + 11 * (iters - 1)
        abytes = passes * es * n
        h_f, h_u = rho.cpu().numpy(), rho_u.cpu().numpy()
        # the one-reduction recurrence in one cooperative launch: start (reads
        # b, d, x; writes r) + first pass (reads d, r, x; writes p, s, x, r)
        # + 9 vectors per later iteration
        rho_c = torch.zeros(2 * iters + 2, dtype=torch.float64, device="cuda")
        ms_c = timed(lambda: salt.salt_cg_diag(d, b, x, r, p, q, iters, rho_c, one_reduction=True))
        cbytes = (4 + 7 + 9 * (iters - 1)) * es * n
        x.zero_()
        form, _ = salt.salt_cg_autotune(d, b, x, r, p, q, iters, rho_c, reps=1)  # setup, untimed
        ms_a = timed(lambda: salt.salt_cg_diag_auto(d, b, x, r, p, q, iters, rho_c))
        out[dt] = {"n": n, "iters": iters, "ms_fused": round(ms_f, 3), "ms_unfused": round(ms_u, 3),
                   "ms_per_iter_fused": round(ms_f / iters, 4),
                   "gbs_fused": round(abytes / (ms_f * 1e-3) / 1e9, 1),
                   "gbs_unfused_same_bytes": round(abytes / (ms_u * 1e-3) / 1e9, 1),
                   "speedup": round(ms_u / ms_f, 3),
                   "launches_fused": 1 + 2 * iters, "launches_unfused": 1 + 6 * iters, "tuned": tuned,
                   "rel_residual": float(np.sqrt(h_f[-1] / h_f[0])),
                   "rho_rel_diff_fused_vs_unfused": float(abs(h_f[-1] - h_u[-1]) / h_f[-1]),
                   "one_reduction": {"ms": round(ms_c, 3), "gbs": round(cbytes / (ms_c * 1e-3) / 1e9, 1),
                                     "speedup_vs_fused": round(ms_f / ms_c, 3),
                                     "rel_residual": float(np.sqrt(rho_c[-2].item() / rho_c[0].item()))},
                   "auto": {"form": ("two_pass", "persistent", "one_reduction")[form], "ms": round(ms_a, 3),
                            "vs_best": round(min(ms_f, ms_c) / ms_a, 3)}}
        del d, b, x, r, p, q, vecs
        torch.cuda.empty_cache()
    return out


def _errors(got: float, exact_value: float, scale: float) -> dict:
    """Error of one reduction result: relative to its exact value (the
    measure the tolerances are stated in) and relative to sum|x_i y_i|."""
    err = abs(got - exact_value)
    return {"rel_value": float(err / abs(exact_value)) if exact_value else float(err),
            "rel_scale": float(err / scale) if scale else float(err)}


def counter_dot_exact(kx: int, ky: int, n: int, npdt, offset: int = 0, piece: int = 1 << 22, offset_y=None):
    """Exact sum x_i y_i and sum |x_i y_i| of counter-based vectors (keys kx,
    ky, elements from `offset` (`offset_y` for y); the same key and offset
    give the sum of squares), by the oracle's fixed-point exact dot on host
    threads."""
    oy = offset if offset_y is None else offset_y
    import concurrent.futures as cf

    from oracle import exact
    from paper_1109_1264_gb300 import inputs
    fb = 52 if npdt.__name__ == "float64" else 23

    def one(lo):
        m = min(piece, n - lo)
        x = inputs.hash_uniform(kx, m, npdt, offset=offset + lo)
        y = x if (ky, oy) == (kx, offset) else inputs.hash_uniform(ky, m, npdt, offset=oy + lo)
        f = exact.FixedPointDot(fb, fb)
        f.add(x, y)
        return f

    with cf.ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        parts = list(ex.map(one, range(0, n, piece)))
    f = exact.FixedPointDot.combine(parts)
    return f.value(), f.abs_value()


def step_precision(step_red: dict, n: int, seed: int = 0) -> dict:
    """The timed step's own reduction results (dot(a, b) and nrm2(c) of the
    counter-based inputs, FP32 and FP64, n = 2^28) against their exact
    values, and the same dot over the first 2^26 elements."""
    import math

    import numpy as np
    out = {}
    for dt, r in step_red.items():
        npdt = np.float32 if dt == "f32" else np.float64
        ka, kb, kc = seed * 16 + 1, seed * 16 + 2, seed * 16 + 3
        ref, scale = counter_dot_exact(ka, kb, n, npdt)
        sq, _ = counter_dot_exact(kc, kc, n, npdt)
        nref = math.sqrt(sq)  # within one rounding of the exact norm
        row = {"dot": _errors(r["dot"], ref, scale), "dot_cond": round(scale / abs(ref), 1),
               "nrm2": _errors(r["nrm2"], nref, nref)}
        if "dot_2e26" in r:
            ref26, scale26 = counter_dot_exact(ka, kb, 1 << 26, npdt)
            row["dot_n2e26"] = _errors(r["dot_2e26"], ref26, scale26)
        out[dt] = row
    return out


def batched_precision(samples: list) -> dict:
    """rho of the sampled batch items against the exact sum of squares of r
    after the update, which the oracle recomputes from the operands."""
    import oracle
    from oracle import exact
    from paper_1109_1264_gb300.programs import PROG_CG
    worst = {}
    for smp in samples:
        want = [v.copy() for v in smp["operands"]]
        oracle.eval_program(PROG_CG, want, smp["ab"])
        ref = exact.exact_sumsq(want[0])
        e = _errors(smp["got"], ref, ref)
        w = worst.setdefault(smp["dt"], {"items": 0, "max_rel_value": 0.0})
        w["items"] += 1
        w["max_rel_value"] = max(w["max_rel_value"], e["rel_value"])
    return worst


def served_precision(samples: list) -> dict:
    """Served dot and norm results against the exact values of the store
    slices the requests read."""
    import math

    import numpy as np
    worst = {}
    for smp in samples:
        npdt = np.float64 if smp["dt"] == "f64" else np.float32
        (kx, ox), (ky, oy) = smp["operands"][0], smp["operands"][-1]
        ref, scale = counter_dot_exact(kx, ky, smp["n"], npdt, offset=ox, offset_y=oy, piece=1 << 20)
        if smp["shape"] == "nrm2":
            ref = scale = math.sqrt(ref)
        e = _errors(smp["got"], ref, scale)
        w = worst.setdefault(f"{smp['shape']}_{smp['dt']}", {"requests": 0, "max_rel_value": 0.0,
                                                             "max_rel_scale": 0.0})
        w["requests"] += 1
        w["max_rel_value"] = max(w["max_rel_value"], e["rel_value"])
        w["max_rel_scale"] = max(w["max_rel_scale"], e["rel_scale"])
    return worst


def precision_measure(torch, salt, log2n: int = 26) -> dict:
    """The precision comparison of the dot product and norm: FP32 inputs of
    random sign and magnitudes 10^U(-3, 3), n = 2^26.  Errors of the
    compensated FP32 path (the default), the plain FP32 path (FP32
    accumulation and combination) and the FP64 path on the widened data,
    relative to the exactly rounded value and to sum|x_i y_i|, beside the CPU
    oracle's own sequential FP64 sum.  Part of the CPU-oracle leg (it uses
    the oracle's exact references)."""
    import numpy as np

    from oracle import exact
    import oracle as orc
    from paper_1109_1264_gb300 import inputs
    n = 1 << log2n
    x, y = inputs.logmag_vectors(0, n, 2, np.float32)
    ref, scale, nref = exact.exact_dot(x, y), exact.abs_dot(x, y), exact.exact_nrm2(x)
    tx, ty = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    salt.salt_dot(tx, ty, out[0:1])
    salt.salt_dot(tx, ty, out[1:2], plain=True)
    salt.salt_dot(tx.double(), ty.double(), out[2:3])
    salt.salt_nrm2(tx, out[3:4])
    salt.salt_nrm2(tx, out[4:5], plain=True)
    salt.salt_nrm2(tx.double(), out[5:6])
    comp, plain, wide, nc, npl, nw = out.cpu().tolist()
    odot, onrm = orc.dot(x, y), orc.nrm2(x)
    return {"n": n, "data": "FP32, random sign x 10^U(-3,3), numpy default_rng(0)",
            "dot_cond": round(scale / abs(ref), 1),
            "dot": {"compensated_f32": _errors(comp, ref, scale), "plain_f32": _errors(plain, ref, scale),
                    "f64_widened": _errors(wide, ref, scale), "cpu_oracle_sequential_f64": _errors(odot, ref, scale)},
            "nrm2": {"compensated_f32": _errors(nc, nref, nref), "plain_f32": _errors(npl, nref, nref),
                     "f64_widened": _errors(nw, nref, nref), "cpu_oracle": _errors(onrm, nref, nref)}}


def config1_measure(torch, salt, reps: int = 100) -> dict:
    """Figure 1's d = a + (b - c), FP64, n = 2^20 (a, b, c from
    default_rng(0).uniform(-1, 1) in order): one plain launch timed with CUDA
    events, median of `reps`, with the 32 MiB working set warm in L2 and with
    L2 flushed (a 256 MiB read) before each launch."""
    import numpy as np

    from paper_1109_1264_gb300 import inputs
    from paper_1109_1264_gb300.programs import PROG_D
    n = 1 << 20
    a, b, c = (torch.from_numpy(v).cuda() for v in inputs.uniform_vectors(0, n, 3, np.float64))
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    flush = torch.zeros(64 << 20, dtype=torch.float32, device="cuda")  # read to flush L2 (clean lines)
    stream = torch.cuda.current_stream()

    def timed(flush_l2):
        ts = []
        for _ in range(reps + 3):
            if flush_l2:
                flush.sum()
            # keep the GPU busy while the host issues the launch, so that the
            # events time the kernel, not the host's launch latency
            torch.cuda._sleep(100_000)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            salt.salt_eval(PROG_D, [a, b, c, d])
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts[3:]))

    warm, cold = timed(False), timed(True)
    nbytes = 32 * n
    return {"n": n, "dtype": "f64", "bytes": nbytes, "reps": reps,
            "l2_warm_us": round(warm * 1e3, 2), "l2_warm_gbs": round(nbytes / (warm * 1e-3) / 1e9, 1),
            "l2_flushed_us": round(cold * 1e3, 2), "l2_flushed_gbs": round(nbytes / (cold * 1e-3) / 1e9, 1),
            "note": "32 MiB fits in the 129 MB L2: the warm figure is not an HBM rate"}


def cg_latency_measure(torch, salt, sizes=(1 << 14, 1 << 17, 1 << 20, 1 << 24), iters: int = 100,
                       reps: int = 3) -> dict:
    """Microseconds per CG iteration, launch-per-pass (salt_cg_diag: two fused
    launches per iteration) against one cooperative launch with grid
    barriers (salt_cg_diag_persistent: two barriers per iteration; and
    salt_cg_diag_one_reduction: one pass and one barrier per iteration), for
    sizes where launches matter."""
    import numpy as np

    stream = torch.cuda.current_stream()
    out = {}
    for dt, tdt in (("f32", torch.float32), ("f64", torch.float64)):
        rows = []
        for n in sizes:
            d, b, x, r, p, q = (torch.empty(n, dtype=tdt, device="cuda") for _ in range(6))
            salt.salt_fill_uniform(d, 31)
            d.add_(1.0).mul_(3.5).add_(1.0)
            salt.salt_fill_uniform(b, 32)
            rho = torch.zeros(2 * iters + 2, dtype=torch.float64, device="cuda")
            row = {"n": n}
            x.zero_()
            form, _ = salt.salt_cg_autotune(d, b, x, r, p, q, iters, rho, reps=2)  # setup, untimed
            row["auto_form"] = ("two_pass", "persistent", "one_reduction")[form]
            for label, fn in (("launch_per_pass_us", lambda: salt.salt_cg_diag(d, b, x, r, p, q, iters, rho)),
                              ("persistent_us", lambda: salt.salt_cg_diag(d, b, x, r, p, q, iters, rho,
                                                                          persistent=True)),
                              ("one_reduction_us", lambda: salt.salt_cg_diag(d, b, x, r, p, q, iters, rho,
                                                                             one_reduction=True)),
                              ("auto_us", lambda: salt.salt_cg_diag_auto(d, b, x, r, p, q, iters, rho))):
                ts = []
                for _ in range(reps + 1):
                    x.zero_()
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                row[label] = round(float(np.median(ts[1:])) * 1e3 / iters, 2)
            row["speedup"] = round(row["launch_per_pass_us"] / row["persistent_us"], 2)
            row["speedup_one_reduction"] = round(row["launch_per_pass_us"] / row["one_reduction_us"], 2)
            row["auto_vs_best"] = round(min(row["launch_per_pass_us"], row["persistent_us"],
                                            row["one_reduction_us"]) / row["auto_us"], 3)
            rows.append(row)
            del d, b, x, r, p, q
        out[dt] = rows
    return {"iters": iters, "rows": out}


def store_place(seed: int, i: int, k: int, n: int, length: int, nstore: int, itemsize: int):
    """(store vector, first element) that operand k of replayed request i
    reads, by the placement rule salt_serve_replay_store documents."""
    m64 = (1 << 64) - 1
    key = (seed * 0x100000001B3 + i * 16 + k + 1) & m64
    h = ((key * 0x9E3779B97F4A7C15) & m64) >> 11
    o = h % (length - n + 1)
    return (i * 5 + k) % nstore, o - o % (32 // itemsize)


def served_measure(salt, count: int = 3000, seed: int = 0, collect: list | None = None) -> dict:
    """Poisson stream of requests over the 5 served shapes (d = a + (b - c),
    axpby, e, dot, nrm2), n log-uniform in [2^8, 2^24], 70% FP32 / 30% FP64.
    Inputs come from a resident store of counter-filled vectors (8 GiB: four
    FP32 and two FP64 vectors of 2^28 elements, each request reading slices
    at hashed offsets); outputs and axpby's read-and-written y live in the
    server's 8 GiB arena.  Saturation throughput first (all requests arrive
    at once), then arrival rates from 10% to 120% of it; then the same stream
    served one request per step, and with every input generated per request
    on the device (standing in for an upload) instead of the store."""
    import numpy as np
    import torch

    from paper_1109_1264_gb300 import inputs
    ops = np.array([4, 3, 5, 2, 1], dtype=np.int64)  # operands read + written per shape
    shapes, is64, lens = inputs.request_mix(seed, count)
    es = np.where(is64, 8, 4)
    total_bytes = int(np.sum(ops[shapes] * es * lens))
    slen = 1 << 28
    store = ([torch.empty(slen, dtype=torch.float32, device="cuda") for _ in range(4)],
             [torch.empty(slen, dtype=torch.float64, device="cuda") for _ in range(2)])
    for j, t in enumerate(store[0] + store[1]):
        salt.salt_fill_uniform(t, inputs.vector_key(seed + 1000, j, 0))
    torch.cuda.synchronize()
    zeros = np.zeros(count)
    d32 = is64.astype(np.int32)

    def saturation(srv, use_store):
        st = store if use_store else None
        srv.replay(zeros[:200], shapes[:200], d32[:200], lens[:200], seed + 99, store=st)  # warm-up
        s0 = srv.stats()["steps"]
        lat, _, wall = srv.replay(zeros, shapes, d32, lens, seed, store=st)
        return lat, wall, srv.stats()["steps"] - s0

    def load_points(srv, sat_rps):
        pts = []
        for k, frac in enumerate((0.1, 0.3, 0.5, 0.7, 0.9, 1.2)):
            rate = frac * sat_rps
            arr = inputs.poisson_arrivals(seed + 1 + k, count, rate) * 1e6
            lat, _, wall_k = srv.replay(arr, shapes, d32, lens, seed, store=store)
            pts.append({"load": frac, "rate_rps": round(rate, 1), "p50_us": round(float(np.percentile(lat, 50)), 1),
                        "p99_us": round(float(np.percentile(lat, 99)), 1),
                        "gbs": round(total_bytes / (wall_k * 1e-6) / 1e9, 1)})
        return pts

    def one_at_a_time(srv, reps=300):
        """One FP32 dot of n = 256 at a time, its operands read in place from
        the store: latency from submission to observed completion."""
        x, y = store[0][0][:256], store[0][1][:256]
        lat = []
        for i in range(reps + 20):
            rid = srv.submit([("VEC", 0), ("VEC", 1), ("DOT", 0)], salt.F32, 256, [0, 0], ptrs=[x, y])
            srv.wait(rid, 10_000_000)
            if i >= 20:
                lat.append(srv.poll(rid)[1])
            srv.release(rid)
        return {"n": 256, "requests": reps, "p50_us": round(float(np.percentile(lat, 50)), 1),
                "p99_us": round(float(np.percentile(lat, 99)), 1)}

    srv = salt.Server()
    try:
        _, wall, steps = saturation(srv, True)
        if collect is not None:
            # dot (shape 3) and norm (shape 4) results of one more saturated replay
            _, red, _ = srv.replay(zeros, shapes, d32, lens, seed, store=store)
            keys = [inputs.vector_key(seed + 1000, j, 0) for j in range(6)]
            for shp in (3, 4):
                for i in [int(i) for i in np.nonzero(shapes == shp)[0][:8]]:
                    f64 = bool(is64[i])
                    ops_ = []
                    for k in range(2 if shp == 3 else 1):
                        j, o = store_place(seed, i, k, int(lens[i]), slen, 2 if f64 else 4, 8 if f64 else 4)
                        ops_.append((keys[4 + j] if f64 else keys[j], int(o)))
                    collect.append({"dt": "f64" if f64 else "f32", "shape": "dot" if shp == 3 else "nrm2",
                                    "n": int(lens[i]), "operands": ops_, "got": float(red[i])})
        sat_rps = count / (wall * 1e-6)
        sat_gbs = total_bytes / (wall * 1e-6) / 1e9
        points = load_points(srv, sat_rps)
        single = one_at_a_time(srv)
        _, wall_f, steps_f = saturation(srv, False)
    finally:
        srv.stop()
    # persistent mode: the same stream, the load points at the default mode's rates
    srvp = salt.Server(persistent=1)
    try:
        _, wall_p, steps_p = saturation(srvp, True)
        points_p = load_points(srvp, sat_rps)
        single_p = one_at_a_time(srvp)
        launches_p = srvp.launches()[0]
    finally:
        srvp.stop()
    persistent = {"saturation_gbs": round(total_bytes / (wall_p * 1e-6) / 1e9, 1), "saturation_steps": steps_p,
                  "points": points_p, "one_at_a_time": single_p, "kernel_launches": launches_p,
                  "note": "one resident launch runs the steps posted to a ring in mapped host memory; load points "
                          "at the default mode's arrival rates"}
    srv1 = salt.Server(max_batch=1)
    try:
        _, wall1, _ = saturation(srv1, True)
    finally:
        srv1.stop()
    srv4 = salt.Server(streams=4)  # beyond the 2 steps in flight of the served configuration
    try:
        _, wall4, _ = saturation(srv4, True)
    finally:
        srv4.stop()
    del store
    torch.cuda.empty_cache()
    unbatched_gbs = total_bytes / (wall1 * 1e-6) / 1e9
    return {"saturation_rps": round(sat_rps, 1), "saturation_gbs": round(sat_gbs, 1), "saturation_steps": steps,
            "unbatched_saturation_gbs": round(unbatched_gbs, 1), "batched_vs_unbatched": round(sat_gbs / unbatched_gbs, 2),
            "fill_per_request_saturation_gbs": round(total_bytes / (wall_f * 1e-6) / 1e9, 1),
            "four_streams_saturation_gbs": round(total_bytes / (wall4 * 1e-6) / 1e9, 1),
            "fill_per_request_steps": steps_f,
            "requests_per_point": count, "bytes_per_point": total_bytes, "points": points,
            "one_at_a_time": single, "persistent": persistent,
            "workload": "5 shapes uniform, n log-uniform [2^8, 2^24], 70% FP32 / 30% FP64; inputs from an 8 GiB "
                        "resident store of counter-filled vectors (slices at hashed offsets), outputs in an 8 GiB "
                        "arena, 2 streams; latency from arrival to observed completion"}


def e2e_measure(torch, salt, loads, args, world, steps, abytes):
    """The same step through the public API with host buffers: per step, the
    inputs are copied from pinned host memory, the ops run, and the results
    (e's output, the updated y, dot and nrm2) are read back."""
    from paper_1109_1264_gb300.programs import PROG_E
    host = {}
    h2d = d2h = 0
    for dt, w in loads.items():
        hs = {k: torch.empty(w.n, dtype=w.a.dtype, pin_memory=True) for k in ("a", "b", "c", "d", "y", "out", "y_out")}
        for k in ("a", "b", "c", "d", "y"):
            hs[k].copy_(getattr(w, k))
        host[dt] = hs
        h2d += 5 * w.n * ES[dt]
        d2h += 2 * w.n * ES[dt] + 16
    stream = torch.cuda.current_stream()
    # The step is pipelined through the public API: each vector is split into
    # chunks; one stream uploads every chunk back to back (the host->device
    # engine never waits on a read-back), a second runs each chunk's ops as
    # soon as its upload has landed, a third reads the chunk's results back.
    # Consecutive steps overlap chunk by chunk: a chunk of the next step is
    # uploaded once this step has read that chunk's results back (its
    # compute, which reads the inputs, is then done too), so the upload
    # engine runs without a gap between steps.  The reduction outputs
    # alternate between two buffers (step parity), so a step's compute never
    # overwrites the sums the previous step still has to read back.
    nchunks = args.e2e_chunks
    up, comp, down = (torch.cuda.Stream() for _ in range(3))
    dred = [{dt: torch.zeros(2 * nchunks, dtype=torch.float64, device="cuda") for dt in loads} for _ in range(2)]
    hred = [{dt: torch.empty(2 * nchunks, dtype=torch.float64, pin_memory=True) for dt in loads} for _ in range(2)]
    d2h += len(loads) * (16 * nchunks - 16)
    work = []
    for dt, w in loads.items():
        n = w.n
        bounds = [n * k // nchunks for k in range(nchunks + 1)]
        bounds = [b - b % 4 for b in bounds[:-1]] + [n]
        for k in range(nchunks):
            work.append((dt, w, k, bounds[k], bounds[k + 1]))
    state = {"read": None, "parity": 0}

    def step(end_event=None):
        par = state["parity"]
        prev_read = state["read"]
        landed = []
        with torch.cuda.stream(up):
            for i, (dt, w, k, lo, hi) in enumerate(work):
                if prev_read is not None:
                    up.wait_event(prev_read[i])
                hs = host[dt]
                for key in ("a", "b", "c", "d", "y"):
                    getattr(w, key)[lo:hi].copy_(hs[key][lo:hi], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(up)
                landed.append(ev)
        done = []
        with torch.cuda.stream(comp):
            for (dt, w, k, lo, hi), ev in zip(work, landed):
                comp.wait_event(ev)
                dv = {key: getattr(w, key)[lo:hi] for key in ("a", "b", "c", "d", "y", "out")}
                red = dred[par][dt]
                salt.salt_eval(PROG_E, [dv["a"], dv["b"], dv["c"], dv["d"], dv["out"]], [ALPHA, BETA], stream=comp)
                salt.salt_axpby(ALPHA, dv["a"], BETA, dv["y"], stream=comp)
                salt.salt_dot(dv["a"], dv["b"], red[2 * k:2 * k + 1], stream=comp)
                salt.salt_nrm2(dv["c"], red[2 * k + 1:2 * k + 2], stream=comp)
                ev2 = torch.cuda.Event()
                ev2.record(comp)
                done.append(ev2)
        read = []
        with torch.cuda.stream(down):
            for (dt, w, k, lo, hi), ev in zip(work, done):
                down.wait_event(ev)
                hs = host[dt]
                hs["out"][lo:hi].copy_(w.out[lo:hi], non_blocking=True)
                hs["y_out"][lo:hi].copy_(w.y[lo:hi], non_blocking=True)
                ev3 = torch.cuda.Event()
                ev3.record(down)
                read.append(ev3)
            for dt in loads:
                hred[par][dt].copy_(dred[par][dt], non_blocking=True)
            if end_event is not None:
                end_event.record(down)
        state["read"] = read
        state["parity"] = 1 - par

    def combine():
        # dot = sum of chunk dots; nrm2 = sqrt(sum of chunk norms squared)
        out = {}
        last = 1 - state["parity"]
        for dt in loads:
            r = hred[last][dt].tolist()
            out[dt] = (sum(r[0::2]), sum(v * v for v in r[1::2]) ** 0.5)
        return out

    k = max(3, min(args.steps, 20))
    for s_ in (up, comp, down):
        s_.wait_stream(stream)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    # Step j ends when its last read-back has landed; with steps overlapping,
    # the interval between consecutive ends is the steady-state step time.
    # The host link is shared with the machine's other GPUs' jobs; the
    # median interval over up to 20 steps is reported (the mean beside it)
    # so that a transient contention does not decide it.
    start = torch.cuda.Event(enable_timing=True)
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    start.record(up)
    for j in range(k):
        step(ends[j])
    torch.cuda.synchronize()
    combine()
    marks = [start] + ends
    step_ms = sorted(marks[j].elapsed_time(marks[j + 1]) for j in range(k))
    ms_mean = start.elapsed_time(ends[-1]) / k
    ms = step_ms[k // 2] if k % 2 else 0.5 * (step_ms[k // 2 - 1] + step_ms[k // 2])
    ms *= k  # the k steps at the median rate
    step_bytes = sum(abytes[(dt, op)] for dt, op, _ in steps)
    # The host link on this machine, measured the same way: one pinned 256 MiB
    # buffer copied host -> device, device -> host, and both directions at
    # once (each direction timed on its own stream).
    lb = 1 << 28
    hb = torch.empty(lb, dtype=torch.uint8, pin_memory=True)
    db = torch.empty(lb, dtype=torch.uint8, device="cuda")
    hb2 = torch.empty(lb, dtype=torch.uint8, pin_memory=True)
    db2 = torch.empty(lb, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        db.copy_(hb, non_blocking=True)
    torch.cuda.synchronize()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(4):
        db.copy_(hb, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = 4 * lb / (c0.elapsed_time(c1) * 1e-3) / 1e9
    c0.record(stream)
    for _ in range(4):
        hb2.copy_(db2, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    d2h_gbs = 4 * lb / (c0.elapsed_time(c1) * 1e-3) / 1e9
    # both directions at once, each timed on its own stream
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    with torch.cuda.stream(side):
        s0.record(side)
        for _ in range(4):
            hb2.copy_(db2, non_blocking=True)
        s1.record(side)
    for _ in range(4):
        db.copy_(hb, non_blocking=True)
    c1.record(stream)
    stream.wait_stream(side)
    c2 = torch.cuda.Event(enable_timing=True)
    c2.record(stream)
    torch.cuda.synchronize()
    both_gbs = 8 * lb / (c0.elapsed_time(c2) * 1e-3) / 1e9
    h2d_conc = 4 * lb / (c0.elapsed_time(c1) * 1e-3) / 1e9
    d2h_conc = 4 * lb / (s0.elapsed_time(s1) * 1e-3) / 1e9
    del hb, db, hb2, db2
    # The step's transfers on this link: both directions at their concurrent
    # rates until one direction is done, then the other at its rate alone
    # (the rate of a direction timed while the other runs includes some time
    # alone at the end, so this bound is slightly optimistic).
    t_h, t_d = h2d / (h2d_conc * 1e9), d2h / (d2h_conc * 1e9)
    if t_d <= t_h:
        two_phase = t_d + (h2d - h2d_conc * 1e9 * t_d) / (h2d_gbs * 1e9)
    else:
        two_phase = t_h + (d2h - d2h_conc * 1e9 * t_h) / (d2h_gbs * 1e9)
    simple_ms = max(h2d / (h2d_gbs * 1e9), (h2d + d2h) / (both_gbs * 1e9)) * 1e3
    bound_ms = max(two_phase * 1e3, simple_ms)
    return {"value": round(world * step_bytes * k / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": k,
            "ms_per_step": round(ms / k, 3), "ms_per_step_mean": round(ms_mean, 3),
            "ms_per_step_min_max": [round(step_ms[0], 3), round(step_ms[-1], 3)],
            "link_h2d_gbs": round(h2d_gbs, 1), "link_d2h_gbs": round(d2h_gbs, 1),
            "link_both_directions_gbs": round(both_gbs, 1),
            "link_concurrent_h2d_d2h_gbs": [round(h2d_conc, 1), round(d2h_conc, 1)],
            "link_bound_ms_per_step": round(bound_ms, 2), "frac_of_link_bound": round(bound_ms / (ms / k), 3),
            "link_bound_simple_ms_per_step": round(simple_ms, 2),
            "pipeline": f"{nchunks} chunks per vector; upload, compute and read-back streams overlap, "
                        "consecutive steps overlap chunk by chunk"}


if __name__ == "__main__":
    main()
