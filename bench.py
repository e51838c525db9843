"""Benchmark of the GB300 float-float library.

Default workload (one "step"): the elementwise float-float operator set on
N = 2^28 values (2 GiB per float-float array, far larger than L2): Add12 and
Mul12 on packed binary32 pairs, then Add22, Mul22, Div22 and Sqrt22 on
float-float arrays -- 6 x 2^28 float-float operator applications (ff-ops) per
step, each one kernel launch of libff.so through its C ABI.

Prints ONE JSON line (rank 0) with the whole-job throughput in ff-op/s, the
roofline of the dominant kernel against the measured HBM copy bandwidth, the
end-to-end rate through host buffers, the oracle timed on the host cores, the
SM clocks seen during the timed region, and per-row measurements of the other
hot-path rows (reductions and their adjoint, GEMV and its adjoint, native
FP64/FP32 baselines on the same GPU).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--rows all|main]
  python bench.py --impl reference      # the CPU oracle, same metric
Multi-GPU (torchrun): every rank runs its own 2^28 batch (weak scaling);
timing is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("float-float ops/s & HBM GB/s vs GB300 peak; batched dot+grad vs plain at ≤2^-44 rel")
UNIT = "ff-op/s"
N_ELEM = 1 << 28
OPS = ["add12", "mul12", "add", "mul", "div", "sqrt"]
# algorithmic HBM bytes per value: packed (a, b) in + (s, e) out = 16;
# two float-float inputs + one output = 24; one input + one output = 16
BYTES_PER_VALUE = {"add12": 16, "mul12": 16, "add": 24, "mul": 24, "div": 24, "sqrt": 16}
WORKLOAD = "elementwise float-float operators on 2^28 values (Add12, Mul12 packed; Add22, Mul22, Div22, Sqrt22)"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured", "sm_max_mhz": d.get("sm_max_mhz")}
    return {"hbm_gbs": 6800.0, "source": "fallback", "sm_max_mhz": 2070.0}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.25)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed plumbing (timing only; no data-path collective)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, local):
    import torch
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return dist if ws > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float) -> float:
    """The slowest rank's time (timing only: the data path has no collective)."""
    if dist is None:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world_size: int, units_per_step: int, steps: int, elapsed_max: float) -> float:
    """Weak scaling: every rank processes its own units; the job's rate is all
    ranks' units over the slowest rank's time."""
    return world_size * units_per_step * steps / elapsed_max


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def make_step(ff, e, outs):
    """One step: the six operators, each one launch; returns per-op closures."""
    return {
        "add12": lambda: ff.add12(e.ab, out=outs[0]),
        "mul12": lambda: ff.mul12(e.ab, out=outs[1]),
        "add": lambda: ff.add(e.a, e.b, out=outs[2]),
        "mul": lambda: ff.mul(e.a, e.b, out=outs[3]),
        "div": lambda: ff.div(e.a, e.b, out=outs[4]),
        "sqrt": lambda: ff.sqrt(e.a_sqrt, out=outs[5]),
    }


def time_fn(torch, fn, reps: int, warm: int = 2) -> float:
    """Mean seconds per call, CUDA events on the current stream."""
    for _ in range(warm):
        fn()
    s = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(s)
    for _ in range(reps):
        fn()
    ev1.record(s)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3 / reps


def time_median(torch, fn, reps: int, warm: int = 2) -> float:
    """Median seconds per call over `reps` calls, each between its own pair
    of CUDA events on the current stream (for calls of a millisecond or more,
    where one call's events cost nothing next to it)."""
    for _ in range(warm):
        fn()
    s = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    for e0, e1 in evs:
        e0.record(s)
        fn()
        e1.record(s)
    torch.cuda.synchronize()
    ts = sorted(e0.elapsed_time(e1) / 1e3 for e0, e1 in evs)
    mid = len(ts) // 2
    return ts[mid] if len(ts) % 2 else 0.5 * (ts[mid - 1] + ts[mid])


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_ops(a, b, ab, asq, threads: int):
    """The six elementwise operators of the oracle over the given arrays, each
    split into `threads` contiguous chunks run on that many host threads (the
    oracle's C loops release the GIL; the oracle itself is unchanged)."""
    import concurrent.futures as cf
    import oracle
    oracle.lib()
    n = a.shape[0]
    cuts = [n * i // threads for i in range(threads + 1)]
    ch = [slice(cuts[i], cuts[i + 1]) for i in range(threads)]
    ops = [lambda s: oracle.add12(ab[s]), lambda s: oracle.mul12(ab[s]), lambda s: oracle.add22(a[s], b[s]),
           lambda s: oracle.mul22(a[s], b[s]), lambda s: oracle.div22(a[s], b[s]), lambda s: oracle.sqrt22(asq[s])]
    if threads == 1:
        return [lambda f=f: f(slice(0, n)) for f in ops], None
    pool = cf.ThreadPoolExecutor(max_workers=threads)
    return [lambda f=f: list(pool.map(f, ch)) for f in ops], pool


def _time_oracle(fns, min_seconds):
    t0 = time.perf_counter()
    reps = 0
    while True:
        for f in fns:
            f()
        reps += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    return reps, time.perf_counter() - t0


def cpu_baseline(e_gpu, min_seconds: float = 8.0):
    """The CPU oracle as it stands on the first 2^26 values of the same
    arrays, repeated until at least min_seconds: on one host core, then on all
    of them (contiguous chunks, one per core)."""
    n = 1 << 26
    a = e_gpu.a[:n].cpu().numpy()
    b = e_gpu.b[:n].cpu().numpy()
    ab = e_gpu.ab[:n].cpu().numpy()
    asq = e_gpu.a_sqrt[:n].cpu().numpy()
    fns1, _ = oracle_ops(a, b, ab, asq, 1)
    reps1, dt1 = _time_oracle(fns1, min_seconds)
    cores = host_cores()
    fnsT, pool = oracle_ops(a, b, ab, asq, cores)
    if pool is not None:
        for f in fnsT:
            f()
    repsT, dtT = _time_oracle(fnsT, min_seconds)
    if pool is not None:
        pool.shutdown()
    single = reps1 * 6 * n / dt1
    return {"value": repsT * 6 * n / dtT, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": single,
            "sample": f"first 2^26 values of the same arrays, all six operators: {repsT} pass(es) in {dtT:.1f} s "
                      f"on {cores} host threads (contiguous chunks); {reps1} pass(es) in {dt1:.1f} s on one"}


# sources that define the elementwise kernels (and their flags)
ELEMENTWISE_SOURCES = ("paper_cs_0603115_gb300/csrc/ff_core.cuh", "paper_cs_0603115_gb300/csrc/ff_stream.cuh",
                       "paper_cs_0603115_gb300/csrc/ff_elementwise.cu", "paper_cs_0603115_gb300/csrc/ff_host.cuh",
                       "paper_cs_0603115_gb300/build.py")


def kernel_fingerprint(files=ELEMENTWISE_SOURCES) -> str:
    """Hash of the kernels' sources with comments and blank space removed, so
    that only a change of code makes a stored profile stale."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        text = open(os.path.join(ROOT, f)).read()
        if f.endswith(".py"):
            text = re.sub(r'"""(.|\n)*?"""', "", text)
            text = re.sub(r"#[^\n]*", "", text)
        else:
            text = re.sub(r"/\*(.|\n)*?\*/", "", text)
            text = re.sub(r"//[^\n]*", "", text)
        h.update(f.encode())
        h.update(re.sub(r"\s+", " ", text).strip().encode())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, n: int):
    """DRAM bytes per launch for `kernel` on n values, from the committed ncu
    summary (profiles/traffic.json), scaled from the captured size in
    proportion to the values processed; None when the kernel's sources
    changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get("kernels", {}).get(kernel)
    if not ent or d.get("fingerprint") != kernel_fingerprint():
        return None
    return ent["dram_bytes_per_launch"] * n / d["n_captured"]


def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(ws, local)
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import build as ffbuild
    from paper_cs_0603115_gb300 import inputs
    if rank == 0:
        ffbuild.build()     # one rank builds; the others wait and load it
    barrier(dist)
    lib = ff.load()
    build_id = lib.ff_build_id().decode()
    peaks = load_peaks()
    dev = torch.device("cuda", local)

    n = N_ELEM
    e = inputs.elementwise(n, inputs.seed_for(1, 16 * rank), device=dev)
    outs = [torch.empty_like(e.a) for _ in OPS]
    step = make_step(ff, e, outs)
    torch.cuda.synchronize()

    for _ in range(args.warmup):
        for op in OPS:
            step[op]()
    torch.cuda.synchronize()

    s = torch.cuda.current_stream()
    evs = {op: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)] for op in OPS}
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    t0.record(s)
    for k in range(args.steps):
        for op in OPS:
            a_, b_ = evs[op][k]
            a_.record(s)
            step[op]()
            b_.record(s)
    t1.record(s)
    torch.cuda.synchronize()
    barrier(dist)
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    elapsed_max = max_over_ranks(dist, elapsed)
    per_op = {op: sum(a_.elapsed_time(b_) for a_, b_ in evs[op]) / 1e3 / args.steps for op in OPS}
    ffops_step = len(OPS) * n
    value = whole_job_value(ws, ffops_step, args.steps, elapsed_max)

    rows = {}
    for op in OPS:
        gbs = BYTES_PER_VALUE[op] * n / per_op[op] / 1e9
        rows[op] = {"ms": round(per_op[op] * 1e3, 4), "GB/s": round(gbs, 1),
                    "frac_hbm": round(gbs / peaks["hbm_gbs"], 4), "ff_op_s": n / per_op[op]}
    dom = max(OPS, key=lambda o: per_op[o])
    ach = BYTES_PER_VALUE[dom] * n / per_op[dom] / 1e9
    kname = {"add12": "ff_add12", "mul12": "ff_mul12", "add": "ff_add", "mul": "ff_mul", "div": "ff_div",
             "sqrt": "ff_sqrt"}[dom]
    traffic = traffic_for(kname, n)
    roofline = {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": traffic, "kernel": kname,
                "algorithmic_bytes_per_launch": BYTES_PER_VALUE[dom] * n,
                "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 2^26-value launch, "
                                "scaled x4 to 2^28 (traffic grows in proportion)",
                "peak_source": peaks["source"] + " copy bandwidth"}

    # end to end through host buffers: every step copies its inputs from
    # pinned host memory, runs the six C-ABI calls and copies every result
    # back.  The step is cut into chunks pipelined over three streams
    # (host-to-device copies, kernels, device-to-host copies) so that both
    # directions of the host link and the GPU work at once.
    e2e = None
    if not args.no_e2e:
        keys = ("a", "b", "ab", "a_sqrt")
        host_in = {k: torch.empty_like(getattr(e, k), device="cpu").pin_memory() for k in keys}
        for k, t in host_in.items():
            t.copy_(getattr(e, k))
        host_out = torch.empty_like(e.a, device="cpu").pin_memory()
        dev_in = {k: torch.empty_like(getattr(e, k)) for k in keys}
        s_h2d, s_cmp, s_d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        chunks = 16
        csz = (n + chunks - 1) // chunks
        e2e_steps = max(1, min(args.steps, 5))
        from types import SimpleNamespace

        def one_e2e():
            # a step may overwrite the device inputs once the previous step's
            # kernels finished, and the outputs once they were copied out
            s_h2d.wait_stream(s_cmp)
            s_cmp.wait_stream(s_d2h)
            for c in range(chunks):
                lo, hi = c * csz, min(n, (c + 1) * csz)
                ev_in, ev_out = torch.cuda.Event(), torch.cuda.Event()
                with torch.cuda.stream(s_h2d):
                    for k in keys:
                        dev_in[k][lo:hi].copy_(host_in[k][lo:hi], non_blocking=True)
                    ev_in.record(s_h2d)
                with torch.cuda.stream(s_cmp):
                    s_cmp.wait_event(ev_in)
                    de = SimpleNamespace(**{k: dev_in[k][lo:hi] for k in keys})
                    step_c = make_step(ff, de, [o[lo:hi] for o in outs])
                    for op in OPS:
                        step_c[op]()
                    ev_out.record(s_cmp)
                with torch.cuda.stream(s_d2h):
                    s_d2h.wait_event(ev_out)
                    for o in outs:
                        host_out[lo:hi].copy_(o[lo:hi], non_blocking=True)
            for st_ in (s_h2d, s_cmp, s_d2h):
                torch.cuda.current_stream().wait_stream(st_)

        one_e2e()
        torch.cuda.synchronize()
        barrier(dist)
        c0 = time.perf_counter()
        for _ in range(e2e_steps):
            one_e2e()
        torch.cuda.synchronize()
        e_el = max_over_ranks(dist, time.perf_counter() - c0)
        h2d = sum(t.numel() * t.element_size() for t in host_in.values())
        d2h = len(OPS) * host_out.numel() * host_out.element_size()
        e2e = {"value": ws * ffops_step * e2e_steps / e_el, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": e2e_steps, "host_buffers": "pinned",
               "pipeline": f"{chunks} chunks over 3 streams", "link_GB/s": round((h2d + d2h) * e2e_steps / e_el / 1e9, 1)}
        del host_in, host_out, dev_in
        torch.cuda.synchronize()

    # the oracle on the host cores: rank 0 of a one-GPU run only (with more
    # ranks the other processes would share the cores it is timed on)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(e)

    if args.rows == "all":
        del outs, step
        rows.update(extra_rows(torch, ff, inputs, e, dev, peaks))
    del e
    torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_values": n, "ops_per_step": OPS,
                   "l2": "inputs larger than L2 (2 GiB per array)", "seed": inputs.seed_for(1, 0)},
        "hbm_gbs_step": round(sum(BYTES_PER_VALUE[o] for o in OPS) * n / (elapsed_max / args.steps) / 1e9, 1),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": len(OPS) * args.steps, "clocks": clk, "build_id": build_id, "rows": rows,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def extra_rows(torch, ff, inputs, e, dev, peaks):
    """Measurements of the other hot-path rows (each timed alone)."""
    out = {}
    hbm = peaks["hbm_gbs"]
    n = e.a.shape[0]
    # the measured FP32 / FP64 peaks first: the FP32-bound rows divide by them
    alu = alu_peaks(torch, ff, dev)
    out["alu_peaks"] = alu
    fp32 = alu["f32_fma_lane_ops_s"]
    # native baselines on the same values (FP64 holds hi + lo exactly)
    a64 = inputs.ff_to_f64(e.a)
    b64 = inputs.ff_to_f64(e.b)
    o64 = torch.empty_like(a64)
    for name, fn, nb in (("f64_add", lambda: ff.f64_add(a64, b64, out=o64), 24),
                         ("f64_mul", lambda: ff.f64_mul(a64, b64, out=o64), 24),
                         ("f64_div", lambda: ff.f64_div(a64, b64, out=o64), 24),
                         ("f64_sqrt", lambda: ff.f64_sqrt(a64.abs(), out=o64), 16)):
        t = time_fn(torch, fn, 5)
        out[name] = {"ms": round(t * 1e3, 4), "GB/s": round(nb * n / t / 1e9, 1), "op_s": n / t}
    del a64, b64, o64
    a32, b32 = e.a[:, 0].contiguous(), e.b[:, 0].contiguous()
    c32 = e.ab[:, 1].contiguous()
    o32 = torch.empty_like(a32)
    for name, fn, nb in (("f32_add", lambda: ff.f32_add(a32, b32, out=o32), 12),
                         ("f32_mul", lambda: ff.f32_mul(a32, b32, out=o32), 12),
                         ("f32_mad", lambda: ff.f32_mad(a32, b32, c32, out=o32), 16)):
        t = time_fn(torch, fn, 5)
        out[name] = {"ms": round(t * 1e3, 4), "GB/s": round(nb * n / t / 1e9, 1), "op_s": n / t}
    del a32, b32, c32, o32
    # accurate float-float addition on the same operands (24 B per value)
    oacc = torch.empty_like(e.a)
    t = time_fn(torch, lambda: ff.add_accurate(e.a, e.b, out=oacc), 5)
    out["add_accurate"] = {"ms": round(t * 1e3, 4), "GB/s": round(24 * n / t / 1e9, 1),
                           "frac_hbm": round(24 * n / t / 1e9 / hbm, 4), "ff_op_s": n / t}
    # AXPY z = Add22(Mul22(alpha, x), y) on the same operands (24 B per value, 2 ff-ops)
    alpha = tuple(float(v) for v in inputs.scalar_ff(inputs.seed_for(1, 5)))
    t = time_fn(torch, lambda: ff.axpy(alpha, e.a, e.b, out=oacc), 5)
    out["axpy"] = {"ms": round(t * 1e3, 4), "GB/s": round(24 * n / t / 1e9, 1),
                   "frac_hbm": round(24 * n / t / 1e9 / hbm, 4), "ff_op_s": 2 * n / t}
    del oacc
    torch.cuda.empty_cache()
    # the reductions at the elementwise size (2^28 values of the same arrays):
    # the fixed cost of a launch (ticket memset, ramp, last-block combine) is
    # a quarter of its share at 2^26
    # reductions: "ms" is the device time per call (20 calls replayed from one
    # CUDA graph, so host launch gaps between calls do not count); "loop_ms"
    # the same calls issued one by one from Python
    red_out = torch.empty(2, dtype=torch.float32, device=dev)

    def red_row(fn, nbytes, nops, key):
        # device time per call from a CUDA graph of 20 calls; and the same
        # calls issued one by one from Python, 50 of them, so that the host's
        # time to issue the first call is spread over many
        t = graph_time(torch, fn, 20)
        tl = time_fn(torch, fn, 50)
        return {"ms": round(t * 1e3, 4), "loop_ms": round(tl * 1e3, 4), "GB/s": round(nbytes / t / 1e9, 1),
                "frac_hbm": round(nbytes / t / 1e9 / hbm, 4), "frac_hbm_loop": round(nbytes / tl / 1e9 / hbm, 4),
                key: nops / t}

    a32, b32 = e.a[:, 0].contiguous(), e.b[:, 0].contiguous()
    for name, fn, nb, ops in (("dot_2^28", lambda: ff.dot(e.a, e.b, out=red_out), 16, 2),
                              ("sum_2^28", lambda: ff.sum(e.a, out=red_out), 8, 1),
                              ("dot2_f32_2^28", lambda: ff.dot2(a32, b32, out=red_out), 8, 2),
                              ("sum2_f32_2^28", lambda: ff.sum2(a32, out=red_out), 4, 1)):
        out[name] = red_row(fn, nb * n, ops * n, "ops_s")
    del a32, b32
    torch.cuda.empty_cache()
    # compensated Sum2 / Dot2 of binary32 vectors, n = 2^26 (4 / 8 B per value)
    nd2 = 1 << 26
    g2 = inputs.ill_dot_f32(nd2, 1e12, inputs.seed_for(5, 12), device=dev)
    out["dot2_f32_2^26"] = red_row(lambda: ff.dot2(g2.x, g2.y, out=red_out), 8 * nd2, nd2, "values_s")
    out["sum2_f32_2^26"] = red_row(lambda: ff.sum2(g2.x, out=red_out), 4 * nd2, nd2, "values_s")
    del g2
    torch.cuda.empty_cache()

    # reductions and the dot adjoint on the ill-conditioned dot, n = 2^26
    nd = 1 << 26
    g = inputs.ill_dot(nd, 1e12, inputs.seed_for(2, 12), device=dev)
    x, y = g.x, g.y
    out["dot_2^26"] = red_row(lambda: ff.dot(x, y, out=red_out), 16 * nd, 2 * nd, "ff_op_s")
    out["sum_2^26"] = red_row(lambda: ff.sum(x, out=red_out), 8 * nd, nd, "ff_op_s")
    dout = torch.tensor([1.0, 0.0], device=dev)
    dx = torch.empty_like(x)
    dy = torch.empty_like(y)
    t = time_fn(torch, lambda: ff.dot_backward(dout, x, y, dx, dy), 10)
    out["dot_backward_2^26"] = {"ms": round(t * 1e3, 4), "GB/s": round(32 * nd / t / 1e9, 1),
                                "frac_hbm": round(32 * nd / t / 1e9 / hbm, 4), "ff_op_s": 2 * nd / t}
    def plain_adjoint():
        db = dout.expand(nd, 2).contiguous()
        ff.mul(db, y, out=dx)
        ff.mul(db, x, out=dy)

    tp = time_fn(torch, plain_adjoint, 10)
    out["dot_backward_2^26"]["plain_two_mul_ms"] = round(tp * 1e3, 4)
    out["dot_backward_2^26"]["speedup_vs_plain"] = round(tp / t, 3)
    x64, y64 = inputs.ff_to_f64(x), inputs.ff_to_f64(y)
    t = time_fn(torch, lambda: ff.f64_dot(x64, y64), 10)
    out["f64_dot_2^26"] = {"ms": round(t * 1e3, 4), "GB/s": round(16 * nd / t / 1e9, 1)}
    del g, x, y, dx, dy, x64, y64
    torch.cuda.empty_cache()

    # GEMV and adjoint, A 32768 x 32768 (8 GiB), the 16 right-hand-side widths
    M = N = 32768
    ks = [1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64]
    gi = inputs.gemv(M, N, 1, inputs.seed_for(4, 0), device=dev)
    A = gi.A
    del gi
    Xall = inputs.to_ff(inputs.loguniform_f64(64 * N, torch.Generator(device=dev).manual_seed(inputs.seed_for(4, 1)),
                                              dev)).reshape(64, N, 2)
    gem = {}
    tot_f = tot_b = 0.0
    dA = torch.empty_like(A)   # the weight gradient dY X^T: one write of every A value
    for k in ks:
        X = Xall[:k].contiguous()
        tf = time_median(torch, lambda: ff.gemv(A, X), 11, warm=2)
        tb = time_median(torch, lambda: ff.gemv_t(A, X), 11, warm=2)
        tw = time_median(torch, lambda: ff.gemv_dA(X, X, out=dA), 11, warm=2)
        tot_f += tf
        tot_b += tb
        t_bound = max(8 * M * N / (hbm * 1e9), 28 * M * N * k / fp32)   # roofline time of one call
        gem[str(k)] = {"fwd_ms": round(tf * 1e3, 3), "adj_ms": round(tb * 1e3, 3), "dA_ms": round(tw * 1e3, 3),
                       "fwd_ff_op_s": 2 * M * N * k / tf, "adj_ff_op_s": 2 * M * N * k / tb,
                       "bound": "hbm" if 8 * M * N / (hbm * 1e9) >= 28 * M * N * k / fp32 else "fp32",
                       "fwd_frac_roofline": round(t_bound / tf, 4), "adj_frac_roofline": round(t_bound / tb, 4),
                       "dA_frac_roofline": round(t_bound / tw, 4)}
    del dA
    out["gemv_32768^2"] = {"per_k": gem, "timing": "median of 11 calls after 2 warm-ups, each call between "
                                                   "its own CUDA events",
                           "sweep_fwd_ms": round(tot_f * 1e3, 2), "sweep_adj_ms": round(tot_b * 1e3, 2),
                           "k1_fwd_GB/s": round(8 * M * N / (gem["1"]["fwd_ms"] / 1e3) / 1e9, 1)}
    A64 = inputs.ff_to_f64(A)
    del A
    torch.cuda.empty_cache()
    X64 = inputs.ff_to_f64(Xall)
    f64 = {}
    for k in (1, 16, 64):
        X = X64[:k].contiguous()
        t = time_fn(torch, lambda: ff.f64_gemv(A64, X), 1, warm=1)
        f64[str(k)] = {"ms": round(t * 1e3, 3)}
    out["f64_gemv_32768^2"] = f64
    del A64, X64, Xall
    torch.cuda.empty_cache()
    out.update(batched_rows(torch, ff, inputs, dev, peaks))
    out.update(gemm_rows(torch, ff, inputs, dev, fp32_measured=alu["f32_fma_lane_ops_s"]))
    return out


def alu_peaks(torch, ff, dev):
    """FP32 and FP64 FMA throughput measured by the library's probe kernel
    (eight independent chains per thread, 8 x 256-thread blocks per SM)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 8 * sms, 256
    out = {}
    for name, f64, iters in (("f32", False, 1 << 15), ("f64", True, 1 << 10)):
        buf = torch.empty(blocks * threads, dtype=torch.float64 if f64 else torch.float32, device=dev)
        t = time_fn(torch, lambda: ff.fma_peak(f64, iters, blocks, threads, out=buf), 5, warm=2)
        flops = 16 * iters * blocks * threads
        out[name + "_fma_flop_s"] = flops / t
        out[name + "_fma_lane_ops_s"] = flops / 2 / t
    out["sms"] = sms
    return out


def gemm_rows(torch, ff, inputs, dev, size=4096, fp32_measured=None):
    """Float-float GEMM, size^3: ff_gemm forward and the two adjoint GEMMs of
    FFGemm, against cuBLAS FP64 and FP32 GEMM (torch.matmul) on the same
    values.  The kernel is bound by FP32 instruction issue: 28 FP32
    instructions per term (Mul22 12, Add22 16) against SMs x 128 lanes x the
    SM clock sampled while it runs."""
    m = n = k = size
    g = inputs.gemm(m, n, k, inputs.seed_for(6, 0), device=dev)
    C = torch.empty((m, n, 2), dtype=torch.float32, device=dev)
    clk = ClockSampler(dev.index or 0)
    clk.start()
    t_fwd = time_fn(torch, lambda: ff.gemm(g.A, g.B, out=C), 5, warm=2)
    clocks = clk.stop()
    dA = torch.empty_like(g.A)
    dB = torch.empty_like(g.B)
    t_dA = time_fn(torch, lambda: ff.gemm(g.dC, g.B, transb=True, out=dA), 3, warm=1)
    t_dB = time_fn(torch, lambda: ff.gemm(g.A, g.dC, transa=True, out=dB), 3, warm=1)
    terms = m * n * k
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_mhz") or 2070.0
    issue = sms * 128 * mhz * 1e6
    A64 = inputs.ff_to_f64(g.A)
    B64 = inputs.ff_to_f64(g.B)
    del g, dA, dB
    torch.cuda.empty_cache()
    t64 = time_fn(torch, lambda: torch.matmul(A64, B64), 3, warm=1)
    A32, B32 = A64.float(), B64.float()
    del A64, B64
    tf32_prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    t32 = time_fn(torch, lambda: torch.matmul(A32, B32), 5, warm=2)
    torch.backends.cuda.matmul.allow_tf32 = tf32_prev
    del A32, B32, C
    torch.cuda.empty_cache()
    return {f"gemm_{size}^3": {
        "fwd_ms": round(t_fwd * 1e3, 3), "dA_ms": round(t_dA * 1e3, 3), "dB_ms": round(t_dB * 1e3, 3),
        "fwd_ff_op_s": 2 * terms / t_fwd, "terms_per_s": terms / t_fwd,
        "frac_fp32_issue": round(28 * terms / t_fwd / issue, 4), "issue_peak_lane_ops_s": issue,
        "frac_of_measured_fp32_fma": round(28 * terms / t_fwd / fp32_measured, 4) if fp32_measured else None,
        "clocks": clocks,
        "cublas_f64_ms": round(t64 * 1e3, 3), "speedup_vs_cublas_f64": round(t64 / t_fwd, 3),
        "cublas_f32_ms": round(t32 * 1e3, 3), "slowdown_vs_cublas_f32": round(t_fwd / t32, 2)}}


def batched_rows(torch, ff, inputs, dev, peaks):
    """4096 dot / AXPY instances, lengths log-uniform over 1e2..1e7 (dots by
    the ill-conditioned generator at cond 1e8, AXPY by the elementwise one
    with its 10% cancelling pairs): one persistent launch (plain run and CUDA
    graph) against 4096 plain calls (loop and CUDA graph); then the same
    dots' forward and adjoint batched against plain ff_dot / ff_dot_backward
    calls; last, the 4096 instances packed without padding, so that every
    instance after an odd length starts 8 bytes off a 16-byte boundary."""
    from paper_cs_0603115_gb300 import batch
    hbm = peaks["hbm_gbs"]
    lengths, kinds = inputs.batch_lengths(4096, inputs.seed_for(3, 0))
    total = sum(lengths)
    offs, o = [], 0
    for n in lengths:
        offs.append(o)
        o += n + (n & 1)                       # keep every instance 16-byte aligned
    X = torch.empty((o, 2), dtype=torch.float32, device=dev)
    Y = torch.empty((o, 2), dtype=torch.float32, device=dev)
    Z = torch.empty((o, 2), dtype=torch.float32, device=dev)   # AXPY outputs / dot gradients dx
    W = torch.empty((o, 2), dtype=torch.float32, device=dev)   # dot gradients dy
    D = torch.empty((4096, 2), dtype=torch.float32, device=dev)
    Dplain = torch.empty_like(D)
    dout = torch.empty((4096, 2), dtype=torch.float32, device=dev)
    alphas = [tuple(float(v) for v in inputs.scalar_ff(inputs.seed_for(3, 3) + i)) for i in range(4096)]
    for i in range(4096):
        dout[i].copy_(inputs.scalar_ff(inputs.seed_for(3, 4) + i))

    def fill(offsets):
        """Every instance's inputs at its offset (the same values whatever the offsets)."""
        for i, (n, kind) in enumerate(zip(lengths, kinds)):
            sl = slice(offsets[i], offsets[i] + n)
            if kind == batch.DOT:
                g = inputs.ill_dot(n, 1e8, inputs.seed_for(3, 1) + 7 * i, device=dev)
                X[sl].copy_(g.x)
                Y[sl].copy_(g.y)
                del g
            else:
                e = inputs.elementwise(n, inputs.seed_for(3, 2) + 7 * i, device=dev)
                X[sl].copy_(e.a)
                Y[sl].copy_(e.b)
                del e
        torch.cuda.synchronize()

    fill(offs)
    sl = [slice(offs[i], offs[i] + lengths[i]) for i in range(4096)]
    specs = [(k, X[sl[i]], Y[sl[i]], D[i] if k == batch.DOT else Z[sl[i]], alphas[i]) for i, k in enumerate(kinds)]
    inst = batch.make_instances(specs)
    bytes_total = sum(16 * n if k == batch.DOT else 24 * n for n, k in zip(lengths, kinds))
    ffops = sum(2 * n for n in lengths)

    tune, tune_ms = batch.autotune(inst, reps=2, cache_path=os.path.join(ROOT, "_build", "autotune.json"),
                                   force=True)
    plan = batch.BatchPlan(inst, tune=tune)
    plan_def = batch.BatchPlan(inst)

    def plain():
        for i, k in enumerate(kinds):
            if k == batch.DOT:
                ff.dot(X[sl[i]], Y[sl[i]], out=Dplain[i])
            else:
                ff.axpy(alphas[i], X[sl[i]], Y[sl[i]], out=Z[sl[i]])

    t_plain = time_fn(torch, plain, 3, warm=1)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plain()
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        plain()
    t_plain_graph = time_fn(torch, g.replay, 3, warm=1)
    t_run = time_fn(torch, plan.run, 5)
    t_run_def = time_fn(torch, plan_def.run, 5)
    plan.capture()
    t_graph = time_fn(torch, plan.launch, 5)
    z_plain = Z.clone()
    plan.launch()
    torch.cuda.synchronize()
    axpy_equal = bool(torch.equal(Z, z_plain))
    # dot agreement with the plain calls, in units of sum |x_i y_i|
    rel = 0.0
    for i, k in enumerate(kinds):
        if k == batch.DOT:
            xv, yv = inputs.ff_to_f64(X[sl[i]]), inputs.ff_to_f64(Y[sl[i]])
            a = float((xv * yv).abs().sum().item())
            d = abs((float(D[i, 0]) - float(Dplain[i, 0])) + (float(D[i, 1]) - float(Dplain[i, 1])))
            rel = max(rel, d / a if a > 0 else d)
    rows = {"batched_4096_dot_axpy": {
        "values": total, "plain_loop_ms": round(t_plain * 1e3, 3), "plain_graph_ms": round(t_plain_graph * 1e3, 3),
        "batched_run_ms": round(t_run * 1e3, 3), "batched_graph_ms": round(t_graph * 1e3, 3),
        "batched_default_tune_ms": round(t_run_def * 1e3, 3),
        "speedup_vs_plain_loop": round(t_plain / t_graph, 3), "speedup_vs_plain_graph": round(t_plain_graph / t_graph, 3),
        "GB/s": round(bytes_total / t_graph / 1e9, 1), "frac_hbm": round(bytes_total / t_graph / 1e9 / hbm, 4),
        "ff_op_s": ffops / t_graph, "tune": list(tune), "tune_ms": tune_ms, "ntiles": plan.ntiles,
        "grid": plan.grid, "axpy_bitequal_plain": axpy_equal,
        "dot_max_absdiff_vs_plain_over_sum_abs": rel}}
    plan.close()
    plan_def.close()
    del g

    # the dots alone: forward and adjoint, batched vs plain
    dots = [i for i, k in enumerate(kinds) if k == batch.DOT]
    fwd = batch.make_instances([(batch.DOT, X[sl[i]], Y[sl[i]], D[i], None) for i in dots])
    bwd = batch.make_instances([(batch.DOT_GRAD, X[sl[i]], Y[sl[i]], Z[sl[i]], None, W[sl[i]], dout[i])
                                for i in dots])
    nd = sum(lengths[i] for i in dots)
    pf = batch.BatchPlan(fwd, tune=batch.autotune(fwd, reps=2, cache_path=None)[0]).capture()
    pb = batch.BatchPlan(bwd, tune=batch.autotune(bwd, reps=2, cache_path=None)[0]).capture()

    def plain_f():
        for j, i in enumerate(dots):
            ff.dot(X[sl[i]], Y[sl[i]], out=Dplain[i])

    def plain_b():
        for j, i in enumerate(dots):
            ff.dot_backward(dout[i], X[sl[i]], Y[sl[i]], Z[sl[i]], W[sl[i]])

    tf_plain = time_fn(torch, plain_f, 3, warm=1)
    tb_plain = time_fn(torch, plain_b, 3, warm=1)
    tf = time_fn(torch, pf.launch, 5)
    tb = time_fn(torch, pb.launch, 5)
    # accuracy of the batched forms against the plain calls: the forward's
    # difference over sum |x_i y_i| (both within the dot bound), the adjoint
    # bit for bit (it is the same Mul22 per value)
    torch.cuda.synchronize()
    fwd_rel, grad_equal = 0.0, True
    for i in dots:
        xv, yv = inputs.ff_to_f64(X[sl[i]]), inputs.ff_to_f64(Y[sl[i]])
        a = float((xv * yv).abs().sum().item())
        d = abs((float(D[i, 0]) - float(Dplain[i, 0])) + (float(D[i, 1]) - float(Dplain[i, 1])))
        fwd_rel = max(fwd_rel, d / a if a > 0 else d)
        dx, dy = ff.dot_backward(dout[i], X[sl[i]], Y[sl[i]])
        grad_equal &= bool(torch.equal(dx.view(torch.int32), Z[sl[i]].view(torch.int32)) and
                           torch.equal(dy.view(torch.int32), W[sl[i]].view(torch.int32)))
        del xv, yv, dx, dy
    rows["batched_2048_dot_fwd_grad"] = {
        "values": nd, "fwd_plain_ms": round(tf_plain * 1e3, 3), "fwd_batched_graph_ms": round(tf * 1e3, 3),
        "bwd_plain_ms": round(tb_plain * 1e3, 3), "bwd_batched_graph_ms": round(tb * 1e3, 3),
        "fwd_speedup": round(tf_plain / tf, 3), "bwd_speedup": round(tb_plain / tb, 3),
        "fwd_frac_hbm": round(16 * nd / tf / 1e9 / hbm, 4), "bwd_frac_hbm": round(32 * nd / tb / 1e9 / hbm, 4),
        "fwd_max_absdiff_vs_plain_over_sum_abs": fwd_rel, "grad_bitequal_plain": grad_equal}
    pf.close()
    pb.close()

    # the same instances packed back to back: an instance that follows an odd
    # length starts 8 bytes off a 16-byte boundary and runs the batched
    # kernel's scalar path (the plain kernels realign with one head value)
    offs_u, o = [], 0
    for n in lengths:
        offs_u.append(o)
        o += n
    fill(offs_u)
    slu = [slice(offs_u[i], offs_u[i] + lengths[i]) for i in range(4096)]
    inst_u = batch.make_instances([(k, X[slu[i]], Y[slu[i]], D[i] if k == batch.DOT else Z[slu[i]], alphas[i])
                                   for i, k in enumerate(kinds)])
    plan_u = batch.BatchPlan(inst_u, tune=tune).capture()

    def plain_u():
        for i, k in enumerate(kinds):
            if k == batch.DOT:
                ff.dot(X[slu[i]], Y[slu[i]], out=Dplain[i])
            else:
                ff.axpy(alphas[i], X[slu[i]], Y[slu[i]], out=Z[slu[i]])

    gu = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plain_u()
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(gu):
        plain_u()
    tu_plain_graph = time_fn(torch, gu.replay, 3, warm=1)
    tu = time_fn(torch, plan_u.launch, 5)
    gu.replay()
    torch.cuda.synchronize()
    z_plain = Z.clone()
    plan_u.launch()
    torch.cuda.synchronize()
    axpy_equal_u = bool(torch.equal(Z.view(torch.int32), z_plain.view(torch.int32)))
    del z_plain
    rel_u = 0.0
    for i, k in enumerate(kinds):
        if k == batch.DOT:
            xv, yv = inputs.ff_to_f64(X[slu[i]]), inputs.ff_to_f64(Y[slu[i]])
            a = float((xv * yv).abs().sum().item())
            d = abs((float(D[i, 0]) - float(Dplain[i, 0])) + (float(D[i, 1]) - float(Dplain[i, 1])))
            rel_u = max(rel_u, d / a if a > 0 else d)
    rows["batched_4096_dot_axpy_unpadded"] = {
        "values": total, "instances_off_16B": sum(1 for v in offs_u if v & 1),
        "plain_graph_ms": round(tu_plain_graph * 1e3, 3), "batched_graph_ms": round(tu * 1e3, 3),
        "speedup_vs_plain_graph": round(tu_plain_graph / tu, 3), "GB/s": round(bytes_total / tu / 1e9, 1),
        "frac_hbm": round(bytes_total / tu / 1e9 / hbm, 4), "tune": list(tune), "axpy_bitequal_plain": axpy_equal_u,
        "dot_max_absdiff_vs_plain_over_sum_abs": rel_u}
    plan_u.close()
    del gu
    del X, Y, Z, W, D, Dplain, dout
    torch.cuda.empty_cache()
    rows.update(batched_gemv_row(torch, ff, inputs, dev, hbm))
    return rows


def batched_gemv_row(torch, ff, inputs, dev, hbm):
    """1024 float-float GEMVs y = A x of uneven shapes (m, n log-uniform over
    32..4096) in one persistent launch, against 1024 plain ff_gemv calls."""
    from paper_cs_0603115_gb300 import batch
    g = torch.Generator().manual_seed(inputs.seed_for(3, 9))
    cnt = 1024
    ms = torch.round(2.0 ** (5 + 7 * torch.rand(cnt, generator=g, dtype=torch.float64))).to(torch.int64).tolist()
    ns = torch.round(2.0 ** (5 + 7 * torch.rand(cnt, generator=g, dtype=torch.float64))).to(torch.int64).tolist()
    ns = [n + (n & 1) for n in ns]
    total = sum(m * n for m, n in zip(ms, ns))
    gA = torch.Generator(device=dev).manual_seed(inputs.seed_for(3, 10))
    Aall = inputs.to_ff(inputs.loguniform_f64(total, gA, dev))
    xall = inputs.to_ff(inputs.loguniform_f64(sum(ns), gA, dev))
    yall = torch.empty((sum(ms), 2), dtype=torch.float32, device=dev)
    yplain = torch.empty_like(yall)
    specs, views = [], []
    oa = ox = oy = 0
    for m, n in zip(ms, ns):
        A = Aall[oa:oa + m * n].view(m, n, 2)
        x = xall[ox:ox + n]
        y = yall[oy:oy + m]
        specs.append((batch.GEMV, A, x, y, None))
        views.append((A, x.view(1, n, 2), yplain[oy:oy + m].view(1, m, 2)))
        oa += m * n
        ox += n
        oy += m
    inst = batch.make_instances(specs)
    tune, _ = batch.autotune(inst, reps=2, cache_path=None)
    plan = batch.BatchPlan(inst, tune=tune).capture()

    def plain():
        for A, x, y in views:
            ff.gemv(A, x, out=y)

    t_plain = time_fn(torch, plain, 3, warm=1)
    gr = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plain()
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(gr):
        plain()
    t_plain_graph = time_fn(torch, gr.replay, 3, warm=1)
    t_b = time_fn(torch, plan.launch, 5)
    # rows agree with the plain GEMV, relative to sum_j |A_rj x_j|
    rel = 0.0
    oy = 0
    for (A, x, yp), (m, n) in zip(views, zip(ms, ns)):
        den = inputs.ff_to_f64(A).abs() @ inputs.ff_to_f64(x[0]).abs()
        d = (inputs.ff_to_f64(yall[oy:oy + m]) - inputs.ff_to_f64(yp[0])).abs()
        rel = max(rel, float((d / den).max()))
        oy += m
    plan.close()
    del Aall, xall, yall, yplain
    torch.cuda.empty_cache()
    nbytes = 8 * total
    return {"batched_1024_gemv": {
        "A_values": total, "plain_loop_ms": round(t_plain * 1e3, 3), "plain_graph_ms": round(t_plain_graph * 1e3, 3),
        "batched_graph_ms": round(t_b * 1e3, 3), "speedup_vs_plain_loop": round(t_plain / t_b, 3),
        "speedup_vs_plain_graph": round(t_plain_graph / t_b, 3), "GB/s": round(nbytes / t_b / 1e9, 1),
        "frac_hbm": round(nbytes / t_b / 1e9 / hbm, 4), "tune": list(tune),
        "max_diff_vs_plain_over_sum_abs": rel}}


# ---------------------------------------------------------------------------
# the reference arm: the CPU oracle, same metric
# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_cs_0603115_gb300 import inputs
    oracle.build()
    n = 1 << 24
    e = inputs.elementwise(n, inputs.seed_for(1, 0))
    a, b, ab, asq = (t.numpy() for t in (e.a, e.b, e.ab, e.a_sqrt))
    cores = host_cores()
    fns, pool = oracle_ops(a, b, ab, asq, cores)
    for _ in range(args.warmup):
        for f in fns:
            f()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for f in fns:
            f()
    dt = time.perf_counter() - t0
    if pool is not None:
        pool.shutdown()
    value = len(fns) * n * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_values": N_ELEM, "ops_per_step": OPS,
                   "sample_per_step": f"2^24 values of the same generator on {cores} host threads (the full "
                                      "2^28 per step would take minutes)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"2^24 values per operator per step, {args.steps} steps, {cores} threads, "
                                   "contiguous chunks"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_case(args):
    """Profiling case: generate n values, run one operator `reps` times, exit.
    Used to capture one kernel under ncu on a small input (no JSON line)."""
    import torch
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import build as ffbuild
    from paper_cs_0603115_gb300 import inputs
    ffbuild.build()
    dev = torch.device("cuda", 0)
    n = args.n
    if args.case in ("dot", "sum", "dot_backward"):
        g = inputs.ill_dot(n, 1e12, inputs.seed_for(2, 12), device=dev)
        x, y = g.x, g.y
        dout = torch.tensor([1.0, 0.0], device=dev)
        fn = {"dot": lambda: ff.dot(x, y), "sum": lambda: ff.sum(x),
              "dot_backward": lambda: ff.dot_backward(dout, x, y)}[args.case]
    elif args.case in ("dot2", "sum2"):
        g = inputs.ill_dot_f32(n, 1e12, inputs.seed_for(5, 12), device=dev)
        fn = (lambda: ff.dot2(g.x, g.y)) if args.case == "dot2" else (lambda: ff.sum2(g.x))
    elif args.case in ("batch", "batch_packed"):
        # 256 dot / AXPY instances, lengths log-uniform over 1e2..1e6 (a small
        # sample of the 4096-instance workload), one persistent launch; with
        # batch_packed the instances lie back to back (every instance after an
        # odd length starts 8 bytes off a 16-byte boundary)
        from paper_cs_0603115_gb300 import batch
        lengths, kinds = inputs.batch_lengths(256, inputs.seed_for(3, 0), hi_exp=6.0)
        offs, o = [], 0
        for ln in lengths:
            offs.append(o)
            o += ln + (ln & 1 if args.case == "batch" else 0)
        gx = torch.Generator(device=dev).manual_seed(inputs.seed_for(3, 11))
        X = inputs.to_ff(inputs.loguniform_f64(o, gx, dev))
        Y = inputs.to_ff(inputs.loguniform_f64(o, gx, dev))
        Z = torch.empty_like(X)
        D = torch.empty((len(lengths), 2), dtype=torch.float32, device=dev)
        specs = []
        for i, (ln, kind) in enumerate(zip(lengths, kinds)):
            sl = slice(offs[i], offs[i] + ln)
            specs.append((kind, X[sl], Y[sl], D[i] if kind == batch.DOT else Z[sl], (1.5, 0.0)))
        plan = batch.BatchPlan(batch.make_instances(specs), tune=(256, 128, 4, 4))
        fn = plan.run
    elif args.case == "batch_gemv":
        from paper_cs_0603115_gb300 import batch
        g = torch.Generator().manual_seed(inputs.seed_for(3, 9))
        cnt = 256
        ms = torch.round(2.0 ** (5 + 7 * torch.rand(cnt, generator=g, dtype=torch.float64))).to(torch.int64).tolist()
        ns = torch.round(2.0 ** (5 + 7 * torch.rand(cnt, generator=g, dtype=torch.float64))).to(torch.int64).tolist()
        ns = [v + (v & 1) for v in ns]
        gA = torch.Generator(device=dev).manual_seed(inputs.seed_for(3, 10))
        Aall = inputs.to_ff(inputs.loguniform_f64(sum(a * b for a, b in zip(ms, ns)), gA, dev))
        xall = inputs.to_ff(inputs.loguniform_f64(sum(ns), gA, dev))
        yall = torch.empty((sum(ms), 2), dtype=torch.float32, device=dev)
        specs, oa, ox, oy = [], 0, 0, 0
        for mm, nn in zip(ms, ns):
            specs.append((batch.GEMV, Aall[oa:oa + mm * nn].view(mm, nn, 2), xall[ox:ox + nn], yall[oy:oy + mm], None))
            oa += mm * nn
            ox += nn
            oy += mm
        # the launch shape the autotuner picks for bench.py's 1024-GEMV batch:
        # 128-thread blocks, as many resident as fit
        plan = batch.BatchPlan(batch.make_instances(specs), tune=(128, 16, 0, 2))
        fn = plan.run
    elif args.case == "gemm":
        # --n is the matrix order here: C (n x n) = A (n x n) B (n x n)
        g = inputs.gemm(n, n, n, inputs.seed_for(6, 0), device=dev)
        C = torch.empty_like(g.A)
        fn = lambda: ff.gemm(g.A, g.B, out=C)
    elif args.case in ("gemv", "gemv_t", "gemv_dA"):
        m = int(math.isqrt(n))
        gi = inputs.gemv(m, m, args.k, inputs.seed_for(4, 0), device=dev)
        if args.case == "gemv":
            fn = lambda: ff.gemv(gi.A, gi.X)
        elif args.case == "gemv_t":
            fn = lambda: ff.gemv_t(gi.A, gi.dY)
        else:
            dA = torch.empty_like(gi.A)
            fn = lambda: ff.gemv_dA(gi.dY, gi.X, out=dA)
    else:
        e = inputs.elementwise(n, inputs.seed_for(1, 0), device=dev)
        outs = [torch.empty_like(e.a) for _ in OPS]
        step = make_step(ff, e, outs)
        if args.case == "step":
            def fn():
                for op in OPS:
                    step[op]()
        else:
            fn = step[args.case]
    torch.cuda.synchronize()
    for _ in range(args.reps):
        fn()
    torch.cuda.synchronize()
    print(f"case {args.case} n={n} reps={args.reps} ok")


def paper_table(args):
    """The paper's timing method (Section 6, Tables 3 and 4) regenerated:
    times of FP32 add / mul / mad, Add12, Mul12, Add22 and Mul22 over 4096 ..
    1048576 values, normalised to the time of 4096 FP32 additions on the same
    device -- on the GB300 (device time per launch: 50 launches replayed from
    one CUDA graph) and on one host core (the oracle's loops, the
    CPU-baseline leg; best of 20)."""
    import torch
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import build as ffbuild
    from paper_cs_0603115_gb300 import inputs
    ffbuild.build()
    dev = torch.device("cuda", 0)
    sizes = [4096, 16384, 65536, 262144, 1048576]
    cols = ["Add", "Mul", "Mad", "Add12", "Mul12", "Add22", "Mul22"]
    gpu_t, cpu_t = {}, {}
    for n in sizes:
        e = inputs.elementwise(n, inputs.seed_for(0, 0), device=dev)
        a32, b32, c32 = e.a[:, 0].contiguous(), e.b[:, 0].contiguous(), e.ab[:, 1].contiguous()
        o32 = torch.empty_like(a32)
        o = torch.empty_like(e.a)
        fns = [lambda: ff.f32_add(a32, b32, out=o32), lambda: ff.f32_mul(a32, b32, out=o32),
               lambda: ff.f32_mad(a32, b32, c32, out=o32), lambda: ff.add12(e.ab, out=o),
               lambda: ff.mul12(e.ab, out=o), lambda: ff.add(e.a, e.b, out=o), lambda: ff.mul(e.a, e.b, out=o)]
        gpu_t[n] = [graph_time(torch, f, 50) for f in fns]
        cpu_t[n] = cpu_paper_row(e)
    base_g, base_c = gpu_t[4096][0], cpu_t[4096][0]
    lines = ["| size | " + " | ".join(cols) + " |", "|---" * (len(cols) + 1) + "|"]
    out = {"gpu": {}, "cpu": {}, "gpu_us_per_4096_adds": base_g * 1e6, "cpu_us_per_4096_adds": base_c * 1e6}
    for which, tab, base in (("gpu", gpu_t, base_g), ("cpu", cpu_t, base_c)):
        lines.append(f"| **{which}** |" + " |" * len(cols))
        for n in sizes:
            norm = [t / base for t in tab[n]]
            out[which][str(n)] = [round(v, 2) for v in norm]
            lines.append(f"| {n} | " + " | ".join(f"{v:.2f}" for v in norm) + " |")
    print("\n".join(lines))
    print(json.dumps(out))


def graph_time(torch, fn, reps: int) -> float:
    """Device time per launch: `reps` launches captured in one CUDA graph and
    replayed, so the host's launch overhead does not count."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            fn()
    return time_fn(torch, g.replay, 5, warm=2) / reps


def cpu_paper_row(e):
    """One host core running the oracle's loops for the paper-table sizes
    (minimum of 20 runs each)."""
    import oracle
    a, b, ab = e.a.cpu().numpy(), e.b.cpu().numpy(), e.ab.cpu().numpy()
    a32, b32, c32 = a[:, 0].copy(), b[:, 0].copy(), ab[:, 1].copy()
    fns = [lambda: oracle.fp32_add(a32, b32), lambda: oracle.fp32_mul(a32, b32),
           lambda: oracle.fp32_mad(a32, b32, c32), lambda: oracle.add12(ab), lambda: oracle.mul12(ab),
           lambda: oracle.add22(a, b), lambda: oracle.mul22(a, b)]
    res = []
    for f in fns:
        best = float("inf")
        for _ in range(20):
            t0 = time.perf_counter()
            f()
            best = min(best, time.perf_counter() - t0)
        res.append(best)
    return res


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    p.add_argument("--rows", choices=["all", "main"], default="all")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--fingerprint", action="store_true", help="print the elementwise kernels' source fingerprint")
    p.add_argument("--paper-table", action="store_true", help="regenerate the paper's normalised timing tables")
    p.add_argument("--case", default=None, help="profiling case: one operator on --n values, --reps launches")
    p.add_argument("--n", type=int, default=1 << 24)
    p.add_argument("--k", type=int, default=1)
    p.add_argument("--reps", type=int, default=3)
    args = p.parse_args()
    if args.fingerprint:
        print(kernel_fingerprint())
        return
    if args.case:
        run_case(args)
        return
    if args.paper_table:
        paper_table(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
