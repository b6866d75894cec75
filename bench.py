"""Benchmark: orbit-steps/s of many-orbit Euler-Maruyama on one GB300.

Workload (one "step" = one pass of the whole hot path over one batch):
stochastic Kuramoto, scalar-sigma layout, n = 8 / 32 / 128 with
2^20 / 2^18 / 2^16 orbits, dt = 0.005, 10^4 Euler-Maruyama steps per orbit,
a frame every 100 steps, Philox seed 0; FP32 with Kahan-compensated state.
Per step: reload the parameters and initial states from device memory, then
integrate all three problems over the full horizon (frames written to HBM).

The JSON line carries the device-timed value (inputs resident in HBM), an
end-to-end value through the C ABI with pinned host buffers (host->device
inputs and device->host frames inside the timed region), the roofline of
the dominant kernel (the forward kernel, bound by the special-function
unit: peak = its rate per SM per clock measured by sdeb_pipe_rate x the SM
count x the median SM clock sampled while it ran), and the other legs:
the same problems in FP64, the discrete adjoint against its forward, the
batched heterogeneous workload, the FitzHugh-Nagumo network (FP32
Euler-Maruyama and Milstein, FP64), the ODE path (Runge-Kutta, implicit
schemes), a run-time compiled user model, the paper's speed and accuracy
protocols and a particle-swarm search.  The CPU leg times the oracle on this
host's cores on a bounded sample and, from the oracle's results on the
legs' first orbits, states each leg's error against the FP64 oracle.  The
line ends with "targets", the figures the design is held to.

With torchrun (N > 1) every rank runs the whole workload as an independent
replica on its own GPU: there is no data exchange, only a barrier and a
max over ranks of the timed region (a gloo process group on the host).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "kuramoto_n8_n32_n128_dt0.005_K1e4_stride100"
CONFIGS = [  # (n, orbits per GPU)
    (8, 1 << 20),
    (32, 1 << 18),
    (128, 1 << 16),
]
DT, STEPS, STRIDE, SEED = 0.005, 10000, 100, 0
METRIC = "orbit-steps/sec"
# SFU (special function unit) operations the method needs per oscillator-step
# in the FP32 path: sin and cos of the phase, and per normal half of the
# Box-Muller (log, sqrt, sin, cos).
SFU_OPS_PER_OSC_STEP = 4
E2E_CHUNKS = 4
ERR_ORBITS = 64          # orbits per leg compared with the oracle
ERR_T = 10.0             # the stated pathwise horizon of the FP32 tolerance
FALLBACK_SM_MHZ = 2070.0

# ncu counters of kernels as they were when captured, keyed by a fingerprint
# of the sources the kernel is compiled from (their code with comments and
# whitespace left out); a counter is reported only while the fingerprint
# matches (null once the kernel's code has changed).
FORWARD_SOURCES = ["em_forward_impl.cuh", "em_device.cuh", "em_models.cuh", "fwd_kuramoto_f32.cu",
                   "fwd_kuramoto_f64.cu", "em_internal.h"]
NCU_COUNTERS = {
    # DRAM bytes (read + write) of one full-size forward launch of the n = 32 problem
    "forward_n32_dram_bytes": {"sha": "b58b7a844f81edb6", "value": 3.488e9},
    # FP64-pipe thread-instructions per oscillator-step of the FP64 forward kernel
    "fp64_pipe_inst_per_osc_step": {"sha": "b58b7a844f81edb6", "value": 65.63},
}


def sources_fingerprint(names):
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_1908_03869_gb300", "csrc", nm)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def counter(name):
    c = NCU_COUNTERS[name]
    return c["value"] if c["sha"] is not None and c["sha"] == sources_fingerprint(FORWARD_SOURCES) else None


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, dist=None):
    """Max of a float over all ranks of a (gloo) process group; the value
    itself without one."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running; medians
    over any interval of the run."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.samples = []          # (time, sm_mhz, max_mhz, reasons)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            reasons = {nm for nm, v in zip(self.NAMES, parts[5:9]) if v.lower() == "active"}
            self.samples.append((time.perf_counter(), sm, mx, reasons))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        s = [x for x in self.samples if (t0 is None or x[0] >= t0) and (t1 is None or x[0] <= t1)]
        if not s:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi sample"], "samples": 0}
        return {"sm_mhz": statistics.median(x[1] for x in s), "sm_max_mhz": max(x[2] for x in s),
                "reasons": sorted(set().union(*[x[3] for x in s])), "samples": len(s)}

    def median_mhz(self, t0=None, t1=None):
        m = self.summary(t0, t1)["sm_mhz"]
        return m if m else FALLBACK_SM_MHZ


def _rel_err(x, ref, axis=None):
    """max |x - ref| / max(|ref|, 1) (over `axis`, or everything)."""
    import numpy as np
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    e = np.abs(x - ref) / np.maximum(np.abs(ref), 1.0)
    return float(e.max()) if axis is None else e.max(axis=axis)


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _timed(fn, stream, reps, flush=None, prep=None):
    """Median over `reps` runs (after one untimed) of fn() on `stream`, CUDA
    events on that stream; prep() (loading the inputs) runs before each run
    and, when a flush buffer is given, the L2 is flushed, both outside the
    events."""
    import torch
    times = []
    for r in range(reps + 1):
        if prep is not None:
            prep()
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(r & 0xFF)
        a, b = _events()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        if r > 0:
            times.append(a.elapsed_time(b))
    return statistics.median(times), times


# ---------------------------------------------------------------------------
# The CPU oracle: baseline timing (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------

def _sample_sizes(cores):
    # 2-3 s per problem on `cores` threads, every thread busy (at least one
    # orbit per thread for each problem): about 8 s for the three
    return [320 * cores, 30 * cores, cores]


def _main_inputs(n, orbits):
    import numpy as np

    from paper_1908_03869_gb300 import inputs
    p, x0 = inputs.kuramoto(n, orbits, seed=1)
    return p.astype(np.float32), x0.astype(np.float32)


def _cpu_sample(nthreads, sizes, mean_field=False, inputs_by_n=None):
    """The oracle (pairwise Kuramoto drift by definition, as it stands; or its
    mean-field form) on the first orbits of each problem, full horizon, on
    the benchmark's own inputs.  Returns (orbit-steps/s over the workload mix,
    description, {n: oracle frames of the sampled orbits})."""
    import numpy as np

    import oracle

    t_total, units_total, desc, frames = 0.0, 0, [], {}
    for (n, orbits), s in zip(CONFIGS, sizes):
        if inputs_by_n is not None:
            p, x0 = inputs_by_n[n]
            p, x0 = p[:s], x0[:s]
        else:
            from paper_1908_03869_gb300 import inputs
            p, x0 = inputs.kuramoto(n, s, seed=1)
            p, x0 = p.astype(np.float32), x0.astype(np.float32)
        pb = oracle.make_problem("kuramoto", n, n, n + 2, DT, STEPS, STRIDE, SEED, mean_field=mean_field)
        t0 = time.perf_counter()
        fr, _ = oracle.integrate(pb, p.astype(np.float64), x0.astype(np.float64), frames=True, nthreads=nthreads)
        dt = time.perf_counter() - t0
        rate = s * STEPS / dt
        t_total += orbits * STEPS / rate          # time the per-GPU problem would take at this rate
        units_total += orbits * STEPS
        desc.append("n=%d: first %d orbits x %d steps in %.2fs" % (n, s, STEPS, dt))
        frames[n] = fr
    return units_total / t_total, "; ".join(desc), frames


def run_reference(args):
    ws, rank, _ = _dist_env()
    if ws > 1 and rank != 0:
        return 0
    cores = os.cpu_count() or 1
    sizes = [max(1, s // 2) for s in _sample_sizes(cores)]
    for _ in range(args.warmup):
        _cpu_sample(cores, [1, 1, 1])
    vals, times = [], []
    desc = ""
    for _ in range(args.steps):
        t0 = time.perf_counter()
        v, desc, _ = _cpu_sample(cores, sizes)
        times.append(time.perf_counter() - t0)
        vals.append(v)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "orbit-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 oracle", "orbits_per_gpu": [o for _, o in CONFIGS]},
        "cpu_baseline": {"value": value, "unit": "orbit-steps/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: " + desc + "; rate scaled to the workload's orbit mix"},
        "e2e": {"value": value, "unit": "orbit-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import build as sdeb_build
    from paper_1908_03869_gb300.integrator import Integrator

    ws, rank, local = _dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")          # timing only: barrier and max over ranks
    if rank == 0 or not os.path.exists(sdeb_build.LIB_PATH):
        sdeb_build.build()
    if dist is not None:
        dist.barrier()
    sdeb.lib()

    stream = torch.cuda.Stream()
    dev = torch.cuda.current_device()
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = ClockSampler(dev)
    clocks.start()
    rates = {p: sdeb.sdeb_pipe_rate(p, 2048 if p.startswith("sfu") else 256, stream)
             for p in ("sfu_sin", "fp64_fma")}

    dtype = torch.float32
    its, dev_inputs, host_inputs, inputs_by_n = [], [], [], {}
    for n, orbits in CONFIGS:
        p, x0 = _main_inputs(n, orbits)
        inputs_by_n[n] = (p, x0)
        pb = sdeb.Problem.make("kuramoto", n, orbits, DT, STEPS, STRIDE, SEED, "fp32")
        its.append(Integrator(pb))
        pt, xt = torch.from_numpy(p), torch.from_numpy(x0)
        dev_inputs.append((pt.cuda(), xt.cuda()))
        host_inputs.append((pt.pin_memory(), xt.pin_memory()))
    # pick each problem's lane-group layout once, outside the timed region
    layouts = {}
    for i, it in enumerate(its):
        it.set_params(*dev_inputs[i], stream=stream)
        if not args.no_autotune:
            it.autotune(trial_steps=64, stream=stream)
        layouts[str(it.pb.n)] = list(it.layout())
    torch.cuda.synchronize()
    units_per_step = sum(o * STEPS for _, o in CONFIGS)
    osc_per_step = sum(n * o * STEPS for n, o in CONFIGS)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")  # 512 MiB > 129 MB L2

    def one_step(kernel_events=None):
        for i, it in enumerate(its):
            it.set_params(*dev_inputs[i], stream=stream)
            if kernel_events is not None:
                kernel_events[i][0].record(stream)
            it.integrate(stream=stream)
            if kernel_events is not None:
                kernel_events[i][1].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            one_step()
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM --------------------
    step_ev = [_events() for _ in range(args.steps)]
    kern_ev = [[_events() for _ in CONFIGS] for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(s & 0xFF)  # evict L2 between timed steps (outside the step's events)
            step_ev[s][0].record(stream)
            one_step(kern_ev[s])
            step_ev[s][1].record(stream)
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    if dist is not None:
        dist.barrier()
    clk = clocks.summary(wall0, wall1)
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    kern_ms = [[a.elapsed_time(b) for a, b in row] for row in kern_ev]
    total_ms = max_over_ranks(sum(step_ms), dist)
    value = units_per_step * ws * args.steps / (total_ms / 1e3)

    # ---- roofline of the dominant kernel (forward EM, FP32) --------------
    sm_mhz = clocks.median_mhz(wall0, wall1)
    kernel_s = sum(sum(r) for r in kern_ms) / 1e3
    sfu_ops = SFU_OPS_PER_OSC_STEP * osc_per_step * args.steps
    achieved = sfu_ops / kernel_s / 1e9
    peak = rates["sfu_sin"] * num_sms * sm_mhz * 1e6 / 1e9
    per_launch_ms = {str(n): statistics.mean(r[i] for r in kern_ms) for i, (n, _) in enumerate(CONFIGS)}
    full_size = args.orbit_scale == 1.0 and args.horizon is None

    # the legs' first orbits for the error against the oracle (outside any timed region)
    samples = {"main": {}}
    for (n, orbits), it in zip(CONFIGS, its):
        fr = it.frames(stream=stream)
        samples["main"][n] = fr[:, :ERR_ORBITS].cpu().numpy()
        del fr
    torch.cuda.synchronize()

    # ---- end to end through the C ABI with pinned host buffers ----------
    e2e = None
    if not args.no_e2e:
        e2e = _time_e2e(its, host_inputs, stream, dist, ws, args.steps, units_per_step, dtype)

    # ---- the other legs --------------------------------------------------
    legs = {}
    if not args.no_fp64:
        legs["fp64"] = _time_fp64(stream, flush, clocks, rates, num_sms, samples)
    if not args.no_adjoint:
        legs["adjoint"] = _time_adjoint(stream, samples)
    if not args.no_fhn:
        legs["fhn"] = _time_fhn(stream, clocks, rates, num_sms, samples)
    if not args.no_rk4:
        legs["ode"] = _time_ode(stream, clocks, rates, num_sms, samples)
    if not args.no_swarm:
        legs["swarm_search"] = _time_swarm(stream)
    if not args.no_user_model:
        legs["user_model"] = _time_user_model(stream, samples)
    if not args.no_paper_protocol:
        legs["paper_speed_protocol"] = _time_paper_protocol(stream, samples)
        legs["paper_accuracy_protocol"] = _paper_accuracy_protocol(stream, samples)
    if not args.no_batched:
        legs["batched"] = _time_batch(stream, clocks, rates, num_sms, samples)
    for it in its:
        it.close()

    # ---- CPU oracle on this host's cores, and the legs' errors against it
    cpu, errors = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, errors = _cpu_leg(inputs_by_n, samples, legs)

    if rank == 0:
        traffic = counter("forward_n32_dram_bytes") if full_size else None
        line = {
            "metric": METRIC, "value": value, "unit": "orbit-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp32 Kahan", "orbits_per_gpu": [o for _, o in CONFIGS],
                       "n": [n for n, _ in CONFIGS], "dt": DT, "steps_per_orbit": STEPS, "stride": STRIDE,
                       "l2": "flushed between steps (512 MiB write)",
                       "parallelism": "one replica of the workload per GPU, no data exchange"},
            "gpu_launches": len(CONFIGS) * args.steps,
            "oscillator_steps_per_sec": value * osc_per_step / units_per_step,
            "wall_s": wall1 - wall0, "per_launch_ms": per_launch_ms, "layouts_G_P": layouts,
            "roofline": {"bound": "alu", "pipe": "SFU (MUFU)", "achieved": achieved, "peak": peak,
                         "unit": "Gop/s", "frac": achieved / peak, "traffic": traffic,
                         "traffic_note": "ncu DRAM bytes of the n=32 launch for the current kernel sources "
                                         "(null if not captured for them); algorithmic 3.52e9",
                         "peak_source": "sdeb_pipe_rate sin %.2f/clk/SM x %d SMs x %.0f MHz (median sampled)"
                                        % (rates["sfu_sin"], num_sms, sm_mhz),
                         "ops_per_osc_step": SFU_OPS_PER_OSC_STEP},
            "pipe_rates_per_clk_per_sm": rates,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        line.update(legs)
        line["err_vs_oracle"] = errors
        line["targets"] = _targets(line, legs, errors)
        print(json.dumps(line), flush=True)
    clocks.stop()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _time_e2e(its, host_inputs, stream, dist, ws, steps, units_per_step, dtype):
    import torch
    host_frames = [torch.empty((it.nframes, it.pb.orbits, it.pb.n), dtype=dtype, pin_memory=True) for it in its]
    h2d = sum(p.numel() * p.element_size() + x.numel() * x.element_size() for p, x in host_inputs)
    d2h = sum(f.numel() * f.element_size() for f in host_frames)
    # The horizon runs in E2E_CHUNKS ranges; each range's frames go to the
    # host on a second stream while the next range (or problem) computes.
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in its]
    for ev in copied:
        ev.record(copy_stream)

    def e2e_step():
        for i, it in enumerate(its):
            stream.wait_event(copied[i])      # the previous step's frames of this problem are out
            it.set_params(*host_inputs[i], stream=stream, async_host=True)
            f_done = 0
            for c in range(E2E_CHUNKS):
                k0, k1 = c * STEPS // E2E_CHUNKS, (c + 1) * STEPS // E2E_CHUNKS
                it.integrate_range(k0, k1, stream=stream)
                ready = torch.cuda.Event()
                ready.record(stream)
                copy_stream.wait_event(ready)
                f_end = k1 // STRIDE + 1
                it.frames(begin=f_done, count=f_end - f_done, out=host_frames[i][f_done:f_end],
                          stream=copy_stream, async_host=True)
                f_done = f_end
            copied[i].record(copy_stream)

    e2e_step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    return {"value": units_per_step * ws * steps / e2e_s, "unit": "orbit-steps/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "pipeline": "%d integrate_range chunks per problem; frames to pinned host memory on a second stream "
                        "while the next chunk computes" % E2E_CHUNKS}


def _time_fp64(stream, flush, clocks, rates, num_sms, samples, steps64=1000, reps=5):
    """The same three problems in FP64 on the first 1000 of the 10^4 steps
    (the cost per step is constant), median of 5 runs, L2 flushed between
    runs.  FP64-pipe roofline: FP64-pipe instructions per oscillator-step
    (ncu, current kernel sources only) x oscillator-steps/s against the
    measured DFMA rate x SMs x the sampled SM clock."""
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300.integrator import Integrator

    out = {"workload": "kuramoto n=8/32/128, 2^20/2^18/2^16 orbits, first %d steps, fp64" % steps64,
           "reps": reps, "per_problem_ms": {}}
    t_sum, units, osc = 0.0, 0, 0
    t0 = time.perf_counter()
    samples["fp64"] = {}
    for n, orbits in CONFIGS:
        p, x0 = _main_inputs(n, orbits)
        pb = sdeb.Problem.make("kuramoto", n, orbits, DT, steps64, STRIDE, SEED, "fp64")
        with Integrator(pb) as it:
            pt, xt = torch.from_numpy(p).double().cuda(), torch.from_numpy(x0).double().cuda()

            ms, _ = _timed(lambda: it.integrate(stream=stream), stream, reps, flush,
                           prep=lambda: it.set_params(pt, xt, stream=stream))
            samples["fp64"][n] = it.frames(stream=stream)[:, :ERR_ORBITS].cpu().numpy()
        out["per_problem_ms"][str(n)] = ms
        t_sum += ms / 1e3
        units += orbits * steps64
        osc += n * orbits * steps64
    mhz = clocks.median_mhz(t0, time.perf_counter())
    out["orbit_steps_per_sec"] = units / t_sum
    out["osc_steps_per_sec"] = osc / t_sum
    inst = counter("fp64_pipe_inst_per_osc_step")
    peak = rates["fp64_fma"] * num_sms * mhz * 1e6
    out["fp64_pipe"] = {"inst_per_osc_step": inst, "peak_inst_per_sec": peak,
                        "frac": (inst * out["osc_steps_per_sec"] / peak) if inst else None,
                        "sm_mhz": mhz}
    return out


def _time_adjoint(stream, samples, reps=5):
    import ctypes

    import numpy as np
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator

    W = inputs.WORKLOADS["kuramoto_adjoint_n32"]
    n, orbits = W["n"], W["orbits"]
    p, x0 = inputs.kuramoto(n, orbits, seed=1, shared=True)
    pt = torch.tensor(p, dtype=torch.float32, device="cuda")
    xt = torch.tensor(x0, dtype=torch.float32, device="cuda")
    mk = lambda ck, o=orbits, shared=True: sdeb.Problem.make(
        "kuramoto", n, o, W["dt"], W["steps"], 1, W["seed"], "fp32", ckpt_every=ck, no_frames=True,
        shared_params=shared)
    with Integrator(mk(0)) as plain, Integrator(mk(W["ckpt_every"])) as ck:
        # each context tuned for what it runs: the plain forward alone, the
        # checkpointed context for forward + adjoint
        for it in (plain, ck):
            it.set_params(pt, xt, stream=stream)
            it.autotune(trial_steps=64, stream=stream)
        lay, fwd_lay = ck.layout(), plain.layout()
        ck_int = sdeb.sdeb_get_checkpoint_interval(ck.ctx)
        ck.integrate(stream=stream)
        xK = ck.final(stream=stream)
        r = torch.empty(orbits, dtype=torch.float32, device="cuda")
        dr = torch.empty_like(xK)
        torch.cuda.synchronize()
        sdeb.sdeb_order_param(ctypes.c_void_p(xK.data_ptr()), orbits, n, 0, ctypes.c_void_p(r.data_ptr()),
                              ctypes.c_void_p(dr.data_ptr()), stream)
        dL = (dr / orbits).contiguous()
        torch.cuda.synchronize()
        t_plain, t_fwd, t_adj = [], [], []
        for _ in range(reps + 1):
            a, b, c, d, e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            plain.set_params(pt, xt, stream=stream)
            a.record(stream)
            plain.integrate(stream=stream)
            b.record(stream)
            ck.set_params(pt, xt, stream=stream)
            c.record(stream)
            ck.integrate(stream=stream)
            d.record(stream)
            ck.grad(dL, stream=stream)
            e.record(stream)
            torch.cuda.synchronize()
            t_plain.append(a.elapsed_time(b))
            t_fwd.append(c.elapsed_time(d))
            t_adj.append(d.elapsed_time(e))
    t_plain, t_fwd, t_adj = [statistics.median(t[1:]) for t in (t_plain, t_fwd, t_adj)]
    # per-orbit gradients of the first orbits for the error against the oracle
    k = 8
    with Integrator(mk(W["ckpt_every"], k, False)) as it:
        it.set_params(torch.tensor(np.tile(p, (k, 1)), dtype=torch.float32, device="cuda"), xt[:k].contiguous(),
                      stream=stream)
        it.integrate(stream=stream)
        xk = it.final(stream=stream)
        dr8 = torch.empty_like(xk)
        r8 = torch.empty(k, dtype=torch.float32, device="cuda")
        sdeb.sdeb_order_param(ctypes.c_void_p(xk.data_ptr()), k, n, 0, ctypes.c_void_p(r8.data_ptr()),
                              ctypes.c_void_p(dr8.data_ptr()), stream)
        torch.cuda.synchronize()          # dr8 is written on `stream`, divided on torch's current stream
        dL8 = (dr8 / orbits).contiguous()
        torch.cuda.synchronize()
        dp, _ = it.grad(dL8, stream=stream)
        torch.cuda.synchronize()
        samples["adjoint"] = {"p": p.astype(np.float32), "x0": x0[:k].astype(np.float32), "dp": dp.cpu().numpy(),
                              "W": W, "orbits": orbits}
    units = orbits * W["steps"]
    return {"workload": "kuramoto n=32, 16384 orbits, shared params, dt=0.01, 2000 steps, ckpt every 100, fp32",
            "layout_G_P": list(lay), "fwd_layout_G_P": list(fwd_lay), "ckpt_interval": ck_int,
            "fwd_ms": t_plain, "fwd_ckpt_ms": t_fwd, "adjoint_ms": t_adj,
            "fwd_plus_adjoint_orbit_steps_per_sec": units / ((t_fwd + t_adj) / 1e3),
            "fwd_orbit_steps_per_sec": units / (t_plain / 1e3),
            "ratio_fwd_plus_adjoint_to_fwd": (t_fwd + t_adj) / t_plain}


def _time_fhn(stream, clocks, rates, num_sms, samples, reps=3, steps=10000, steps64=1000):
    """The FitzHugh-Nagumo network (64 units, n = 128, 2^18 orbits, dt =
    0.01, frame every 1000 steps): FP32 Euler-Maruyama and Milstein on the
    first 10^4 of its 10^5 steps, FP64 Euler-Maruyama on the first 10^3 (the
    cost per step is constant)."""
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator

    W = inputs.WORKLOADS["fhn_64units"]
    n, orbits = W["n"], W["orbits"]
    p, x0 = inputs.fhn(n // 2, orbits, seed=1)
    out = {"workload": "FitzHugh-Nagumo network, 64 units (n = 128), 2^18 orbits, dt = 0.01, frame every %d steps"
                       % W["stride"]}
    samples["fhn"] = {"p": p[:ERR_ORBITS], "x0": x0[:ERR_ORBITS]}
    t0 = time.perf_counter()
    for name, mil, prec, k in (("euler_maruyama", False, "fp32", steps), ("milstein", True, "fp32", steps),
                               ("euler_maruyama_fp64", False, "fp64", steps64)):
        dt_t = torch.float64 if prec == "fp64" else torch.float32
        pt, xt = torch.tensor(p, dtype=dt_t, device="cuda"), torch.tensor(x0, dtype=dt_t, device="cuda")
        pb = sdeb.Problem.make("fhn_net", n, orbits, W["dt"], k, W["stride"], W["seed"], prec, milstein=mil)
        with Integrator(pb) as it:
            ms, _ = _timed(lambda: it.integrate(stream=stream), stream, reps,
                           prep=lambda: it.set_params(pt, xt, stream=stream))
            fr = it.frames(stream=stream)
            samples["fhn"][name] = fr[:, :ERR_ORBITS].cpu().numpy()       # frames at t = 0, 10, ...
            del fr
        out[name] = {"steps": k, "ms": ms, "unit_steps_per_sec": orbits * (n // 2) * k / (ms / 1e3)}
    mhz = clocks.median_mhz(t0, time.perf_counter())
    out["milstein_time_over_em"] = out["milstein"]["ms"] / out["euler_maruyama"]["ms"]
    # one normal per unit-step: half of (log2, sqrt, sin, cos) = 2 SFU operations
    out["sfu_roofline_frac_em"] = 2.0 * out["euler_maruyama"]["unit_steps_per_sec"] / (
        rates["sfu_sin"] * num_sms * mhz * 1e6)
    return out


# A FitzHugh-Nagumo network written as a user-defined model (the run-time
# compiled path, diagonal-noise form; x = (v_1..v_u, w_1..w_u),
# p = (a, b, eps, I, c, sigma)).
USER_FHN_SOURCE = r"""
#define SDEB_DIAGONAL_NOISE 1
__device__ void sdeb_drift(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *f) {
    const int u = SDEB_N / 2;
    sdeb_real mean = 0;
    for (int i = 0; i < u; ++i) mean += x[i];
    mean /= u;
    for (int i = 0; i < u; ++i) {
        const sdeb_real v = x[i], w = x[u + i];
        f[i] = v - v * v * v / 3 - w + p[3] + p[4] * mean - p[4] * v;
        f[u + i] = p[2] * (v + p[0] - p[1] * w);
    }
}
__device__ void sdeb_diffusion(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *g) {
    for (int j = 0; j < SDEB_M; ++j) g[j] = p[5] * x[j];
}
"""


def _time_user_model(stream, samples, reps=3, steps=1000):
    """A FitzHugh-Nagumo network of 16 units (n = 32) on 2^18 orbits, dt =
    0.01, 1000 steps, FP32: compile time of the run-time compiled user model
    and its unit-steps/s beside the built-in model's."""
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits = 32, 1 << 18
    p, x0 = inputs.fhn(n // 2, orbits, seed=1)
    pt = torch.tensor(p, dtype=torch.float32, device="cuda")
    xt = torch.tensor(x0, dtype=torch.float32, device="cuda")
    out = {"workload": "FitzHugh-Nagumo network, 16 units (n = 32), 2^18 orbits, dt = 0.01, %d steps, fp32" % steps}
    samples["user_model"] = {"p": p[:ERR_ORBITS].astype("float32"), "x0": x0[:ERR_ORBITS].astype("float32"),
                             "steps": steps}
    for name in ("built_in", "user_source"):
        user = name == "user_source"
        pb = sdeb.Problem.make("user" if user else "fhn_net", n, orbits, 0.01, steps, 100, 0, "fp32", m=n // 2, d=6)
        t0 = time.perf_counter()
        it = Integrator(pb, user_source=USER_FHN_SOURCE if user else None)
        create_s = time.perf_counter() - t0
        try:
            ms, _ = _timed(lambda: it.integrate(stream=stream), stream, reps,
                           prep=lambda: it.set_params(pt, xt, stream=stream))
            if user:
                samples["user_model"]["frames"] = it.frames(stream=stream)[:, :ERR_ORBITS].cpu().numpy()
        finally:
            it.close()
        out[name] = {"create_s": create_s, "ms": ms, "unit_steps_per_sec": orbits * (n // 2) * steps / (ms / 1e3)}
    out["user_time_over_built_in"] = out["user_source"]["ms"] / out["built_in"]["ms"]
    return out


# The paper's runtimes of its speed protocol on an NVIDIA P100 (Tables S1-S3,
# M = 163840 orbits, FP64, including OpenCL set-up and host transfers): context
# for the same protocol here, not a target.
PAPER_P100_SECONDS = {5: 4.719, 10: 9.315, 15: 17.656}


def _time_paper_protocol(stream, samples):
    """The paper's speed protocol (Sec. 2.2.1): stochastic Kuramoto in the
    paper's parameter layout p = (K, omega_1..omega_N, p_1..p_N), K = 1,
    omega ~ U(0.01, 0.03), p ~ U(0.001, 0.003), theta(0) ~ U(-pi, pi),
    N = 5 / 10 / 15 oscillators, M = 163840 orbits, dt = 0.05, T = 400 s
    (8000 steps), FP64; a frame every 100 steps.  Device time of the whole
    horizon, and end to end through the C ABI (host inputs in, all frames
    to pinned host memory)."""
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator

    orbits, dt, steps, stride = 163840, 0.05, 8000, 100
    out = {"workload": "paper speed protocol: Kuramoto paper layout, M = 163840, dt = 0.05, 8000 steps, "
                       "frame every 100 steps, fp64",
           "paper_p100_seconds_context": PAPER_P100_SECONDS, "runs": {}}
    samples["paper_speed"] = {}
    for n in (5, 10, 15):
        p, x0 = inputs.kuramoto_paper_speed(n, orbits, seed=1)
        ph, xh = torch.tensor(p).pin_memory(), torch.tensor(x0).pin_memory()
        pd, xd = ph.cuda(), xh.cuda()
        pb = sdeb.Problem.make("kuramoto_paper", n, orbits, dt, steps, stride, 0, "fp64")
        with Integrator(pb) as it:
            host_frames = torch.empty((it.nframes, orbits, n), dtype=torch.float64, pin_memory=True)
            it.set_params(pd, xd, stream=stream)
            it.integrate_range(0, 100, stream=stream)          # warm-up
            torch.cuda.synchronize()
            it.set_params(pd, xd, stream=stream)
            a, b = _events()
            a.record(stream)
            it.integrate(stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            dev_s = a.elapsed_time(b) / 1e3
            t0 = time.perf_counter()
            it.set_params(ph, xh, stream=stream)
            it.integrate(stream=stream)
            it.frames(out=host_frames, stream=stream)
            torch.cuda.synchronize()
            e2e_s = time.perf_counter() - t0
        samples["paper_speed"][n] = {"p": p[:16], "x0": x0[:16], "frames": host_frames[:, :16].numpy().copy()}
        del host_frames
        out["runs"][str(n)] = {"device_s": dev_s, "e2e_s": e2e_s,
                               "orbit_steps_per_sec": orbits * steps / dev_s,
                               "e2e_orbit_steps_per_sec": orbits * steps / e2e_s}
    return out


def _paper_accuracy_protocol(stream, samples):
    """The paper's accuracy protocol (Sec. 2.3.1): N = 100, 64 realisations,
    omega ~ U(0.2, 0.4), theta(0) ~ U(-pi, pi), p ~ U(0.01, 0.03),
    K = 0.02 and 0.2, 400 s, dt = 2^(l-5)/5 for l = 1..5, FP64: the mean and
    standard deviation over realisations of the coherence r(t_MAX) (Eq. 7),
    from the FP64 moment accumulators on the GPU (sdeb_frame_moments), and
    the device time of each run."""
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits = 100, 64
    out = {"workload": "paper accuracy protocol: Kuramoto paper layout, N = 100, 64 realisations, 400 s, fp64",
           "runs": []}
    samples["paper_accuracy"] = []
    for K in (0.02, 0.2):
        p, x0 = inputs.kuramoto_paper_accuracy(K, orbits=orbits, n=n, seed=1)
        pd, xd = torch.tensor(p).cuda(), torch.tensor(x0).cuda()
        for l in range(1, 6):
            dt = 2.0 ** (l - 5) / 5
            steps = int(round(400 / dt))
            pb = sdeb.Problem.make("kuramoto_paper", n, orbits, dt, steps, steps, 0, "fp64")
            with Integrator(pb) as it:
                it.set_params(pd, xd, stream=stream)
                a, b = _events()
                a.record(stream)
                it.integrate(stream=stream)
                b.record(stream)
                _, rmom = it.moments(begin=1, count=1, state=False, order_param=True, stream=stream)
                torch.cuda.synchronize()
                rmean, rvar = [float(v) for v in rmom[0].cpu()]
            out["runs"].append({"K": K, "dt": dt, "r_mean": rmean, "r_sd": math.sqrt(rvar),
                                "device_ms": a.elapsed_time(b)})
            if l == 5:
                samples["paper_accuracy"].append({"K": K, "dt": dt, "steps": steps, "p": p, "x0": x0,
                                                  "r_mean": rmean, "r_sd": math.sqrt(rvar)})
    return out


def _time_swarm(stream, generations=5, particles=1024, realisations=64, n=32, steps=1000):
    """Particle swarm search over (K, sigma) of the Kuramoto model: 1024
    particles x 64 realisations = 2^16 orbits of n = 32, dt = 0.005, 1000
    steps, FP32, target order parameter 0.8.  A generation is expand +
    set_params + integrate + read_final + fitness + update on one stream;
    timed over 5 generations after one untimed one, beside set_params +
    integrate alone."""
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.swarm import SwarmSearch

    p, x0 = inputs.kuramoto(n, realisations, seed=11)
    base = p[0].copy()
    pb = sdeb.Problem.make("kuramoto", n, 1, DT, steps, steps, SEED, "fp32")
    g = torch.Generator().manual_seed(3)
    x_init = torch.rand((particles, 2), generator=g, dtype=torch.float64) * torch.tensor([4.0, 0.5])
    v_init = torch.zeros((particles, 2), dtype=torch.float64)
    orbit_steps = particles * realisations * steps
    out = {"workload": "Kuramoto n = %d, %d particles x %d realisations, dt = %g, %d steps, fp32, search over "
                       "(K, sigma), target r = 0.8" % (n, particles, realisations, DT, steps)}
    with SwarmSearch(pb, base, x0, [0, 1], [0.0, 0.0], [4.0, 0.5], particles, r_target=0.8, swarm_seed=7) as s:
        s.reset(x_init, v_init)
        with torch.cuda.stream(stream):
            s.step(stream)
            torch.cuda.synchronize()
            a, b = _events()
            a.record(stream)
            for _ in range(generations):
                s.step(stream)
            b.record(stream)
            torch.cuda.synchronize()
            gen_ms = a.elapsed_time(b) / generations
            a.record(stream)
            for _ in range(generations):
                s.it.set_params(s.params, s.x0_all, stream=stream)
                s.it.integrate(stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            integ_ms = a.elapsed_time(b) / generations
            _, best_fit = s.best()
    out.update({"ms_per_generation": gen_ms, "orbit_steps_per_sec": orbit_steps / (gen_ms / 1e3),
                "integration_ms": integ_ms, "integration_share": integ_ms / gen_ms,
                "best_fitness_after": best_fit, "generations_run": generations + 1})
    return out


def _time_ode(stream, clocks, rates, num_sms, samples, reps=3, steps=1000):
    """The ODE path: classical fourth-order Runge-Kutta, implicit Euler and
    the implicit midpoint rule (4 Newton iterations a step) on the drift of
    the n = 32 benchmark problem (2^18 orbits, dt = 0.005, frame every 100
    steps), FP32, first 1000 steps, beside Euler-Maruyama on the same steps."""
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits = 32, 1 << 18
    p, x0 = _main_inputs(n, orbits)
    pt, xt = torch.from_numpy(p).cuda(), torch.from_numpy(x0).cuda()
    out = {"workload": "Kuramoto n = 32, 2^18 orbits, dt = %g, first %d steps, frame every %d steps, fp32"
                       % (DT, steps, STRIDE)}
    samples["ode"] = {"p": p[:ERR_ORBITS], "x0": x0[:ERR_ORBITS], "steps": steps}
    schemes = (("euler_maruyama", {}), ("rk4", {"rk4": True}), ("implicit_euler", {"implicit": "euler"}),
               ("implicit_midpoint", {"implicit": "midpoint"}))
    t0 = time.perf_counter()
    for name, kw in schemes:
        pb = sdeb.Problem.make("kuramoto", n, orbits, DT, steps, STRIDE, SEED, "fp32", **kw)
        with Integrator(pb) as it:
            ms, _ = _timed(lambda: it.integrate(stream=stream), stream, reps,
                           prep=lambda: it.set_params(pt, xt, stream=stream))
            if name != "euler_maruyama":
                samples["ode"][name] = it.frames(stream=stream)[:, :ERR_ORBITS].cpu().numpy()
        out[name] = {"ms": ms, "orbit_steps_per_sec": orbits * steps / (ms / 1e3)}
    peak = rates["sfu_sin"] * num_sms * clocks.median_mhz(t0, time.perf_counter()) * 1e6
    # four drift evaluations per step, each a sin and a cos per oscillator
    out["sfu_roofline_frac_rk4"] = 8.0 * n * out["rk4"]["orbit_steps_per_sec"] / peak
    out["rk4_time_over_em"] = out["rk4"]["ms"] / out["euler_maruyama"]["ms"]
    # four Newton iterations per step, each a sin, a cos and a reciprocal per oscillator
    for name in ("implicit_euler", "implicit_midpoint"):
        out["sfu_roofline_frac_" + name] = 12.0 * n * out[name]["orbit_steps_per_sec"] / peak
        out[name + "_time_over_em"] = out[name]["ms"] / out["euler_maruyama"]["ms"]
    return out


def _time_batch(stream, clocks, rates, num_sms, samples, reps=5):
    import numpy as np
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import BatchIntegrator

    W = inputs.WORKLOADS["batched_4096"]
    insts = inputs.batched_instances(W["count"], seed=1)
    pbs = [sdeb.Problem.make("kuramoto", d["n"], 1, d["dt"], d["steps"], W["stride"], W["seed"], "fp32",
                             orbit_offset=i) for i, d in enumerate(insts)]
    ps = [d["params"][None, :].astype(np.float32) for d in insts]
    xs = [d["x0"][None, :].astype(np.float32) for d in insts]
    orbit_steps = sum(d["steps"] for d in insts)
    osc_steps = sum(d["steps"] * d["n"] for d in insts)
    work = [d["n"] * d["steps"] for d in insts]
    pick = sorted(set([0, 1, 2047, 4095, int(np.argmax(work)), int(np.argmax([d["steps"] for d in insts]))]))
    with BatchIntegrator(pbs) as b:
        b.set_params(ps, xs, stream=stream)
        info = b.autotune(stream=stream)
        t0 = time.perf_counter()

        ms, _ = _timed(lambda: b.integrate(stream=stream), stream, reps,
                       prep=lambda: b.set_params(ps, xs, stream=stream))
        mhz = clocks.median_mhz(t0, time.perf_counter())
        samples["batched"] = [{"i": i, "n": insts[i]["n"], "dt": insts[i]["dt"], "steps": insts[i]["steps"],
                               "p": ps[i], "x0": xs[i], "stride": W["stride"], "seed": W["seed"],
                               "frames": b.frames(i, stream=stream).cpu().numpy()} for i in pick]
    peak = rates["sfu_sin"] * num_sms * mhz * 1e6
    return {"workload": "4096 Kuramoto instances, n~U{2..256}, steps~logU[1e3,1e5], dt in {0.001,0.01}, stride 100, "
                        "fp32", "ms": ms, "orbit_steps_per_sec": orbit_steps / (ms / 1e3),
            "osc_steps_per_sec": osc_steps / (ms / 1e3),
            "sfu_roofline_frac": SFU_OPS_PER_OSC_STEP * osc_steps / (ms / 1e3) / peak,
            "total_osc_steps": osc_steps, "longest_instance_osc_steps": max(work), "schedule": info}


# ---------------------------------------------------------------------------
# The CPU leg: the oracle timed on this host, and the legs' errors against it
# ---------------------------------------------------------------------------

def _adjoint_errors(a):
    """Per-orbit gradients of the adjoint leg (a["dp"], FP32) against the FP64
    oracle adjoint of the same orbits, relative to each orbit's largest
    component; beside each, how far the oracle's own gradient moves when x0
    moves by one FP32 ulp (signs fixed per component): an FP32 gradient
    carries a rounding in each of its steps, so an orbit whose one-ulp
    sensitivity is large cannot be followed to 1e-3."""
    import numpy as np

    import oracle

    W, k = a["W"], a["x0"].shape[0]
    n = a["x0"].shape[1]
    pb = oracle.make_problem("kuramoto", n, n, n + 2, W["dt"], W["steps"], 1, W["seed"])
    sign = np.where(np.sin(np.arange(n) * 7.1) >= 0, 1.0, -1.0)

    def oracle_grad(x, o):
        _, xK = oracle.integrate(pb, a["p"][None, :], x, orbit_begin=o, frames=False)
        _, dr = oracle.order_param(xK[0])
        dp, _ = oracle.adjoint(pb, a["p"][None, :], x, (dr / a["orbits"])[None, :], orbit_begin=o)
        return dp[0]

    per, sens = [], []
    for o in range(k):
        x = a["x0"][o:o + 1].astype(np.float64)
        ref = oracle_grad(x, o)
        per.append(float(np.abs(a["dp"][o] - ref).max() / np.abs(ref).max()))
        sens.append(float(np.abs(oracle_grad(x * (1.0 + 2.0 ** -24 * sign), o) - ref).max() / np.abs(ref).max()))
    return {"orbits": k, "max_rel_to_orbit_max": max(per), "per_orbit": per, "oracle_one_ulp_sensitivity": sens,
            "over_1e-3": [{"orbit": o, "err": per[o], "oracle_one_ulp_sensitivity": sens[o]}
                          for o in range(k) if per[o] >= 1e-3]}


def _cpu_leg(inputs_by_n, samples, legs):
    import numpy as np

    import oracle

    cores = os.cpu_count() or 1
    sizes = _sample_sizes(cores)
    v, desc, ofr = _cpu_sample(cores, sizes, inputs_by_n=inputs_by_n)
    v1, desc1, _ = _cpu_sample(1, [max(1, s // cores) for s in sizes], inputs_by_n=inputs_by_n)
    vmf, descmf, _ = _cpu_sample(cores, sizes, mean_field=True, inputs_by_n=inputs_by_n)
    cpu = {"value": v, "unit": "orbit-steps/s", "cores": cores, "kind": "oracle",
           "sample": desc + "; rate scaled to the workload's orbit mix",
           "single_thread": {"value": v1, "cores": 1, "sample": desc1},
           "mean_field_form": {"value": vmf, "cores": cores, "sample": descmf,
                               "note": "the oracle's O(n) mean-field drift instead of the pairwise definition"}}

    t_frames = int(ERR_T / DT) // STRIDE + 1                 # frames up to t = 10
    err = {"metric": "max |x - x_oracle| / max(|x_oracle|, 1) over the first orbits of each leg, frames up to "
                     "t = %g unless stated" % ERR_T}
    # main workload, FP32: the baseline's own oracle results (its first orbits, whole horizon)
    main = {}
    for n, _ in CONFIGS:
        k = min(ERR_ORBITS, ofr[n].shape[1])
        g = samples["main"][n][:, :k]
        per_orbit = _rel_err(g[:t_frames], ofr[n][:t_frames, :k], axis=(0, 2))
        main[str(n)] = {"orbits": k, "t_le_10": float(per_orbit.max()),
                        "t_le_10_median": float(np.median(per_orbit)),
                        "horizon_t_50": _rel_err(g, ofr[n][:, :k])}
        # orbits past the FP32 tolerance: how far the oracle itself departs
        # when its state is rounded like an FP32 state every step
        over = [int(o) for o in np.flatnonzero(per_orbit > 1e-4)]
        main[str(n)]["over_1e-4"] = [
            {"orbit": o, "err": float(per_orbit[o]),
             "oracle_fp32_rounding_departure": _fp32_rounding_departure(n, inputs_by_n[n], o, t_frames)}
            for o in over[:4]]
    err["forward_fp32"] = main
    thr = max(1, cores)

    def run_oracle(model, n, p, x0, dt, steps, stride, seed=0, mean_field=False, orbit_begin=0, **kw):
        m, d = {"kuramoto": (n, n + 2), "kuramoto_paper": (n, 2 * n + 1), "fhn_net": (n // 2, 6)}[model]
        pb = oracle.make_problem(model, n, m, d, dt, steps, stride, seed, mean_field=mean_field, **kw)
        fr, _ = oracle.integrate(pb, np.asarray(p, np.float64), np.asarray(x0, np.float64), orbit_begin=orbit_begin,
                                 nthreads=thr)
        return fr

    if "fp64" in samples:
        e = {}
        for n, _ in CONFIGS:
            g = samples["fp64"][n]
            e[str(n)] = _rel_err(g, run_oracle("kuramoto", n, inputs_by_n[n][0][:ERR_ORBITS],
                                               inputs_by_n[n][1][:ERR_ORBITS], DT, (g.shape[0] - 1) * STRIDE,
                                               STRIDE, mean_field=True))
        err["forward_fp64_t_le_5"] = e
    if "adjoint" in samples:
        err["adjoint_fp32_per_orbit_T20"] = _adjoint_errors(samples["adjoint"])
    if "fhn" in samples:
        f = samples["fhn"]
        W = {"dt": 0.01, "stride": 1000}
        p32, x32 = f["p"].astype(np.float32), f["x0"].astype(np.float32)
        ref32 = run_oracle("fhn_net", 128, p32, x32, W["dt"], 1000, W["stride"])
        ref_mil = run_oracle("fhn_net", 128, p32, x32, W["dt"], 1000, W["stride"], milstein=True)
        ref64 = run_oracle("fhn_net", 128, f["p"], f["x0"], W["dt"], 1000, W["stride"])
        err["fhn"] = {"euler_maruyama_fp32": _rel_err(f["euler_maruyama"][:2], ref32),
                      "milstein_fp32": _rel_err(f["milstein"][:2], ref_mil),
                      "euler_maruyama_fp64": _rel_err(f["euler_maruyama_fp64"][:2], ref64)}
    if "ode" in samples:
        o = samples["ode"]
        e = {}
        for name, kw in (("rk4", {"rk4": True}), ("implicit_euler", {"implicit": "euler"}),
                         ("implicit_midpoint", {"implicit": "midpoint"})):
            ref = run_oracle("kuramoto", 32, o["p"], o["x0"], DT, o["steps"], STRIDE, **kw)
            e[name + "_t_le_2"] = _rel_err(o[name][:5], ref[:5])
            e[name + "_t_le_5"] = _rel_err(o[name], ref)
        err["ode_fp32"] = e
    if "user_model" in samples:
        u = samples["user_model"]
        ref = run_oracle("fhn_net", 32, u["p"], u["x0"], 0.01, u["steps"], 100)
        err["user_model_fhn_fp32"] = _rel_err(u["frames"], ref)
    if "paper_speed" in samples:
        e = {}
        for n, s in samples["paper_speed"].items():
            ref = run_oracle("kuramoto_paper", n, s["p"], s["x0"], 0.05, 8000, 100)
            e[str(n)] = {"t_le_10": _rel_err(s["frames"][:3], ref[:3]), "horizon_t_400": _rel_err(s["frames"], ref)}
        err["paper_speed_fp64"] = e
    if "paper_accuracy" in samples:
        e = []
        for s in samples["paper_accuracy"]:
            ref = run_oracle("kuramoto_paper", 100, s["p"], s["x0"], s["dt"], s["steps"], s["steps"],
                             mean_field=True)
            _, rm = oracle.frame_moments(ref[1:], order_parameter=True)
            e.append({"K": s["K"], "dt": s["dt"], "r_mean_abs_err": abs(s["r_mean"] - rm[0, 0]),
                      "r_sd_abs_err": abs(s["r_sd"] - math.sqrt(rm[0, 1]))})
        err["paper_accuracy_fp64_r_stats"] = e
    if "batched" in samples:
        e = {}
        for s in samples["batched"]:
            kmax = min(s["steps"], int(round(ERR_T / s["dt"])))
            kmax -= kmax % s["stride"]
            ref = run_oracle("kuramoto", s["n"], s["p"], s["x0"], s["dt"], kmax, s["stride"], seed=s["seed"],
                             mean_field=True, orbit_begin=s["i"]) if kmax > 0 else None
            e[str(s["i"])] = _rel_err(s["frames"][:ref.shape[0]], ref) if ref is not None else 0.0
        err["batched_fp32_sampled_instances"] = e
    return cpu, err


def _fp32_rounding_departure(n, inputs_n, orbit, frames):
    """max over the first `frames` frames of the departure of the oracle
    (mean-field form) from itself when its state is multiplied by
    (1 + s 2^-24), s a random sign per component, after every step: the
    error the dynamics alone give an orbit integrated with FP32 roundings."""
    import numpy as np

    import oracle

    p, x0 = inputs_n
    pr = p[orbit:orbit + 1].astype(np.float64)
    x = x0[orbit:orbit + 1].astype(np.float64)
    steps = (frames - 1) * STRIDE
    pb = oracle.make_problem("kuramoto", n, n, n + 2, DT, steps, 1, SEED, mean_field=True)
    ref, _ = oracle.integrate(pb, pr, x, orbit_begin=orbit)
    rng = np.random.Generator(np.random.PCG64(orbit))
    d = 0.0
    for k in range(steps):
        x = x * (1.0 + 2.0 ** -24 * rng.choice([-1.0, 1.0], size=x.shape))
        _, x = oracle.integrate(pb, pr, x, orbit_begin=orbit, k_begin=k, k_end=k + 1, frames=False)
        d = max(d, _rel_err(x, ref[k + 1]))
    return d


def _targets(line, legs, errors):
    """The figures the design is held to, in one short object at the end of
    the line."""
    def g(d, *keys):
        for k in keys:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    t = {"fp32_forward_sfu_frac": g(line, "roofline", "frac"),
         "fp32_forward_orbit_steps_per_sec": line["value"],
         "e2e_orbit_steps_per_sec": g(line, "e2e", "value"),
         "fp64_orbit_steps_per_sec": g(legs, "fp64", "orbit_steps_per_sec"),
         "fp64_pipe_frac": g(legs, "fp64", "fp64_pipe", "frac"),
         "adjoint_ratio_fwd_plus_adj_to_fwd": g(legs, "adjoint", "ratio_fwd_plus_adjoint_to_fwd"),
         "batched_sfu_frac": g(legs, "batched", "sfu_roofline_frac"),
         "fhn_fp32_unit_steps_per_sec": g(legs, "fhn", "euler_maruyama", "unit_steps_per_sec"),
         "fhn_fp64_unit_steps_per_sec": g(legs, "fhn", "euler_maruyama_fp64", "unit_steps_per_sec")}
    if errors:
        m = errors.get("forward_fp32", {})
        t["err_fp32_t_le_10"] = max((v["t_le_10"] for v in m.values()), default=None)
        t["err_fp64_t_le_5"] = max(errors.get("forward_fp64_t_le_5", {}).values(), default=None)
        t["err_adjoint_fp32_T20"] = g(errors, "adjoint_fp32_per_orbit_T20", "max_rel_to_orbit_max")
        t["err_fhn_fp32_fp64"] = [g(errors, "fhn", "euler_maruyama_fp32"), g(errors, "fhn", "euler_maruyama_fp64")]
        t["err_batched_fp32"] = max(errors.get("batched_fp32_sampled_instances", {}).values(), default=None)
    return t


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    for leg in ("e2e", "fp64", "cpu-baseline", "adjoint", "autotune", "batched", "fhn", "rk4", "paper-protocol",
                "user-model", "swarm"):
        ap.add_argument("--no-" + leg, action="store_true")
    ap.add_argument("--orbit-scale", type=float, default=1.0,
                    help="scale the orbit counts (profiling runs only; the benchmark uses 1)")
    ap.add_argument("--horizon", type=int, default=None,
                    help="steps per orbit (profiling runs only; the benchmark uses 10^4)")
    args = ap.parse_args()
    global CONFIGS, STEPS, WORKLOAD
    if args.orbit_scale != 1.0 or args.horizon is not None:
        CONFIGS = [(n, max(1, int(o * args.orbit_scale))) for n, o in CONFIGS]
        STEPS = args.horizon if args.horizon is not None else STEPS
        WORKLOAD = "profiling case: n=8/32/128, orbits %s, %d steps" % ([o for _, o in CONFIGS], STEPS)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
