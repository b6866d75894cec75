"""Benchmark: orbit-steps/s of many-orbit Euler-Maruyama on one GB300.

Workload (one "step" = one pass of the whole hot path over one batch):
stochastic Kuramoto, scalar-sigma layout, n = 8 / 32 / 128 with
2^20 / 2^18 / 2^16 orbits, dt = 0.005, 10^4 Euler-Maruyama steps per orbit,
a frame every 100 steps, Philox seed 0; FP32 with Kahan-compensated state.
Per step: reload the parameters and initial states from device memory, then
integrate all three problems over the full horizon (frames written to HBM).

The JSON line carries: the device-timed value (inputs resident in HBM), an
end-to-end value through the C ABI with pinned host buffers (host->device
inputs and device->host frames inside the timed region), a roofline entry
for the dominant kernel (the forward Euler-Maruyama kernel, bound by the
SFU / special-function pipe), the same workload in FP64 on a 1000-step
prefix of the horizon, the discrete adjoint against its forward, the
batched heterogeneous workload, the FitzHugh-Nagumo network under
Euler-Maruyama and Milstein, the ODE path (fourth-order Runge-Kutta), a
user-defined model compiled at run time, the paper's own speed and accuracy
protocols in FP64, and the CPU oracle timed on this host's cores on a
bounded sample.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
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
SFU_PER_SM_PER_CLK = 16
NUM_SMS = 152
SM_MAX_MHZ = 2070.0
# DRAM bytes (read + write) of one forward launch of the n = 32 problem, from
# the ncu capture summarised in profiles/em_forward_kuramoto_fp32_n32_dram_full_size.md;
# set to None whenever the forward kernel changes until it is measured again.
FORWARD_N32_DRAM_BYTES = 3.50e9
E2E_CHUNKS = 4


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_sample(nthreads, budget_orbits, mean_field=False):
    """Oracle (pairwise Kuramoto drift by definition, as it stands; or its
    mean-field form) on the first orbits of each problem, full horizon.
    Returns (orbit-steps/s over the workload mix, description)."""
    import numpy as np

    import oracle
    from paper_1908_03869_gb300 import inputs

    t_total, units_total = 0.0, 0
    desc = []
    for (n, orbits), s in zip(CONFIGS, budget_orbits):
        p, x0 = inputs.kuramoto(n, s, seed=1)
        pb = oracle.make_problem("kuramoto", n, n, n + 2, DT, STEPS, STRIDE, SEED, mean_field=mean_field)
        t0 = time.perf_counter()
        oracle.integrate(pb, p.astype(np.float32).astype(np.float64), x0.astype(np.float32).astype(np.float64),
                         frames=True, nthreads=nthreads)
        dt = time.perf_counter() - t0
        rate = s * STEPS / dt
        # time the full per-GPU problem would take at this rate (workload mix)
        t_total += orbits * STEPS / rate
        units_total += orbits * STEPS
        desc.append("n=%d: first %d orbits x %d steps in %.2fs" % (n, s, STEPS, dt))
    return units_total / t_total, "; ".join(desc)


def _sample_sizes(cores):
    # 2-3 s per problem on `cores` threads, every thread busy (at least one
    # orbit per thread for each problem): about 8 s for the three
    return [320 * cores, 30 * cores, cores]


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
        v, desc = _cpu_sample(cores, sizes)
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


def run_ours(args):
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import build as sdeb_build
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator
    from paper_1908_03869_gb300.sharding import max_over_ranks, weak_scaling_offset

    ws, rank, local = _dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(sdeb_build.LIB_PATH):
        sdeb_build.build()
    if dist is not None:
        dist.barrier()
    sdeb.lib()

    stream = torch.cuda.Stream()
    dtype = torch.float32
    its, dev_inputs, host_inputs = [], [], []
    for n, orbits in CONFIGS:
        p, x0 = inputs.kuramoto(n, orbits, seed=1 + rank)
        pb = sdeb.Problem.make("kuramoto", n, orbits, DT, STEPS, STRIDE, SEED, "fp32",
                               orbit_offset=weak_scaling_offset(orbits, rank))
        its.append(Integrator(pb))
        pt, xt = torch.tensor(p, dtype=dtype), torch.tensor(x0, dtype=dtype)
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
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in CONFIGS]
               for _ in range(args.steps)]
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
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    kern_ms = [[a.elapsed_time(b) for a, b in row] for row in kern_ev]
    total_ms = max_over_ranks(sum(step_ms), dist, device="cuda")
    value = units_per_step * ws * args.steps / (total_ms / 1e3)

    # ---- roofline of the dominant kernel (forward EM, FP32) --------------
    kernel_s = sum(sum(r) for r in kern_ms) / 1e3
    sfu_ops = SFU_OPS_PER_OSC_STEP * osc_per_step * args.steps
    achieved = sfu_ops / kernel_s / 1e9
    peak = SFU_PER_SM_PER_CLK * NUM_SMS * SM_MAX_MHZ * 1e6 / 1e9
    per_launch_ms = {str(n): statistics.mean(r[i] for r in kern_ms) for i, (n, _) in enumerate(CONFIGS)}

    # ---- end to end through the C ABI with pinned host buffers ----------
    e2e = None
    if not args.no_e2e:
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
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, device="cuda")
        e2e = {"value": units_per_step * ws * args.steps / e2e_s, "unit": "orbit-steps/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "pipeline": "%d integrate_range chunks per problem; frames copied to pinned host memory on a "
                           "second stream while the next chunk computes" % E2E_CHUNKS}
        del host_frames

    # ---- FP64 on a 1000-step prefix of the same problems -----------------
    fp64 = None
    if not args.no_fp64:
        steps64 = 1000
        t64, u64 = 0.0, 0
        for n, orbits in CONFIGS:
            p, x0 = inputs.kuramoto(n, orbits, seed=1 + rank)
            pb = sdeb.Problem.make("kuramoto", n, orbits, DT, steps64, STRIDE, SEED, "fp64",
                                   orbit_offset=weak_scaling_offset(orbits, rank))
            with Integrator(pb) as it64:
                pt, xt = torch.tensor(p, device="cuda"), torch.tensor(x0, device="cuda")
                it64.set_params(pt, xt, stream=stream)
                it64.integrate(stream=stream)  # warm-up
                it64.set_params(pt, xt, stream=stream)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                it64.integrate(stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                t64 += a.elapsed_time(b) / 1e3
                u64 += orbits * steps64
        fp64 = {"value": u64 / t64, "unit": "orbit-steps/s", "steps_per_orbit": steps64,
                "note": "same orbits, first 1000 of the 10^4 steps; cost per step is constant over the horizon"}

    # ---- forward + adjoint (n = 32, 16384 orbits sharing one parameter
    # vector, 2000 steps, checkpoints every 100, loss = mean order parameter)
    adjoint = None
    if not args.no_adjoint:
        adjoint = _time_adjoint(stream, rank)

    # ---- FitzHugh-Nagumo network, Euler-Maruyama and Milstein ------------
    fhn = None
    if not args.no_fhn:
        fhn = _time_fhn(stream, rank)

    # ---- the ODE path: Runge-Kutta and the implicit schemes on the Kuramoto drift
    rk4 = None
    if not args.no_rk4:
        rk4 = _time_rk4(stream, rank)

    # ---- particle swarm search over the coupling: whole generations on the GPU
    swarm = None
    if not args.no_swarm:
        swarm = _time_swarm(stream, rank)

    # ---- a user-defined model compiled at run time, beside the built-in one --
    user = None
    if not args.no_user_model:
        user = _time_user_model(stream, rank)

    # ---- the paper's own speed and accuracy protocols (Sec. 2.2.1, 2.3.1) ----
    paper, paper_acc = None, None
    if not args.no_paper_protocol:
        paper = _time_paper_protocol(stream, rank)
        paper_acc = _paper_accuracy_protocol(stream, rank)

    # ---- batched heterogeneous instances (one persistent graph launch) -----
    batched = None
    if not args.no_batched:
        batched = _time_batch(stream, rank)

    # ---- CPU oracle on this host's cores --------------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        sizes = _sample_sizes(cores)
        v, desc = _cpu_sample(cores, sizes)
        v1, desc1 = _cpu_sample(1, [max(1, s // cores) for s in sizes])
        vmf, descmf = _cpu_sample(cores, sizes, mean_field=True)
        cpu = {"value": v, "unit": "orbit-steps/s", "cores": cores, "kind": "oracle",
               "sample": desc + "; rate scaled to the workload's orbit mix",
               "single_thread": {"value": v1, "cores": 1, "sample": desc1},
               "mean_field_form": {"value": vmf, "cores": cores, "sample": descmf,
                                   "note": "the oracle's O(n) mean-field drift instead of the pairwise definition"}}

    for it in its:
        it.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "orbit-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp32 Kahan", "orbits_per_gpu": [o for _, o in CONFIGS],
                       "n": [n for n, _ in CONFIGS], "dt": DT, "steps_per_orbit": STEPS, "stride": STRIDE,
                       "l2": "flushed between steps (512 MiB write)", "parallelism": "orbits sharded, no collective"},
            "oscillator_steps_per_sec": value * osc_per_step / units_per_step,
            "wall_s": wall,
            "per_launch_ms": per_launch_ms, "layouts_G_P": layouts,
            "roofline": {"bound": "alu", "pipe": "SFU (MUFU)", "achieved": achieved, "peak": peak,
                         "unit": "Gop/s", "frac": achieved / peak,
                         "traffic": FORWARD_N32_DRAM_BYTES if args.orbit_scale == 1.0 and args.horizon is None else None,
                         "traffic_note": "DRAM bytes of the n=32 launch (ncu); algorithmic 3.52e9",
                         "peak_source": "16 SFU results/clk/SM x 152 SMs x 2070 MHz",
                         "ops_per_osc_step": SFU_OPS_PER_OSC_STEP},
            "e2e": e2e, "fp64": fp64, "adjoint": adjoint, "batched": batched, "fhn": fhn, "rk4": rk4,
            "user_model": user, "swarm_search": swarm, "paper_speed_protocol": paper, "paper_accuracy_protocol": paper_acc,
            "cpu_baseline": cpu,
            "clocks": clk,
            "gpu_launches": len(CONFIGS) * args.steps,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _time_batch(stream, rank, reps=5):
    import numpy as np
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import BatchIntegrator

    W = inputs.WORKLOADS["batched_4096"]
    insts = inputs.batched_instances(W["count"], seed=1)
    base = rank * W["count"]
    pbs = [sdeb.Problem.make("kuramoto", d["n"], 1, d["dt"], d["steps"], W["stride"], W["seed"], "fp32",
                             orbit_offset=base + i) for i, d in enumerate(insts)]
    ps = [d["params"][None, :].astype(np.float32) for d in insts]
    xs = [d["x0"][None, :].astype(np.float32) for d in insts]
    orbit_steps = sum(d["steps"] for d in insts)
    osc_steps = sum(d["steps"] * d["n"] for d in insts)
    times = []
    with BatchIntegrator(pbs) as b:
        b.set_params(ps, xs, stream=stream)
        info = b.autotune(stream=stream)
        for _ in range(reps + 1):
            b.set_params(ps, xs, stream=stream)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.integrate(stream=stream)
            e.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(e))
    ms = statistics.median(times[1:])
    peak = SFU_PER_SM_PER_CLK * NUM_SMS * SM_MAX_MHZ * 1e6
    longest = max(d["steps"] * d["n"] for d in insts)
    return {"workload": "4096 Kuramoto instances, n~U{2..256}, steps~logU[1e3,1e5], dt in {0.001,0.01}, stride 100, fp32",
            "ms": ms, "orbit_steps_per_sec": orbit_steps / (ms / 1e3), "osc_steps_per_sec": osc_steps / (ms / 1e3),
            "sfu_roofline_frac": SFU_OPS_PER_OSC_STEP * osc_steps / (ms / 1e3) / peak,
            "total_osc_steps": osc_steps, "longest_instance_osc_steps": longest, "schedule": info}


def _time_fhn(stream, rank, reps=3, steps=10000):
    """The FitzHugh-Nagumo network workload (64 units, n = 128, 2^18 orbits,
    dt = 0.01, frame every 1000 steps), FP32, on the first 10^4 of its 10^5
    steps (the cost per step is constant), Euler-Maruyama and Milstein."""
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator
    from paper_1908_03869_gb300.sharding import weak_scaling_offset

    W = inputs.WORKLOADS["fhn_64units"]
    n, orbits = W["n"], W["orbits"]
    p, x0 = inputs.fhn(n // 2, orbits, seed=1 + rank)
    pt = torch.tensor(p, dtype=torch.float32, device="cuda")
    xt = torch.tensor(x0, dtype=torch.float32, device="cuda")
    out = {"workload": "FitzHugh-Nagumo network, 64 units (n = 128), 2^18 orbits, dt = 0.01, first %d of the "
                       "10^5 steps, frame every %d steps, fp32" % (steps, W["stride"])}
    unit_steps = orbits * (n // 2) * steps
    for name, mil in (("euler_maruyama", False), ("milstein", True)):
        pb = sdeb.Problem.make("fhn_net", n, orbits, W["dt"], steps, W["stride"], W["seed"], "fp32",
                               orbit_offset=weak_scaling_offset(orbits, rank), milstein=mil)
        times = []
        with Integrator(pb) as it:
            for _ in range(reps + 1):
                it.set_params(pt, xt, stream=stream)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                it.integrate(stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
        ms = statistics.median(times[1:])
        out[name] = {"ms": ms, "unit_steps_per_sec": unit_steps / (ms / 1e3)}
    out["milstein_time_over_em"] = out["milstein"]["ms"] / out["euler_maruyama"]["ms"]
    peak = SFU_PER_SM_PER_CLK * NUM_SMS * SM_MAX_MHZ * 1e6
    # one normal per unit-step: half of (log2, sqrt, sin, cos) = 2 SFU operations
    out["sfu_roofline_frac_em"] = 2.0 * out["euler_maruyama"]["unit_steps_per_sec"] / peak
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


def _time_user_model(stream, rank, reps=3, steps=1000):
    """A FitzHugh-Nagumo network of 16 units (n = 32) on 2^18 orbits, dt =
    0.01, 1000 steps, FP32: compile time of the run-time compiled user model
    and its unit-steps/s beside the built-in model's."""
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator
    from paper_1908_03869_gb300.sharding import weak_scaling_offset

    n, orbits = 32, 1 << 18
    p, x0 = inputs.fhn(n // 2, orbits, seed=1 + rank)
    pt = torch.tensor(p, dtype=torch.float32, device="cuda")
    xt = torch.tensor(x0, dtype=torch.float32, device="cuda")
    out = {"workload": "FitzHugh-Nagumo network, 16 units (n = 32), 2^18 orbits, dt = 0.01, %d steps, fp32"
                       % steps}
    for name in ("built_in", "user_source"):
        user = name == "user_source"
        pb = sdeb.Problem.make("user" if user else "fhn_net", n, orbits, 0.01, steps, 100, 0, "fp32",
                               orbit_offset=weak_scaling_offset(orbits, rank), m=n // 2, d=6)
        t0 = time.perf_counter()
        it = Integrator(pb, user_source=USER_FHN_SOURCE if user else None)
        create_s = time.perf_counter() - t0
        times = []
        try:
            for _ in range(reps + 1):
                it.set_params(pt, xt, stream=stream)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                it.integrate(stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
        finally:
            it.close()
        ms = statistics.median(times[1:])
        out[name] = {"create_s": create_s, "ms": ms, "unit_steps_per_sec": orbits * (n // 2) * steps / (ms / 1e3)}
    out["user_time_over_built_in"] = out["user_source"]["ms"] / out["built_in"]["ms"]
    return out


# The paper's runtimes of its speed protocol on an NVIDIA P100 (Tables S1-S3,
# M = 163840 orbits, FP64, including OpenCL set-up and host transfers): context
# for the same protocol here, not a target.
PAPER_P100_SECONDS = {5: 4.719, 10: 9.315, 15: 17.656}


def _time_paper_protocol(stream, rank):
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
    from paper_1908_03869_gb300.sharding import weak_scaling_offset

    orbits, dt, steps, stride = 163840, 0.05, 8000, 100
    out = {"workload": "paper speed protocol: Kuramoto paper layout, M = 163840, dt = 0.05, 8000 steps, "
                       "frame every 100 steps, fp64",
           "paper_p100_seconds_context": PAPER_P100_SECONDS, "runs": {}}
    for n in (5, 10, 15):
        p, x0 = inputs.kuramoto_paper_speed(n, orbits, seed=1 + rank)
        ph, xh = torch.tensor(p).pin_memory(), torch.tensor(x0).pin_memory()
        pd, xd = ph.cuda(), xh.cuda()
        pb = sdeb.Problem.make("kuramoto_paper", n, orbits, dt, steps, stride, 0, "fp64",
                               orbit_offset=weak_scaling_offset(orbits, rank))
        with Integrator(pb) as it:
            host_frames = torch.empty((it.nframes, orbits, n), dtype=torch.float64, pin_memory=True)
            it.set_params(pd, xd, stream=stream)
            it.integrate_range(0, 100, stream=stream)          # warm-up
            torch.cuda.synchronize()
            it.set_params(pd, xd, stream=stream)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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
        out["runs"][str(n)] = {"device_s": dev_s, "e2e_s": e2e_s,
                               "orbit_steps_per_sec": orbits * steps / dev_s,
                               "e2e_orbit_steps_per_sec": orbits * steps / e2e_s}
    return out


def _paper_accuracy_protocol(stream, rank):
    """The paper's accuracy protocol (Sec. 2.3.1): N = 100, 64 realisations,
    omega ~ U(0.2, 0.4), theta(0) ~ U(-pi, pi), p ~ U(0.01, 0.03),
    K = 0.02 and 0.2, 400 s, dt = 2^(l-5)/5 for l = 1..5, FP64: the mean and
    standard deviation over realisations of the coherence r(t_MAX) (Eq. 7)
    and the device time of each run."""
    import numpy as np
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits = 100, 64
    out = {"workload": "paper accuracy protocol: Kuramoto paper layout, N = 100, 64 realisations, 400 s, fp64",
           "runs": []}
    for K in (0.02, 0.2):
        p, x0 = inputs.kuramoto_paper_accuracy(K, orbits=orbits, n=n, seed=1 + rank)
        pd, xd = torch.tensor(p).cuda(), torch.tensor(x0).cuda()
        for l in range(1, 6):
            dt = 2.0 ** (l - 5) / 5
            steps = int(round(400 / dt))
            pb = sdeb.Problem.make("kuramoto_paper", n, orbits, dt, steps, steps, 0, "fp64")
            with Integrator(pb) as it:
                it.set_params(pd, xd, stream=stream)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                it.integrate(stream=stream)
                b.record(stream)
                fin = it.final(stream=stream)
                torch.cuda.synchronize()
                r = np.abs(np.exp(1j * fin.cpu().numpy()).mean(axis=1))
            out["runs"].append({"K": K, "dt": dt, "r_mean": float(r.mean()), "r_sd": float(r.std()),
                                "device_ms": a.elapsed_time(b)})
    return out


def _time_swarm(stream, rank, generations=5, particles=1024, realisations=64, n=32, steps=1000):
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

    p, x0 = inputs.kuramoto(n, realisations, seed=11 + rank)
    base = p[0].copy()
    pb = sdeb.Problem.make("kuramoto", n, 1, DT, steps, steps, SEED, "fp32")
    g = torch.Generator().manual_seed(3 + rank)
    x_init = torch.rand((particles, 2), generator=g, dtype=torch.float64) * torch.tensor([4.0, 0.5])
    v_init = torch.zeros((particles, 2), dtype=torch.float64)
    orbit_steps = particles * realisations * steps
    out = {"workload": "Kuramoto n = %d, %d particles x %d realisations (%d orbits), dt = %g, %d steps, fp32, "
                       "search over (K, sigma), target r = 0.8" % (n, particles, realisations,
                                                                   particles * realisations, DT, steps)}
    with SwarmSearch(pb, base, x0, [0, 1], [0.0, 0.0], [4.0, 0.5], particles, r_target=0.8, swarm_seed=7) as s:
        s.reset(x_init, v_init)
        with torch.cuda.stream(stream):
            s.step(stream)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
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


def _time_rk4(stream, rank, reps=3, steps=1000):
    """The ODE path: classical fourth-order Runge-Kutta, implicit Euler and
    the implicit midpoint rule (4 Newton iterations a step) on the drift of
    the n = 32 benchmark problem (2^18 orbits, dt = 0.005, frame every 100
    steps), FP32, first 1000 steps, beside Euler-Maruyama on the same steps."""
    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator
    from paper_1908_03869_gb300.sharding import weak_scaling_offset

    n, orbits = 32, 1 << 18
    p, x0 = inputs.kuramoto(n, orbits, seed=1 + rank)
    pt = torch.tensor(p, dtype=torch.float32, device="cuda")
    xt = torch.tensor(x0, dtype=torch.float32, device="cuda")
    out = {"workload": "Kuramoto n = 32, 2^18 orbits, dt = %g, first %d steps, frame every %d steps, fp32"
                       % (DT, steps, STRIDE)}
    schemes = (("euler_maruyama", {}), ("rk4", {"rk4": True}), ("implicit_euler", {"implicit": "euler"}),
               ("implicit_midpoint", {"implicit": "midpoint"}))
    for name, kw in schemes:
        pb = sdeb.Problem.make("kuramoto", n, orbits, DT, steps, STRIDE, SEED, "fp32",
                               orbit_offset=weak_scaling_offset(orbits, rank), **kw)
        times = []
        with Integrator(pb) as it:
            for _ in range(reps + 1):
                it.set_params(pt, xt, stream=stream)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                it.integrate(stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
        ms = statistics.median(times[1:])
        out[name] = {"ms": ms, "orbit_steps_per_sec": orbits * steps / (ms / 1e3)}
    peak = SFU_PER_SM_PER_CLK * NUM_SMS * SM_MAX_MHZ * 1e6
    # four drift evaluations per step, each a sin and a cos per oscillator
    out["sfu_roofline_frac_rk4"] = 8.0 * n * out["rk4"]["orbit_steps_per_sec"] / peak
    out["rk4_time_over_em"] = out["rk4"]["ms"] / out["euler_maruyama"]["ms"]
    # four Newton iterations per step, each a sin, a cos and a reciprocal per oscillator
    for name in ("implicit_euler", "implicit_midpoint"):
        out["sfu_roofline_frac_" + name] = 12.0 * n * out[name]["orbit_steps_per_sec"] / peak
        out[name + "_time_over_em"] = out[name]["ms"] / out["euler_maruyama"]["ms"]
    return out


def _time_adjoint(stream, rank, reps=5):
    import ctypes

    import torch

    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator
    from paper_1908_03869_gb300.sharding import weak_scaling_offset

    W = inputs.WORKLOADS["kuramoto_adjoint_n32"]
    n, orbits = W["n"], W["orbits"]
    p, x0 = inputs.kuramoto(n, orbits, seed=1, shared=True)
    pt = torch.tensor(p, dtype=torch.float32, device="cuda")
    xt = torch.tensor(x0, dtype=torch.float32, device="cuda")
    mk = lambda ck: sdeb.Problem.make("kuramoto", n, orbits, W["dt"], W["steps"], 1, W["seed"], "fp32",
                                      ckpt_every=ck, no_frames=True, shared_params=True,
                                      orbit_offset=weak_scaling_offset(orbits, rank))
    ev = lambda: torch.cuda.Event(enable_timing=True)
    with Integrator(mk(0)) as plain, Integrator(mk(W["ckpt_every"])) as ck:
        # dL/dX^K of the mean order parameter at T, from the library's kernel
        # each context tuned for what it runs: the plain forward alone, the
        # checkpointed context for forward + adjoint
        for it in (plain, ck):
            it.set_params(pt, xt, stream=stream)
            it.autotune(trial_steps=64, stream=stream)
        lay, fwd_lay = ck.layout(), plain.layout()
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
            a, b, c, d, e = ev(), ev(), ev(), ev(), ev()
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
    units = orbits * W["steps"]
    return {"workload": "kuramoto n=32, 16384 orbits, shared params, dt=0.01, 2000 steps, ckpt every 100, fp32",
            "layout_G_P": list(lay), "fwd_layout_G_P": list(fwd_lay),
            "fwd_ms": t_plain, "fwd_ckpt_ms": t_fwd, "adjoint_ms": t_adj,
            "fwd_plus_adjoint_orbit_steps_per_sec": units / ((t_fwd + t_adj) / 1e3),
            "fwd_orbit_steps_per_sec": units / (t_plain / 1e3),
            "ratio_fwd_plus_adjoint_to_fwd": (t_fwd + t_adj) / t_plain}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-fhn", action="store_true")
    ap.add_argument("--no-rk4", action="store_true")
    ap.add_argument("--no-paper-protocol", action="store_true")
    ap.add_argument("--no-user-model", action="store_true")
    ap.add_argument("--no-swarm", action="store_true")
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
