"""Benchmark of the PIC hot path (sort + gather + push + deposit + Yee) on GB300.

Default workload: the uniform thermal plasma of the paper's scaling runs
(Sec. 4.1.1): 256^3 periodic cells, 8 particles per cell (134,217,728
particles), order-3 shapes, u ~ N(0, 0.05), density 1, dt = 0.99 CFL,
synthetic seeded inputs.  One step = counting sort + fused gather/push/
deposit tile kernel + Yee update, in FP32-mixed (the headline) and FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica of the workload on its own GPU (the path has no exchange step on one
box): value = all ranks' particle-steps / the slowest rank's time.
"""
import argparse
import hashlib
import re
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "uniform_256"
METRIC = "particle-steps/s (gather+push+deposit+Yee), FP32-mixed vs FP64 at stated error"
UNIT = "particle-steps/s"


def derived_fp32_tflops(sms, mhz):
    """FP32 ALU roof from the device: SMs x 128 FP32 lanes x 2 flop (FMA) x SM clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def derived_smem_gbs(sms, mhz):
    """Shared-memory roof from the device: SMs x 32 banks x 4 B per clock x SM clock."""
    return sms * 128 * mhz * 1e6 / 1e9


def device_roofs(torch, pic, local, clock_summary, peaks):
    """SM count and maximum SM clock read from the device and nvidia-smi, the
    derived FP32 and shared-memory roofs, and the FP32 / FP64 FMA throughput
    measured by the library's microbenchmark (the ALU peaks used)."""
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = clock_summary.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    return {"sms": sms, "sm_max_mhz": mhz,
            "fp32_derived_tflops": derived_fp32_tflops(sms, mhz),
            "smem_derived_gbs": derived_smem_gbs(sms, mhz),
            "fp32_measured_tflops": pic.measure_fma_peak(pic.FP32_MIXED),
            "fp64_measured_tflops": pic.measure_fma_peak(pic.FP64)}


def flops_per_particle(p: int) -> int:
    """Algorithmic flops of gather + Boris + advance + Esirkepov per particle
    (FMA = 2).  S = p+1 stencil nodes per axis, NW = p+2 Esirkepov window."""
    S, NW = p + 1, p + 2
    shape_cost = {1: 1, 2: 9, 3: 14}[p]
    gather = 12 * (S ** 3 + S ** 2 + S)
    weights = 12 * shape_cost
    boris, advance = 60, 16
    esirk = 3 * NW + 3 * (2 * (NW - 1) + 8 * NW * NW + 2 * NW * NW * (NW - 1))
    return gather + weights + boris + advance + esirk



def smem_bytes_per_particle(p: int, prec: str) -> int:
    """Algorithmic shared-memory bytes of one particle in the tile kernel:
    the gather reads 6 (p+1)^3 staged field values, the narrow Esirkepov
    deposit adds 3 p (p+1)^2 current values (FP32-mixed: two int32 words
    each, the fixed-point hi and lo; FP64: one double)."""
    rs = 4 if prec == "fp32" else 8
    gather = 6 * (p + 1) ** 3 * rs
    deposit = 3 * p * (p + 1) ** 2 * 8
    return gather + deposit


def bytes_per_launch(np_, C, prec):
    """Algorithmic HBM bytes of one fused tile-kernel launch: each particle's
    state read once and written once (FP32-mixed: key + 3 offsets + 3 u + w
    read, key + 3 offsets + 3 u written = 60 B; FP64: 7 doubles read, 6
    written = 104 B), E and B read once and J written once per cell."""
    if prec == "fp32":
        return np_ * 60 + C * (24 + 12)
    return np_ * 104 + C * (48 + 24)


def kernel_bytes(name, np_, C, prec):
    """Algorithmic HBM bytes of one launch of each kernel of the step, with a
    statement of what they count; None for kernels without a fixed amount."""
    rs = 4 if prec == "fp32" else 8
    table = {
        "k_tile_step": (bytes_per_launch(np_, C, prec), "particle state read and written once, E/B read and J "
                        "written once per cell"),
        "k_yee_fused": (C * rs * 15, "E, B, J read and E, B written once per cell"),
        "k_yee_b": (C * rs * 9, "E, B read and B written once per cell"),
        "k_yee_e": (C * rs * 12, "E, B, J read and E written once per cell"),
        "k_hist": (np_ * 4 + C * 4, "keys read, counts written"),
        "k_scan": (C * 8, "counts read, offsets written"),
        "k_scatter_perm": (np_ * 8 + C * 4, "keys read, slots written, offsets read"),
        "k_scatter": (np_ * (72 if prec == "fp32" else 128), "every particle array read and written once"),
    }
    return table.get(name)


def kernel_rooflines(timings, np_, C, prec, hbm_gbs):
    """Each timed kernel's algorithmic bytes over its mean launch time (CUDA
    events on the launching stream) against the measured HBM copy rate."""
    out = {}
    for name, (ms, n) in timings.items():
        kb = kernel_bytes(name, np_, C, prec)
        if not kb or not n or ms <= 0:
            continue
        gbs = kb[0] / (ms / n / 1e3) / 1e9
        out[name] = {"bytes_per_launch": kb[0], "achieved_gbs": gbs, "frac_of_hbm": gbs / hbm_gbs, "bytes": kb[1]}
    return out


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash():
    """Hash of the code (comments and layout stripped) of the sources the tile
    kernel is built from: its DRAM counters in profiles/ hold only while
    this matches."""
    h = hashlib.sha256()
    for f in ("pic_kernels.cu", "pic_device.cuh", "pic_step_common.cuh"):
        with open(os.path.join(ROOT, "paper_2101_12149_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, prec, workload=WORKLOAD):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    summary is absent or was taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}_{prec}.md")
    if not os.path.exists(path):
        return None
    src_hash, traffic = None, None
    for line in open(path):
        if line.startswith("kernel_source_hash:"):
            src_hash = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch_full_size:"):
            traffic = float(line.split(":", 1)[1].strip())
    if src_hash != kernel_source_hash():
        return None
    return traffic


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.uuid}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([v.strip() for v in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, s[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def pinned_particles(n_cells_ppc, torch):
    """Pinned host float64 arrays for the particle SoA (numpy views)."""
    out, keep = {}, []
    for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
        t = torch.empty(n_cells_ppc, dtype=torch.float64, pin_memory=True)
        keep.append(t)
        out[k] = t.numpy()
    return out, keep


def cpu_baseline(seconds_target=15.0):
    """The oracle as it stands on a bounded sample of the workload: the same
    recipe (8 ppc, order 3, u ~ N(0, 0.05), density 1, dt = 0.99 CFL) on a
    32^3 periodic box, a few full steps, single host core."""
    from oracle import Oracle
    from paper_2101_12149_gb300 import inputs
    w = inputs.WORKLOADS[WORKLOAD]
    n = (32, 32, 32)
    O = Oracle()
    g = O.grid(n)
    dt = inputs.dt_from_cfl((1, 1, 1), w["cfl"])
    parts = inputs.uniform_plasma(w["seed"], n, w["ppc"], sigma_u=w["sigma_u"], density=w["density"])
    F = np.zeros((9,) + n)
    N = parts["x"].size
    t0 = time.perf_counter()
    steps = 0
    while True:
        O.pic_step(g, w["order"], dt, -1.0, 1.0, parts, F)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds_target or steps >= 50:
            break
    return {"value": N * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle on the same recipe at 32^3 ({N} particles, order 3, 8 ppc), {steps} steps, "
                      f"{el:.1f} s, 1 host core"}


def cpu_baseline_mt(seconds_target=15.0, workload=WORKLOAD, n=(64, 64, 64)):
    """The multi-threaded CPU baseline (oracle/pic_oracle_mt.c: OpenMP,
    private current arrays summed in thread order, the CPU deposition of
    Sec. 3.4.1) on every host core, on a bounded sample of the workload (the
    same recipe on a 64^3 box), a few full steps."""
    from oracle import Oracle, OracleMT
    from paper_2101_12149_gb300 import inputs
    w = inputs.WORKLOADS[workload]
    M = OracleMT(os.cpu_count() or 1)
    g = Oracle.grid(n)
    dt = inputs.dt_from_cfl((1, 1, 1), w["cfl"])
    parts = inputs.uniform_plasma(w["seed"], n, w["ppc"], sigma_u=w["sigma_u"], density=w["density"])
    F = np.zeros((9,) + n)
    N = parts["x"].size
    M.pic_step(g, w["order"], dt, -1.0, 1.0, parts, F)  # first touch of the private arrays
    t0 = time.perf_counter()
    steps = 0
    while True:
        M.pic_step(g, w["order"], dt, -1.0, 1.0, parts, F, 0.0, 0.0, (steps + 1) * dt)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds_target or steps >= 50:
            break
    return {"value": N * steps / el, "unit": UNIT, "cores": M.nthreads, "kind": "oracle_mt",
            "sample": f"OpenMP baseline on the same recipe at {n[0]}^3 ({N} particles, order {w['order']}, "
                      f"{w['ppc']} ppc), {steps} steps, {el:.1f} s, {M.nthreads} threads on "
                      f"{os.cpu_count()} host cores"}


def cpu_baselines_per_config():
    """CPU timings of the oracle (1 core) and the OpenMP baseline (every host
    core) on each workload, as stated baselines (not tuned): the 32^3 parity
    run in full (50 steps, serial oracle); the 256^3 x 8 ppc run, 2 full-size
    steps (OpenMP); the 128 x 128 x 1024 wakefield grid, 2 full-size steps of
    the step itself (OpenMP, z open, no window shift); the 96-box ensemble, 5
    steps of every box (OpenMP); the 64^3 differentiation run's forward pass,
    200 steps with the drive (OpenMP), and the serial oracle's adjoint of 20
    steps on its 16^3 copy.  Prints one JSON line; several minutes."""
    from oracle import Oracle, OracleMT
    from paper_2101_12149_gb300 import inputs
    M = OracleMT(os.cpu_count() or 1)
    O = Oracle()
    res = {"host_cores": os.cpu_count(), "threads": M.nthreads}

    def timed(fn, steps, N, C, what):
        t0 = time.perf_counter()
        fn()
        t = time.perf_counter() - t0
        return {"particle_steps_per_s": N * steps / t, "cell_steps_per_s": C * steps / t, "seconds": t,
                "steps": steps, "particles": N, "what": what}

    w = inputs.WORKLOADS["uniform_32"]
    n = w["n"]
    parts = inputs.workload_particles("uniform_32")
    F = np.zeros((9,) + n)
    g = O.grid(n)
    dt = inputs.dt_from_cfl((1, 1, 1), w["cfl"])
    res["uniform_32"] = timed(lambda: [O.pic_step(g, w["order"], dt, -1.0, 1.0, parts, F, 0.0, 0.0, s * dt)
                                       for s in range(w["steps"])], w["steps"], parts["x"].size, int(np.prod(n)),
                              "oracle, 1 core, the full 50-step run")
    for name in ("uniform_256",):
        w = inputs.WORKLOADS[name]
        n = w["n"]
        parts = inputs.workload_particles(name)
        F = np.zeros((9,) + n)
        g = O.grid(n)
        dt = inputs.dt_from_cfl((1, 1, 1), w["cfl"])
        res[name] = timed(lambda: [M.pic_step(g, w["order"], dt, -1.0, 1.0, parts, F) for _ in range(2)], 2,
                          parts["x"].size, int(np.prod(n)), f"OpenMP, {M.nthreads} threads, 2 full-size steps")
        del parts, F
    cfg = inputs.WAKEFIELD
    parts = inputs.wakefield_particles(cfg)
    F = inputs.laser_fields(cfg)
    g = O.grid(cfg["n"], zopen=True)
    dt = inputs.dt_from_cfl((1, 1, 1), cfg["cfl"])
    res["wakefield"] = timed(lambda: [M.pic_step(g, cfg["order"], dt, -1.0, 1.0, parts, F) for _ in range(2)], 2,
                             parts["x"].size, int(np.prod(cfg["n"])),
                             f"OpenMP, {M.nthreads} threads, 2 full-size steps (z open, no window shift)")
    del parts, F
    boxes = inputs.ensemble_boxes()
    _, counts, bparts = inputs.ensemble_particles(boxes)
    bF = [np.zeros((9,) + b["n"]) for b in boxes]
    dt = inputs.dt_from_cfl((1, 1, 1), inputs.ENSEMBLE["cfl"])

    def ens():
        for _ in range(5):
            for b, p_, f_ in zip(boxes, bparts, bF):
                M.pic_step(O.grid(b["n"]), b["order"], dt, -1.0, 1.0, p_, f_)
    res["ensemble"] = timed(ens, 5, int(counts.sum()), sum(int(np.prod(b["n"])) for b in boxes),
                            f"OpenMP, {M.nthreads} threads, 5 steps of all 96 boxes")
    w = inputs.WORKLOADS["adjoint_64"]
    parts = inputs.workload_particles("adjoint_64")
    F = np.zeros((9,) + w["n"])
    g = O.grid(w["n"])
    dt = inputs.dt_from_cfl((1, 1, 1), w["cfl"])
    A, kd = inputs.drive_amplitude(w["seed"]), 2 * np.pi / w["n"][0]
    res["adjoint_64_forward"] = timed(
        lambda: [M.pic_step(g, w["order"], dt, -1.0, 1.0, parts, F, A, kd, s * dt) for s in range(w["steps"])],
        w["steps"], parts["x"].size, int(np.prod(w["n"])), f"OpenMP, {M.nthreads} threads, the 200-step forward run")
    n16 = (16, 16, 16)
    p16 = inputs.uniform_plasma(w["seed"], n16, w["ppc"], sigma_u=w["sigma_u"])
    g16 = O.grid(n16)
    res["adjoint_16_copy"] = timed(
        lambda: O.pic_adjoint(g16, w["order"], dt, -1.0, 1.0, p16, np.zeros((9,) + n16), 20, A, 2 * np.pi / 16),
        20, p16["x"].size, int(np.prod(n16)), "oracle, 1 core, forward + adjoint of 20 steps on the 16^3 copy")
    print(json.dumps({"cpu_baselines": res}), flush=True)


def dist_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(t, dist, device):
    """The whole job's time: the slowest rank's (every rank gets it)."""
    if dist is None:
        return t
    import torch
    tt = torch.tensor([float(t)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(world, units_per_rank, steps, t):
    """Units all ranks processed (independent replicas, same work each) per second of the job."""
    return world * units_per_rank * steps / t


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, one host core, on a
    bounded sample of the same workload (a 32^3 box of the recipe, 262,144
    particles); W untimed steps, then K timed steps.  Rank 0 only."""
    rank, _, _ = dist_env()
    if rank != 0:
        return
    # this arm builds and loads only the oracle and the input generator
    from oracle import build as obuild
    from paper_2101_12149_gb300.inputs import build as ibuild
    obuild.build()
    ibuild()
    from oracle import Oracle
    from paper_2101_12149_gb300 import inputs
    w = inputs.WORKLOADS[WORKLOAD]
    n = (32, 32, 32)
    parts = inputs.uniform_plasma(w["seed"], n, w["ppc"], sigma_u=w["sigma_u"], density=w["density"])
    O = Oracle()
    g = O.grid(n)
    dt = inputs.dt_from_cfl((1, 1, 1), w["cfl"])
    F = np.zeros((9,) + n)
    for s in range(args.warmup):
        O.pic_step(g, w["order"], dt, -1.0, 1.0, parts, F, 0.0, 0.0, s * dt)
    t0 = time.perf_counter()
    for s in range(args.steps):
        O.pic_step(g, w["order"], dt, -1.0, 1.0, parts, F, 0.0, 0.0, (args.warmup + s) * dt)
    t = time.perf_counter() - t0
    N = parts["x"].size
    value = N * args.steps / t
    sample = f"oracle on a 32^3 box of the same recipe ({N} particles, order 3, 8 ppc), {args.steps} timed steps"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": "256^3", "ppc": 8, "order": 3, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_run(ctx, steps, stream, torch):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def field_error_statement(torch, steps=100):
    """FP32-mixed against FP64 on a 64^3 copy of the recipe for `steps` steps
    (relative L2 of E and B), with the FP64 sensitivity floor: FP64 rerun with
    momenta perturbed by 1e-7 relative."""
    from paper_2101_12149_gb300 import inputs, pic
    w = inputs.WORKLOADS[WORKLOAD]
    n = (64, 64, 64)
    parts = inputs.uniform_plasma(w["seed"], n, w["ppc"], sigma_u=w["sigma_u"], density=w["density"])
    res = {}
    s = torch.cuda.Stream()

    def run(prec, p):
        with pic.Context(n, cfl=w["cfl"], order=w["order"], precision=prec, stream=s) as ctx:
            ctx.load_particles(-1.0, 1.0, p)
            ctx.step(steps)
            return ctx.get_fields()[:6]

    F64 = run(pic.FP64, parts)
    F32 = run(pic.FP32_MIXED, parts)
    pert = {k: v.copy() for k, v in parts.items()}
    for k in ("ux", "uy", "uz"):
        pert[k] *= 1.0 + 1e-7 * (2 * inputs.uniform(99, 0, pert[k].size, 3) - 1)
    Fp = run(pic.FP64, pert)
    nrm = np.linalg.norm(F64)
    res["fp32_field_rel_l2"] = float(np.linalg.norm(F32 - F64) / nrm)
    res["fp64_floor_rel_l2"] = float(np.linalg.norm(Fp - F64) / nrm)
    res["steps"] = steps
    res["grid"] = "64^3 copy of the recipe (8 ppc, order 3)"
    return res


def step_bytes(np_, C, prec="fp32", sort=True):
    """Algorithmic HBM bytes of one whole step, as the method's minimum: the
    tile kernel's (particle state read and written once, E/B read and J
    written once per cell), the field update's (E, B, J read and E, B written
    once per cell) and, when the particles are sorted that step, a sort
    moving every particle once more (FP32-mixed 76 B, FP64 144 B a particle;
    the library's permutation sort moves less)."""
    rs = 4 if prec == "fp32" else 8
    yee = C * rs * (9 + 6)
    srt = np_ * (76 if prec == "fp32" else 144) if sort else 0
    return bytes_per_launch(np_, C, prec) + yee + srt


def hbm_leg_statement(torch, stream, peaks, steps=20, warmup=3):
    """The memory-bound end of the method: order 1, 2 particles per cell on the
    full 256^3 grid (33,554,432 particles), FP32-mixed.  The step loop timed
    as the library runs it (CUDA events on the launching stream), then again
    with per-kernel events; the tile kernel's algorithmic bytes (60 B a
    particle, 36 B a cell) over its time against the measured HBM copy rate,
    and the whole step's (tile kernel, sort and field update)."""
    from paper_2101_12149_gb300 import inputs, pic
    w = inputs.WORKLOADS["uniform_256_o1"]
    n, ppc = w["n"], w["ppc"]
    C = n[0] * n[1] * n[2]
    N = C * ppc
    parts = inputs.workload_particles("uniform_256_o1")
    dev = {k: torch.from_numpy(v).to(torch.cuda.current_device()) for k, v in parts.items()}
    with pic.Context(n, cfl=w["cfl"], order=w["order"], precision=pic.FP32_MIXED, stream=stream) as ctx:
        ctx.load_particles(-1.0, 1.0, dev)
        del dev
        ctx.step(warmup)
        t = timed_run(ctx, steps, stream, torch)
        ctx.set_timing(True)
        timed_run(ctx, steps, stream, torch)
        tm = ctx.get_timing()
    torch.cuda.empty_cache()
    ms_tile, n_tile = tm.get("k_tile_step", (0.0, 0))
    t_tile = ms_tile / max(n_tile, 1) / 1e3
    tile_gbs = bytes_per_launch(N, C, "fp32") / t_tile / 1e9
    step_gbs = step_bytes(N, C) * steps / t / 1e9
    return {"workload": "uniform_256_o1", "grid": "256^3", "ppc": ppc, "order": 1, "particles": N,
            "precision": "fp32_mixed", "steps": steps, "ms_per_step": 1e3 * t / steps,
            "particle_steps_per_s": N * steps / t, "cell_steps_per_s": C * steps / t,
            "fom_per_gpu": C * (0.1 + 0.9 * ppc) / (t / steps),
            "kernels_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in tm.items()},
            "kernel_rooflines": kernel_rooflines(tm, N, C, "fp32", peaks["hbm_gbs"]),
            "roofline": {"bound": "hbm", "kernel": "k_tile_step", "achieved": tile_gbs, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": tile_gbs / peaks["hbm_gbs"],
                         "traffic": profiled_traffic("k_tile_step", "fp32", "uniform_256_o1"),
                         "bytes": "60 B a particle + 36 B a cell per launch"},
            "step_roofline": {"achieved": step_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                              "frac": step_gbs / peaks["hbm_gbs"],
                              "bytes": "tile kernel + sort (76 B a particle) + field update (60 B a cell)"}}


def ensemble_statement(torch, stream, steps=20):
    """The batched ensemble (96 uneven periodic boxes, FP32-mixed): autotuned,
    then `steps` steps timed as one graph replay with CUDA events on the
    batch's stream; FP64 timed beside it."""
    from paper_2101_12149_gb300 import inputs, pic
    boxes = inputs.ensemble_boxes()
    cat, counts, _ = inputs.ensemble_particles(boxes)
    N = int(counts.sum())
    C = sum(int(np.prod(b["n"])) for b in boxes)
    dt = inputs.dt_from_cfl((1.0, 1.0, 1.0), inputs.ENSEMBLE["cfl"])
    res = {"boxes": len(boxes), "particles": N, "cells": C,
           "orders": {str(o): sum(b["order"] == o for b in boxes) for o in (1, 3)}}
    for prec, name in ((pic.FP32_MIXED, "fp32_mixed"), (pic.FP64, "fp64")):
        with pic.Batch([b["n"] for b in boxes], [b["order"] for b in boxes], dt=dt, precision=prec,
                       stream=stream) as B:
            B.load_particles(-1.0, 1.0, cat, counts)
            if prec == pic.FP32_MIXED:
                best, best_ms = B.autotune(trial_steps=3)
                res["tuning"] = best
            k = steps if prec == pic.FP32_MIXED else max(3, steps // 5)
            B.step(k)  # captures the k-step graph, warms up
            l0 = B.launch_count()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            B.step(k)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            res[name] = {"particle_steps_per_s": N * k / t, "cell_steps_per_s": C * k / t,
                         "ms_per_step": 1e3 * t / k, "steps": k, "gpu_launches": B.launch_count() - l0}
    res["fp32_mixed_speedup"] = res["fp32_mixed"]["particle_steps_per_s"] / res["fp64"]["particle_steps_per_s"]
    return res


def wakefield_statement(torch, steps_cmp=50, steps_fp32=150):
    """The laser-wakefield-shaped run (128 x 128 x 1024, window moving at c,
    laser a0 = 2, ramped plasma at 2 ppc, order 2): FP64 and FP32-mixed for
    `steps_cmp` steps from the same start, then their field difference
    (relative L2 of E and B) and each run's energy drift (field + kinetic,
    relative to the start); FP32-mixed then runs `steps_fp32` more steps,
    timed with CUDA events on its stream."""
    from paper_2101_12149_gb300 import inputs, pic
    cfg = inputs.WAKEFIELD
    parts = inputs.wakefield_particles(cfg)
    F0 = inputs.laser_fields(cfg)
    n0 = inputs.wakefield_plasma_density(cfg)
    C = int(np.prod(cfg["n"]))
    res = {"grid": "128x128x1024", "particles_start": int(parts["x"].size), "order": cfg["order"],
           "ppc": cfg["ppc"], "a0": cfg["a0"]}
    s = torch.cuda.Stream()
    fields = {}
    for prec, name in ((pic.FP64, "fp64"), (pic.FP32_MIXED, "fp32_mixed")):
        with pic.Context(cfg["n"], cfl=cfg["cfl"], order=cfg["order"], precision=prec, window_speed=cfg["speed"],
                         stream=s) as c:
            c.set_window_plasma(cfg["ppc"], n0, cfg["ramp_start"], cfg["ramp_length"])
            c.set_fields(F0)
            c.load_particles(-1.0, 1.0, parts)
            d0 = c.diagnostics()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(s)
            c.step(steps_cmp)
            e1.record(s)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            d1 = c.diagnostics()
            fields[name] = np.stack([c.get_field(i) for i in range(6)])
            r = {"ms_per_step": 1e3 * t / steps_cmp, "steps": steps_cmp,
                 "particle_steps_per_s": 0.5 * (parts["x"].size + c.num_particles()) * steps_cmp / t,
                 "cell_steps_per_s": C * steps_cmp / t, "shifts": c.window()["shifts"],
                 "particles_end": c.num_particles(),
                 "energy_drift": (d1["field_energy"] + d1["kinetic_energy"]) / (d0["field_energy"] + d0["kinetic_energy"]) - 1.0}
            if prec == pic.FP32_MIXED and steps_fp32 > 0:
                np0 = c.num_particles()
                torch.cuda.synchronize()
                e0.record(s)
                c.step(steps_fp32)
                e1.record(s)
                torch.cuda.synchronize()
                t2 = e0.elapsed_time(e1) / 1e3
                r["timed_steps"] = steps_fp32
                r["ms_per_step"] = 1e3 * t2 / steps_fp32
                r["particle_steps_per_s"] = 0.5 * (np0 + c.num_particles()) * steps_fp32 / t2
                r["cell_steps_per_s"] = C * steps_fp32 / t2
                r["shifts_end"] = c.window()["shifts"]
                # the whole step's algorithmic bytes (tile kernel, sort, field
                # update; the window shift's field and particle moves left out)
                # against the measured HBM copy rate
                npm = 0.5 * (np0 + c.num_particles())
                gbs = step_bytes(npm, C) / (t2 / steps_fp32) / 1e9
                peak = measured_peaks()[0]["hbm_gbs"]
                r["step_roofline"] = {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                      "bytes": "tile kernel + sort + field update"}
            res[name] = r
    res["fp32_field_rel_l2_vs_fp64"] = float(np.linalg.norm(fields["fp32_mixed"] - fields["fp64"]) /
                                             np.linalg.norm(fields["fp64"]))
    res["compared_after_steps"] = steps_cmp
    # the paper's particle and field options for this run (Sec. 4.2): Vay pusher,
    # energy-conserving gather, CKC solver at dt = 0.99 dx
    if steps_fp32 <= 0:
        return res
    with pic.Context(cfg["n"], dt=0.99, order=cfg["order"], precision=pic.FP32_MIXED, window_speed=cfg["speed"],
                     stream=s, solver="ckc") as c:
        c.set_particle_algorithms("vay", "energy")
        c.set_window_plasma(cfg["ppc"], n0, cfg["ramp_start"], cfg["ramp_length"])
        c.set_fields(F0)
        c.load_particles(-1.0, 1.0, parts)
        c.step(5)
        np0 = c.num_particles()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        c.step(steps_fp32)
        e1.record(s)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        res["fp32_mixed_vay_energy_ckc"] = {"dt": 0.99, "steps": steps_fp32, "ms_per_step": 1e3 * t / steps_fp32,
                                            "particle_steps_per_s": 0.5 * (np0 + c.num_particles()) * steps_fp32 / t,
                                            "shifts": c.window()["shifts"]}
    return res


def sort_study_statement(torch, stream, parts, n, steps32=8, steps64=4):
    """The sort-interval x bin-size study and the shared-vs-global deposit
    ablation (Sec. 3.4.2, 4.1.1) on the uniform-plasma workload (fields and
    particles far larger than L2): ms per step of (a) the fused tile kernel
    sorting by cell every k steps (between sorts the particles that left
    their tile take the global-atomic outsider path), (b) the split path of
    the paper's GPU design (gather+push kernel, then a deposit kernel with
    global atomics) from a random particle order, never re-sorted or
    re-sorted every k steps by bins of 2^s consecutive tile-major cells, and
    from cell order never re-sorted.  Each configuration: 2 untimed steps,
    then the timed steps with CUDA events on the launching stream (sorts
    included)."""
    from paper_2101_12149_gb300 import inputs, pic
    w = inputs.WORKLOADS[WORKLOAD]
    dev = {k: torch.from_numpy(v).to(torch.cuda.current_device()) for k, v in parts.items()}
    N = parts["x"].size
    res = {"grid": "x".join(str(v) for v in n), "particles": N, "order": w["order"], "ppc": w["ppc"]}

    def timed(body, steps):
        for s_ in range(2):
            body(s_)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for s_ in range(steps):
            body(s_ + 2)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def split_body(ctx, every, shift):
        def body(s_):
            if every and s_ % every == 0:
                ctx.sort_particles(shift)
            ctx.gather_push()
            ctx.deposit()
            ctx.yee_step()
        return body

    for prec, name, steps in ((pic.FP32_MIXED, "fp32_mixed", steps32), (pic.FP64, "fp64", steps64)):
        r = {}
        everies = (1, 2, 4, 8, 16) if prec == pic.FP32_MIXED else (1, 4)
        for k in everies:
            with pic.Context(n, cfl=w["cfl"], order=w["order"], precision=prec, sort_every=k, stream=stream) as ctx:
                ctx.load_particles(-1.0, 1.0, dev)
                r[f"fused, cell sort every {k}"] = timed(lambda s_: ctx.step(1), steps)
        split = [(0, None)] + ([(k, sh) for k in (1, 4, 16) for sh in (0, 5, 9, 12)] if prec == pic.FP32_MIXED
                                 else [(1, 0), (1, 5)])
        for start in ("random", "cell"):
            for every, shift in split:
                if start == "cell" and every:
                    continue
                with pic.Context(n, cfl=w["cfl"], order=w["order"], precision=prec, stream=stream) as ctx:
                    ctx.load_particles(-1.0, 1.0, dev)
                    if start == "random":
                        ctx.sort_particles(pic.ORDER_RANDOM)
                    key = (f"split, {start} start, " +
                           (f"bins of 2^{shift} cells every {every}" if every else "never re-sorted"))
                    r[key] = timed(split_body(ctx, every, shift), steps)
        r = {k: round(v, 3) for k, v in r.items()}
        best_split = min(v for k, v in r.items() if k.startswith("split"))
        res[name] = {"steps": steps, "ms_per_step": r,
                     "split_random_never_over_best_split": r["split, random start, never re-sorted"] / best_split,
                     "global_over_shared_deposit_sorted_every_step":
                         r["split, random start, bins of 2^0 cells every 1"] / r["fused, cell sort every 1"]}
    del dev
    torch.cuda.empty_cache()
    return res


def adjoint_statement(torch):
    """The differentiation workload: 64^3, 4 ppc, order 2, drive A from seed 4,
    200 steps with checkpoints every 20; forward + checkpointed reverse timed
    on the host around pic_step_adjoint (it waits), FP32-mixed and FP64."""
    from paper_2101_12149_gb300 import inputs, pic
    w = inputs.WORKLOADS["adjoint_64"]
    parts = inputs.workload_particles("adjoint_64")
    A = inputs.drive_amplitude(w["seed"])
    kd = 2 * np.pi / w["n"][0]
    N = parts["x"].size
    res = {"grid": "64^3", "particles": N, "steps": w["steps"], "ckpt_every": 20, "A": A}
    s = torch.cuda.Stream()
    for prec, name in ((pic.FP32_MIXED, "fp32_mixed"), (pic.FP64, "fp64")):
        with pic.Context(w["n"], cfl=w["cfl"], order=w["order"], precision=prec, stream=s) as ctx:
            ctx.load_particles(-1.0, 1.0, parts)
            ctx.set_external_drive(A, kd)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            loss, dA, du = ctx.step_adjoint(w["steps"], 20)
            t = time.perf_counter() - t0
            res[name] = {"seconds": t, "loss": loss, "dL_dA": dA, "dL_du_norm": float(np.linalg.norm(du)),
                         "forward_equiv_particle_steps_per_s": N * w["steps"] / t}
    res["fp32_vs_fp64_dL_dA_rel"] = abs(res["fp32_mixed"]["dL_dA"] - res["fp64"]["dL_dA"]) / abs(res["fp64"]["dL_dA"])
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-extras", action="store_true", help="skip FP64, error statement, e2e and CPU legs")
    ap.add_argument("--grid", type=int, default=0,
                    help="run the same recipe on an N^3 grid instead of 256^3 (small cases for profiling)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="precision of the timed headline run")
    ap.add_argument("--sort-every", type=int, default=1, help="sort cadence of the timed run")
    ap.add_argument("--workload", default=WORKLOAD, choices=["uniform_256", "uniform_256_o1"],
                    help="recipe of the timed run (uniform_256: order 3, 8 ppc; uniform_256_o1: order 1, 2 ppc)")
    ap.add_argument("--cpu-baselines", action="store_true",
                    help="time the oracle and the OpenMP baseline on every workload (CPU only, several minutes)")
    args = ap.parse_args()
    if args.cpu_baselines:
        from oracle import build as obuild
        from paper_2101_12149_gb300.inputs import build as ibuild
        obuild.build()
        obuild.build_mt()
        ibuild()
        cpu_baselines_per_config()
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from __graft_entry__ import build
    if rank == 0 or world == 1:
        build()
    if dist:
        dist.barrier()
        build()
    from paper_2101_12149_gb300 import inputs, pic

    w = inputs.WORKLOADS[args.workload]
    n, ppc, order = w["n"], w["ppc"], w["order"]
    if args.grid:
        n = (args.grid,) * 3
    C = n[0] * n[1] * n[2]
    N = C * ppc
    host, _keep = pinned_particles(N, torch)
    inputs.uniform_plasma(w["seed"] + rank * 7919, n, ppc, sigma_u=w["sigma_u"], density=w["density"], out=host)

    stream = torch.cuda.Stream()

    def make_ctx(prec, sort_every=1):
        ctx = pic.Context(n, cfl=w["cfl"], order=order, precision=prec, stream=stream, sort_every=sort_every)
        dev = {k: torch.from_numpy(v).to(f"cuda:{local}", non_blocking=False) for k, v in host.items()}
        ctx.load_particles(-1.0, 1.0, dev)
        del dev
        torch.cuda.empty_cache()
        return ctx

    # ---- headline: FP32-mixed, device-resident inputs ---------------------
    head_prec = pic.FP32_MIXED if args.precision == "fp32" else pic.FP64
    ctx = make_ctx(head_prec, args.sort_every)
    ctx.step(args.warmup)
    l0 = ctx.launch_count()
    uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid) if hasattr(
        torch.cuda.get_device_properties(local), "uuid") else str(local)
    if dist:
        dist.barrier()
    # the timed steps run as the library runs them (pairs of steps replayed as
    # one CUDA graph, no per-kernel events)
    with ClockSampler(uuid) as clk:
        t = timed_run(ctx, args.steps, stream, torch)
    launches = ctx.launch_count() - l0
    # per-kernel times: the same number of steps again, with CUDA events around
    # every kernel on the launching stream
    ctx.set_timing(True)
    t_evented = timed_run(ctx, args.steps, stream, torch)
    timings = ctx.get_timing()
    ctx.set_timing(False)
    t = max_over_ranks(t, dist, f"cuda:{local}")
    if dist:
        dist.barrier()
    value = job_throughput(world, N, args.steps, t)
    ms_step = 1e3 * t / args.steps
    ctx.close()

    peaks, peak_kind = measured_peaks()
    clocks = clk.summary()
    roofs = device_roofs(torch, pic, local, clocks, peaks)
    ms_tile, n_tile = timings.get("k_tile_step", (0.0, 0))
    avg_tile_s = ms_tile / max(n_tile, 1) / 1e3
    flops = N * flops_per_particle(order)
    alu_peak = roofs["fp32_measured_tflops"] if args.precision == "fp32" else roofs["fp64_measured_tflops"]
    alu_tf = flops / avg_tile_s / 1e12 if avg_tile_s > 0 else None
    hbm = bytes_per_launch(N, C, args.precision) / avg_tile_s / 1e9 if avg_tile_s > 0 else None
    alu_frac = alu_tf / alu_peak if alu_tf else None
    hbm_frac = hbm / peaks["hbm_gbs"] if hbm else None
    traffic = profiled_traffic("k_tile_step", args.precision, args.workload) if not args.grid else None
    roof_alu = {"bound": "alu", "achieved": alu_tf, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_frac,
                "traffic": traffic, "kernel": "k_tile_step",
                "peak_source": ("measured FP32 FMA microbenchmark (pic_measure_fma_peak)" if args.precision == "fp32"
                                else "measured FP64 FMA microbenchmark (pic_measure_fma_peak)"),
                "note": f"derived FP32 roof {roofs['fp32_derived_tflops']:.1f} TFLOP/s ({roofs['sms']} SMs x 128 "
                        f"lanes x 2 x {roofs['sm_max_mhz']:.0f} MHz); algorithmic flops "
                        f"{flops_per_particle(order)} per particle"}
    roof_hbm = {"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": hbm_frac,
                "traffic": traffic, "kernel": "k_tile_step", "peak_source": f"{peak_kind} hbm_gbs"}
    smem_peak = roofs["smem_derived_gbs"]
    smem = N * smem_bytes_per_particle(order, args.precision) / avg_tile_s / 1e9 if avg_tile_s > 0 else None
    roof_smem = {"bound": "smem", "achieved": smem, "peak": smem_peak, "unit": "GB/s",
                 "frac": smem / smem_peak if smem else None, "kernel": "k_tile_step",
                 "note": f"shared-memory roof derived from {roofs['sms']} SMs x 128 B/clock x "
                         f"{roofs['sm_max_mhz']:.0f} MHz; algorithmic bytes "
                         f"{smem_bytes_per_particle(order, args.precision)} per particle (gather loads + narrow "
                         "deposit reductions); the ncu profile gives the pipe's busy fraction including bank "
                         "conflicts and the two cycles of each reduction"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32-mixed" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": args.workload if not args.grid else f"{args.workload} recipe at {args.grid}^3",
                   "grid": f"{n[0]}^3", "ppc": ppc, "particles": N, "order": order,
                   "sigma_u": w["sigma_u"], "cfl": w["cfl"], "sort_every": args.sort_every,
                   "precision": "fp32_mixed" if args.precision == "fp32" else "fp64",
                   "l2": f"inputs larger than L2 ({N * 36 / 1e9:.1f} GB of particle state per step)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof_alu if (alu_frac or 0) >= (hbm_frac or 0) else roof_hbm,
        "roofline_alt": roof_hbm if (alu_frac or 0) >= (hbm_frac or 0) else roof_alu,
        "roofline_smem": roof_smem,
        "kernels_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in timings.items()},
        "ms_per_step_with_kernel_events": 1e3 * t_evented / args.steps,
        "kernel_share": {k: v[0] / max(sum(x[0] for x in timings.values()), 1e-30) for k, v in timings.items()},
        "kernel_rooflines": kernel_rooflines(timings, N, C, args.precision, peaks["hbm_gbs"]),
        "gpu_launches": int(launches),
        "clocks": clocks,
        "device_roofs": roofs,
        # context metrics: cells advanced per second and the paper's figure of
        # merit per GPU, cells (0.1 + 0.9 ppc) / time per step (Sec. 4.2)
        "cell_steps_per_s": job_throughput(world, C, args.steps, t),
        "fom_per_gpu": C * (0.1 + 0.9 * ppc) / (t / args.steps),
    }

    if not args.no_extras:
        # ---- end to end through the C-ABI with host buffers ----------------
        e2e_steps = args.steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2 = pic.Context(n, cfl=w["cfl"], order=order, precision=pic.FP32_MIXED, stream=stream)
        t1 = time.perf_counter()
        ctx2.load_particles(-1.0, 1.0, host)
        t2 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx2.step(1)
            ctx2.diagnostics()
        t3 = time.perf_counter()
        ex = ctx2.get_field("Ex")
        t_e2e = time.perf_counter() - t0
        phases = {"create": t1 - t0, "load": t2 - t1, "steps_with_diagnostics": t3 - t2,
                  "field_readback": t0 + t_e2e - t3}
        ctx2.close()
        h2d = 7 * 8 * N
        d2h = e2e_steps * 4 * 8 + ex.nbytes
        t_e2e = max_over_ranks(t_e2e, dist, f"cuda:{local}")
        line["e2e"] = {"value": job_throughput(world, N, e2e_steps, t_e2e), "unit": UNIT,
                       "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps,
                       "what": "context creation + pic_load_particles from pinned host FP64 arrays + "
                               f"{e2e_steps} x (pic_step + pic_diagnostics read-back) + E_x field read-back",
                       "phases_s": {k: round(v, 4) for k, v in phases.items()}}
        # ---- FP64 on the same workload -----------------------------------
        ctx64 = make_ctx(pic.FP64)
        ctx64.step(1)
        ctx64.set_timing(True)
        t64 = timed_run(ctx64, args.fp64_steps, stream, torch)
        tm64 = ctx64.get_timing()
        ctx64.close()
        torch.cuda.empty_cache()
        ms64, n64 = tm64.get("k_tile_step", (0.0, 0))
        fl64 = N * flops_per_particle(order) / (ms64 / max(n64, 1) / 1e3) / 1e12 if n64 else None
        t64 = max_over_ranks(t64, dist, f"cuda:{local}")
        line["fp64"] = {"value": job_throughput(world, N, args.fp64_steps, t64),
                        "ms_per_step": 1e3 * t64 / args.fp64_steps,
                        "steps": args.fp64_steps, "tile_kernel_tflops": fl64,
                        "tile_kernel_frac_of_fp64_peak": fl64 / roofs["fp64_measured_tflops"] if fl64 else None,
                        "fp32_mixed_speedup": value / job_throughput(world, N, args.fp64_steps, t64)}
        # ---- stated error of FP32-mixed ----------------------------------
        if rank == 0:
            line["error"] = field_error_statement(torch)
        # ---- the plasma-acceleration run's particle options on the same workload
        ctxa = make_ctx(pic.FP32_MIXED)
        ctxa.set_particle_algorithms("vay", "energy")
        ctxa.step(2)
        ta = timed_run(ctxa, args.fp64_steps * 3, stream, torch)
        ctxa.close()
        torch.cuda.empty_cache()
        line["vay_energy_gather"] = {"value": job_throughput(world, N, args.fp64_steps * 3, ta),
                                     "ms_per_step": 1e3 * ta / (args.fp64_steps * 3), "steps": args.fp64_steps * 3,
                                     "what": "FP32-mixed, Vay pusher and energy-conserving gather"}
        if rank == 0:
            line["hbm_bound"] = hbm_leg_statement(torch, stream, peaks)
            line["ensemble"] = ensemble_statement(torch, stream)
            line["adjoint"] = adjoint_statement(torch)
            line["sort_study"] = sort_study_statement(torch, stream, host, n)
            line["wakefield"] = wakefield_statement(torch)
        if rank == 0 and world == 1:
            line["cpu_baseline"] = cpu_baseline()
            line["cpu_baseline_mt"] = cpu_baseline_mt()

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
