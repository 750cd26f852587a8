#!/usr/bin/env python3
"""Throughput benchmark of the CCZ4 FD4 hot path on GB300.

Workload: the single static puncture of mass M = 1 at the origin (Brill-
Lindquist data, 1+log slicing, Gamma-driver shift with eta = 2, Kreiss-Oliger
0.1, Sommerfeld boundary), [-8, 8]^3 as 16^3 patches of 9^3 points
(144^3 = 2,985,984 points, dx = 1/9), classic RK4 with dt = 0.1 dx.
A step is one RK4 step over the whole grid: for each of the four stages the
halo fill and the fused right-hand-side + stage-update kernel (plus the
Sommerfeld ghost-cell kernel). Metric: point-stages per second
(interior points x 4 stages x steps / time).

Prints one JSON line. --impl reference times the CPU oracle instead (the
plain FP64 restatement of the paper that the parity tests use) on a bounded
sample of the same physics.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CCZ4 RHS+RK point-stages/s at 1 GB300, mixed vs FP64 at stated error; % roofline"
UNIT = "point-stages/s"
# FP64 pipe of GB300: 152 SMs x 2 FP64 FMA per clock x 2 flops at the 2070 MHz
# maximum SM clock (the nominal 1.25 TFLOP/s FP64 rate).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
KERNEL_SOURCES = ("paper_2406_11626_gb300/csrc/stage_kernels.cuh", "paper_2406_11626_gb300/csrc/ccz4_algebra.cuh",
                  "paper_2406_11626_gb300/csrc/ccz4_internal.cuh")


def measure_fma_peaks():
    """FP64 and FP32 FMA throughput of this GPU (TFLOP/s), from the probe in
    paper_2406_11626_gb300/measure (eight independent FMA chains per thread,
    eight blocks of 256 threads per SM), or None if its library is missing."""
    import ctypes
    path = os.path.join(ROOT, "paper_2406_11626_gb300", "lib", "libccz4_peaks.so")
    if not os.path.exists(path):
        return None
    L = ctypes.CDLL(path)
    f = L.ccz4_probe_fma_rate
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    out = {}
    for prec, iters in ((64, 4000), (32, 200000)):
        best = 0.0
        for _ in range(3):
            t, ms = ctypes.c_double(), ctypes.c_double()
            if f(prec, 8, iters, ctypes.byref(t), ctypes.byref(ms)) != 0:
                return None
            best = max(best, t.value)
        out["fp%d_tflops" % prec] = best
    out["how"] = "FMA-chain probe (measure/fma_peaks.cu), best of 3 launches of 8 x 256-thread blocks per SM"
    return out


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--workload", default="puncture144",
                    choices=["puncture144", "puncture3level", "binary", "mid", "small", "mesh-mid"],
                    help="the same physics on fewer points, for profiler captures: mid = 90^3 (10^3 patches), "
                         "small = 54^3 (6^3 patches), mesh-mid = two levels (2240 patches)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision comparison")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.5)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r[2] > 200.0] or rows
        sm = sorted(r[0] for r in load)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(load), "power_w_max": max(r[2] for r in rows)}


# ----------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------
def oracle_sample_config(workload="puncture144"):
    """Same physics and grid spacing as the workload on a sub-box around the
    puncture: 36^3 points (4^3 patches of 9^3, [-2, 2]^3); for the
    three-level workload, those 4^3 level-0 patches with the central 2^3
    refined once and one level-1 patch refined again (307 patches)."""
    from paper_2406_11626_gb300 import inputs as I
    if workload in ("puncture3level", "binary", "mesh-mid"):
        # the binary uses the same multi-level sample: the oracle's rate per
        # point-stage does not depend on the data
        return I.multilevel_puncture_config(n_side=4, half_width=2.0,
                                            boxes=[((1, 1, 1), (3, 3, 3)), ((4, 4, 4), (5, 5, 5))])
    return I.single_puncture_config(n_side=4, half_width=2.0)


def sample_text(cfg):
    if getattr(cfg, "level", None) is not None:
        return "%d patches of 9^3 on 3 levels around the puncture ([-2,2]^3, dx = 1/9, 1/27, 1/81)" % cfg.n_patches
    return "%d^3 points (4^3 patches of 9^3, [-2,2]^3)" % cfg.N[0]


def time_oracle(n_steps, n_warm=0, workload="puncture144"):
    import oracle as O
    from paper_2406_11626_gb300 import inputs as I
    cfg = oracle_sample_config(workload)
    og = O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc, level=getattr(cfg, "level", None))
    U, G = I.initial_state(cfg)
    P = O.make_params(**cfg.params)
    for _ in range(n_warm):
        U, G = og.rk4_step(P, cfg.dt, U, G, G)
    t0 = time.perf_counter()
    Gini = G
    for _ in range(n_steps):
        U, G = og.rk4_step(P, cfg.dt, U, G, Gini)
    dt = time.perf_counter() - t0
    return cfg, dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle_threads(n_steps, n_threads, workload="puncture144"):
    """The oracle on all host cores: n_threads threads, each stepping its
    own copy of the sample n_steps times (the oracle's C code holds no
    shared mutable state, and ctypes releases the interpreter lock during
    each call, so the copies run in parallel). Returns (cfg, wall seconds)."""
    import threading
    import oracle as O
    from paper_2406_11626_gb300 import inputs as I
    cfg = oracle_sample_config(workload)
    P = O.make_params(**cfg.params)
    U0, G0 = I.initial_state(cfg)
    grids = [O.Grid(cfg.p, cfg.np, cfg.ijk(), cfg.origin, cfg.dx, cfg.bc, level=getattr(cfg, "level", None))
             for _ in range(n_threads)]
    start = threading.Barrier(n_threads + 1)
    done = threading.Barrier(n_threads + 1)

    def work(og):
        U, G = U0, G0
        start.wait()
        for _ in range(n_steps):
            U, G = og.rk4_step(P, cfg.dt, U, G, G0)
        done.wait()

    th = [threading.Thread(target=work, args=(og,)) for og in grids]
    for t in th:
        t.start()
    start.wait()
    t0 = time.perf_counter()
    done.wait()
    wall = time.perf_counter() - t0
    for t in th:
        t.join()
    return cfg, wall


def cpu_baseline(target_s=12.0, workload="puncture144"):
    """The oracle on the host: all cores (one sample per core, in parallel)
    as the value, and one core beside it."""
    cfg, t1 = time_oracle(1, workload=workload)
    n = max(1, int(target_s / 2 / max(t1, 1e-3)))
    cfg, t = time_oracle(n, workload=workload)
    v1 = cfg.n_points * 4 * n / t
    cores = host_cores()
    cfg, tw = time_oracle_threads(n, cores, workload=workload)
    v = cfg.n_points * 4 * n * cores / tw
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d RK4 steps of the same puncture physics and dx on %s per core, plain C FP64, "
                      "one independent copy per host core in parallel" % (n, sample_text(cfg)),
            "single_core": {"value": v1, "cores": 1, "sample": "%d RK4 steps on one copy, one thread" % n}}


def run_reference(args):
    """The oracle as it stands, on all host cores: each timed step is one
    RK4 step of the bounded sample on every core (one independent copy per
    core, in parallel)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = args.workload
    cores = host_cores()
    if args.warmup > 0:
        time_oracle_threads(args.warmup, cores, workload=wl)
    steps = max(args.steps, 1)
    cfg, t = time_oracle_threads(steps, cores, workload=wl)
    v = cfg.n_points * 4 * steps * cores / t
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(None, workload=wl),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "each step: one RK4 step of the puncture physics on " + sample_text(cfg)
                                   + " on each of the %d host cores (one copy per core, in parallel)" % cores},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(g, precision="fp64", K=None, workload="puncture144"):
    import numpy as np
    from paper_2406_11626_gb300 import inputs as I
    if workload == "small":
        cfg = I.single_puncture_config(n_side=6, half_width=3.0)
        name = "single puncture M=1, [-3,3]^3, 6^3 patches of 9^3 (54^3 points), profiling case"
    elif workload == "mid":
        cfg = I.single_puncture_config(n_side=10, half_width=5.0)
        name = "single puncture M=1, [-5,5]^3, 10^3 patches of 9^3 (90^3 points), profiling case"
    elif workload == "mesh-mid":
        cfg = I.multilevel_puncture_config(n_side=8, half_width=4.0, boxes=[((2, 2, 2), (6, 6, 6))])
        name = ("single puncture M=1 on 2 static ratio-3 levels: [-4,4]^3 as 8^3 patches of 9^3 (dx 1/9), "
                "central 4^3 refined to 12^3 patches (dx 1/27): 2240 patches, profiling case")
    elif workload == "binary":
        cfg = I.binary_puncture_config()
        name = ("rotating binary puncture: bare masses 0.487 at x = -3, +3, momenta (0, -+0.0934, 0), no spin, "
                "Bowen-York data (u by the plain relaxation solve, over-relaxed by 1.98, on 192^3 cells of "
                "[-32,32]^3, then on nested boxes of h = 1/8, 1/16, 1/64 around the punctures, each to residual "
                "1e-10); [-32,32]^3 on 4 ratio-3 levels of 9^3 patches (4096/5832/3456/6912, dx 4/9 .. 4/243); "
                "1+log, Gamma-driver f=0.75 eta=1, KO 0.1, Sommerfeld, RK4 dt=0.1 dx_finest")
    elif workload == "puncture3level":
        cfg = I.multilevel_puncture_config()
        name = ("single puncture M=1 on 3 static ratio-3 levels: [-8,8]^3 as 16^3 patches of 9^3 (dx 1/9), "
                "central 4^3 refined to 12^3 patches (dx 1/27), their central 4^3 refined to 12^3 patches "
                "(dx 1/81); 1+log, Gamma-driver eta=2, KO 0.1, Sommerfeld, RK4 dt=0.1 dx_finest, "
                "restriction after every step")
    else:
        cfg = I.single_puncture_config()
        name = ("single puncture M=1, [-8,8]^3, 16^3 patches of 9^3 (144^3 points), "
                "1+log, Gamma-driver eta=2, KO 0.1, Sommerfeld, RK4 dt=0.1dx")
    c = {"workload": name,
         "patches": cfg.n_patches, "p": cfg.p, "points": cfg.n_points, "dx": cfg.dx,
         "precision": precision,
         "l2": "inputs larger than L2 (129 MB): each state buffer is 25 x %.2fM doubles = %.0f MB, "
               "the halo tiles %.0f MB" % ((cfg.n_points + 0) / 1e6, 8 * 25 * cfg.n_points / 1e6,
                                         8 * 25 * cfg.n_patches * (cfg.p + 6) ** 3 / 1e6)}
    if getattr(cfg, "level", None) is not None:
        c["levels"] = cfg.n_levels
        c["patches_per_level"] = [int(v) for v in np.bincount(cfg.level)]
        c["leaf_points"] = int(sum(cfg.p ** 3 for n in range(cfg.n_patches) if not _has_children(cfg, n)))
        c["units"] = "every evolved point of every level (coarse points under finer patches included)"
    if g is not None:
        c["ghost_cells"] = g.n_ghost
    return c


def _has_children(cfg, n):
    l = cfg.level[n]
    if l + 1 >= cfg.n_levels:
        return False
    kids = cfg.ijk()[cfg.level == l + 1] // 3
    return bool((kids == cfg.ijk()[n]).all(axis=1).any())


# ----------------------------------------------------------------------------
# GB300 arm
# ----------------------------------------------------------------------------
def load_traffic(n_points, precision="fp64", mesh=False):
    """DRAM bytes of one stage-kernel launch over n_points, from the ncu
    capture of the single-level instance of that precision recorded in
    profiles/traffic.json, scaled by points; None for a refined mesh, for a
    precision without a record, or once the kernel sources have changed."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("kernel_hash") != kernel_hash() or mesh:
        return None
    cap = d.get(precision, {})
    if not cap.get("points"):
        return None
    return (cap["dram_bytes_read"] + cap["dram_bytes_write"]) * n_points / cap["points"]


def bench_config(args):
    from paper_2406_11626_gb300 import inputs as I
    if args.workload == "small":
        return I.single_puncture_config(n_side=6, half_width=3.0)
    if args.workload == "mid":
        return I.single_puncture_config(n_side=10, half_width=5.0)
    if args.workload == "mesh-mid":
        return I.multilevel_puncture_config(n_side=8, half_width=4.0, boxes=[((2, 2, 2), (6, 6, 6))])
    if args.workload == "puncture3level":
        return I.multilevel_puncture_config()
    if args.workload == "binary":
        return I.binary_puncture_config()
    return I.single_puncture_config()


_ID_CACHE = {}


def init_state(C, I, cfg, g):
    """Initial state into U and INI: closed-form data uploaded from the host,
    or, for the binary, the state assembled on the device from the
    initial-data solve (solved once per process, outside any timed region)."""
    if cfg.name == "binary_puncture":
        from paper_2406_11626_gb300 import initial_data as ID
        if "binary" not in _ID_CACHE:
            _ID_CACHE["binary"] = ID.solve_nested(cfg)
        solvers, B, _ = _ID_CACHE["binary"]
        ID.assemble_nested(solvers, B, g, "U")
        ID.assemble_nested(solvers, B, g, "INI")
        return
    U0, G0 = I.initial_state(cfg)
    g.upload(U0, G0)
    g.upload(U0, G0, buf="INI")


def time_path(C, I, cfg, precision, K, W, stream, dist, clocks_index=None):
    """Builds a grid, runs W warm-up and K timed RK4 steps; returns the grid,
    the time of the K steps and the per-stage kernel times (ms)."""
    import torch
    g = C.Grid.from_config(cfg)
    init_state(C, I, cfg, g)
    P = C.make_params(**cfg.params, precision=precision)
    bufs = [C.stage_buffers(s) for s in range(4)]

    def step(ev=None):
        for s in range(4):
            g.fill_halos(bufs[s][0], stream, P)
            if ev is not None:
                ev[s][0].record(stream)
            g.rk_stage(P, s, cfg.dt, stream, fill=False)
            if ev is not None:
                ev[s][1].record(stream)

    for _ in range(W):
        step()
    torch.cuda.synchronize()
    kev = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(4)] for _ in range(K)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(clocks_index) if clocks_index is not None else None
    if clk:
        clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(K):
        step(kev[k])
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop() if clk else None
    ms = e0.elapsed_time(e1)
    stage_ms = [kev[k][s][0].elapsed_time(kev[k][s][1]) for k in range(K) for s in range(4)]
    return g, P, ms, stage_ms, clocks


def time_graph(g, P, dt, K, W, stream, dist):
    """K RK4 steps through ccz4_step_graph (one captured CUDA graph per step,
    the path a time loop of the library runs), after W warm-up replays (the
    first one captures the graph); returns milliseconds."""
    import torch
    g.step_graph(P, dt, max(W, 1), stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    g.step_graph(P, dt, K, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return e0.elapsed_time(e1)


def time_first_order(C, I, cfg, K, W, stream):
    """The paper's two other formulations on the same workload (single
    level): the first-order one (58 variables evolved, red terms) and the
    second-order one with the reconstruction sweep of the auxiliary
    variables, K RK4 steps after W warm-up steps each; ms per step."""
    import torch
    g = C.Grid.from_config(cfg)
    U, G = I.fo_initial_state(cfg)
    P = C.make_params(**cfg.params)
    out = {}
    for variant in ("fo", "so-recon"):
        fo = C.FirstOrder(g, variant)
        fo.upload(U, G)
        if g.n_ghost:
            fo.upload(U, G, buf="INI")
        fo.step(P, cfg.dt, W, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fo.step(P, cfg.dt, K, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out[variant] = e0.elapsed_time(e1) / K
        fo.close()
    g.close()
    return out


def max_over_ranks(x, dist, device):
    """The largest value of x over the ranks (the slowest rank sets the job time)."""
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, n_points, stages, seconds):
    """Whole-job point-stages/s: the units all ranks processed (weak scaling,
    each rank its own copy of the workload) over the job time."""
    return world * n_points * stages / seconds


def run_gb300(args):
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2406_11626_gb300 import ccz4 as C
    from paper_2406_11626_gb300 import inputs as I
    cfg = bench_config(args)
    stream = torch.cuda.current_stream()
    K = args.steps
    g, P, ms, stage_ms, clocks = time_path(C, I, cfg, args.precision, K, args.warmup, stream, dist, local)
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_rate(world, cfg.n_points, 4 * K, ms * 1e-3)
    out = g.constraints("U", raise_nonfinite=False)
    ms_graph = max_over_ranks(time_graph(g, P, cfg.dt, K, args.warmup, stream, dist), dist, "cuda")
    peaks = measure_fma_peaks() if rank == 0 else None

    # end to end through the C ABI from pinned host memory, one step per call
    n_state = g.n_points + g.n_ghost
    Uh = torch.empty((I.NV, g.n_points), dtype=torch.float64, pin_memory=True).numpy()
    Gh = torch.empty((I.NV, max(g.n_ghost, 1)), dtype=torch.float64, pin_memory=True).numpy()[:, :g.n_ghost]
    Ud, Gd = g.download("U")
    Uh[...] = Ud.reshape(I.NV, -1)
    Gh[...] = Gd
    E = max(1, args.e2e_steps)
    g.evolve_host(P, cfg.dt, 1, Uh, Gh, Uh, Gh, stream)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(E):
        g.evolve_host(P, cfg.dt, 1, Uh, Gh, Uh, Gh, stream)
    t_e2e = time.perf_counter() - t0
    e2e_value = job_rate(world, cfg.n_points, 4 * E, max_over_ranks(t_e2e, dist, "cuda"))

    mixed = None
    if not args.no_mixed and args.precision == "fp64":
        # the mixed path on the same workload, same steps; its state is
        # compared with the FP64 state after the same W + K steps
        g64, _, _, _, _ = time_path(C, I, cfg, "fp64", K, args.warmup, stream, None)
        gmx, _, ms_mx, stage_mx, _ = time_path(C, I, cfg, "mixed", K, args.warmup, stream, None)
        a, _ = g64.download("U")
        b, _ = gmx.download("U")
        a = a.reshape(I.NV, -1)
        b = b.reshape(I.NV, -1)
        err = np.abs(b - a).max(axis=1) / np.maximum(np.abs(a).max(axis=1), 1.0)
        # root-mean-square difference over all interior points, same scaling
        rms = lambda x: np.sqrt(np.mean(np.square(x), axis=1))
        err2 = rms(b - a) / np.maximum(rms(a), 1.0)
        c64 = g64.constraints("U", raise_nonfinite=False)
        cmx = gmx.constraints("U", raise_nonfinite=False)
        flm = C.flops_per_point_stage("mixed")
        t_stage_mx = sum(stage_mx) / len(stage_mx) * 1e-3
        t_roof_mx = max(flm["fp64"] * cfg.n_points / (FP64_PEAK_TFLOPS * 1e12),
                        flm["fp32"] * cfg.n_points / (FP32_PEAK_TFLOPS * 1e12))
        mixed = {"value": world * cfg.n_points * 4 * K / (ms_mx * 1e-3), "unit": UNIT,
                 "speedup_vs_fp64": ms / ms_mx, "ms_per_step": ms_mx / K,
                 "dtype": "f64 state/1-over-phi terms/update + f64-accurate differences on split f32 pairs + f32 algebra",
                 "max_rel_state_error_vs_fp64": float(err.max()),
                 "worst_field": I.FIELDS[int(err.argmax())],
                 "rel_state_error_per_field": {f: float(e) for f, e in zip(I.FIELDS, err)},
                 "rms_state_error_per_field": {f: float(e) for f, e in zip(I.FIELDS, err2)},
                 "after_steps": K + args.warmup,
                 "L2_H": cmx[0], "L2_H_fp64": c64[0], "L2_M": cmx[1], "L2_M_fp64": c64[1],
                 "roofline_frac": t_roof_mx / t_stage_mx, "stage_kernel_ms": t_stage_mx * 1e3,
                 "traffic": load_traffic(cfg.n_points, "mixed", g.n_levels > 1),
                 "fp64_flops_per_point_stage": flm["fp64"], "fp32_flops_per_point_stage": flm["fp32"]}
        del g64, gmx

    first_order = None
    if not args.no_mixed and args.precision == "fp64" and getattr(cfg, "level", None) is None:
        fo_ms = time_first_order(C, I, cfg, K, args.warmup, stream)
        first_order = {
            variant: {"value": world * cfg.n_points * 4 / (t * 1e-3), "unit": UNIT, "ms_per_step": t,
                      "vs_second_order_path": (ms / K) / t}
            for variant, t in fo_ms.items()}
        first_order["how"] = ("ccz4_fo_step on the same workload and steps: 'fo' the first-order formulation "
                              "(58 variables evolved, red terms), 'so-recon' the second-order formulation over "
                              "the 58 variables with the auxiliary variables reconstructed before every stage; "
                              "vs_second_order_path = this build's second-order step time / this one's (>1: faster)")

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    fl = C.flops_per_point_stage(args.precision)
    t_stage = sum(stage_ms) / len(stage_ms) * 1e-3
    f64 = fl["fp64"] * cfg.n_points
    f32 = fl["fp32"] * cfg.n_points
    if args.precision == "fp64" or f32 == 0:
        roof = {"bound": "alu", "achieved": f64 / t_stage / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": f64 / t_stage / 1e12 / FP64_PEAK_TFLOPS, "traffic": load_traffic(cfg.n_points, args.precision, g.n_levels > 1),
                "kernel": "interior_kernel (fused RHS + RK stage) with the ghost-cell kernel of the same stage",
                "flops_per_point_stage": fl["fp64"], "units_per_launch": cfg.n_points,
                "peak_source": "FP64 pipe: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz",
                "peak_measured": peaks}
    else:
        t_roof = max(f64 / (FP64_PEAK_TFLOPS * 1e12), f32 / (FP32_PEAK_TFLOPS * 1e12))
        roof = {"bound": "alu", "achieved": f64 / t_stage / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": t_roof / t_stage, "traffic": load_traffic(cfg.n_points, args.precision, g.n_levels > 1),
                "fp64_flops_per_point_stage": fl["fp64"], "fp32_flops_per_point_stage": fl["fp32"],
                "fp32_tflops": f32 / t_stage / 1e12,
                "note": "frac = max(F64/P64, F32/P32) / kernel time", "peak_measured": peaks}
    launches_per_stage = 2 + (1 if g.n_ghost > 0 else 0)
    restrict_per_step = g.n_levels - 1
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64 state + f32 algebra",
        "data": ("synthetic (Bowen-York binary data from the initial-data solve)" if args.workload == "binary"
                 else "synthetic (Brill-Lindquist puncture data generated in closed form)"),
        "config": workload_config(g, args.precision, K, args.workload),
        "stage_kernel_ms": sum(stage_ms) / len(stage_ms),
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * I.NV * n_state,
                "d2h_bytes_per_step": 8 * I.NV * n_state,
                "how": "ccz4_evolve_host per step: pinned host state -> device, one RK4 step, device -> host"},
        "gpu_launches": (launches_per_stage * 4 + restrict_per_step) * K,
        "graph": {"value": job_rate(world, cfg.n_points, 4 * K, ms_graph * 1e-3), "unit": UNIT,
                  "ms_per_step": ms_graph / K, "gpu_launches": (launches_per_stage * 4 + restrict_per_step) * K,
                  "how": "ccz4_step_graph: each RK4 step one replay of a captured CUDA graph (the halo fills, "
                         "stage kernels, ghost kernels and restriction of the step), the same K steps after the "
                         "launch-path run; value and the kernel times above come from the launch path"},
        "constraints_after": {"L2_H": out[0], "L2_M": out[1], "max_H": out[2], "nonfinite": out[4]},
    }
    if mixed is not None:
        line["mixed"] = mixed
    if first_order is not None:
        line["first_order"] = first_order
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(workload=args.workload)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
