"""Autotuner for the patch edge and the launch shapes of a step.

The cost of a step depends on
- the patch edge p (single level only; the halo'd tile of a patch holds
  (p+6)^3 points for p^3 interior ones: 8x at p = 6, 4.6x at p = 9, 3.4x
  at p = 12, 2.6x at p = 17, so small patches move more halo data while
  large ones give the halo fill fewer, larger blocks);
- the launch of the stage kernel: a flat grid of one thread per point, a
  persistent launch whose warps take 32-point items from a device queue,
  or (p = 9) the fill and the stage in one cooperative launch per RK stage;
- the stage kernel's launch shape: the default number of resident
  128-thread blocks per SM, one more (fewer registers per thread, more
  warps to hide latency, more register spills), one fewer, or (mixed
  precision) two phases in one launch, the stencil values of each point
  parked in shared memory before the algebra runs on them;
- the halo fill's launch shape: threads per patch block and the number of
  independent loads per thread in its gather.
The tuner times one RK4 step (replays of the step captured as a CUDA graph,
the way a production loop runs it, CUDA events) of each candidate on the
workload itself and descends one coordinate at a time: first p and the
launch (every pair), then the stage shape, then the fill shape, each with
the others at their best so far. It keeps the fastest by point-stages per
second. Results are cached as JSON, keyed by the GPU, the library build,
the workload and the precision, so a production run pays for the sweep
once.

Workloads: the 144^3 single puncture (p swept at about the same number of
points), the three-level puncture and the four-level binary puncture mesh
(p = 9, the patch edge their level boxes are laid out for). The meshes are
timed on closed-form Brill-Lindquist data (the binary's two bare masses at
its puncture positions): the cost of a step does not depend on the values.
"""
import hashlib
import json
import os
import time

from . import inputs as I

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ccz4_gb300", "autotune.json")
# the patch edges of the paper's patch-size study, plus the largest edge the fill kernel takes
CANDIDATES = (6, 9, 12, 17, 18)
LAUNCHES = ("flat", "queue", "fused")
STAGE_SHAPES = (0, 1, 2, 3)   # default, one resident block more, one fewer, two phases (mixed)
FILL_SHAPES = (0, 1, 2, 3)    # 256 threads x 8 loads, 512 x 8, 256 x 16, 128 x 8
WORKLOADS = ("puncture144", "puncture3level", "binary")


def layouts(n_target, candidates=CANDIDATES, max_p=18):
    """(p, n_side) pairs with n_side * p closest to n_target points per axis,
    one per candidate p (n_side >= 1)."""
    out = []
    for p in candidates:
        if p < 1 or p > max_p:
            continue
        n_side = max(1, int(round(n_target / p)))
        out.append((p, n_side))
    return out


def workload_configs(workload, n_target=144, h=1.0 / 9.0, candidates=CANDIDATES):
    """The configurations a workload is tuned over: one per candidate patch
    edge for the single puncture, the mesh itself otherwise."""
    if workload == "puncture144":
        out = []
        for p, n_side in layouts(n_target, candidates):
            out.append(I.single_puncture_config(p=p, n_side=n_side, half_width=0.5 * n_side * p * h))
        return out
    if workload == "puncture3level":
        return [I.multilevel_puncture_config()]
    if workload == "binary":
        return [I.binary_puncture_config()]
    raise ValueError("unknown workload %r" % (workload,))


def timing_state(cfg):
    """(U, G) to time a configuration with: its closed-form data, or for the
    binary mesh Brill-Lindquist data of its two bare masses."""
    if cfg.name != "binary_puncture":
        return I.initial_state(cfg)
    m, d = cfg.extra["m1"], 0.5 * cfg.extra["d"]
    cen = ((-d, 0.0, 0.0), (d, 0.0, 0.0))
    x, y, z = I.mesh_point_coords(cfg.p, cfg.level, cfg.ijk(), cfg.origin, cfg.dx)
    gx, gy, gz = I.ghost_positions(cfg.N, cfg.origin, cfg.dx)
    return I.brill_lindquist(x, y, z, (m, m), cen), I.brill_lindquist(gx, gy, gz, (m, m), cen)


def _lib_hash():
    from .ccz4 import LIB_PATH
    h = hashlib.sha256()
    with open(LIB_PATH, "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def time_config(cfg, precision="fp64", steps=3, warmup=2, launch="flat", stage_shape=0, fill_shape=0):
    """Seconds per RK4 step of a configuration with the given launch and
    shapes (graph replay, CUDA events), and its number of points."""
    import torch
    from . import ccz4 as C
    g = C.Grid.from_config(cfg)
    g.set_launch(launch)
    g.set_tuning(stage_shape, fill_shape)
    U, G = timing_state(cfg)
    g.upload(U, G)
    if g.n_ghost:
        g.upload(U, G, buf="INI")
    P = C.make_params(**cfg.params, precision=precision)
    stream = torch.cuda.current_stream()
    g.step_graph(P, cfg.dt, warmup, stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    g.step_graph(P, cfg.dt, steps, stream)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) * 1e-3 / steps
    n_points = cfg.n_points
    g.close()
    return sec, n_points


def _name(p, launch, stage_shape, fill_shape):
    return "p%d/%s/stage%d/fill%d" % (p, launch, stage_shape, fill_shape)


def tune(workload="puncture144", precision="fp64", n_target=144, h=1.0 / 9.0, candidates=CANDIDATES, steps=3,
         warmup=2, cache=DEFAULT_CACHE, timer=None, key_extra=None, refresh=False, launches=LAUNCHES,
         stage_shapes=STAGE_SHAPES, fill_shapes=FILL_SHAPES):
    """Chooses p, the launch and the launch shapes for a workload. Returns
    {"workload", "p", "n_side", "launch", "stage_shape", "fill_shape",
    "point_stages_per_s", "results": {name: {...}}, "key"}.

    timer(cfg, precision, steps, warmup, launch, stage_shape, fill_shape)
    -> (seconds per step, points) may replace the GPU timing (tests use a
    fake one); key_extra replaces the GPU/library part of the cache key."""
    if timer is None:
        timer = time_config
        key_extra = key_extra or "%s|%s" % (_gpu_name(), _lib_hash())
    key = "%s|%s|%s|n=%d|h=%.17g|p=%s|%s|s=%s|f=%s" % (
        key_extra, workload, precision, n_target, h, ",".join(map(str, candidates)), ",".join(launches),
        ",".join(map(str, stage_shapes)), ",".join(map(str, fill_shapes)))
    store = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            store = json.load(f)
        if key in store and not refresh:
            return store[key]
    cfgs = {c.p: c for c in workload_configs(workload, n_target, h, candidates)}
    results = {}

    def run(p, launch, s, f):
        name = _name(p, launch, s, f)
        if name not in results:
            cfg = cfgs[p]
            sec, n_points = timer(cfg, precision, steps, warmup, launch, s, f)
            results[name] = {"p": p, "launch": launch, "stage_shape": s, "fill_shape": f,
                             "n_side": cfg.np[0], "points": n_points, "s_per_step": sec,
                             "point_stages_per_s": 4.0 * n_points / sec}
        return results[name]["point_stages_per_s"]

    # 1. patch edge and launch, shapes at their defaults
    pairs = [(p, l) for p in cfgs for l in launches if l != "fused" or p == 9]
    best = max(pairs, key=lambda q: run(q[0], q[1], 0, 0))
    p, launch = best
    # 2. the stage kernel's shape (the shapes apply to the flat launch)
    stage = 0
    if launch == "flat":
        stage = max(stage_shapes, key=lambda s: run(p, launch, s, 0))
    # 3. the fill's shape (the fused launch has its own)
    fill = 0 if launch == "fused" else max(fill_shapes, key=lambda f: run(p, launch, stage, f))
    win = results[_name(p, launch, stage, fill)]
    entry = {"workload": workload, "precision": precision, "p": p, "n_side": win["n_side"], "launch": launch,
             "stage_shape": stage, "fill_shape": fill, "point_stages_per_s": win["point_stages_per_s"],
             "results": results, "key": key, "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if cache:
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        store[key] = entry
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return entry


def compare(workload, precision, launches, p=9, steps=10, warmup=3, repeats=2, timer=None):
    """Milliseconds per RK4 step of each launch on a workload at patch edge
    p with the default shapes, timed `repeats` times in turn (graph replay,
    CUDA events): {"workload", "precision", "p", "points", launch: [ms, ...]}."""
    timer = timer or time_config
    cfg = {c.p: c for c in workload_configs(workload, candidates=(p,))}[p]
    row = {"workload": workload, "precision": precision, "p": p, "points": cfg.n_points}
    for _ in range(repeats):
        for launch in launches:
            sec, _n = timer(cfg, precision, steps, warmup, launch, 0, 0)
            row.setdefault(launch, []).append(round(sec * 1e3, 3))
    return row


def apply(grid, entry):
    """Sets a grid's launch and launch shapes to a tuner entry."""
    grid.set_launch(entry["launch"])
    grid.set_tuning(entry["stage_shape"], entry["fill_shape"])


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="tune the launch of the CCZ4 step on this GPU")
    ap.add_argument("--workload", nargs="+", default=list(WORKLOADS), choices=WORKLOADS)
    ap.add_argument("--precision", nargs="+", default=["fp64", "mixed"], choices=["fp64", "mixed"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--cache", default=DEFAULT_CACHE)
    ap.add_argument("--refresh", action="store_true")
    ap.add_argument("--compare", nargs="+", choices=LAUNCHES, metavar="LAUNCH",
                    help="no tuning: time these launches at p = 9 with the default shapes")
    ap.add_argument("--repeats", type=int, default=2)
    a = ap.parse_args(argv)
    if a.compare:
        for w in a.workload:
            for prec in a.precision:
                print(json.dumps(compare(w, prec, a.compare, steps=a.steps, warmup=a.warmup, repeats=a.repeats)),
                      flush=True)
        return 0
    for w in a.workload:
        for prec in a.precision:
            e = tune(w, prec, steps=a.steps, warmup=a.warmup, cache=a.cache, refresh=a.refresh)
            print(json.dumps(e), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
