"""Evolution driver: runs one of the workloads for a number of RK4 steps on
the current GPU (CUDA-graph replays of one step) in FP64 or in the mixed
precision, and reports the constraint monitors (Sec. "Hamiltonian and
momentum constraints": L2 of H, L2 of |M|, max |H|, max |M| over the points
of leaf patches, and the count of non-finite values) every `every` steps,
one JSON line per report. With --track, puncture trackers (Sec. "Particle
tracers": tracers dropped at the black holes that move with the opposite
shift by explicit Euler steps of the solver's dt, projected by trilinear
interpolation) follow the punctures, and each report carries their
positions. With --psi4 R1 R2 ..., each report carries the modes of psi_4
(appendix "psi_4 in ExaGRyPE") on spheres of those radii around the origin.

    python -m paper_2406_11626_gb300.evolve --workload binary --steps 500 --every 50 --precision mixed --track
"""
import json
import time

import numpy as np

from . import inputs as I

WORKLOADS = {
    "gauge_wave": lambda: I.gauge_wave_config(),
    "puncture144": lambda: I.single_puncture_config(),
    "mid": lambda: I.single_puncture_config(n_side=10, half_width=5.0),
    "puncture3level": lambda: I.multilevel_puncture_config(),
    "mesh-mid": lambda: I.multilevel_puncture_config(n_side=8, half_width=4.0, boxes=[((2, 2, 2), (6, 6, 6))]),
    "binary": lambda: I.binary_puncture_config(),
}


def initial_state(cfg, g):
    """Writes the initial state into U and (Sommerfeld) INI: the closed-form
    data of the configuration, or for the binary the Bowen-York state
    assembled on the device from the initial-data solve."""
    if cfg.name == "binary_puncture":
        from . import initial_data as ID
        t0 = time.perf_counter()
        solvers, B, sweeps = ID.solve_nested(cfg)
        ID.assemble_nested(solvers, B, g, "U")
        ID.assemble_nested(solvers, B, g, "INI")
        for s in solvers:
            s.close()
        return {"initial_data_sweeps": sweeps, "initial_data_boxes": [list(b) for b in cfg.extra["id_boxes"]],
                "initial_data_seconds": time.perf_counter() - t0}
    U0, G0 = I.initial_state(cfg)
    g.upload(U0, G0)
    if g.n_ghost:
        g.upload(U0, G0, buf="INI")
    return {}


def interface_mask(cfg):
    """(leaf, near) per interior point, each (n_patches, p, p, p) in the
    state's order (z, y, x within a patch): leaf marks the points of leaf
    patches (those the constraint norms run over); near marks the leaf
    points whose stencil (three points along each axis) reaches a halo point
    that the mesh interpolates from the coarser level, i.e. a neighbouring
    patch slot of the same level inside the domain that holds no patch. On a
    single level nothing is near."""
    p = cfg.p
    lev = np.asarray(getattr(cfg, "level", None) if getattr(cfg, "level", None) is not None
                     else np.zeros(cfg.n_patches, int))
    ijk = np.asarray(cfg.ijk()).reshape(-1, 3)
    nl = int(lev.max()) + 1
    slots = [set(map(tuple, ijk[lev == l])) for l in range(nl)]
    extent = [np.asarray(cfg.np) * 3 ** l for l in range(nl)]
    leaf = np.ones((len(lev), p, p, p), bool)
    near = np.zeros((len(lev), p, p, p), bool)
    loc = np.arange(p)
    side = {-1: loc < 3, 0: np.ones(p, bool), 1: loc > p - 4}
    for n in range(len(lev)):
        l = int(lev[n])
        if l + 1 < nl and tuple(3 * ijk[n]) in slots[l + 1]:
            leaf[n] = False
            continue
        if l == 0:
            continue
        for ox in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for oz in (-1, 0, 1):
                    nb = ijk[n] + (ox, oy, oz)
                    if (ox, oy, oz) == (0, 0, 0) or tuple(nb) in slots[l]:
                        continue
                    if (nb < 0).any() or (nb >= extent[l]).any():
                        continue  # the domain's ghost shell, not an interpolation
                    near[n] |= side[oz][:, None, None] & side[oy][None, :, None] & side[ox][None, None, :]
    return leaf, near


def interface_split(cfg, H, masks=None, centres=(), radius=1.0):
    """The L2 norm of H (sqrt of the mean of H^2, as the monitor) over the
    leaf points near a coarse-fine interface, over the others, and over the
    others at distance >= radius from every centre."""
    leaf, near = masks if masks is not None else interface_mask(cfg)
    h = np.asarray(H).reshape(leaf.shape)
    far = leaf & ~near
    out = {"L2_H_cf": float(np.sqrt((h[near] ** 2).mean())) if near.any() else 0.0,
           "L2_H_off_cf": float(np.sqrt((h[far] ** 2).mean())) if far.any() else 0.0,
           "points_cf": int(near.sum()), "points_off_cf": int(far.sum())}
    if centres:
        x, y, z = I.mesh_point_coords(cfg.p, cfg.level, cfg.ijk(), cfg.origin, cfg.dx) \
            if getattr(cfg, "level", None) is not None else I.point_coords(cfg.p, cfg.ijk(), cfg.origin, cfg.dx)
        r = np.full(leaf.shape, np.inf)
        for c in centres:
            r = np.minimum(r, np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2).reshape(leaf.shape))
        m = far & (r >= radius)
        out["L2_H_off_cf_r1"] = float(np.sqrt((h[m] ** 2).mean())) if m.any() else 0.0
    return out


def puncture_positions(cfg):
    """Initial puncture positions of a workload: the binary's two punctures
    at x = -d/2 and +d/2, the single puncture at the origin."""
    if cfg.name == "binary_puncture":
        h = 0.5 * cfg.extra["d"]
        return [(-h, 0.0, 0.0), (h, 0.0, 0.0)]
    if cfg.name == "single_puncture":
        return [(0.0, 0.0, 0.0)]
    return []


def run(workload="gauge_wave", steps=10, every=1, precision="fp64", launch="flat", log=None, track=False,
        id_boxes=None, split=False, psi4_radii=(), psi4_lmax=4):
    """Returns the reports: step 0 and every `every` steps up to `steps`,
    each {"step", "time", "L2_H", "L2_M", "max_H", "max_M", "nonfinite",
    "wall_s"}, for puncture workloads the same norms over the points at
    r >= 1 from every puncture ("..._r1"), and with track=True "punctures"
    (tracker positions, which then also centre the r >= 1 norms). id_boxes
    replaces the binary's nested initial-data boxes (() for the single
    global solve). split=True adds the L2 norm of H near and away from the
    coarse-fine interfaces (interface_split) to every report of a puncture
    workload. psi4_radii: for each radius, the modes l <= psi4_lmax of psi_4
    on the sphere of that radius around the origin (psi4.extract, the RHS
    buffer as scratch) in every report, as "psi4": {radius: {"l,m": [re, im]}}."""
    import torch
    from . import ccz4 as C
    if steps < 0 or every < 1:
        raise ValueError("steps must be >= 0 and every >= 1")
    cfg = WORKLOADS[workload]()
    if id_boxes is not None and "id_boxes" in cfg.extra:
        cfg.extra["id_boxes"] = tuple(id_boxes)
    g = C.Grid.from_config(cfg)
    g.set_launch(launch)
    extra = initial_state(cfg, g)
    P = C.make_params(**cfg.params, precision=precision)
    reports = []
    tracker = None
    if track and puncture_positions(cfg):
        tracker = C.Tracers(g, puncture_positions(cfg), velocity="shift")

    centres = puncture_positions(cfg)
    masks = interface_mask(cfg) if split and centres else None
    if centres:
        # per-point monitors, for the norms away from the punctures
        H = torch.empty(g.n_points, dtype=torch.float64, device="cuda")
        M = torch.empty(3 * g.n_points, dtype=torch.float64, device="cuda")

    def report(n, wall):
        nonlocal centres
        if centres:
            out = g.constraints("U", H.data_ptr(), M.data_ptr(), raise_nonfinite=False)
        else:
            out = g.constraints("U", raise_nonfinite=False)
        r = {"step": n, "time": n * cfg.dt, "L2_H": out[0], "L2_M": out[1], "max_H": out[2], "max_M": out[3],
             "nonfinite": out[4], "wall_s": wall}
        if tracker is not None:
            r["punctures"] = tracker.read()[0].tolist()
            centres = r["punctures"]
        if psi4_radii:
            from . import psi4 as PS
            r["psi4"] = {}
            for rad in psi4_radii:
                md, _ = PS.extract(g, float(rad), "U", "RHS", lmax=psi4_lmax)
                r["psi4"][str(rad)] = {"%d,%d" % k: [v.real, v.imag] for k, v in md.items()}
        if centres:
            # the norms without the points within r < 1 of a puncture (at its tracked position)
            ex = g.constraints_excluding(H.data_ptr(), M.data_ptr(), centres, 1.0)
            r.update({"L2_H_r1": ex[0], "L2_M_r1": ex[1], "max_H_r1": ex[2], "max_M_r1": ex[3]})
            if split:
                r.update(interface_split(cfg, H.cpu().numpy(), masks, centres))
        reports.append(r)
        if log:
            log(r)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    report(0, 0.0)
    n = 0
    while n < steps:
        k = min(every, steps - n)
        if tracker is None:
            g.step_graph(P, cfg.dt, k)
        else:
            # x^{t+dt} = x^t - dt beta(x^t): the tracker moves with the state at the start of each step
            for _ in range(k):
                tracker.step("U", cfg.dt)
                g.step_graph(P, cfg.dt, 1)
        n += k
        torch.cuda.synchronize()
        report(n, time.perf_counter() - t0)
    if tracker is not None:
        tracker.close()
    g.close()
    if log and extra:
        log(extra)
    return reports


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="evolve a CCZ4 workload on the GPU and monitor its constraints")
    ap.add_argument("--workload", default="gauge_wave", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--every", type=int, default=1)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--launch", default="flat", choices=["flat", "queue", "fused"])
    ap.add_argument("--track", action="store_true", help="follow the punctures with puncture trackers")
    ap.add_argument("--single-id-solve", action="store_true",
                    help="binary: initial data from the global solve alone, without the nested boxes")
    ap.add_argument("--interface-split", action="store_true",
                    help="puncture workloads: L2 of H near and away from the coarse-fine interfaces")
    ap.add_argument("--psi4", type=float, nargs="*", default=[],
                    help="radii of psi_4 extraction spheres around the origin (modes up to l = 4 per report)")
    a = ap.parse_args(argv)
    reps = run(a.workload, a.steps, a.every, a.precision, a.launch, log=lambda r: print(json.dumps(r), flush=True),
               track=a.track, id_boxes=() if a.single_id_solve else None, split=a.interface_split,
               psi4_radii=tuple(a.psi4))
    return 0 if reps and reps[-1]["nonfinite"] == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
