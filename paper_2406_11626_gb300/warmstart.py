"""Learned warm start of the puncture initial-data solve.

Binding of include/ccz4_mlp.h (argument marshalling only: the network's
forward pass, back-propagation, Adam, feature assembly and the hand-over of
its output to the solver run in the library's CUDA kernels) and the
orchestration of the experiment:

1. draws: a scrambled Sobol sequence (seed 0) over the binary parameters
   m1, m2 in [0.3, 0.7], d in [2, 12], P in [0, 0.2], S in [0, 0.3];
2. data: the plain relaxation solve (initial_data.Solver, from u = 0, to a
   max residual of 1e-10) of every training draw on n^3 cells of
   [-L, L]^3, kept on the device in FP32;
3. training: Adam on the mean squared error of the scaled correction at
   cells drawn uniformly (host-seeded) from the stored solutions;
4. evaluation: on held-out draws, sweeps to the same tolerance from the
   network's guess against sweeps from u = 0, with the same relaxation (by
   default red-black Newton-SOR with the factor that needs the fewest sweeps
   on three training draws; omega = 1 gives plain Gauss-Seidel). The plain
   solve stays the arbiter: a guess is only a starting point, and a solve
   that does not reach the tolerance reports -1.
"""
import ctypes
import math
import time

import numpy as np

from .ccz4 import _check, _stream, _wrap_device, lib as _lib
from . import initial_data as ID

N_FEATURES = 8
U_SCALE = 10.0
RANGES = ((0.3, 0.7), (0.3, 0.7), (2.0, 12.0), (0.0, 0.2), (0.0, 0.3))  # m1, m2, d, P, S


def _sig():
    L = _lib()
    if getattr(L, "_mlp_ready", False):
        return L
    vp = ctypes.c_void_p
    fp = ctypes.POINTER(ctypes.c_float)
    ll = ctypes.POINTER(ctypes.c_longlong)
    sigs = {
        "ccz4_mlp_create": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)],
        "ccz4_mlp_free": [vp],
        "ccz4_mlp_params": [vp, ctypes.POINTER(fp), ll],
        "ccz4_mlp_grads": [vp, ctypes.POINTER(fp), ll],
        "ccz4_mlp_forward": [vp, vp, ctypes.c_int, vp, vp],
        "ccz4_mlp_loss_grad": [vp, vp, vp, ctypes.c_int, vp, vp],
        "ccz4_mlp_adam": [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, vp],
        "ccz4_mlp_features_grid": [ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double), vp, vp],
        "ccz4_mlp_features_sample": [ctypes.c_int, ctypes.c_double, vp, vp, vp, ctypes.c_int, vp, vp, vp],
        "ccz4_mlp_output_to_u": [vp, ctypes.c_longlong, vp, vp],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L._mlp_ready = True
    return L


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def init_params(n_in=8, width=128, depth=4, seed=0):
    """Layer-wise uniform initialisation, bound 1/sqrt(fan_in), in the flat
    layout of the network (FP32)."""
    rng = np.random.default_rng(seed)
    dims = [n_in] + [width] * depth + [1]
    out = []
    for l in range(depth + 1):
        bound = 1.0 / np.sqrt(dims[l])
        out.append(rng.uniform(-bound, bound, dims[l + 1] * dims[l]))
        out.append(rng.uniform(-bound, bound, dims[l + 1]))
    return np.concatenate(out).astype(np.float32)


class MLP:
    """The perceptron on the current CUDA device (FP32)."""

    def __init__(self, n_in=8, width=128, depth=4, max_batch=65536):
        self.n_in, self.width, self.depth, self.max_batch = n_in, width, depth, max_batch
        h = ctypes.c_void_p()
        _check(_sig().ccz4_mlp_create(n_in, width, depth, max_batch, ctypes.byref(h)))
        self._h = h
        import torch
        p, n = ctypes.POINTER(ctypes.c_float)(), ctypes.c_longlong()
        _check(_sig().ccz4_mlp_params(h, ctypes.byref(p), ctypes.byref(n)))
        self.n_params = n.value
        self.theta = _wrap_device(ctypes.cast(p, ctypes.c_void_p).value, (n.value,), torch.float32)
        _check(_sig().ccz4_mlp_grads(h, ctypes.byref(p), ctypes.byref(n)))
        self.grad = _wrap_device(ctypes.cast(p, ctypes.c_void_p).value, (n.value,), torch.float32)
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def close(self):
        if getattr(self, "_h", None):
            _sig().ccz4_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        import torch
        self.theta.copy_(torch.as_tensor(np.asarray(theta, dtype=np.float32), device="cuda"))

    def forward(self, x, stream=None):
        """y (batch,) for x (batch, n_in) float32 on the device."""
        import torch
        B = x.shape[0]
        y = torch.empty(B, dtype=torch.float32, device="cuda")
        for r0 in range(0, B, self.max_batch):
            r1 = min(B, r0 + self.max_batch)
            _check(_sig().ccz4_mlp_forward(self._h, _p(x[r0:r1]), r1 - r0, _p(y[r0:r1]), _stream(stream)))
        return y

    def loss_grad(self, x, t, stream=None):
        """Loss (device scalar tensor); the gradient lands in self.grad."""
        _check(_sig().ccz4_mlp_loss_grad(self._h, _p(x), _p(t), x.shape[0], _p(self._loss), _stream(stream)))
        return self._loss

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        _check(_sig().ccz4_mlp_adam(self._h, lr, b1, b2, eps, _stream(stream)))


def features_grid(n, L, p5, stream=None):
    import torch
    x = torch.empty((n ** 3, N_FEATURES), dtype=torch.float32, device="cuda")
    arr = (ctypes.c_double * 5)(*[float(v) for v in p5])
    _check(_sig().ccz4_mlp_features_grid(n, float(L), arr, _p(x), _stream(stream)))
    return x


def features_sample(n, L, p5, u_store, idx, stream=None):
    """x (B, 8) and t (B,) for flat indices idx = solution * n^3 + cell."""
    import torch
    B = idx.shape[0]
    x = torch.empty((B, N_FEATURES), dtype=torch.float32, device="cuda")
    t = torch.empty(B, dtype=torch.float32, device="cuda")
    _check(_sig().ccz4_mlp_features_sample(n, float(L), _p(p5), _p(u_store), _p(idx), B, _p(x), _p(t),
                                           _stream(stream)))
    return x, t


def output_to_u(y, u_ptr, stream=None):
    _check(_sig().ccz4_mlp_output_to_u(_p(y), y.shape[0], ctypes.c_void_p(u_ptr), _stream(stream)))


# ---------------------------------------------------------------------------
# the experiment
# ---------------------------------------------------------------------------
def sobol_draws(count, seed=0):
    """count x 5 parameter draws (m1, m2, d, P, S) from a scrambled Sobol sequence."""
    import torch
    eng = torch.quasirandom.SobolEngine(dimension=5, scramble=True, seed=seed)
    q = eng.draw(count).double().numpy()
    lo = np.array([r[0] for r in RANGES])
    hi = np.array([r[1] for r in RANGES])
    return lo + q * (hi - lo)


def optimal_omega(n):
    """Over-relaxation factor of red-black SOR for the 7-point Laplacian on
    n cells per axis (Young: 2 / (1 + sqrt(1 - rho^2)) with the Jacobi
    spectral radius rho = cos(pi / n))."""
    return 2.0 / (1.0 + np.sin(np.pi / n))


OMEGAS = (1.95, 1.96, 1.97, 1.975, 1.98)


def tune_omega(draws, n, L, candidates=OMEGAS, tol=1e-10, check=20):
    """The relaxation factor with the fewest total sweeps from u = 0 on the
    given draws (the optimum of the model problem ignores the fall-off
    ghosts); returns (omega, {omega: total sweeps or None if one failed})."""
    totals = {}
    for w in candidates:
        _, sw, _ = solve_draws(draws, n, L, tol=tol, check=check, keep=False, omega=w, max_sweeps=20000)
        totals[w] = int(sw.sum()) if (sw > 0).all() else None
    ok = {w: t for w, t in totals.items() if t is not None}
    return (min(ok, key=ok.get) if ok else 1.0), totals


def solve_draws(draws, n, L, tol=1e-10, check=100, max_sweeps=2000000, keep=True, omega=1.0):
    """Plain solves from u = 0; returns (u_store (len, n^3) float32 or None, sweeps, seconds)."""
    import torch
    s = ID.Solver(n, L)
    s.set_relaxation(omega)
    store = torch.empty((len(draws), n ** 3), dtype=torch.float32, device="cuda") if keep else None
    sweeps = []
    t0 = time.perf_counter()
    for k, d in enumerate(draws):
        s.set_punctures(ID.binary(*d))
        s.u_tensor().zero_()
        it, _ = s.solve(tol=tol, check=check, max_sweeps=max_sweeps)
        sweeps.append(it)
        if keep:
            store[k] = s.u_tensor().reshape(-1).float()
    torch.cuda.synchronize()
    return store, np.array(sweeps), time.perf_counter() - t0


def lr_at(k, steps, lr, lr_final=None):
    """Learning rate of step k: cosine decay from lr to lr_final over the
    run (constant lr when lr_final is None)."""
    if lr_final is None or steps <= 1:
        return lr
    return lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * k / (steps - 1)))


def train(mlp, u_store, draws, n, L, steps, batch=16384, lr=1e-3, seed=1, log_every=0, lr_final=None):
    """Adam on uniformly drawn (solution, cell) rows, learning rate from
    lr_at; returns the loss history. The rows are drawn on the device (a
    seeded CUDA generator), so a step makes no host-device copy."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    p5 = torch.as_tensor(np.asarray(draws, dtype=np.float32), device="cuda").contiguous()
    n3 = n ** 3
    hist = []
    for k in range(steps):
        idx = torch.randint(0, len(draws) * n3, (batch,), generator=gen, device="cuda", dtype=torch.int64)
        x, t = features_sample(n, L, p5, u_store, idx)
        loss = mlp.loss_grad(x, t)
        mlp.adam(lr_at(k, steps, lr, lr_final))
        if log_every and (k % log_every == 0 or k == steps - 1):
            hist.append((k, float(loss.item())))
    return hist


def evaluate(mlp, draws, n, L, tol=1e-10, check=100, max_sweeps=2000000, omega=1.0):
    """Per held-out draw: (sweeps from u = 0, sweeps from the network's guess,
    max |guess - solution| / max |solution|)."""
    import torch
    s = ID.Solver(n, L)
    s.set_relaxation(omega)
    out = []
    for d in draws:
        s.set_punctures(ID.binary(*d))
        s.u_tensor().zero_()
        k0, _ = s.solve(tol=tol, check=check, max_sweeps=max_sweeps)
        sol = s.u_tensor().clone()
        y = mlp.forward(features_grid(n, L, d))
        output_to_u(y, s.u_ptr)
        guess = s.u_tensor().clone()
        k1, _ = s.solve(tol=tol, check=check, max_sweeps=max_sweeps)
        err = float((guess - sol).abs().max() / sol.abs().max())
        out.append((k0, k1, err))
    return np.array(out)


def run_experiment(n=96, L=16.0, n_train=2000, n_test=200, steps=400000, batch=65536, lr=1e-3, tol=1e-10,
                   check=20, seed=0, omega=None, gs_draws=10, log=print, lr_final=1e-6):
    """The whole experiment; returns a JSON-ready report."""
    import torch
    draws = sobol_draws(n_train + n_test, seed=seed)
    train_d, test_d = draws[:n_train], draws[n_train:]
    t0 = time.perf_counter()
    omega_scan = None
    if omega is None:
        omega, omega_scan = tune_omega(train_d[:3], n, L, tol=tol, check=check)
        log("relaxation factor %.4f (sweeps on 3 draws: %s)" % (omega, omega_scan))
    store, sweeps, t_solve = solve_draws(train_d, n, L, tol=tol, check=check, omega=omega)
    log("plain solves: %d draws in %.1f s, sweeps mean %.0f (min %d, max %d)"
        % (n_train, t_solve, sweeps.mean(), sweeps.min(), sweeps.max()))
    net = MLP(N_FEATURES, 128, 4, batch)
    net.set_params(init_params(N_FEATURES, 128, 4, seed=seed))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = train(net, store, train_d, n, L, steps, batch=batch, lr=lr, seed=seed + 1,
                 log_every=max(1, steps // 20), lr_final=lr_final)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    log("training: %d steps of %d rows in %.1f s, loss %s" % (steps, batch, t_train, hist[-1]))
    t2 = time.perf_counter()
    res = evaluate(net, test_d, n, L, tol=tol, check=check, omega=omega)
    t_eval = time.perf_counter() - t2
    ok = (res[:, 0] > 0) & (res[:, 1] > 0)
    # the same evaluation with plain Gauss-Seidel (omega = 1) on the first held-out draws
    gs = evaluate(net, test_d[:gs_draws], n, L, tol=tol, check=200, omega=1.0) if gs_draws else None
    gs_ok = (gs[:, 0] > 0) & (gs[:, 1] > 0) if gs is not None else None
    report = {
        "grid": {"n": n, "L": L, "tol": tol, "check_every": check, "omega": omega,
                 "omega_scan": {str(k): v for k, v in (omega_scan or {}).items()}},
        "draws": {"train": n_train, "test": n_test, "sobol_seed": seed, "ranges": dict(zip(
            ("m1", "m2", "d", "P", "S"), RANGES))},
        "network": {"layers": "8 -> 4 x 128 SiLU -> 1", "params": net.n_params, "steps": steps, "batch": batch,
                    "lr": lr, "lr_final": lr_final, "loss_history": hist},
        "train_solves": {"seconds": t_solve, "sweeps_mean": float(sweeps.mean())},
        "train_seconds": t_train,
        "eval": {"seconds": t_eval, "all_converged": bool(ok.all()),
                 "sweeps_from_zero_mean": float(res[ok, 0].mean()),
                 "sweeps_from_network_mean": float(res[ok, 1].mean()),
                 "sweep_ratio_mean": float((res[ok, 1] / res[ok, 0]).mean()),
                 "guess_rel_error_median": float(np.median(res[:, 2])),
                 "guess_rel_error_max": float(res[:, 2].max())},
        "eval_gauss_seidel": None if gs is None else {
            "draws": int(gs_draws), "all_converged": bool(gs_ok.all()),
            "sweeps_from_zero_mean": float(gs[gs_ok, 0].mean()) if gs_ok.any() else None,
            "sweeps_from_network_mean": float(gs[gs_ok, 1].mean()) if gs_ok.any() else None,
            "sweep_ratio_mean": float((gs[gs_ok, 1] / gs[gs_ok, 0]).mean()) if gs_ok.any() else None},
        "total_seconds": time.perf_counter() - t0,
    }
    log("held-out: sweeps from u=0 %.0f, from the network %.0f (ratio %.3f), guess error median %.2e"
        % (report["eval"]["sweeps_from_zero_mean"], report["eval"]["sweeps_from_network_mean"],
           report["eval"]["sweep_ratio_mean"], report["eval"]["guess_rel_error_median"]))
    if gs is not None:
        log("held-out, Gauss-Seidel on %d draws: %s" % (gs_draws, report["eval_gauss_seidel"]))
    return report


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned warm start of the puncture initial-data solve")
    ap.add_argument("--n", type=int, default=96)
    ap.add_argument("--L", type=float, default=16.0)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--steps", type=int, default=400000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=1e-6,
                    help="end of a cosine learning-rate decay (a negative value: a constant rate)")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--omega", type=float, default=None,
                    help="relaxation factor (default: the fastest of a short scan; 1 = Gauss-Seidel)")
    ap.add_argument("--check", type=int, default=20, help="sweeps between residual checks")
    ap.add_argument("--gs-draws", type=int, default=10,
                    help="held-out draws also evaluated with plain Gauss-Seidel (omega = 1)")
    ap.add_argument("--out", default=None, help="write the report as JSON here")
    a = ap.parse_args(argv)
    rep = run_experiment(a.n, a.L, a.train, a.test, a.steps, a.batch, a.lr, a.tol, check=a.check, omega=a.omega,
                         gs_draws=a.gs_draws, log=lambda s: print(s, flush=True),
                         lr_final=a.lr_final if a.lr_final >= 0 else None)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rep, f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
