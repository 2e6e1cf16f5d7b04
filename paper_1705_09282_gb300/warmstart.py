"""Learned warm start (front end of the igamg_nn_* and igamg_warm_start calls).

A small CNN maps the forcing sampled on the streamfunction control grid and
log10(sigma/nu) to a scaled streamfunction; the exact discrete curl of its prediction is a
divergence-free initial guess for the V-cycle.  Training targets are streamfunctions of
solutions computed by the multigrid itself.  Marshalling only: every step runs in the
library's kernels.
"""
import ctypes

import numpy as np
import torch

from . import _lib, inputs
from ._lib import check, lib
from .solver import Solver, solve_batch


def _fptr(t):
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 tensor")
    return ctypes.c_void_p(t.data_ptr())


class Network:
    """The 4-layer, 32-channel network (BF16 weights, FP32 accumulation)."""

    DEFAULT_DILATIONS = (1, 2, 4, 8)

    def __init__(self, seed=1, device="cuda", stream=None, dilations=DEFAULT_DILATIONS):
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.dilations = tuple(dilations)
        d = (ctypes.c_int * 4)(*self.dilations)
        h = ctypes.c_void_p()
        check(lib().igamg_nn_create(3, 32, d, ctypes.c_ulonglong(seed), ctypes.c_void_p(self.stream.cuda_stream),
                                    ctypes.byref(h)), "igamg_nn_create")
        self._h = h
        self.n_params = lib().igamg_nn_num_params(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().igamg_nn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        check(lib().igamg_nn_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p), out.size), "get_params")
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        check(lib().igamg_nn_set_params(self._h, flat.ctypes.data_as(ctypes.c_void_p), flat.size), "set_params")

    def forward(self, x):
        B, _, H, W = x.shape
        out = torch.empty((B, 2, H, W), dtype=torch.float32, device=self.device)
        check(lib().igamg_nn_forward(self._h, B, H, W, _fptr(x), _fptr(out)), "igamg_nn_forward")
        return out

    def loss_grad(self, x, target):
        B, _, H, W = x.shape
        loss = ctypes.c_double()
        g = np.zeros(self.n_params, dtype=np.float32)
        check(lib().igamg_nn_loss_grad(self._h, B, H, W, _fptr(x), _fptr(target), ctypes.byref(loss),
                                       g.ctypes.data_as(ctypes.c_void_p)), "igamg_nn_loss_grad")
        return loss.value, g

    def train_step(self, x, target, lr, want_loss=True):
        """One Adam step; returns the minibatch loss (a host synchronisation) or None."""
        B, _, H, W = x.shape
        loss = ctypes.c_double()
        check(lib().igamg_nn_train_step(self._h, B, H, W, _fptr(x), _fptr(target), ctypes.c_float(lr),
                                        ctypes.byref(loss) if want_loss else None), "igamg_nn_train_step")
        return loss.value if want_loss else None


def streamfunction(solver, U):
    """Discrete streamfunction (interior, FP64) of a divergence-free velocity."""
    s = solver.sizes()
    nint = s.nx_ux
    psi = torch.empty(nint * nint, dtype=torch.float64, device=solver.device)
    check(lib().igamg_streamfunction(solver._h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(psi.data_ptr())),
          "igamg_streamfunction")
    return psi


def warm_start(solver, grid, psi_scale, p_scale, out=None):
    """U0 = (curl(psi_scale * grid[0] interior), p_scale * grid[1], 0) for one network output
    grid (2, H, W) float32."""
    U = solver.empty() if out is None else out
    check(lib().igamg_warm_start(solver._h, _fptr(grid.contiguous()), float(psi_scale), float(p_scale),
                                 ctypes.c_void_p(U.data_ptr())), "igamg_warm_start")
    return U


def warm_start_minres(solver, grid, psi_scale, p_scale, F, out=None):
    """As warm_start, with the velocity and pressure fields scaled by the pair of factors
    that minimises ||F - K U|| (igamg_warm_start_minres); returns (U, alpha, beta)."""
    U = solver.empty() if out is None else out
    a, b = ctypes.c_double(), ctypes.c_double()
    check(lib().igamg_warm_start_minres(solver._h, _fptr(grid.contiguous()), float(psi_scale), float(p_scale),
                                        ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                                        ctypes.byref(a), ctypes.byref(b)), "igamg_warm_start_minres")
    return U, a.value, b.value


def solve_abs(solver, U, F, atol, max_cycles=100):
    rep, hist = Solver._report(max_cycles)
    rc = check(lib().igamg_solve_abs(solver._h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(F.data_ptr()),
                                     float(atol), int(max_cycles), ctypes.byref(rep)), "igamg_solve_abs")
    return Solver._report_dict(rep, hist, rc)


def solve_batch_abs(solvers, Us, Fs, atols, max_cycles=100):
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s._h.value for s in solvers])
    up = (ctypes.c_void_p * n)(*[u.data_ptr() for u in Us])
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in Fs])
    at = (ctypes.c_double * n)(*[float(a) for a in atols])
    reps = (_lib.Report * n)()
    status = (ctypes.c_int * n)()
    check(lib().igamg_solve_batch_abs(n, hs, up, fp, at, int(max_cycles), reps, status), "igamg_solve_batch_abs")
    return [{"converged": status[i] == 0, "cycles": reps[i].cycles, "res0": reps[i].res0,
             "rel_residual": reps[i].rel_residual, "div_inf": reps[i].div_inf} for i in range(n)]


class Problem:
    """One generalized Stokes problem of a batch: solver, forcing, network input."""

    def __init__(self, p, n, levels, sigma, nu, seed, device="cuda", stream=None, precision=_lib.IGAMG_FP64):
        self.p, self.n, self.sigma, self.nu, self.seed = p, n, sigma, nu, seed
        self.solver = Solver(p, n, levels, sigma, nu, device=device, stream=stream, precision=precision)
        f = torch.tensor(inputs.grf_forcing(p, n, seed), device=device)
        self.F = self.solver.load_vector(f)
        self.x = torch.tensor(inputs.warm_start_input(p, n, seed, sigma, nu), device=device)
        self.scale = inputs.warm_start_scale(sigma, nu)
        self.p_scale = inputs.warm_start_pressure_scale()
        self.U = self.solver.empty()


def levels_for(n, coarsest=4):
    """Number of grids down to a coarsest mesh of at most `coarsest` elements."""
    L = 1
    while n % 2 == 0 and n // 2 >= coarsest and n // 2 >= 2:
        n //= 2
        L += 1
    return L


def targets(problems, rtol=1e-10, max_cycles=80):
    """Solve every problem with the multigrid (side by side) and return, per problem, its
    streamfunction (channel 0, interior) and pressure (channel 1, leading (n+p-1)^2 points)
    on the network grid, each divided by its output scale (float32, (2, H, W))."""
    for pr in problems:
        pr.U.zero_()
    reps = solve_batch([pr.solver for pr in problems], [pr.U for pr in problems], [pr.F for pr in problems],
                       rtol=rtol, max_cycles=max_cycles)
    out = []
    for pr, rep in zip(problems, reps):
        assert rep["converged"], rep
        psi = streamfunction(pr.solver, pr.U)
        s = pr.solver.sizes()
        nint = pr.n + pr.p - 2
        grid = torch.zeros((2, nint + 2, nint + 2), dtype=torch.float32, device=pr.U.device)
        grid[0, 1:-1, 1:-1] = (psi.view(nint, nint) / pr.scale).to(torch.float32)
        pres = pr.U[s.n_ux + s.n_uy: s.n_ux + s.n_uy + s.n_p].view(s.n_pdir, s.n_pdir)
        grid[1, :nint + 1, :nint + 1] = (pres / pr.p_scale).to(torch.float32)
        out.append(grid)
    return out


def train(net, problems, grids, steps, batch=8, lr=2e-3, seed=0, lr_final=None, loss_every=50):
    """Adam on minibatches of equal-size problems (the network is fully convolutional);
    the step size decays geometrically from lr to lr_final (default lr / 20).  Returns the
    minibatch losses of the first 5 steps, of every loss_every-th step and of the last 20, in
    step order: only those steps wait for the device, the others are queued back to back."""
    lr_final = lr / 20.0 if lr_final is None else lr_final
    by_size = {}
    for i, pr in enumerate(problems):
        by_size.setdefault(pr.x.shape[-1], []).append(i)
    keys = sorted(by_size)
    rng = inputs.SplitMix64(seed)
    losses = []
    for s in range(steps):
        idx = by_size[keys[s % len(keys)]]
        pick = [idx[int(u * len(idx))] for u in rng.uniform(min(batch, len(idx)))]
        x = torch.stack([problems[i].x for i in pick]).contiguous()
        t = torch.stack([grids[i] for i in pick]).contiguous()
        rate = lr * (lr_final / lr) ** (s / max(1, steps - 1))
        want = s < 5 or s >= steps - 20 or s % loss_every == 0
        loss = net.train_step(x, t, rate, want_loss=want)
        if want:
            losses.append(loss)
    return losses


def predict_guesses(net, problems, scaled=False):
    """Warm-start initial guesses U0 (written into each problem's U); with scaled the two
    predicted fields are rescaled against each problem's F (igamg_warm_start_minres)."""
    for pr in problems:
        g = net.forward(pr.x.unsqueeze(0).contiguous())[0]
        if scaled:
            warm_start_minres(pr.solver, g, pr.scale, pr.p_scale, pr.F, out=pr.U)
        else:
            warm_start(pr.solver, g, pr.scale, pr.p_scale, out=pr.U)
