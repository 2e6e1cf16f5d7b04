"""Thin Python front end of the C ABI (include/igamg.h) on PyTorch device memory.

Marshalling only: tensors are passed to the library as raw device pointers on the
current PyTorch stream; every numerical step runs in the library's CUDA kernels.
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, lib


def _ptr(t, dtype=torch.float64):
    if t is None:
        return None
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """Owns one igamg_handle: the level hierarchy of Sec. 5.1 for a 2D (unit square) or
    3D (unit cube, dim=3) problem."""

    def __init__(self, p, n_fine, n_levels, sigma, nu, smoother="mult", eta=0.0, nu1=2, nu2=2,
                 c_penalty=0.0, precision=_lib.IGAMG_FP64, device="cuda", stream=None, beta=None, dim=2,
                 restart=0, gamma=1, fmg=False, geometry=_lib.IGAMG_GEOM_SQUARE, r_inner=0.0, r_outer=0.0):
        """beta: advection at the quadrature points (host array (2, nG, nG)) for the
        generalized Oseen problem, or None for generalized Stokes.  gamma = 2 selects the
        W-cycle; fmg starts every solve with one full-multigrid pass.  geometry =
        IGAMG_GEOM_QUARTER_ANNULUS solves on the quarter annulus (2D Stokes)."""
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise RuntimeError("the igamg solver runs on a CUDA device only")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._beta = None if beta is None else np.ascontiguousarray(beta, dtype=np.float64)
        self.problem = _lib.make_problem(p, n_fine, n_levels, sigma, nu, smoother, eta, nu1, nu2,
                                         c_penalty, precision, beta=self._beta, dim=dim, restart=restart,
                                         gamma=gamma, fmg=fmg, geometry=geometry, r_inner=r_inner,
                                         r_outer=r_outer)
        self.p, self.n_fine, self.n_levels, self.dim = p, n_fine, n_levels, dim
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().igamg_create(ctypes.byref(self.problem), ctypes.c_void_p(self.stream.cuda_stream),
                                     ctypes.byref(h)), "igamg_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().igamg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- sizes / points ----------------------------------------------------------
    def sizes(self, level=None):
        level = self.n_levels - 1 if level is None else level
        s = _lib.Sizes()
        check(lib().igamg_get_sizes(self._h, level, ctypes.byref(s)), "igamg_get_sizes")
        return s

    def ndof(self, level=None):
        return self.sizes(level).n_total

    def quad_points(self):
        n = ctypes.c_size_t()
        check(lib().igamg_quad_points(self._h, None, 0, ctypes.byref(n)), "igamg_quad_points")
        x = np.zeros(n.value)
        check(lib().igamg_quad_points(self._h, x.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)),
              "igamg_quad_points")
        return x

    def quad_points_xy(self):
        """Physical quadrature points: 2D (2, nG, nG) [x or y][eta][xi], 3D (3, nG, nG, nG)."""
        n = ctypes.c_size_t()
        check(lib().igamg_quad_points_xy(self._h, None, 0, ctypes.byref(n)), "igamg_quad_points_xy")
        xy = np.zeros(n.value)
        check(lib().igamg_quad_points_xy(self._h, xy.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)),
              "igamg_quad_points_xy")
        if self.dim == 3:
            nG = int(round((n.value // 3) ** (1.0 / 3.0)))
            return xy.reshape(3, nG, nG, nG)
        nG = int(round(np.sqrt(n.value // 2)))
        return xy.reshape(2, nG, nG)

    def empty(self, level=None):
        return torch.zeros(self.ndof(level), dtype=torch.float64, device=self.device)

    # ---- operators ---------------------------------------------------------------
    def load_vector(self, f_qp, out=None):
        F = self.empty() if out is None else out
        check(lib().igamg_load_vector(self._h, _ptr(f_qp), _ptr(F)), "igamg_load_vector")
        return F

    def residual(self, U, F, level=None, out=None, norm=False):
        level = self.n_levels - 1 if level is None else level
        R = self.empty(level) if out is None else out
        nrm = ctypes.c_double()
        check(lib().igamg_residual(self._h, level, _ptr(U), _ptr(F), _ptr(R),
                                   ctypes.byref(nrm) if norm else None), "igamg_residual")
        return (R, nrm.value) if norm else R

    def smooth(self, U, F, level=None, sweeps=1):
        level = self.n_levels - 1 if level is None else level
        check(lib().igamg_smooth(self._h, level, _ptr(U), _ptr(F), sweeps), "igamg_smooth")
        return U

    def level_form(self, level=None):
        """The sweep form the autotuner chose for a level (2D): dict(lanes, threads, tiles, chains)."""
        level = self.n_levels - 1 if level is None else level
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().igamg_level_form(self._h, level, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
              "igamg_level_form")
        d = ctypes.c_int()
        check(lib().igamg_level_chains(self._h, level, ctypes.byref(d)), "igamg_level_chains")
        return {"lanes": a.value, "threads": b.value, "tiles": c.value, "chains": d.value}

    def smooth32(self, U, F, level=None, sweeps=1):
        """FP32 smoothing sweeps (FP32-in-FP64 handles): U, F float32 device tensors."""
        level = self.n_levels - 1 if level is None else level
        check(lib().igamg_smooth_f32(self._h, level, _ptr(U, torch.float32), _ptr(F, torch.float32), sweeps),
              "igamg_smooth_f32")
        return U

    def residual32(self, U, F, level=None, out=None, norm=False):
        """FP32 residual (FP32-in-FP64 handles): U, F float32 device tensors."""
        level = self.n_levels - 1 if level is None else level
        R = torch.empty(self.ndof(level), dtype=torch.float32, device=self.device) if out is None else out
        nrm = ctypes.c_double()
        check(lib().igamg_residual_f32(self._h, level, _ptr(U, torch.float32), _ptr(F, torch.float32),
                                       _ptr(R, torch.float32), ctypes.byref(nrm) if norm else None),
              "igamg_residual_f32")
        return (R, nrm.value) if norm else R

    def residual_form(self):
        """The finest residual's operator form per precision: {"fp64": f, "fp32": f}, f = 0 class
        stencils, 1 per-row records, 2 matrix-free advection (-1: no FP32 V-cycle)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        check(lib().igamg_residual_form(self._h, ctypes.byref(a), ctypes.byref(b)), "igamg_residual_form")
        return {"fp64": a.value, "fp32": b.value}

    def set_residual_form(self, fp64=0, fp32=0):
        """Pin the finest residual's form (1 records, 2 matrix-free advection, 0 unchanged)."""
        check(lib().igamg_set_residual_form(self._h, fp64, fp32), "igamg_set_residual_form")

    def restrict(self, r_fine, level, out=None):
        g = self.empty(level - 1) if out is None else out
        check(lib().igamg_restrict(self._h, level, _ptr(r_fine), _ptr(g)), "igamg_restrict")
        return g

    def prolong_add(self, u_coarse, u_fine, level):
        check(lib().igamg_prolong_add(self._h, level, _ptr(u_coarse), _ptr(u_fine)), "igamg_prolong_add")
        return u_fine

    def coarse_solve(self, G, out=None):
        U = self.empty(0) if out is None else out
        check(lib().igamg_coarse_solve(self._h, _ptr(G), _ptr(U)), "igamg_coarse_solve")
        return U

    def vcycle(self, U, F):
        check(lib().igamg_vcycle(self._h, _ptr(U), _ptr(F)), "igamg_vcycle")
        return U

    def solve(self, U, F, rtol=1e-8, max_cycles=100, history=True):
        rep, hist = self._report(max_cycles if history else 0)
        rc = check(lib().igamg_solve(self._h, _ptr(U), _ptr(F), float(rtol), int(max_cycles),
                                     ctypes.byref(rep)), "igamg_solve")
        return self._report_dict(rep, hist, rc)

    def solve_host(self, f_qp_host, U_host, rtol=1e-8, max_cycles=100):
        """End-to-end solve from host numpy arrays (f at the quadrature points, U in/out)."""
        f = np.ascontiguousarray(f_qp_host, dtype=np.float64)
        if U_host.dtype != np.float64 or not U_host.flags.c_contiguous:
            raise ValueError("U_host must be a contiguous float64 array")
        rep, hist = self._report(max_cycles)
        rc = check(lib().igamg_solve_host(self._h, f.ctypes.data_as(ctypes.c_void_p),
                                          U_host.ctypes.data_as(ctypes.c_void_p), float(rtol),
                                          int(max_cycles), ctypes.byref(rep)), "igamg_solve_host")
        return self._report_dict(rep, hist, rc)

    @staticmethod
    def _report(cap):
        rep = _lib.Report()
        hist = (ctypes.c_double * max(cap, 1))()
        rep.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if cap else None
        rep.history_cap = cap
        return rep, hist

    @staticmethod
    def _report_dict(rep, hist, rc):
        n = min(rep.cycles, rep.history_cap)
        return {"converged": rc == _lib.IGAMG_OK, "cycles": rep.cycles, "res0": rep.res0,
                "rel_residual": rep.rel_residual, "div_inf": rep.div_inf,
                "history": [hist[i] for i in range(n)]}

    def div_inf(self, U):
        out = ctypes.c_double()
        check(lib().igamg_div_inf(self._h, _ptr(U), ctypes.byref(out)), "igamg_div_inf")
        return out.value

    def curl(self, psi, out=None):
        U = self.empty() if out is None else out
        check(lib().igamg_curl(self._h, _ptr(psi), _ptr(U)), "igamg_curl")
        return U


def solve_batch(solvers, Us, Fs, rtol=1e-8, max_cycles=100, history=False):
    """Independent solves (igamg_solve_batch): groups of eight or more FP64 solves of one
    cycle shape step in lockstep; the others run side by side, each on its handle's own
    stream, and each advances to its next cycle as soon as its own residual norm is back."""
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s._h.value for s in solvers])
    up = (ctypes.c_void_p * n)(*[_ptr(u).value for u in Us])
    fp = (ctypes.c_void_p * n)(*[_ptr(f).value for f in Fs])
    reps = (_lib.Report * n)()
    hists = []
    for i in range(n):
        cap = max_cycles if history else 0
        hist = (ctypes.c_double * max(cap, 1))()
        reps[i].history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if cap else None
        reps[i].history_cap = cap
        hists.append(hist)
    status = (ctypes.c_int * n)()
    check(lib().igamg_solve_batch(n, hs, up, fp, float(rtol), int(max_cycles), reps, status), "igamg_solve_batch")
    return [Solver._report_dict(reps[i], hists[i], status[i]) for i in range(n)]


# ---- host-only inspection (no GPU) ----------------------------------------------------
def host_level_matrix(p, n_fine, n_levels, sigma, nu, level, c_penalty=0.0, beta=None, dim=2, geometry=0):
    beta = None if beta is None else np.ascontiguousarray(beta, dtype=np.float64)
    pr = _lib.make_problem(p, n_fine, n_levels, sigma, nu, c_penalty=c_penalty, beta=beta, dim=dim,
                           geometry=geometry)
    n = ctypes.c_longlong()
    check(lib().igamg_host_level_matrix(ctypes.byref(pr), level, None, 0, ctypes.byref(n)), "host_level_matrix")
    K = np.zeros((n.value, n.value))
    check(lib().igamg_host_level_matrix(ctypes.byref(pr), level, K.ctypes.data_as(ctypes.c_void_p), K.size,
                                        ctypes.byref(n)), "host_level_matrix")
    return K


def host_operator_rows(p, n_fine, n_levels, sigma, nu, level, beta=None, dim=2, geometry=0):
    beta = None if beta is None else np.ascontiguousarray(beta, dtype=np.float64)
    pr = _lib.make_problem(p, n_fine, n_levels, sigma, nu, beta=beta, dim=dim, geometry=geometry)
    n = ctypes.c_longlong()
    check(lib().igamg_host_operator_rows(ctypes.byref(pr), level, None, 0, ctypes.byref(n)), "host_operator_rows")
    K = np.zeros((n.value, n.value))
    check(lib().igamg_host_operator_rows(ctypes.byref(pr), level, K.ctypes.data_as(ctypes.c_void_p), K.size,
                                         ctypes.byref(n)), "host_operator_rows")
    return K


def host_operator_apply(p, n_fine, n_levels, sigma, nu, level, V, beta=None, dim=2, geometry=0):
    """K_l V through the kernels' row evaluation, on the host (V: float64 numpy vector)."""
    beta = None if beta is None else np.ascontiguousarray(beta, dtype=np.float64)
    pr = _lib.make_problem(p, n_fine, n_levels, sigma, nu, beta=beta, dim=dim, geometry=geometry)
    V = np.ascontiguousarray(V, dtype=np.float64)
    KV = np.zeros_like(V)
    check(lib().igamg_host_operator_apply(ctypes.byref(pr), level, V.ctypes.data_as(ctypes.c_void_p),
                                          KV.ctypes.data_as(ctypes.c_void_p), V.size), "host_operator_apply")
    return KV


def host_prolongation(p, n_fine, n_levels, level, dim=2):
    pr = _lib.make_problem(p, n_fine, n_levels, 1.0, 1.0, dim=dim)
    r, c = ctypes.c_longlong(), ctypes.c_longlong()
    check(lib().igamg_host_prolongation(ctypes.byref(pr), level, None, 0, ctypes.byref(r), ctypes.byref(c)),
          "host_prolongation")
    P = np.zeros((r.value, c.value))
    check(lib().igamg_host_prolongation(ctypes.byref(pr), level, P.ctypes.data_as(ctypes.c_void_p), P.size,
                                        ctypes.byref(r), ctypes.byref(c)), "host_prolongation")
    return P


def host_patches(p, n_fine, n_levels, level, dim=2):
    pr = _lib.make_problem(p, n_fine, n_levels, 1.0, 1.0, dim=dim)
    npat, maxl = ctypes.c_int(), ctypes.c_int()
    check(lib().igamg_host_patches(ctypes.byref(pr), level, None, None, 0, 0, ctypes.byref(npat),
                                   ctypes.byref(maxl)), "host_patches")
    col = np.zeros(npat.value, dtype=np.int32)
    dofs = np.zeros(npat.value * maxl.value, dtype=np.int32)
    check(lib().igamg_host_patches(ctypes.byref(pr), level, col.ctypes.data_as(ctypes.c_void_p),
                                   dofs.ctypes.data_as(ctypes.c_void_p), col.size, dofs.size,
                                   ctypes.byref(npat), ctypes.byref(maxl)), "host_patches")
    return col, dofs.reshape(npat.value, maxl.value)
