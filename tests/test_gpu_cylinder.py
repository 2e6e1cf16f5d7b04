"""GPU parity on the hollow cylinder section (Sec. 4.3 push-forwards, Sec. 6.4): quadrature
points, load vector, level operators, smoother, V-cycles and solves against the mapped 3D
oracle on the same inputs.  Tolerances as for the cube: single operator applications 1e-13
relative, V-cycle and solve iterates 1e-10 with identical cycle counts."""
import numpy as np
import pytest

from oracle import cylinder3d as C
from oracle import stokes3d as o3
from paper_1705_09282_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL_OP = 1e-13
RTOL_IT = 1e-10
GEOM = C.HollowCylinder()


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _solver(p, n, L, sigma=1.0, nu=1.0, **kw):
    from paper_1705_09282_gb300 import _lib
    from paper_1705_09282_gb300.solver import Solver
    _torch()
    return Solver(p, n, L, sigma, nu, dim=3, geometry=_lib.IGAMG_GEOM_HOLLOW_CYLINDER, **kw)


def _t(x):
    torch = _torch()
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


_H = {}


def _hier(p, n, L, sigma=1.0, nu=1.0):
    key = (p, n, L, sigma, nu)
    if key not in _H:
        fine = C.MappedStokes3D(p, n, sigma, nu, GEOM)
        _H[key] = o3.Hierarchy3D(p, n, L, sigma, nu, fine=fine)
    return _H[key]


def _forcing(X, sigma=1.0, nu=1.0):
    return inputs.cylinder_forcing(X[0], X[1], X[2], sigma, nu)


@pytest.mark.parametrize("p,n,L", [(2, 4, 2), (3, 2, 2)])
def test_points_load_residual_and_smoother(p, n, L):
    S = _solver(p, n, L)
    H = _hier(p, n, L)
    Xo = H.fine.quad_points_xyz()
    assert np.abs(S.quad_points_xy() - Xo).max() <= 1e-15
    f = _forcing(Xo)
    assert _rel(_np(S.load_vector(_t(f))), H.fine.load_vector(f)) < RTOL_OP
    for lev in range(L):
        nd = H.levels[lev].K.shape[0]
        U = inputs.random_vector(nd, seed=lev + 1)
        F = inputs.random_vector(nd, seed=lev + 50)
        R, nrm = S.residual(_t(U), _t(F), level=lev, norm=True)
        Ro = F - H.levels[lev].K @ U
        assert _rel(_np(R), Ro) < RTOL_OP * 100, lev
        if lev >= 1:
            Ug = _t(U)
            S.smooth(Ug, _t(F), level=lev, sweeps=2)
            Uo = U.copy()
            H.smooth(lev, Uo, F)
            H.smooth(lev, Uo, F)
            assert _rel(_np(Ug), Uo) < 1e-12, lev


@pytest.mark.parametrize("p,n,L", [(2, 8, 3), (2, 4, 2)])
def test_vcycles_and_solve(p, n, L):
    S = _solver(p, n, L)
    H = _hier(p, n, L)
    f = _forcing(H.fine.quad_points_xyz())
    F = H.fine.load_vector(f)
    Fg = S.load_vector(_t(f))
    U, Ug = np.zeros_like(F), S.empty()
    for k in range(2):
        H.vcycle(U, F)
        S.vcycle(Ug, Fg)
        assert _rel(_np(Ug), U) < RTOL_IT, k
    Uo = np.zeros_like(F)
    ko, hist = H.solve(Uo, F, 1e-8, 80)
    Ug = S.empty()
    rep = S.solve(Ug, Fg, rtol=1e-8, max_cycles=80)
    assert rep["converged"] and rep["cycles"] == ko
    assert _rel(_np(Ug), Uo) < RTOL_IT
    assert rep["div_inf"] <= 1e-11 * np.abs(Uo).max()


def test_mixed_precision_and_fgmres_on_the_cylinder():
    from paper_1705_09282_gb300 import _lib
    p, n, L = 2, 8, 3
    S64 = _solver(p, n, L)
    f = _t(_forcing(S64.quad_points_xy()))
    U64 = S64.empty()
    assert S64.solve(U64, S64.load_vector(f), rtol=1e-8, max_cycles=80)["converged"]
    for prec in (_lib.IGAMG_FP32_IR, _lib.IGAMG_FGMRES_FP64):
        S = _solver(p, n, L, precision=prec)
        U = S.empty()
        rep = S.solve(U, S.load_vector(f), rtol=1e-8, max_cycles=80)
        assert rep["converged"], prec
        assert rep["div_inf"] <= 1e-10 * float(U.abs().max()), prec
        assert _rel(_np(U), _np(U64)) < 1e-6, prec
