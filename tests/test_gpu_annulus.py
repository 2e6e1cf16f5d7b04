"""GPU parity on the quarter annulus (Sec. 4.3 push-forwards, Sec. 6.2): quadrature points,
load vector, level operators, smoother, V-cycles and whole solves against the mapped-domain
oracle, on the same seeded inputs.  Tolerances as for the unit square: single operator
applications 1e-13 relative, V-cycle and solve iterates 1e-10 with identical cycle counts."""
import numpy as np
import pytest

from oracle import annulus2d as A
from oracle import stokes2d as o2
from paper_1705_09282_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL_OP = 1e-13
RTOL_IT = 1e-10
GEOM = A.QuarterAnnulus()


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _solver(p, n, L, sigma=1.0, nu=1.0, **kw):
    from paper_1705_09282_gb300 import _lib
    from paper_1705_09282_gb300.solver import Solver
    _torch()
    return Solver(p, n, L, sigma, nu, geometry=_lib.IGAMG_GEOM_QUARTER_ANNULUS, **kw)


def _t(x):
    torch = _torch()
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


_H = {}


def _hier(p, n, L, sigma=1.0, nu=1.0, **kw):
    key = (p, n, L, sigma, nu, tuple(sorted(kw.items())))
    if key not in _H:
        fine = A.MappedStokes2D(p, n, sigma, nu, GEOM)
        _H[key] = o2.Hierarchy(p, n, L, sigma, nu, fine=fine, **kw)
    return _H[key]


def _forcing(S, sigma=1.0, nu=1.0):
    X = S.quad_points_xy()
    return inputs.annulus_forcing(X[0], X[1], sigma, nu)


CASES = [(2, 8, 3), (3, 8, 2), (2, 12, 2), (3, 12, 3)]


@pytest.mark.parametrize("p,n,L", CASES)
def test_points_and_load_vector(p, n, L):
    S = _solver(p, n, L)
    H = _hier(p, n, L)
    Xo = H.fine.quad_points_xy()
    assert np.abs(S.quad_points_xy() - Xo).max() <= 1e-15
    f = inputs.annulus_forcing(Xo[0], Xo[1], 1.0, 1.0)
    assert _rel(_np(S.load_vector(_t(f))), H.fine.load_vector(f)) < RTOL_OP


@pytest.mark.parametrize("p,n,L", CASES)
def test_residual_every_level(p, n, L):
    S = _solver(p, n, L)
    H = _hier(p, n, L)
    for lev in range(L):
        nd = H.levels[lev].K.shape[0]
        U = inputs.random_vector(nd, seed=lev + 1)
        F = inputs.random_vector(nd, seed=lev + 50)
        R, nrm = S.residual(_t(U), _t(F), level=lev, norm=True)
        Ro = F - H.levels[lev].K @ U
        assert _rel(_np(R), Ro) < RTOL_OP * 100, lev
        assert abs(nrm - np.linalg.norm(Ro)) <= 1e-12 * np.linalg.norm(Ro)


@pytest.mark.parametrize("p,n,L", CASES)
def test_smoother_every_level(p, n, L):
    S = _solver(p, n, L)
    H = _hier(p, n, L)
    for lev in range(1, L):
        nd = H.levels[lev].K.shape[0]
        U = inputs.random_vector(nd, seed=7 * lev)
        F = inputs.random_vector(nd, seed=7 * lev + 1)
        Ug = _t(U)
        S.smooth(Ug, _t(F), level=lev, sweeps=2)
        Uo = U.copy()
        H.smooth(lev, Uo, F)
        H.smooth(lev, Uo, F)
        assert _rel(_np(Ug), Uo) < 1e-12, lev


@pytest.mark.parametrize("p,n,L", [(2, 16, 3), (3, 16, 3), (2, 12, 2)])
def test_vcycle_iterates(p, n, L):
    S = _solver(p, n, L)
    H = _hier(p, n, L)
    f = _forcing(S)
    F = H.fine.load_vector(f)
    Fg = S.load_vector(_t(f))
    U, Ug = np.zeros_like(F), S.empty()
    for k in range(3):
        H.vcycle(U, F)
        S.vcycle(Ug, Fg)
        assert _rel(_np(Ug), U) < RTOL_IT, k


@pytest.mark.parametrize("p,sigma", [(2, 1.0), (2, 1e3), (3, 1.0)])
def test_solve_cycle_counts_and_iterates(p, sigma):
    n, L = 32, 4
    S = _solver(p, n, L, sigma=sigma)
    H = _hier(p, n, L, sigma=sigma)
    f = _forcing(S, sigma)
    F = H.fine.load_vector(f)
    U = np.zeros_like(F)
    k, hist = H.solve(U, F, 1e-8, 80)
    Ug = S.empty()
    rep = S.solve(Ug, S.load_vector(_t(f)), rtol=1e-8, max_cycles=80)
    assert rep["converged"] and rep["cycles"] == k
    assert _rel(_np(Ug), U) < RTOL_IT
    assert np.allclose(rep["history"], np.array(hist[1:]) / hist[0], rtol=1e-6)
    assert rep["div_inf"] < 1e-10 * np.abs(U).max()


def test_mixed_precision_w_and_fmg_on_the_annulus():
    from paper_1705_09282_gb300 import _lib
    p, n, L = 2, 64, 5
    S64 = _solver(p, n, L)
    f = _forcing(S64)
    U64 = S64.empty()
    r64 = S64.solve(U64, S64.load_vector(_t(f)), rtol=1e-8, max_cycles=80)
    for kw in (dict(precision=_lib.IGAMG_FP32_IR), dict(gamma=2), dict(fmg=True, precision=_lib.IGAMG_FP32_IR),
               dict(precision=_lib.IGAMG_FGMRES_FP64)):
        S = _solver(p, n, L, **kw)
        U = S.empty()
        rep = S.solve(U, S.load_vector(_t(f)), rtol=1e-8, max_cycles=80)
        assert rep["converged"], kw
        assert rep["div_inf"] < 1e-10 * float(U.abs().max()), kw
        assert _rel(_np(U), _np(U64)) < 1e-6, kw
    assert r64["converged"]


def test_solve_host_on_the_annulus():
    p, n, L = 2, 32, 4
    S = _solver(p, n, L)
    f = _forcing(S)
    Uh = np.zeros(S.ndof())
    rep_h = S.solve_host(f, Uh, rtol=1e-8, max_cycles=80)
    Ud = S.empty()
    rep_d = S.solve(Ud, S.load_vector(_t(f)), rtol=1e-8, max_cycles=80)
    assert rep_h["cycles"] == rep_d["cycles"]
    assert np.array_equal(Uh, _np(Ud))


@pytest.mark.parametrize("p,n,L", [(2, 12, 3), (3, 8, 2)])
def test_additive_smoother_and_vcycle_on_the_annulus(p, n, L):
    # eq. ASM with per-patch inverses on the mapped operator
    S = _solver(p, n, L, smoother="add", eta=0.3)
    fine = A.MappedStokes2D(p, n, 1.0, 1.0, GEOM)
    H = o2.Hierarchy(p, n, L, 1.0, 1.0, smoother="add", eta=0.3, fine=fine)
    for lev in range(1, L):
        nd = H.levels[lev].K.shape[0]
        U = inputs.random_vector(nd, seed=11 * lev)
        F = inputs.random_vector(nd, seed=11 * lev + 1)
        Ug = _t(U)
        S.smooth(Ug, _t(F), level=lev, sweeps=1)
        Uo = U.copy()
        H.smooth(lev, Uo, F)
        assert _rel(_np(Ug), Uo) < 1e-12, lev
    f = _forcing(S)
    F = fine.load_vector(f)
    Fg = S.load_vector(_t(f))
    U, Ug = np.zeros_like(F), S.empty()
    for k in range(2):
        H.vcycle(U, F)
        S.vcycle(Ug, Fg)
        assert _rel(_np(Ug), U) < RTOL_IT, k
