"""W-cycles and full multigrid on the GPU against the oracle (Sec. 5 opening paragraph:
the method also runs inside a W-cycle or a full-multigrid framework).

FP64 iterates agree to 1e-10 relative (max-norm) with identical cycle counts, as for the
V-cycle; FP32-in-FP64 solves reach the same FP64 tolerance with divergence-free iterates."""
import numpy as np
import pytest

from oracle import stokes2d as o2
from oracle import stokes3d as o3
from paper_1705_09282_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL_IT = 1e-10


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _solver(p, n, L, sigma=1.0, nu=1.0, **kw):
    from paper_1705_09282_gb300.solver import Solver
    _torch()
    return Solver(p, n, L, sigma, nu, **kw)


def _t(x):
    torch = _torch()
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("p,n,L", [(2, 16, 3), (3, 16, 3), (2, 32, 4), (3, 20, 3)])
def test_w_cycle_iterates_2d(p, n, L):
    S = _solver(p, n, L, gamma=2)
    H = o2.Hierarchy(p, n, L, 1.0, 1.0, gamma=2)
    f = inputs.grf_forcing(p, n, seed=31)
    F = H.fine.load_vector(f)
    Fg = S.load_vector(_t(f))
    U, Ug = np.zeros_like(F), S.empty()
    for k in range(3):
        H.vcycle(U, F)
        S.vcycle(Ug, Fg)
        assert _rel(_np(Ug), U) < RTOL_IT, k


@pytest.mark.parametrize("p,n,L,gamma", [(2, 16, 3, 1), (3, 16, 3, 1), (2, 32, 4, 2), (3, 32, 4, 1)])
def test_fmg_first_step_2d(p, n, L, gamma):
    # one solve step with fmg from zero is U = FMG(F); the next ones are ordinary cycles
    S = _solver(p, n, L, gamma=gamma, fmg=True)
    H = o2.Hierarchy(p, n, L, 1.0, 1.0, gamma=gamma)
    f = inputs.grf_forcing(p, n, seed=32)
    F = H.fine.load_vector(f)
    Ug = S.empty()
    rep = S.solve(Ug, S.load_vector(_t(f)), rtol=1e-30, max_cycles=1)
    assert rep["cycles"] == 1
    Uf = H.fmg(F)
    assert _rel(_np(Ug), Uf) < RTOL_IT
    # from a nonzero start: U += FMG(F - K U)
    U0 = inputs.random_vector(len(F), seed=33)
    Ug = _t(U0)
    S.solve(Ug, S.load_vector(_t(f)), rtol=1e-30, max_cycles=1)
    Uo = U0 + H.fmg(F - H.fine.K @ U0)
    assert _rel(_np(Ug), Uo) < RTOL_IT


@pytest.mark.parametrize("p,sigma,gamma,fmg", [(2, 1.0, 2, False), (3, 1.0, 2, False), (2, 1e4, 1, True),
                                               (3, 1e-4, 2, True)])
def test_w_and_fmg_solves_match_oracle_2d(p, sigma, gamma, fmg):
    n, L = 32, 4
    S = _solver(p, n, L, sigma=sigma, gamma=gamma, fmg=fmg)
    H = o2.Hierarchy(p, n, L, sigma, 1.0, gamma=gamma)
    f = inputs.grf_forcing(p, n, seed=34)
    F = H.fine.load_vector(f)
    U = np.zeros_like(F)
    k, hist = H.solve(U, F, 1e-8, 50, fmg=fmg)
    Ug = S.empty()
    rep = S.solve(Ug, S.load_vector(_t(f)), rtol=1e-8, max_cycles=50)
    assert rep["converged"] and rep["cycles"] == k
    assert _rel(_np(Ug), U) < RTOL_IT
    assert np.allclose(rep["history"], np.array(hist[1:]) / hist[0], rtol=1e-6)
    assert rep["div_inf"] < 1e-10 * np.abs(U).max()


@pytest.mark.parametrize("gamma,fmg", [(2, False), (1, True), (2, True)])
def test_mixed_precision_w_and_fmg_2d(gamma, fmg):
    from paper_1705_09282_gb300 import _lib
    p, n, L = 2, 64, 5
    f = inputs.grf_forcing(p, n, seed=35)
    S64 = _solver(p, n, L, gamma=gamma, fmg=fmg)
    S32 = _solver(p, n, L, gamma=gamma, fmg=fmg, precision=_lib.IGAMG_FP32_IR)
    U64, U32 = S64.empty(), S32.empty()
    r64 = S64.solve(U64, S64.load_vector(_t(f)), rtol=1e-8, max_cycles=50)
    r32 = S32.solve(U32, S32.load_vector(_t(f)), rtol=1e-8, max_cycles=50)
    assert r64["converged"] and r32["converged"]
    assert r32["cycles"] <= r64["cycles"] + 2
    assert r32["div_inf"] < 1e-10 * float(U32.abs().max())
    assert _rel(_np(U32), _np(U64)) < 1e-6


def test_w_cycle_iterates_and_fmg_3d():
    p, n, L = 2, 8, 3
    S = _solver(p, n, L, dim=3, gamma=2, fmg=True)
    H = o3.Hierarchy3D(p, n, L, 1.0, 1.0, gamma=2)
    F = H.fine.load_vector(inputs.manufactured_forcing_3d(p, n, 1.0, 1.0))
    Fg = _t(F)
    # FMG first step, then W-cycles
    Ug = S.empty()
    S.solve(Ug, Fg, rtol=1e-30, max_cycles=1)
    U = H.fmg(F)
    assert _rel(_np(Ug), U) < RTOL_IT
    for k in range(2):
        H.vcycle(U, F)
        S.vcycle(Ug, Fg)
        assert _rel(_np(Ug), U) < RTOL_IT, k
    # a whole solve: same cycle count as the oracle
    Uo = np.zeros_like(F)
    ko, _ = H.solve(Uo, F, 1e-8, 40, fmg=True)
    Ug = S.empty()
    rep = S.solve(Ug, Fg, rtol=1e-8, max_cycles=40)
    assert rep["converged"] and rep["cycles"] == ko
    assert _rel(_np(Ug), Uo) < RTOL_IT
    assert rep["div_inf"] <= 1e-11 * np.abs(Uo).max()


def test_mixed_precision_fmg_3d():
    from paper_1705_09282_gb300 import _lib
    p, n, L = 2, 16, 3
    S = _solver(p, n, L, dim=3, fmg=True, precision=_lib.IGAMG_FP32_IR)
    F = S.load_vector(_t(inputs.manufactured_forcing_3d(p, n, 1.0, 1.0)))
    U = S.empty()
    rep = S.solve(U, F, rtol=1e-8, max_cycles=40)
    assert rep["converged"]
    assert rep["div_inf"] <= 1e-10 * float(U.abs().max())
