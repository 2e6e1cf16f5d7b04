"""FGMRES(m) around the V-cycle (precision wrapper): FP64 and FP32 preconditioners reach
the FP64 oracle's solution, keep every iterate divergence-free at round-off, and need no
more V-cycles than the plain iteration (2D and 3D)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import stokes2d as o2
from oracle import stokes3d as o3
from paper_1705_09282_gb300 import inputs

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _t(x):
    return _torch().tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("p,n,L,sigma", [(2, 32, 4, 1.0), (3, 32, 4, 1.0), (2, 32, 4, 1e-4), (2, 24, 3, 1e3)])
@pytest.mark.parametrize("prec", [2, 3])
def test_fgmres_2d_matches_direct_solve(p, n, L, sigma, prec):
    _torch()
    from paper_1705_09282_gb300.solver import Solver
    S0 = Solver(p, n, L, sigma, 1.0)
    SK = Solver(p, n, L, sigma, 1.0, precision=prec, restart=12)
    f = inputs.grf_forcing(p, n, seed=70 + n)
    Ko = o2.Stokes2D(p, n, sigma, 1.0)
    F = Ko.load_vector(f)
    Ux = spla.spsolve(Ko.K.tocsc(), F)
    Fg = _t(F)
    U0, UK = S0.empty(), SK.empty()
    r0 = S0.solve(U0, Fg, rtol=1e-10, max_cycles=100)
    rk = SK.solve(UK, Fg, rtol=1e-10, max_cycles=100)
    assert r0["converged"] and rk["converged"], (r0["cycles"], rk)
    assert rk["rel_residual"] <= 1e-10
    assert _rel(_np(UK), Ux) < 1e-8
    assert rk["div_inf"] <= 1e-12 * np.abs(Ux).max()
    assert rk["cycles"] <= r0["cycles"]
    # the reported history is the Krylov estimate, decreasing
    h = rk["history"]
    assert len(h) == rk["cycles"] and all(b <= a * (1 + 1e-12) for a, b in zip(h, h[1:]))


@pytest.mark.parametrize("prec", [2, 3])
def test_fgmres_restarts(prec):
    # a small restart length forces several restart cycles; the result does not change
    _torch()
    from paper_1705_09282_gb300.solver import Solver
    p, n, L = 2, 32, 4
    S = Solver(p, n, L, 1.0, 1.0, precision=prec, restart=3)
    f = inputs.grf_forcing(p, n, seed=5)
    Ko = o2.Stokes2D(p, n, 1.0, 1.0)
    F = Ko.load_vector(f)
    U = S.empty()
    rep = S.solve(U, _t(F), rtol=1e-10, max_cycles=100)
    assert rep["converged"] and rep["cycles"] > 3
    assert _rel(_np(U), spla.spsolve(Ko.K.tocsc(), F)) < 1e-8


@pytest.mark.parametrize("prec", [2, 3])
def test_fgmres_3d(prec):
    _torch()
    from paper_1705_09282_gb300.solver import Solver
    p, n, L = 2, 8, 3
    S0 = Solver(p, n, L, 1.0, 1.0, dim=3)
    SK = Solver(p, n, L, 1.0, 1.0, precision=prec, dim=3, restart=10)
    H = o3.Hierarchy3D(p, n, L, 1.0, 1.0)
    F = H.fine.load_vector(inputs.manufactured_forcing_3d(p, n, 1.0, 1.0))
    Ux = spla.spsolve(H.levels[-1].K.tocsc(), F)
    U0, UK = S0.empty(), SK.empty()
    r0 = S0.solve(U0, _t(F), rtol=1e-10, max_cycles=60)
    rk = SK.solve(UK, _t(F), rtol=1e-10, max_cycles=60)
    assert rk["converged"] and rk["cycles"] <= r0["cycles"]
    assert _rel(_np(UK), Ux) < 1e-8
    assert rk["div_inf"] <= 1e-12 * np.abs(Ux).max()
