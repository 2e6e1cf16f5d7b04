"""Generalized Oseen (advection beta . grad u, Sec. 3.1) on the GPU against the oracle.

The operator is non-symmetric and not a Kronecker sum, so every level is held as one
stencil record per row, the coarse operators are the Galerkin products R K P of Sec. 5.1,
and every patch has its own bordered local inverse.
"""
import numpy as np
import pytest

from oracle import stokes2d as o2
from paper_1705_09282_gb300 import inputs

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("p,n,L,sigma,nu,vmax", [(2, 32, 4, 1.0, 0.01, 0.5), (3, 16, 3, 10.0, 0.01, 0.5), (2, 16, 3, 1000.0, 1.0, 1.0)])
def test_oseen_operator_smoother_and_solve(p, n, L, sigma, nu, vmax):
    # Re = vmax / nu <= Da / 2: the regime where the paper reports convergence (Sec. 6.5)
    torch = _torch()
    from paper_1705_09282_gb300.solver import Solver
    beta = inputs.oseen_advection(p, n, vmax)
    S = Solver(p, n, L, sigma, nu, beta=beta)
    H = o2.Hierarchy(p, n, L, sigma, nu, beta=beta)
    for lev in range(L):
        nd = H.levels[lev].K.shape[0]
        U = inputs.random_vector(nd, seed=lev + 3)
        F = inputs.random_vector(nd, seed=lev + 13)
        R = S.residual(torch.tensor(U, device="cuda"), torch.tensor(F, device="cuda"), level=lev).cpu().numpy()
        assert _rel(R, F - H.levels[lev].K @ U) < 1e-11, lev
        if lev >= 1:
            Ug = torch.tensor(U, device="cuda")
            S.smooth(Ug, torch.tensor(F, device="cuda"), level=lev, sweeps=1)
            Uo = U.copy()
            H.smooth(lev, Uo, F)
            assert _rel(Ug.cpu().numpy(), Uo) < 1e-11, lev
    f = inputs.grf_forcing(p, n, seed=77)
    Fo = H.fine.load_vector(f)
    Uo = np.zeros_like(Fo)
    k, hist = H.solve(Uo, Fo, 1e-8, 60)
    Ug = S.empty()
    rep = S.solve(Ug, S.load_vector(torch.tensor(f, device="cuda")), rtol=1e-8, max_cycles=60)
    assert rep["converged"] and rep["cycles"] == k
    assert _rel(Ug.cpu().numpy(), Uo) < 1e-10
    assert rep["div_inf"] < 1e-12 * np.abs(Uo).max()


def test_oseen_mixed_precision():
    torch = _torch()
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR
    from paper_1705_09282_gb300.solver import Solver
    p, n, L, sigma, nu = 2, 32, 4, 1.0, 0.01
    beta = inputs.oseen_advection(p, n, 0.5)
    H = o2.Hierarchy(p, n, L, sigma, nu, beta=beta)
    f = inputs.grf_forcing(p, n, seed=78)
    Fo = H.fine.load_vector(f)
    Uo = np.zeros_like(Fo)
    H.solve(Uo, Fo, 1e-12, 80)
    S = Solver(p, n, L, sigma, nu, beta=beta, precision=IGAMG_FP32_IR)
    U = S.empty()
    rep = S.solve(U, S.load_vector(torch.tensor(f, device="cuda")), rtol=1e-8, max_cycles=60)
    assert rep["converged"]
    assert _rel(U.cpu().numpy(), Uo) < 1e-6
    assert rep["div_inf"] < 1e-12 * np.abs(Uo).max()


def test_oseen_advection_dominated_diverges_on_both_sides():
    # Re = Da = 100 (max |beta| = 1, sigma = 1, nu = 0.01): the V-cycle diverges -- the paper
    # reports convergence only when the problem is not advection-dominated; the GPU shows
    # the same growth as the oracle (it is a property of the method here, not of the port)
    torch = _torch()
    from paper_1705_09282_gb300.solver import Solver
    p, n, L, sigma, nu = 2, 32, 4, 1.0, 0.01
    beta = inputs.oseen_advection(p, n, 1.0)
    H = o2.Hierarchy(p, n, L, sigma, nu, beta=beta)
    f = inputs.grf_forcing(p, n, seed=77)
    Fo = H.fine.load_vector(f)
    Uo = np.zeros_like(Fo)
    H.solve(Uo, Fo, 1e-8, 3)
    S = Solver(p, n, L, sigma, nu, beta=beta)
    U = S.empty()
    rep = S.solve(U, S.load_vector(torch.tensor(f, device="cuda")), rtol=1e-8, max_cycles=3)
    assert not rep["converged"] and rep["rel_residual"] > 10.0
    assert _rel(U.cpu().numpy(), Uo) < 1e-9
