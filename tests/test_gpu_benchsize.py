"""GPU parity against the oracle at the sizes and launch configurations that bench.py times.

The other parity files use small meshes; these cases run the benchmarked configurations
themselves (or the largest member of their operator family the oracle assembles in about a
minute), element by element, at the FP64 tolerance the method's statement fixes (1e-10
relative for iterates) and 1e-6 for the FP32-refined mode:
  * the headline sweep's problems: 2D generalized Stokes, 256 x 256, 7 grids, V(2,2),
    Gaussian-random-field forcing with the bench's seed, sigma/nu at the sweep's ends;
  * the generalized Oseen family (nu = 1e-2, sigma = 1, max |beta| = 0.5) at 128 x 128;
  * the 3D cube (config family of the 64^3 workload) at 16^3 with 3 grids;
  * a lockstep batch (two size classes of eight solves each, the default group threshold)
    against one oracle solve per member;
  * the 3D FP32-in-FP64 refinement against the oracle's converged solution.
"""
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


def _t(x):
    return _torch().tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("p,sigma,cycles", [(2, 1e-4, 2), (3, 1e4, 1)])
def test_headline_problems_vcycle_iterates(p, sigma, cycles):
    # bench.py's sweep problem (256^2, 7 grids, V(2,2), seed 1706) in the bench's launch
    # configuration (default solver, autotuned coarse end): V-cycle iterates from zero
    from paper_1705_09282_gb300.solver import Solver
    n, L, seed = 256, 7, 1706
    f = inputs.grf_forcing(p, n, seed=seed)
    S = Solver(p, n, L, sigma, 1.0, nu1=2, nu2=2)
    Fg = S.load_vector(_t(f))
    H = o2.Hierarchy(p, n, L, sigma, 1.0, nu1=2, nu2=2)
    F = H.fine.load_vector(f)
    assert _rel(_np(Fg), F) < 1e-13
    U, Ug = np.zeros_like(F), S.empty()
    for k in range(cycles):
        H.vcycle(U, F)
        S.vcycle(Ug, Fg)
        assert _rel(_np(Ug), U) < RTOL_IT, k
    R, nrm = S.residual(Ug, Fg, norm=True)
    Ro = F - H.fine.K @ U
    assert abs(nrm - np.linalg.norm(Ro)) <= 1e-8 * np.linalg.norm(Ro)
    S.close()


def test_oseen_family_128_vcycle_iterates():
    # the Oseen workload's operator family (nu = 1e-2, sigma = 1, beta = curl of
    # sin^2 sin^2 scaled to max |beta| = 0.5, GRF forcing seed 1707) at 128^2, 6 grids
    from paper_1705_09282_gb300.solver import Solver
    p, n, L, sigma, nu = 2, 128, 6, 1.0, 1e-2
    beta = inputs.oseen_advection(p, n, 0.5)
    f = inputs.grf_forcing(p, n, seed=1707)
    S = Solver(p, n, L, sigma, nu, beta=beta)
    H = o2.Hierarchy(p, n, L, sigma, nu, beta=beta)
    F = H.fine.load_vector(f)
    Fg = S.load_vector(_t(f))
    U, Ug = np.zeros_like(F), S.empty()
    for k in range(2):
        H.vcycle(U, F)
        S.vcycle(Ug, Fg)
        assert _rel(_np(Ug), U) < RTOL_IT, k
    S.close()


def test_cube_16_vcycle_iterates():
    # the 64^3 cube workload's family (p = 2, manufactured forcing, coarsest 4^3) at 16^3
    from paper_1705_09282_gb300.solver import Solver
    p, n, L = 2, 16, 3
    f = inputs.manufactured_forcing_3d(p, n, 1.0, 1.0)
    S = Solver(p, n, L, 1.0, 1.0, nu1=2, nu2=2, dim=3)
    H = o3.Hierarchy3D(p, n, L, 1.0, 1.0, nu1=2, nu2=2)
    F = H.fine.load_vector(f)
    Fg = S.load_vector(_t(f))
    assert _rel(_np(Fg), F) < 1e-13
    U, Ug = np.zeros_like(F), S.empty()
    for k in range(2):
        H.vcycle(U, F)
        S.vcycle(Ug, Fg)
        assert _rel(_np(Ug), U) < RTOL_IT, k
    S.close()


def test_lockstep_batch_against_oracle_solves():
    # sixteen solves in two size classes (8 x 32^2, 8 x 48^2; sigma/nu log-uniform as in the
    # 1024-solve batch) through igamg_solve_batch with the default lockstep threshold of 8:
    # every member's cycle count and iterate equal the oracle's own solve
    from paper_1705_09282_gb300.solver import Solver, solve_batch
    p = 2
    specs = []
    for j in range(16):
        n, L = (32, 4) if j % 2 == 0 else (48, 5)
        sigma = float(10.0 ** (-2.0 + 6.0 * ((j * 7) % 16) / 15.0))
        specs.append((n, L, sigma, 2100 + j))
    solvers, Us, Fs, oracle = [], [], [], []
    for n, L, sigma, seed in specs:
        f = inputs.grf_forcing(p, n, seed=seed)
        S = Solver(p, n, L, sigma, 1.0)
        solvers.append(S)
        Fs.append(S.load_vector(_t(f)))
        Us.append(S.empty())
        H = o2.Hierarchy(p, n, L, sigma, 1.0)
        F = H.fine.load_vector(f)
        U = np.zeros_like(F)
        k, _ = H.solve(U, F, 1e-8, 60)
        oracle.append((k, U))
    reps = solve_batch(solvers, Us, Fs, rtol=1e-8, max_cycles=60)
    for j, (rep, Ug, (k, U)) in enumerate(zip(reps, Us, oracle)):
        assert rep["converged"] and rep["cycles"] == k, (j, rep["cycles"], k)
        assert _rel(_np(Ug), U) < RTOL_IT, j
    for S in solvers:
        S.close()


@pytest.mark.parametrize("sigma", [1.0, 1e3])
def test_cube_fp32_refinement_against_oracle(sigma):
    # FP32 V-cycles inside FP64 refinement reach the oracle's FP64 solution to 1e-6, with
    # the divergence at FP64 round-off
    from paper_1705_09282_gb300 import _lib
    from paper_1705_09282_gb300.solver import Solver
    p, n, L = 2, 8, 2
    f = inputs.manufactured_forcing_3d(p, n, sigma, 1.0)
    H = o3.Hierarchy3D(p, n, L, sigma, 1.0)
    F = H.fine.load_vector(f)
    U = np.zeros_like(F)
    H.solve(U, F, 1e-12, 80)
    S32 = Solver(p, n, L, sigma, 1.0, dim=3, precision=_lib.IGAMG_FP32_IR)
    Ug = S32.empty()
    rep = S32.solve(Ug, S32.load_vector(_t(f)), rtol=1e-8, max_cycles=60)
    assert rep["converged"] and rep["rel_residual"] <= 1e-8
    assert _rel(_np(Ug), U) < 1e-6
    assert rep["div_inf"] <= 1e-11 * np.abs(U).max()
    S32.close()
