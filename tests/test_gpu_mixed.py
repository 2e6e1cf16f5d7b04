"""FP32 V-cycles inside FP64 iterative refinement (the precision wrapper), on the GPU.

Bar: the same 1e-8 relative residual as the FP64 solve, the solution within 1e-6 of the
FP64 oracle's converged iterate, and a velocity that stays pointwise divergence-free at
FP64 round-off (the correction is applied as the exact discrete curl of a streamfunction).
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


@pytest.mark.parametrize("p,sigma,smoother", [(2, 1.0, "mult"), (3, 1.0, "mult"), (2, 1e4, "mult"),
                                               (2, 1e-4, "mult"), (2, 1.0, "add")])
def test_fp32_refinement_reaches_fp64_solution(p, sigma, smoother):
    torch = _torch()
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR
    from paper_1705_09282_gb300.solver import Solver
    n, L = 32, 4
    eta = 0.3 if smoother == "add" else 0.5
    H = o2.Hierarchy(p, n, L, sigma, 1.0, smoother=smoother, eta=eta)
    f = inputs.grf_forcing(p, n, seed=29)
    F = H.fine.load_vector(f)
    U = np.zeros_like(F)
    k64, _ = H.solve(U, F, 1e-10, 80)
    S = Solver(p, n, L, sigma, 1.0, smoother=smoother, eta=eta, precision=IGAMG_FP32_IR)
    Fg = S.load_vector(torch.tensor(f, device="cuda"))
    Ug = S.empty()
    rep = S.solve(Ug, Fg, rtol=1e-8, max_cycles=80)
    assert rep["converged"] and rep["rel_residual"] <= 1e-8
    Ugn = Ug.cpu().numpy()
    assert np.abs(Ugn - U).max() <= 1e-6 * np.abs(U).max()
    assert rep["div_inf"] <= 1e-12 * np.abs(U).max()
    # not many more cycles than the FP64 solve to the same tolerance
    S64 = Solver(p, n, L, sigma, 1.0, smoother=smoother, eta=eta)
    U64 = S64.empty()
    rep64 = S64.solve(U64, S64.load_vector(torch.tensor(f, device="cuda")), rtol=1e-8, max_cycles=80)
    assert rep["cycles"] <= rep64["cycles"] + 2
    # refinement keeps going below the FP32 accuracy of one inner cycle
    Ug.zero_()
    rep = S.solve(Ug, Fg, rtol=1e-11, max_cycles=80)
    assert rep["converged"]
    assert np.abs(Ug.cpu().numpy() - U).max() <= 1e-9 * np.abs(U).max()


def test_fp32_vcycle_entry_point_is_one_refinement_step():
    torch = _torch()
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR
    from paper_1705_09282_gb300.solver import Solver
    p, n, L = 2, 16, 3
    S = Solver(p, n, L, 1.0, 1.0, precision=IGAMG_FP32_IR)
    F = S.load_vector(torch.tensor(inputs.grf_forcing(p, n, seed=3), device="cuda"))
    U = S.empty()
    r = [S.residual(U, F, norm=True)[1]]
    for _ in range(4):
        S.vcycle(U, F)
        r.append(S.residual(U, F, norm=True)[1])
    assert all(r[i + 1] < 0.5 * r[i] for i in range(4))
    assert S.div_inf(U) <= 1e-12 * float(U.abs().max())


@pytest.mark.parametrize("p,sigma", [(2, 1.0), (3, 1e-4), (2, 1e4)])
def test_bf16_operand_refinement_reaches_fp64_solution(p, sigma, monkeypatch):
    # FP32 V-cycles whose operator records and local inverses are rounded to bfloat16 (FP32
    # accumulation) inside FP64 refinement: the outer FP64 residual still reaches 1e-8, the
    # velocity stays divergence-free at FP64 round-off, and the solution is the oracle's to 1e-6
    torch = _torch()
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR
    from paper_1705_09282_gb300.solver import Solver
    n, L = 32, 4
    H = o2.Hierarchy(p, n, L, sigma, 1.0)
    f = inputs.grf_forcing(p, n, seed=31)
    F = H.fine.load_vector(f)
    U = np.zeros_like(F)
    H.solve(U, F, 1e-11, 80)
    monkeypatch.setenv("IGAMG_BF16_OPERANDS", "1")
    S16 = Solver(p, n, L, sigma, 1.0, precision=IGAMG_FP32_IR)
    monkeypatch.delenv("IGAMG_BF16_OPERANDS")
    S32 = Solver(p, n, L, sigma, 1.0, precision=IGAMG_FP32_IR)
    reps = []
    for S in (S16, S32):
        Ug = S.empty()
        rep = S.solve(Ug, S.load_vector(torch.tensor(f, device="cuda")), rtol=1e-8, max_cycles=80)
        assert rep["converged"] and rep["rel_residual"] <= 1e-8
        assert rep["div_inf"] <= 1e-11 * np.abs(U).max()
        assert np.abs(Ug.cpu().numpy() - U).max() <= 1e-6 * np.abs(U).max()
        reps.append(rep)
    # bf16 operands cost cycles but not many (their inner V-cycle is a coarser approximation)
    assert reps[0]["cycles"] <= 2 * reps[1]["cycles"] + 2, (reps[0]["cycles"], reps[1]["cycles"])
    S16.close()
    S32.close()
