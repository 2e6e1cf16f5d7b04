"""Lockstep batches (igamg_solve_batch): FP64 handles of one cycle shape step their V-cycles
together (one group per mesh, and one mixed-size group of the left-over meshes, its V-cycles
aligned from the finest grid down), each colour / residual / transfer / coarse solve one
launch over up to 24 solves, larger groups as parallel graph branches, converged solves
switched off by a device flag.
Per solve the arithmetic is the single solve's up to the order of each row's sum (the
throughput-bound batch kernels keep one multiply-add chain per stencil box, the latency-bound
single-solve kernels four), so with per-level launches on every level (IGAMG_FUSED_LEVELS=-1
for the single solves) cycle counts are equal and iterates and histories agree to round-off."""
import numpy as np
import pytest

from paper_1705_09282_gb300 import inputs

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(cases, monkeypatch, abs_tol=False, zero=()):
    torch = _torch()
    from paper_1705_09282_gb300 import warmstart as ws
    from paper_1705_09282_gb300.solver import Solver, solve_batch
    monkeypatch.setenv("IGAMG_FUSED_LEVELS", "-1")
    monkeypatch.setenv("IGAMG_LOCKSTEP_MIN", "2")       # small groups too (default: 8 or more)
    solvers, Fs, Us, singles, atol = [], [], [], [], []
    for j, (p, n, L, sigma, kw) in enumerate(cases):
        S = Solver(p, n, L, sigma, 1.0, **kw)
        if kw.get("geometry", 0) == 1:
            X = S.quad_points_xy()
            f = inputs.annulus_forcing(X[0], X[1], sigma, 1.0)
        else:
            f = inputs.grf_forcing(p, n, seed=300 + j)
        F = S.load_vector(torch.tensor(f, device="cuda"))
        if j in zero:
            F.zero_()
        a = 1e-8 * float(torch.linalg.norm(F)) if abs_tol else None
        U1 = S.empty()
        if abs_tol:
            r1 = ws.solve_abs(S, U1, F, a, 80)
        else:
            r1 = S.solve(U1, F, rtol=1e-8, max_cycles=80)
        singles.append((r1, U1.cpu().numpy()))
        solvers.append(S); Fs.append(F); Us.append(S.empty()); atol.append(a)
    if abs_tol:
        reps = ws.solve_batch_abs(solvers, Us, Fs, atol, 80)
    else:
        reps = solve_batch(solvers, Us, Fs, rtol=1e-8, max_cycles=80, history=True)
    for j, ((r1, U1), rep, U) in enumerate(zip(singles, reps, Us)):
        assert rep["converged"] == r1["converged"] and rep["cycles"] == r1["cycles"], j
        Ub = U.cpu().numpy()
        assert np.abs(Ub - U1).max() <= 1e-12 * max(np.abs(U1).max(), 1e-300), j
        if not abs_tol:
            assert rep["history"] == pytest.approx(r1["history"], rel=1e-8), j
        assert rep["div_inf"] <= 1e-12 * max(np.abs(U1).max(), 1.0), j
    return reps


def test_mixed_groups_and_stragglers(monkeypatch):
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR
    cases = [(2, 32, 4, s, {}) for s in (1e-4, 1e-2, 1.0, 1e2, 1e4)]            # one group of 5
    cases += [(3, 32, 4, s, {}) for s in (1e-2, 1e2)]                          # a second group
    cases += [(2, 16, 3, 1.0, {})]                                             # a singleton
    cases += [(2, 32, 4, 1.0, {"precision": IGAMG_FP32_IR})]                   # not batched (FP32)
    cases += [(2, 32, 4, 3.0, {"gamma": 2})]                                   # not batched (W-cycle)
    _run(cases, monkeypatch)


def test_group_larger_than_one_launch(monkeypatch):
    # 30 solves: two branches (15 + 15) of at most 24 solves, side by side in the batch graph
    rng = np.random.default_rng(5)
    cases = [(2, 16, 3, float(10 ** rng.uniform(-2, 4)), {}) for _ in range(30)]
    reps = _run(cases, monkeypatch)
    assert len({r["cycles"] for r in reps}) >= 1


def test_mixed_size_group(monkeypatch):
    # one solve per mesh (none forms a group of its own): the left-over solves share one
    # mixed-size group whose launches cover meshes of 16^2 .. 48^2 with 3 and 4 grids, their
    # V-cycles aligned from the finest grid down; plus a Stokes-Oseen pair that must not mix
    cases = [(2, 16, 3, 1.0, {}), (2, 24, 3, 1e2, {}), (2, 32, 4, 1e-2, {}), (2, 40, 3, 10.0, {}),
             (2, 48, 4, 1e3, {})]
    cases += [(3, 16, 3, 1.0, {}), (3, 32, 4, 1e2, {})]                       # a p = 3 mixed group
    reps = _run(cases, monkeypatch)
    assert all(r["converged"] for r in reps)


def test_absolute_tolerance_and_zero_rhs(monkeypatch):
    cases = [(2, 32, 4, s, {}) for s in (1e-2, 1.0, 1e3)] + [(3, 16, 3, s, {}) for s in (1.0, 10.0)]
    reps = _run(cases, monkeypatch, abs_tol=True, zero=(1,))
    assert reps[1]["cycles"] == 0 and reps[1]["converged"]


def test_annulus_group(monkeypatch):
    cases = [(2, 16, 3, s, {"geometry": 1}) for s in (1.0, 1e3, 1e-2)]
    _run(cases, monkeypatch)


def test_member_handle_recreated_between_batches(monkeypatch):
    # the group's captured graphs belong to the batch's list of handles; a member destroyed and
    # replaced (possibly at the same address) must not reuse them
    torch = _torch()
    from paper_1705_09282_gb300.solver import Solver, solve_batch
    monkeypatch.setenv("IGAMG_FUSED_LEVELS", "-1")
    monkeypatch.setenv("IGAMG_LOCKSTEP_MIN", "2")
    p, n, L = 2, 16, 3
    f = torch.tensor(inputs.grf_forcing(p, n, seed=77), device="cuda")
    A = Solver(p, n, L, 1.0, 1.0)
    B = Solver(p, n, L, 10.0, 1.0)
    FA, FB = A.load_vector(f), B.load_vector(f)
    UA, UB = A.empty(), B.empty()
    solve_batch([A, B], [UA, UB], [FA, FB], rtol=1e-8, max_cycles=60)
    B.close()
    del B
    C = Solver(p, n, L, 1e3, 1.0)                     # same structure, other operator
    FC = C.load_vector(f)
    UA.zero_()
    UC = UB                                          # the same vector buffers as before
    UC.zero_()
    FB.copy_(FC)
    reps = solve_batch([A, C], [UA, UC], [FA, FB], rtol=1e-8, max_cycles=60)
    U1 = C.empty()
    r1 = C.solve(U1, FC, rtol=1e-8, max_cycles=60)
    assert reps[1]["cycles"] == r1["cycles"]
    a, b = UC.cpu().numpy(), U1.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
