"""Forms of the multiplicative colour sweep: the pipelined sweep (k_sweep_tiles) against one
launch per colour, and the two-lanes-per-row patch form against one lane per row.

The pipelined form runs all colours of a level's sweeps in one cooperative launch, tile by
tile, each tile waiting only for its eight neighbours (Sec. 5.2's colour-major order kept
locally).  Every patch computes the same arithmetic from the same values as in the
colour-by-colour sweep, so results are identical bit for bit, for any tile width.  The
timeout path is exercised by a tile that never reports progress: the waits give up, the
host reports IGAMG_ETIMEOUT, and the context stays usable.
"""
import numpy as np
import pytest

from paper_1705_09282_gb300 import inputs

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _pair(monkeypatch, mult, p, n, L, sigma=1.0, nu=1.0, **kw):
    from paper_1705_09282_gb300.solver import Solver
    monkeypatch.setenv("IGAMG_PIPELINE", "0")
    monkeypatch.setenv("IGAMG_ROW_LANES", "1")      # the lane form the tile kernel uses
    S0 = Solver(p, n, L, sigma, nu, **kw)
    monkeypatch.delenv("IGAMG_ROW_LANES")
    monkeypatch.setenv("IGAMG_PIPELINE", "1")
    monkeypatch.setenv("IGAMG_TILE_MULT", str(mult))
    S1 = Solver(p, n, L, sigma, nu, **kw)
    monkeypatch.delenv("IGAMG_TILE_MULT")
    return S0, S1


@pytest.mark.parametrize("p,n,L,mult", [(2, 64, 4, 1), (2, 64, 4, 4), (3, 64, 4, 1), (3, 40, 3, 2),
                                        (2, 50, 2, 1)])
def test_pipelined_sweeps_equal_colour_launches(p, n, L, mult, monkeypatch):
    torch = _torch()
    S0, S1 = _pair(monkeypatch, mult, p, n, L)
    for lev in range(1, L):
        nd = S0.ndof(lev)
        U = torch.tensor(inputs.random_vector(nd, seed=70 + lev), device="cuda")
        F = torch.tensor(inputs.random_vector(nd, seed=80 + lev), device="cuda")
        for sweeps in (1, 2):
            U0, U1 = U.clone(), U.clone()
            S0.smooth(U0, F, level=lev, sweeps=sweeps)
            S1.smooth(U1, F, level=lev, sweeps=sweeps)
            assert torch.equal(U0, U1), (lev, sweeps)
    S0.close()
    S1.close()


@pytest.mark.parametrize("kind", ["oseen", "fp32", "annulus"])
def test_pipelined_solves_equal_colour_launches(kind, monkeypatch):
    torch = _torch()
    from paper_1705_09282_gb300 import _lib
    p, n, L = 2, 32, 4
    kw, sigma, nu = {}, 1.0, 1.0
    if kind == "oseen":
        kw["beta"] = inputs.oseen_advection(p, n, 0.5)
        sigma, nu = 10.0, 0.05
    elif kind == "fp32":
        kw["precision"] = _lib.IGAMG_FP32_IR
    else:
        kw["geometry"] = _lib.IGAMG_GEOM_QUARTER_ANNULUS
    S0, S1 = _pair(monkeypatch, 1, p, n, L, sigma, nu, **kw)
    if kind == "annulus":
        X = S0.quad_points_xy()
        f = inputs.annulus_forcing(X[0], X[1], sigma, nu)
    else:
        f = inputs.grf_forcing(p, n, seed=91)
    out = []
    for S in (S0, S1):
        F = S.load_vector(torch.tensor(f, device="cuda"))
        U = S.empty()
        rep = S.solve(U, F, rtol=1e-9, max_cycles=80)
        assert rep["converged"]
        out.append((rep["cycles"], U.cpu().numpy()))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])
    S0.close()
    S1.close()


def test_sweep_timeout_is_reported_and_the_context_stays_usable(monkeypatch):
    torch = _torch()
    from paper_1705_09282_gb300._lib import IgamgError
    from paper_1705_09282_gb300.solver import Solver
    p, n, L = 2, 48, 3
    monkeypatch.setenv("IGAMG_FUSED_LEVELS", "-1")     # no tuning runs at creation
    monkeypatch.setenv("IGAMG_PIPELINE", "1")
    monkeypatch.setenv("IGAMG_TILE_MULT", "1")
    monkeypatch.setenv("IGAMG_TEST_STALL_TILE", "0")  # tile 0 never reports its progress
    S = Solver(p, n, L, 1.0, 1.0)
    monkeypatch.delenv("IGAMG_TEST_STALL_TILE")
    f = inputs.grf_forcing(p, n, seed=5)
    F = S.load_vector(torch.tensor(f, device="cuda"))
    U = S.empty()
    with pytest.raises(IgamgError) as ei:
        S.solve(U, F, rtol=1e-8, max_cycles=5)
    assert ei.value.code == -6                        # IGAMG_ETIMEOUT
    torch.cuda.synchronize()
    S.close()
    # the same problem on a healthy handle solves normally afterwards
    monkeypatch.delenv("IGAMG_PIPELINE")
    S2 = Solver(p, n, L, 1.0, 1.0)
    U2 = S2.empty()
    rep = S2.solve(U2, S2.load_vector(torch.tensor(f, device="cuda")), rtol=1e-8, max_cycles=40)
    assert rep["converged"]
    S2.close()


@pytest.mark.parametrize("p,n,L", [(2, 64, 4), (3, 48, 3)])
def test_two_lanes_per_row_form_matches_one_lane(p, n, L, monkeypatch):
    # the same sweep with each 8-DOF patch row's multiply-adds split over two lanes: only the
    # summation order changes (1e-13), and solves take the same cycles to the same iterates
    torch = _torch()
    from paper_1705_09282_gb300.solver import Solver
    S = {}
    for lanes in ("1", "2"):
        monkeypatch.setenv("IGAMG_ROW_LANES", lanes)
        S[lanes] = Solver(p, n, L, 1.0, 1.0)
    monkeypatch.delenv("IGAMG_ROW_LANES")
    for lev in range(1, L):
        nd = S["1"].ndof(lev)
        U = torch.tensor(inputs.random_vector(nd, seed=170 + lev), device="cuda")
        F = torch.tensor(inputs.random_vector(nd, seed=180 + lev), device="cuda")
        U1, U2 = U.clone(), U.clone()
        S["1"].smooth(U1, F, level=lev, sweeps=2)
        S["2"].smooth(U2, F, level=lev, sweeps=2)
        a, b = U2.cpu().numpy(), U1.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), lev
    f = inputs.grf_forcing(p, n, seed=93)
    res = []
    for k in ("1", "2"):
        Ug = S[k].empty()
        rep = S[k].solve(Ug, S[k].load_vector(torch.tensor(f, device="cuda")), rtol=1e-9, max_cycles=60)
        res.append((rep["cycles"], Ug.cpu().numpy()))
        S[k].close()
    assert res[0][0] == res[1][0]
    assert np.abs(res[0][1] - res[1][1]).max() <= 1e-12 * np.abs(res[0][1]).max()


@pytest.mark.parametrize("p,n,L", [(2, 64, 4), (3, 48, 3)])
def test_two_chain_form_matches_four_chains(p, n, L, monkeypatch):
    # the one-lane colour kernel with two multiply-add chains per row and local inverse instead
    # of four: only the summation order changes, so sweeps agree to 1e-13 and solves take the
    # same cycles to the same iterates
    torch = _torch()
    from paper_1705_09282_gb300.solver import Solver
    S = {}
    for form in ("lanes1_b64", "lanes1_b64_c2"):
        monkeypatch.setenv("IGAMG_SWEEP_FORM", form)
        S[form] = Solver(p, n, L, 1.0, 1.0)
    monkeypatch.delenv("IGAMG_SWEEP_FORM")
    assert S["lanes1_b64"].level_form()["chains"] == 4
    assert S["lanes1_b64_c2"].level_form() == {"lanes": 1, "threads": 64, "tiles": 0, "chains": 2}
    for lev in range(1, L):
        nd = S["lanes1_b64"].ndof(lev)
        U = torch.tensor(inputs.random_vector(nd, seed=270 + lev), device="cuda")
        F = torch.tensor(inputs.random_vector(nd, seed=280 + lev), device="cuda")
        U4, U2 = U.clone(), U.clone()
        S["lanes1_b64"].smooth(U4, F, level=lev, sweeps=2)
        S["lanes1_b64_c2"].smooth(U2, F, level=lev, sweeps=2)
        a, b = U2.cpu().numpy(), U4.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), lev
    f = inputs.grf_forcing(p, n, seed=94)
    res = []
    for k in ("lanes1_b64", "lanes1_b64_c2"):
        Ug = S[k].empty()
        rep = S[k].solve(Ug, S[k].load_vector(torch.tensor(f, device="cuda")), rtol=1e-9, max_cycles=60)
        res.append((rep["cycles"], Ug.cpu().numpy()))
        S[k].close()
    assert res[0][0] == res[1][0]
    assert np.abs(res[0][1] - res[1][1]).max() <= 1e-12 * np.abs(res[0][1]).max()
