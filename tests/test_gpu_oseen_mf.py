"""The finest generalized-Oseen level's residual with the advection term applied matrix-free.

Sec. 3.1's advection integrals (beta . grad u, v) are evaluated element by element at the
(p+2)^2 Gauss points (sum-factorised per direction, k_residual_adv) instead of read from
stored per-row records.  Both forms are compared with the oracle's assembled K (F - K U) and
with each other, in FP64 and in the FP32 V-cycle's precision, on meshes that span several
tiles of the kernel and end in a ragged one, with a random advection field (no symmetry to
hide a transposed or mirrored index) and with the workload's smooth field.
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


def _random_beta(p, n, seed):
    nG = n * (p + 2)
    return inputs.random_vector(2 * nG * nG, seed).reshape(2, nG, nG)


def _solver(monkeypatch, form, *args, **kw):
    from paper_1705_09282_gb300.solver import Solver
    monkeypatch.setenv("IGAMG_ADV_FORM", form)
    S = Solver(*args, **kw)
    monkeypatch.delenv("IGAMG_ADV_FORM")
    return S


# tiles of 14 (p = 2) and 13 (p = 3) index positions: 41 -> 3 tiles, 50 -> 4, 14 -> 1 (exact),
# 8 -> one tile larger than the mesh
@pytest.mark.parametrize("p,n,L", [(2, 40, 3), (3, 48, 3), (2, 12, 2), (3, 6, 2)])
def test_matrix_free_residual_matches_oracle(p, n, L, monkeypatch):
    torch = _torch()
    sigma, nu = 2.0, 0.05
    beta = _random_beta(p, n, seed=500 + n)
    S_mf = _solver(monkeypatch, "mf", p, n, L, sigma, nu, beta=beta)
    S_rec = _solver(monkeypatch, "records", p, n, L, sigma, nu, beta=beta)
    assert S_mf.residual_form()["fp64"] == 2
    assert S_rec.residual_form()["fp64"] == 1
    H = o2.Hierarchy(p, n, L, sigma, nu, beta=beta)
    K = H.fine.K
    nd = K.shape[0]
    U = inputs.random_vector(nd, seed=600 + n)
    F = inputs.random_vector(nd, seed=700 + n)
    Ug, Fg = torch.tensor(U, device="cuda"), torch.tensor(F, device="cuda")
    Rm, nm = S_mf.residual(Ug, Fg, norm=True)
    Rr, nr = S_rec.residual(Ug, Fg, norm=True)
    Ro = F - K @ U
    assert _rel(Rm.cpu().numpy(), Ro) < 1e-11
    assert _rel(Rm.cpu().numpy(), Rr.cpu().numpy()) < 1e-12
    assert abs(nm - np.linalg.norm(Ro)) <= 1e-11 * np.linalg.norm(Ro)
    assert abs(nm - nr) <= 1e-12 * nr
    # coarse levels keep their Galerkin records: unchanged
    for lev in range(L - 1):
        ndl = H.levels[lev].K.shape[0]
        Ul = torch.tensor(inputs.random_vector(ndl, seed=lev + 3), device="cuda")
        Fl = torch.tensor(inputs.random_vector(ndl, seed=lev + 13), device="cuda")
        assert torch.equal(S_mf.residual(Ul, Fl, level=lev), S_rec.residual(Ul, Fl, level=lev))
    S_mf.close()
    S_rec.close()


@pytest.mark.parametrize("p,n", [(2, 40), (3, 24)])
def test_matrix_free_residual_fp32(p, n, monkeypatch):
    torch = _torch()
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR
    sigma, nu, L = 1.0, 0.01, 3
    beta = inputs.oseen_advection(p, n, 0.5)
    S_mf = _solver(monkeypatch, "mf", p, n, L, sigma, nu, beta=beta, precision=IGAMG_FP32_IR)
    S_rec = _solver(monkeypatch, "records", p, n, L, sigma, nu, beta=beta, precision=IGAMG_FP32_IR)
    assert S_mf.residual_form() == {"fp64": 2, "fp32": 2}
    assert S_rec.residual_form() == {"fp64": 1, "fp32": 1}
    H = o2.Hierarchy(p, n, L, sigma, nu, beta=beta)
    nd = H.fine.K.shape[0]
    U32 = inputs.random_vector(nd, seed=41).astype(np.float32)
    F32 = inputs.random_vector(nd, seed=42).astype(np.float32)
    Ro = F32.astype(np.float64) - H.fine.K @ U32.astype(np.float64)
    Ug, Fg = torch.tensor(U32, device="cuda"), torch.tensor(F32, device="cuda")
    Rm = S_mf.residual32(Ug, Fg).cpu().numpy().astype(np.float64)
    Rr = S_rec.residual32(Ug, Fg).cpu().numpy().astype(np.float64)
    # FP32 arithmetic on FP32-rounded operator values: a few units of 2^-24 of the row sums
    assert _rel(Rm, Ro) < 2e-5
    assert _rel(Rr, Ro) < 2e-5
    S_mf.close()
    S_rec.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32ir"])
def test_matrix_free_solves_match_records(precision, monkeypatch):
    torch = _torch()
    from paper_1705_09282_gb300._lib import IGAMG_FP32_IR, IGAMG_FP64
    p, n, L, sigma, nu = 2, 64, 5, 1.0, 0.01
    prec = IGAMG_FP64 if precision == "fp64" else IGAMG_FP32_IR
    beta = inputs.oseen_advection(p, n, 0.5)
    f = inputs.grf_forcing(p, n, seed=1707)
    out = []
    for form in ("mf", "records"):
        S = _solver(monkeypatch, form, p, n, L, sigma, nu, beta=beta, precision=prec)
        U = S.empty()
        rep = S.solve(U, S.load_vector(torch.tensor(f, device="cuda")), rtol=1e-8, max_cycles=60)
        assert rep["converged"] and rep["div_inf"] < 1e-12 * U.abs().max().item()
        out.append((rep["cycles"], U.cpu().numpy()))
        S.close()
    assert out[0][0] == out[1][0]
    assert _rel(out[0][1], out[1][1]) < (1e-10 if precision == "fp64" else 1e-6)


def test_matrix_free_oseen_128_vcycle_iterates(monkeypatch):
    # the Oseen workload's operator family (nu = 1e-2, sigma = 1, max |beta| = 0.5, GRF forcing
    # seed 1707) at 128^2, 6 grids, with the matrix-free fine residual: two V-cycles equal the
    # oracle's
    torch = _torch()
    p, n, L, sigma, nu = 2, 128, 6, 1.0, 1e-2
    beta = inputs.oseen_advection(p, n, 0.5)
    f = inputs.grf_forcing(p, n, seed=1707)
    S = _solver(monkeypatch, "mf", p, n, L, sigma, nu, beta=beta)
    H = o2.Hierarchy(p, n, L, sigma, nu, beta=beta)
    F = H.fine.load_vector(f)
    Fg = S.load_vector(torch.tensor(f, device="cuda"))
    U, Ug = np.zeros_like(F), S.empty()
    for k in range(2):
        H.vcycle(U, F)
        S.vcycle(Ug, Fg)
        assert _rel(Ug.cpu().numpy(), U) < 1e-10, k
    S.close()


def test_matrix_free_residual_at_512(monkeypatch):
    # the Oseen workload's full size (512^2, 8 grids): every row of the matrix-free residual
    # equals the oracle's assembled fine operator applied to U (F - K U), and the record form
    torch = _torch()
    p, n, L, sigma, nu = 2, 512, 8, 1.0, 1e-2
    beta = inputs.oseen_advection(p, n, 0.5)
    S_mf = _solver(monkeypatch, "mf", p, n, L, sigma, nu, beta=beta)
    S_rec = _solver(monkeypatch, "records", p, n, L, sigma, nu, beta=beta)
    nd = S_mf.ndof()
    U = inputs.random_vector(nd, seed=8)
    F = inputs.random_vector(nd, seed=9)
    Ug, Fg = torch.tensor(U, device="cuda"), torch.tensor(F, device="cuda")
    Rm, nm = S_mf.residual(Ug, Fg, norm=True)
    Rr = S_rec.residual(Ug, Fg).cpu().numpy()
    Rm = Rm.cpu().numpy()
    S_mf.close()
    S_rec.close()
    assert _rel(Rm, Rr) < 1e-12
    K = o2.Stokes2D(p, n, sigma, nu, beta=beta).K
    Ro = F - K @ U
    assert _rel(Rm, Ro) < 1e-11
    assert abs(nm - np.linalg.norm(Ro)) <= 1e-11 * np.linalg.norm(Ro)


def test_residual_form_setter(monkeypatch):
    # the autotuned handle switched by igamg_set_residual_form computes what a handle pinned
    # to that form computes; a Stokes handle (no advection term) refuses
    torch = _torch()
    from paper_1705_09282_gb300._lib import IgamgError
    from paper_1705_09282_gb300.solver import Solver
    p, n, L, sigma, nu = 2, 32, 3, 1.0, 0.01
    beta = inputs.oseen_advection(p, n, 0.5)
    S = Solver(p, n, L, sigma, nu, beta=beta)
    assert S.residual_form()["fp64"] in (1, 2) and S.residual_form()["fp32"] == -1
    nd = S.ndof()
    U = torch.tensor(inputs.random_vector(nd, seed=1), device="cuda")
    F = torch.tensor(inputs.random_vector(nd, seed=2), device="cuda")
    out = {}
    for form in (1, 2):
        S.set_residual_form(fp64=form)
        assert S.residual_form()["fp64"] == form
        out[form] = S.residual(U, F).cpu().numpy()
        P = _solver(monkeypatch, "mf" if form == 2 else "records", p, n, L, sigma, nu, beta=beta)
        assert np.array_equal(out[form], P.residual(U, F).cpu().numpy())
        P.close()
    assert _rel(out[2], out[1]) < 1e-12
    # a solve after switching re-captures its graphs with the new form
    S.set_residual_form(fp64=2)
    Ug = S.empty()
    rep = S.solve(Ug, S.load_vector(torch.tensor(inputs.grf_forcing(p, n, seed=3), device="cuda")), rtol=1e-8)
    assert rep["converged"]
    S.close()
    T = Solver(p, n, L, 1.0, 1.0)
    assert T.residual_form() == {"fp64": 0, "fp32": -1}
    with pytest.raises(IgamgError):
        T.set_residual_form(fp64=2)
    T.close()
