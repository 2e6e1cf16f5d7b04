"""CPU checks of the C-ABI library: it loads, exports every declared symbol, and its
host-side set-up (1D Kronecker factors, knot-insertion transfers, patch tables) agrees
with the oracle's independent assembly.  No GPU is needed."""
import os
import re

import numpy as np
import pytest

from oracle import stokes2d as o2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1705_09282_gb300 import _lib
    return _lib


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"\b(igamg_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    L = _lib().lib()
    names = _declared_symbols()
    assert len(names) >= 19
    for n in names:
        assert hasattr(L, n), n
    assert set(_lib().SIGNATURES) >= names


def test_strerror():
    L = _lib().lib()
    assert L.igamg_strerror(-1) == b"invalid argument"
    assert L.igamg_strerror(1).startswith(b"not converged")


def test_bad_arguments_rejected_on_host():
    import ctypes
    L = _lib().lib()
    pr = _lib().make_problem(2, 6, 3, 1.0, 1.0)       # 6 not divisible by 4
    h = ctypes.c_void_p()
    assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -1
    pr = _lib().make_problem(4, 8, 2, 1.0, 1.0)       # p = 4 not built
    assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -2
    pr = _lib().make_problem(2, 8, 2, -1.0, 1.0)      # sigma <= 0
    assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -1
    for dim in (2, 3):
        pr = _lib().make_problem(2, 8, 2, 1.0, 1.0, dim=dim, gamma=5)   # at most 4 coarse cycles
        assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -1
        pr = _lib().make_problem(2, 8, 2, 1.0, 1.0, dim=dim, fmg=True,  # FMG is not an FGMRES option
                                 precision=_lib().IGAMG_FGMRES_FP64)
        assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -2


@pytest.mark.parametrize("p,sigma,nu", [(2, 1.0, 1.0), (3, 100.0, 0.3), (2, 1e-4, 1.0)])
def test_level_operators_match_oracle_galerkin(p, sigma, nu):
    from paper_1705_09282_gb300.solver import host_level_matrix
    n, L = 8, 3
    H = o2.Hierarchy(p, n, L, sigma, nu)
    for lev in range(L):
        Kg = host_level_matrix(p, n, L, sigma, nu, lev)
        Ko = H.levels[lev].K.toarray()
        scale = np.abs(Ko).max()
        assert Kg.shape == Ko.shape
        assert np.abs(Kg - Ko).max() <= 1e-12 * scale, (lev, np.abs(Kg - Ko).max() / scale)


@pytest.mark.parametrize("p,n,L", [(2, 8, 3), (3, 8, 3), (2, 32, 2), (3, 24, 2), (3, 2, 2)])
def test_kernel_row_stencils_reproduce_operator(p, n, L):
    # the class-stencil row evaluation the kernels run, executed on the host, against the
    # oracle's Galerkin operators (covers the wall classes and the interior class)
    from paper_1705_09282_gb300.solver import host_operator_rows
    H = o2.Hierarchy(p, n, L, 2.0, 0.5)
    for lev in range(L):
        Kr = host_operator_rows(p, n, L, 2.0, 0.5, lev)
        Ko = H.levels[lev].K.toarray()
        assert np.abs(Kr - Ko).max() <= 1e-12 * np.abs(Ko).max(), lev


@pytest.mark.parametrize("p", [2, 3])
def test_prolongations_match_oracle(p):
    from paper_1705_09282_gb300.solver import host_prolongation
    n, L = 16, 4
    for lev in range(1, L):
        Pg = host_prolongation(p, n, L, lev)
        Po = o2.prolongation(p, n >> (L - lev)).toarray()
        assert Pg.shape == Po.shape
        assert np.abs(Pg - Po).max() <= 1e-13


@pytest.mark.parametrize("p,n", [(2, 8), (3, 8), (2, 4), (3, 4)])
def test_patch_tables_match_oracle(p, n):
    from paper_1705_09282_gb300.solver import host_patches
    col, dofs = host_patches(p, n, 2, 1)
    S = o2.Stokes2D(p, n, 1, 1)
    lev = o2.Level(p, n, S.K, S.m, S)
    lev.build_patches()
    # same colour of every patch and same DOF lists; the order inside a colour is free
    # (same-colour patches share no DOF and are not coupled)
    want = sorted((P.colour, tuple(P.dofs)) for P in lev.patches)
    got = [(int(c), tuple(int(g) for g in d if g >= 0)) for c, d in zip(col, dofs)]
    assert [c for c, _ in got] == sorted(c for c, _ in got)
    assert sorted(got) == want


@pytest.mark.parametrize("p,n,L", [(2, 8, 3), (3, 8, 3), (2, 16, 3)])
def test_oseen_operators_match_oracle_galerkin(p, n, L):
    # generalized Oseen: fine operator with the advection term, coarse operators = R K P
    # (not re-assembly); the kernels' per-row records reproduce them on every level
    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300.solver import host_level_matrix, host_operator_rows
    beta = inputs.oseen_advection(p, n, 1.0)
    sigma, nu = 1.0, 0.01
    H = o2.Hierarchy(p, n, L, sigma, nu, beta=beta)
    for lev in range(L):
        Ko = H.levels[lev].K.toarray()
        scale = np.abs(Ko).max()
        Kg = host_level_matrix(p, n, L, sigma, nu, lev, beta=beta)
        assert np.abs(Kg - Ko).max() <= 1e-12 * scale, (lev, np.abs(Kg - Ko).max() / scale)
        Kr = host_operator_rows(p, n, L, sigma, nu, lev, beta=beta)
        assert np.abs(Kr - Ko).max() <= 1e-12 * scale, lev
    # and the operator is not symmetric (the advection term is present)
    K = H.levels[-1].K.toarray()
    assert np.abs(K - K.T).max() > 1e-6 * np.abs(K).max()


# ---- quarter annulus (Sec. 4.3 push-forwards, Sec. 6.2) ----------------------------------

@pytest.mark.parametrize("p,n,L,sigma,nu", [(2, 8, 3, 1.3, 0.7), (3, 8, 2, 1.0, 1.0), (2, 12, 2, 1e3, 1.0)])
def test_annulus_operators_match_oracle(p, n, L, sigma, nu):
    # the host assembly on the mapped domain (third record box for the u_x - u_y coupling)
    # and its Galerkin coarse levels, entry by entry and through the kernels' row evaluation
    from oracle import annulus2d as A
    from paper_1705_09282_gb300.solver import host_level_matrix, host_operator_rows
    fine = A.MappedStokes2D(p, n, sigma, nu, A.QuarterAnnulus())
    H = o2.Hierarchy(p, n, L, sigma, nu, fine=fine)
    for lev in range(L):
        Ko = H.levels[lev].K.toarray()
        scale = np.abs(Ko).max()
        assert np.abs(host_level_matrix(p, n, L, sigma, nu, lev, geometry=1) - Ko).max() <= 1e-13 * scale, lev
        assert np.abs(host_operator_rows(p, n, L, sigma, nu, lev, geometry=1) - Ko).max() <= 1e-13 * scale, lev


def test_annulus_arguments_rejected_on_host():
    import ctypes
    L = _lib().lib()
    h = ctypes.c_void_p()
    pr = _lib().make_problem(2, 8, 2, 1.0, 1.0, geometry=2)                       # no such domain
    assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -1
    pr = _lib().make_problem(2, 8, 2, 1.0, 1.0, geometry=1, r_inner=0.3, r_outer=0.2)
    assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -1
    beta = np.zeros((2, 32, 32))
    pr = _lib().make_problem(2, 8, 2, 1.0, 1.0, geometry=1, beta=beta)           # Stokes only
    assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -2
    pr = _lib().make_problem(2, 8, 2, 1.0, 1.0, geometry=1, dim=3)               # 2D only
    assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -2


def test_batch_entry_points_reject_bad_lists_on_host():
    # argument checks of the batch entry points run before any device work
    import ctypes
    L = _lib().lib()
    assert L.igamg_solve_batch(0, None, None, None, 1e-8, 10, None, None) == 0          # empty batch
    assert L.igamg_solve_batch(-1, None, None, None, 1e-8, 10, None, None) == -1
    hs = (ctypes.c_void_p * 2)(None, None)
    us = (ctypes.c_void_p * 2)(None, None)
    assert L.igamg_solve_batch(2, hs, us, us, 1e-8, 10, None, None) == -1              # null handles
    assert L.igamg_solve_batch(0, None, None, None, -1.0, 10, None, None) == -1        # rtol < 0
    at = (ctypes.c_double * 1)(1e-8)
    assert L.igamg_solve_batch_abs(0, None, None, None, at, 10, None, None) == 0


def test_form_entry_points_reject_bad_arguments_on_host():
    # the residual-form, chain-count and FP32-residual entry points check their arguments
    # before touching a handle or the device
    import ctypes
    L = _lib().lib()
    a, b = ctypes.c_int(), ctypes.c_int()
    assert L.igamg_residual_form(None, ctypes.byref(a), ctypes.byref(b)) == -1
    assert L.igamg_set_residual_form(None, 1, 0) == -1
    assert L.igamg_level_chains(None, 0, ctypes.byref(a)) == -1
    assert L.igamg_residual_f32(None, 0, None, None, None, None) == -1
