"""Pins for the mapped 3D oracle (Sec. 4.3 push-forwards on the hollow cylinder section of
Sec. 6.4): the identity map reproduces the unit-cube oracle, the map is the extruded quarter
annulus, the pushed-forward spaces keep the discrete complex, the discrete solution
converges to a closed-form solution, and V-cycles converge to the direct solve."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bspline as bs
from oracle import cylinder3d as C
from oracle import stokes3d as o3
from paper_1705_09282_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")
GEOM = C.HollowCylinder()


def _table(name):
    rows, cur = {}, None
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.isalpha() or line.startswith("table"):
            cur = line
            rows[cur] = []
            continue
        rows[cur].append([int(v) for v in line.split()])
    return rows[name]


def test_map_is_the_extruded_quarter_annulus():
    rng = np.random.default_rng(0)
    xi, eta, zeta = rng.uniform(0, 1, 50), rng.uniform(0, 1, 50), rng.uniform(0, 1, 50)
    X, DF, dDF = GEOM.eval(xi, eta, zeta)
    r = np.hypot(X[:, 0], X[:, 1])
    assert np.allclose(r, 0.075 + 0.15 * xi, atol=1e-15)
    assert np.allclose(X[:, 2], 0.1 * zeta, atol=1e-16)
    assert np.all(X[:, :2] >= -1e-16)
    h = 1e-6
    for k in range(3):
        d = np.zeros(3); d[k] = h
        Xp, DFp, _ = GEOM.eval(xi + d[0], eta + d[1], zeta + d[2])
        Xm, DFm, _ = GEOM.eval(xi - d[0], eta - d[1], zeta - d[2])
        assert np.allclose((Xp - Xm) / (2 * h), DF[:, :, k], atol=1e-8)
        assert np.allclose((DFp - DFm) / (2 * h), dDF[:, :, :, k], atol=1e-7)
    assert np.all(np.linalg.det(DF) > 0)


@pytest.mark.parametrize("p,n", [(2, 2), (2, 3), (3, 2)])
def test_identity_map_reproduces_the_unit_cube(p, n):
    S0 = o3.Stokes3D(p, n, 1.3, 0.7)
    S1 = C.MappedStokes3D(p, n, 1.3, 0.7, C.IdentityMap3())
    assert abs(S0.K - S1.K).max() <= 1e-14 * abs(S0.K).max()
    G = n * (p + 2)
    f = np.random.default_rng(1).standard_normal((3, G, G, G))
    assert np.abs(S0.load_vector(f) - S1.load_vector(f)).max() <= 1e-15


def test_pushed_forward_spaces_keep_the_complex():
    p, n = 2, 3
    S = C.MappedStokes3D(p, n, 1.0, 1.0, GEOM)
    psi = np.random.default_rng(2).standard_normal(S.n_psi())
    Uc = S.curl(psi)
    assert np.abs((S.K @ Uc)[S.n_u: S.n_u + S.n_p]).max() <= 1e-13 * np.abs(Uc).max()
    Au = S.K[: S.n_u, : S.n_u]
    assert abs(Au - Au.T).max() <= 1e-13 * abs(Au).max()
    Bup, Bpu = S.K[: S.n_u, S.n_u: S.n_u + S.n_p], S.K[S.n_u: S.n_u + S.n_p, : S.n_u]
    assert abs(Bup + Bpu.T).max() <= 1e-14 * abs(Bup).max()


def _l2_velocity_error(S, U):
    p, n = S.p, S.n
    g, w = bs.gauss_legendre(p + 3)
    xs = ((np.arange(n)[:, None] + g[None, :]) / n).ravel()
    ws = np.tile(w / n, n)
    ZZ, YY, XX = np.meshgrid(xs, xs, xs, indexing="ij")
    uh, X = S.velocity_at(U, XX.ravel(), YY.ravel(), ZZ.ravel())
    ue, _ = inputs.cylinder_solution(X[:, 0], X[:, 1], X[:, 2])
    _, DF, _ = GEOM.eval(XX.ravel(), YY.ravel(), ZZ.ravel())
    W = (ws[:, None, None] * ws[None, :, None] * ws[None, None, :]).ravel() * np.linalg.det(DF)
    return np.sqrt(np.sum(W * np.sum((uh - ue.T) ** 2, axis=1)) / np.sum(W * np.sum(ue.T ** 2, axis=1)))


def test_manufactured_convergence_on_the_cylinder():
    # p = 2: rate 1.80 from n = 4 to 8 (still below its asymptotic 2 at these sizes)
    errs = []
    for n in (4, 8):
        S = C.MappedStokes3D(2, n, 1.0, 1.0, GEOM)
        X = S.quad_points_xyz()
        F = S.load_vector(inputs.cylinder_forcing(X[0], X[1], X[2], 1.0, 1.0))
        U = spla.spsolve(S.K.tocsc(), F)
        errs.append(_l2_velocity_error(S, U))
        assert S.div_inf(U) <= 1e-10 * np.abs(U[: S.n_u]).max()
        assert abs(S.m @ U) <= 1e-12
    rate = np.log2(errs[0] / errs[1])
    assert 1.5 <= rate <= 2.6, (rate, errs)
    assert errs[1] < 0.3


def test_vcycles_on_the_cylinder_converge_to_direct_solve():
    p, n = 2, 4
    fine = C.MappedStokes3D(p, n, 1.0, 1.0, GEOM)
    H = o3.Hierarchy3D(p, n, 2, 1.0, 1.0, fine=fine)
    X = fine.quad_points_xyz()
    F = fine.load_vector(inputs.cylinder_forcing(X[0], X[1], X[2], 1.0, 1.0))
    Ux = spla.spsolve(fine.K.tocsc(), F)
    U = np.zeros_like(F)
    H.solve(U, F, 1e-13, 100)
    assert np.abs(U - Ux).max() <= 1e-10 * np.abs(Ux).max()


def test_paper_cylinder_cycle_counts_loosely():
    # the hollow-cylinder table's protocol (V(1,2), random divergence-free guess, 1e6
    # reduction, coarsest mesh one element): n_l = 1 as printed; n_l = 2 needs a few cycles
    # more than printed (as for the cube, whose counts the oracle also exceeds)
    tab = {r[0]: r for r in _table("tablecylinder")}
    for nl, bound in ((1, None), (2, 6)):
        n = 2 ** nl
        for sigma, col in ((1.0, 2), (1000.0, 3)):
            fine = C.MappedStokes3D(2, n, sigma, 1.0, GEOM)
            H = o3.Hierarchy3D(2, n, nl + 1, sigma, 1.0, nu1=1, nu2=2, fine=fine)
            psi, pr = inputs.random_divfree_guess_3d(2, n, seed=nl)
            U = fine.curl(psi)
            U[fine.n_u: fine.n_u + fine.n_p] = pr
            X = fine.quad_points_xyz()
            F = fine.load_vector(inputs.cylinder_forcing(X[0], X[1], X[2], sigma, 1.0))
            k, _ = H.solve(U, F, 1e-6, 40)
            if bound is None:
                assert k == tab[nl][col], (nl, sigma, k)
            else:
                assert k <= bound, (nl, sigma, k)
