"""Pins for the CPU oracle: each test checks it against something other than itself
(closed forms, textbook identities, exactness of the discrete complex, brute-force
direct solves, the paper's printed DOF counts and cycle counts)."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bspline as bs
from oracle import stokes2d as o2
from paper_1705_09282_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


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


# ---------------------------------------------------------------- B-splines --

@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_partition_of_unity_and_derivative(deg):
    t = bs.uniform_open_knots(deg, 7)
    x = np.linspace(0.0, 1.0, 301)
    N = bs.basis_values(t, deg, x)
    assert np.allclose(N.sum(axis=1), 1.0, atol=1e-14)
    assert N.min() >= -1e-15
    if deg >= 1:
        h = 1e-6
        xi = np.linspace(0.013, 0.987, 97)
        fd = (bs.basis_values(t, deg, xi + h) - bs.basis_values(t, deg, xi - h)) / (2 * h)
        assert np.allclose(bs.basis_derivs(t, deg, xi), fd, atol=1e-6 * 7 ** 2)


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_marsden_linear_reproduction(deg):
    # sum_i (Greville abscissa)_i N_i(x) = x  (textbook identity)
    t = bs.uniform_open_knots(deg, 6)
    n = bs.n_basis(t, deg)
    grev = np.array([t[i + 1: i + deg + 1].mean() for i in range(n)])
    x = np.linspace(0, 1, 101)
    assert np.allclose(bs.basis_values(t, deg, x) @ grev, x, atol=1e-14)


def test_cardinal_quadratic_mass_and_stiffness_rows():
    # interior row of the quadratic B-spline mass matrix = h * [1, 26, 66, 26, 1] / 120
    # and stiffness = (1/h) * [-1/6, -1/3, 1, -1/3, -1/6]  (cardinal B-spline closed forms)
    n = 10
    t = bs.uniform_open_knots(2, n)
    x, w = o2.quad_points_1d(2, n)
    V = bs.basis_values(t, 2, x)
    D = bs.basis_derivs(t, 2, x)
    M = V.T @ (w[:, None] * V)
    S = D.T @ (w[:, None] * D)
    i = 5
    assert np.allclose(M[i, i - 2: i + 3], np.array([1, 26, 66, 26, 1]) / 120 / n, atol=1e-15)
    assert np.allclose(S[i, i - 2: i + 3], np.array([-1 / 6, -1 / 3, 1, -1 / 3, -1 / 6]) * n, atol=1e-12)


def test_knot_insertion_figure_example():
    # Sec. 4.4 figure: Xi = (0,0,0,.2,.4,.6,.8,1,1,1) refined at the midpoints gives
    # (0,0,0,.1,...,.9,1,1,1); the function is the same before and after.
    t = np.array([0, 0, 0, .2, .4, .6, .8, 1, 1, 1.0])
    tf, P = bs.refinement_matrix(t, 2, [.1, .3, .5, .7, .9])
    assert np.allclose(tf, [0, 0, 0, .1, .2, .3, .4, .5, .6, .7, .8, .9, 1, 1, 1])
    c = np.random.default_rng(1).standard_normal(7)
    x = np.random.default_rng(2).uniform(0, 1, 200)
    assert np.allclose(bs.basis_values(t, 2, x) @ c, bs.basis_values(tf, 2, x) @ (P @ c), atol=1e-14)


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_dyadic_prolongation_interior_is_binomial(deg):
    # uniform midpoint refinement: interior columns are 2^-deg * C(deg+1, k)  (Lane-Riesenfeld)
    from math import comb
    P = bs.dyadic_prolongation(deg, 8)
    col = P[:, 4]
    nz = col[np.abs(col) > 0]
    assert np.allclose(nz, [comb(deg + 1, k) / 2 ** deg for k in range(deg + 2)])


# ------------------------------------------------------- discretization --

@pytest.mark.parametrize("p", [2, 3])
def test_paper_dof_column(p):
    # Table 1 "DOFs" = (2^n_l + p)^2 = the unconstrained streamfunction space dimension
    tab = _table("table1")
    for row in tab:
        nl = row[0]
        dofs = row[1] if p == 2 else row[4]
        assert (2 ** nl + p) ** 2 == dofs


@pytest.mark.parametrize("p,n", [(2, 4), (2, 7), (3, 5)])
def test_discrete_complex_exact(p, n):
    S = o2.Stokes2D(p, n, 1.0, 1.0)
    # dim V - dim Psi = dim Q - 1 (exactness of Psi -> V -> Q with the mean constraint)
    assert S.n_u - S.n_psi_interior() == S.n_p - 1
    psi = np.random.default_rng(0).uniform(-1, 1, S.n_psi_interior())
    U = S.curl(psi)
    assert S.div_inf(U) <= 1e-12 * n
    # the curl really is d psi/dy, -d psi/dx: evaluate both at random points
    xs = np.random.default_rng(3).uniform(0, 1, 40)
    ys = np.random.default_rng(4).uniform(0, 1, 40)
    Pf = np.zeros((n + p, n + p))
    Pf[1:-1, 1:-1] = psi.reshape(n + p - 2, n + p - 2)
    Vx, Dx = bs.basis_values(S.tp, p, xs), bs.basis_derivs(S.tp, p, xs)
    Vy, Dy = bs.basis_values(S.tp, p, ys), bs.basis_derivs(S.tp, p, ys)
    dpsi_dy = np.einsum('ki,kj,ji->k', Vx, Dy, Pf)
    cx = np.zeros((n + p - 1, n + p))
    cx[:, 1:-1] = U[: S.n_ux].reshape(n + p - 1, n + p - 2)
    Wy = bs.basis_values(S.tq, p - 1, ys)
    ux = np.einsum('ki,kj,ji->k', Vx, Wy, cx)
    assert np.allclose(ux, dpsi_dy, atol=1e-11)


@pytest.mark.parametrize("p", [2, 3])
def test_divergence_pairing_is_b(p):
    # q^T (B^T u) = int (div u_h) q_h, with the integral done by a 2x finer, higher
    # order quadrature on function values (independent of the assembly tables)
    n = 5
    S = o2.Stokes2D(p, n, 1.0, 1.0)
    rng = np.random.default_rng(7)
    U = np.zeros(S.ndof)
    U[: S.n_u] = rng.standard_normal(S.n_u)
    qv = rng.standard_normal(S.n_p)
    lhs = qv @ (S.K[S.n_u: S.n_u + S.n_p, : S.n_u] @ U[: S.n_u])
    g, w = bs.gauss_legendre(p + 4)
    m = 2 * n
    x = np.concatenate([(e + g) / m for e in range(m)])
    wx = np.concatenate([w / m for _ in range(m)])
    Dv = bs.basis_values(S.tq, p - 1, x)
    divc = S.div_coeffs(U)                                   # (iy, ix)
    divh = Dv @ divc @ Dv.T
    qh = Dv @ qv.reshape(n + p - 1, n + p - 1) @ Dv.T
    rhs = np.sum(np.outer(wx, wx) * divh * qh)
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))


@pytest.mark.parametrize("p,sigma,nu", [(2, 1.0, 1.0), (3, 1.0, 1.0), (2, 1000.0, 1.0), (2, 1.0, 0.01)])
def test_manufactured_convergence_rate(p, sigma, nu):
    # velocity L2 error ~ h^p for the divergence-conforming pair; pressure has zero mean
    errs = []
    for n in (8, 16):
        S = o2.Stokes2D(p, n, sigma, nu)
        F = S.load_vector(inputs.manufactured_forcing(p, n, sigma, nu))
        U = spla.spsolve(S.K.tocsc(), F)
        ux_e, uy_e, p_e = inputs.manufactured_solution(p, n)
        x, w = o2.quad_points_1d(p, n)
        Vp, Vq = bs.basis_values(S.tp, p, x), bs.basis_values(S.tq, p - 1, x)
        cx = np.zeros((n + p - 1, n + p)); cx[:, 1:-1] = U[: S.n_ux].reshape(n + p - 1, n + p - 2)
        cy = np.zeros((n + p, n + p - 1)); cy[1:-1, :] = U[S.n_ux: S.n_u].reshape(n + p - 2, n + p - 1)
        uxh, uyh = Vq @ cx @ Vp.T, Vp @ cy @ Vq.T
        ph = Vq @ U[S.n_u: S.n_u + S.n_p].reshape(n + p - 1, n + p - 1) @ Vq.T
        W = np.outer(w, w)
        errs.append((np.sqrt(np.sum(W * ((uxh - ux_e) ** 2 + (uyh - uy_e) ** 2))),
                     np.sqrt(np.sum(W * (ph - p_e) ** 2)), abs(np.sum(W * ph)), S.div_inf(U)))
    rate = np.log2(errs[0][0] / errs[1][0])
    assert p - 0.35 <= rate <= p + 0.6, (rate, errs)
    assert errs[1][1] < 0.05                      # pressure converges to the exact one
    assert errs[1][2] < 1e-12                     # zero-mean pressure (Lagrange multiplier)
    assert errs[1][3] < 1e-10                     # pointwise divergence-free (Lemma, Sec. 4.1)


def test_oseen_manufactured_convergence():
    # generalized Oseen with beta = manufactured-type divergence-free field
    p, sigma, nu = 2, 1.0, 0.1
    errs = []
    for n in (8, 16):
        beta = inputs.oseen_advection(p, n, 1.0)
        S = o2.Stokes2D(p, n, sigma, nu, beta=beta)
        ux_e, uy_e, _ = inputs.manufactured_solution(p, n)
        x = inputs.quad_points_1d(p, n)
        X, Y = np.meshgrid(x, x)
        pi = np.pi
        # beta . grad u for the manufactured u (closed form derivatives)
        dux_dx = pi * 2 * pi * np.sin(pi * X) * np.cos(pi * X) * np.sin(2 * pi * Y)
        dux_dy = pi * np.sin(pi * X) ** 2 * 2 * pi * np.cos(2 * pi * Y)
        duy_dx = -pi * 2 * pi * np.cos(2 * pi * X) * np.sin(pi * Y) ** 2
        duy_dy = -pi * np.sin(2 * pi * X) * 2 * pi * np.sin(pi * Y) * np.cos(pi * Y)
        f = inputs.manufactured_forcing(p, n, sigma, nu)
        f[0] += beta[0] * dux_dx + beta[1] * dux_dy
        f[1] += beta[0] * duy_dx + beta[1] * duy_dy
        U = spla.spsolve(S.K.tocsc(), S.load_vector(f))
        _, w = o2.quad_points_1d(p, n)
        Vp, Vq = bs.basis_values(S.tp, p, x), bs.basis_values(S.tq, p - 1, x)
        cx = np.zeros((n + p - 1, n + p)); cx[:, 1:-1] = U[: S.n_ux].reshape(n + p - 1, n + p - 2)
        cy = np.zeros((n + p, n + p - 1)); cy[1:-1, :] = U[S.n_ux: S.n_u].reshape(n + p - 2, n + p - 1)
        W = np.outer(w, w)
        errs.append(np.sqrt(np.sum(W * ((Vq @ cx @ Vp.T - ux_e) ** 2 + (Vp @ cy @ Vq.T - uy_e) ** 2))))
    rate = np.log2(errs[0] / errs[1])
    assert 1.65 <= rate <= 2.6, (rate, errs)


@pytest.mark.parametrize("p,n", [(2, 5), (3, 4)])
def test_oseen_advection_block_exact(p, n):
    # The advection term of Sec. 3.1, (beta . grad u, v) over the velocity blocks, against an
    # independent evaluation: scipy's B-splines on the same open uniform knots, 1D integrals by
    # 12-point Gauss-Legendre per element (exact here), and beta = (c1 + a1 y, c2 + a2 x), for
    # which each block is a sum of Kronecker products of 1D integrals.  A non-constant,
    # direction-dependent field catches a transposed quadrature layout or swapped components;
    # it need not be divergence-free for the bilinear form's definition.
    from scipy.interpolate import BSpline
    c1, a1, c2, a2 = 0.7, -1.3, -0.4, 2.1
    x = inputs.quad_points_1d(p, n)
    X, Y = np.meshgrid(x, x)
    beta = np.stack([c1 + a1 * Y, c2 + a2 * X])
    K = (o2.Stokes2D(p, n, 1.0, 1.0, beta=beta).K - o2.Stokes2D(p, n, 1.0, 1.0).K).toarray()
    q = p - 1
    gx, gw = np.polynomial.legendre.leggauss(12)

    def knots(d):
        return np.concatenate([np.zeros(d + 1), np.arange(1, n) / n, np.ones(d + 1)])

    def integral(di, dj, derivative_j, weight):
        # M[i, j] = int_0^1 weight(s) N^di_i(s) (N^dj_j)^(derivative_j)(s) ds
        ti, tj = knots(di), knots(dj)
        ni, nj = n + di, n + dj
        M = np.zeros((ni, nj))
        for e in range(n):
            s = (e + 0.5 * (gx + 1)) / n
            w = 0.5 * gw / n * weight(s)
            Bi = np.array([BSpline(ti, np.eye(ni)[i], di, extrapolate=False)(s) for i in range(ni)])
            Bj = np.array([BSpline(tj, np.eye(nj)[j], dj, extrapolate=False).derivative(derivative_j)(s)
                           if derivative_j else BSpline(tj, np.eye(nj)[j], dj, extrapolate=False)(s)
                           for j in range(nj)])
            M += (np.nan_to_num(Bi) * w) @ np.nan_to_num(Bj).T
        return M

    one = lambda s: np.ones_like(s)   # noqa: E731
    lin = lambda s: s                 # noqa: E731
    S = o2.Stokes2D(p, n, 1.0, 1.0)
    # u_x block (x-degree p, y-degree q; x indices 1..n+p-2 free): rows (iy, ix), columns (jy, jx)
    #   b1 d/dx: (c1 + a1 y) -> [int N_ix N'_jx dx] (x) [int (c1 + a1 y) N_iy N_jy dy]
    #   b2 d/dy: (c2 + a2 x) -> [int (c2 + a2 x) N_ix N_jx dx] (x) [int N_iy N'_jy dy]
    Dx_p, Mx_p, Mx_p_lin = integral(p, p, 1, one), integral(p, p, 0, one), integral(p, p, 0, lin)
    My_q, My_q_lin, Dy_q = integral(q, q, 0, one), integral(q, q, 0, lin), integral(q, q, 1, one)
    fx = slice(1, n + p - 1)
    Axx = (np.kron(c1 * My_q + a1 * My_q_lin, Dx_p[fx, fx]) + np.kron(Dy_q, c2 * Mx_p[fx, fx] + a2 * Mx_p_lin[fx, fx]))
    ux = slice(0, S.n_ux)
    assert np.abs(K[ux, ux] - Axx).max() <= 1e-13 * np.abs(Axx).max()
    # u_y block (x-degree q, y-degree p; y indices 1..n+p-2 free)
    Dx_q, Mx_q, Mx_q_lin = integral(q, q, 1, one), integral(q, q, 0, one), integral(q, q, 0, lin)
    My_p, My_p_lin, Dy_p = integral(p, p, 0, one), integral(p, p, 0, lin), integral(p, p, 1, one)
    Ayy = (np.kron((c1 * My_p + a1 * My_p_lin)[fx, fx], Dx_q) + np.kron(Dy_p[fx, fx], c2 * Mx_q + a2 * Mx_q_lin))
    uy = slice(S.n_ux, S.n_u)
    assert np.abs(K[uy, uy] - Ayy).max() <= 1e-13 * np.abs(Ayy).max()
    # nothing else: no coupling between the components, the pressure or the multiplier (up to
    # the rounding of the two assemblies' Stokes parts, which the difference cancels)
    K[ux, ux] = 0.0
    K[uy, uy] = 0.0
    assert np.abs(K).max() <= 1e-15 * np.abs(Axx).max()


@pytest.mark.parametrize("p,n", [(2, 5), (3, 4)])
def test_load_vector_exact(p, n):
    # The load vector (f, v) of Sec. 3.1 for f = (a + b x y, c + d x^2) sampled at the Gauss
    # points, against an independent evaluation: each velocity row is a sum of products of 1D
    # moments int s^k N_i(s) ds of scipy's B-splines on the same knots (12-point Gauss-Legendre
    # per element, exact); the pressure and multiplier rows are zero.
    from scipy.interpolate import BSpline
    a, b, c, d = 0.3, -1.7, 0.9, 2.4
    x = inputs.quad_points_1d(p, n)
    X, Y = np.meshgrid(x, x)
    f = np.stack([a + b * X * Y, c + d * X * X])
    S = o2.Stokes2D(p, n, 1.0, 1.0)
    F = S.load_vector(f)
    q = p - 1
    gx, gw = np.polynomial.legendre.leggauss(12)

    def moments(deg, k):
        # m[i] = int_0^1 s^k N^deg_i(s) ds
        t = np.concatenate([np.zeros(deg + 1), np.arange(1, n) / n, np.ones(deg + 1)])
        m = np.zeros(n + deg)
        for e in range(n):
            s_ = (e + 0.5 * (gx + 1)) / n
            w = 0.5 * gw / n * s_ ** k
            for i in range(n + deg):
                m[i] += np.dot(w, np.nan_to_num(BSpline(t, np.eye(n + deg)[i], deg, extrapolate=False)(s_)))
        return m

    free = slice(1, n + p - 1)
    # u_x rows (x-degree p free, y-degree q), y-major: F = a m0p(x) m0q(y) + b m1p(x) m1q(y)
    Fx = a * np.outer(moments(q, 0), moments(p, 0)[free]) + b * np.outer(moments(q, 1), moments(p, 1)[free])
    # u_y rows (x-degree q, y-degree p free): F = c m0q(x) m0p(y) + d m2q(x) m0p(y)
    Fy = np.outer(moments(p, 0)[free], c * moments(q, 0) + d * moments(q, 2))
    expect = np.concatenate([Fx.ravel(), Fy.ravel()])
    assert np.abs(F[: S.n_u] - expect).max() <= 1e-14 * np.abs(expect).max()
    assert np.abs(F[S.n_u:]).max() == 0.0
    # the pressure-mean multiplier (Sec. 4.3 footnote): its row and column hold m_j = int N^q_j,
    # the products of the 1D moments, and nothing else
    K = S.K.toarray()
    m = np.kron(moments(q, 0), moments(q, 0))
    pr = slice(S.n_u, S.n_u + S.n_p)
    assert np.abs(K[-1, pr] - m).max() <= 1e-14 * m.max()
    assert np.abs(K[pr, -1] - m).max() <= 1e-14 * m.max()
    assert np.abs(K[-1, : S.n_u]).max() == 0.0 and K[-1, -1] == 0.0


@pytest.mark.parametrize("p,n,sigma,nu", [(2, 5, 1.7, 0.3), (3, 4, 0.2, 2.5)])
def test_velocity_blocks_with_nitsche_terms_exact(p, n, sigma, nu):
    # The velocity blocks of a_h (Sec. 3.3): sigma (v, u) + nu (grad v : grad u) minus the two
    # normal-derivative wall integrals plus (C_I nu / h) (v, u) on the walls where the
    # component is tangential (the normal one is zero strongly), C_I = 4(p-1), h = 1/n.  Each
    # block is a sum of Kronecker products of 1D matrices: mass and stiffness by 12-point
    # Gauss-Legendre per element, wall terms by point values and derivatives at 0 and 1, all
    # from scipy's B-splines (independent of the oracle's element assembly).  There is no
    # u_x-u_y coupling on the square.
    from scipy.interpolate import BSpline
    S = o2.Stokes2D(p, n, sigma, nu)
    K = S.K.toarray()
    q = p - 1
    gx, gw = np.polynomial.legendre.leggauss(12)
    c_pen, h = 4.0 * (p - 1), 1.0 / n

    def basis(deg):
        t = np.concatenate([np.zeros(deg + 1), np.arange(1, n) / n, np.ones(deg + 1)])
        return [BSpline(t, np.eye(n + deg)[i], deg) for i in range(n + deg)]

    def mats(deg):
        B = basis(deg)
        m = len(B)
        M, St = np.zeros((m, m)), np.zeros((m, m))
        for e in range(n):
            s_ = (e + 0.5 * (gx + 1)) / n
            w = 0.5 * gw / n
            V = np.array([b(s_) for b in B])
            D = np.array([b.derivative()(s_) for b in B])
            M += (V * w) @ V.T
            St += (D * w) @ D.T
        # wall terms at s = 0 (outward normal -1) and s = 1 (+1)
        Wl = np.zeros((m, m))
        for s0, sign in ((0.0, -1.0), (1.0, 1.0)):
            v = np.array([float(b(s0)) for b in B])
            dv = np.array([float(b.derivative()(s0)) for b in B])
            Wl += -sign * (np.outer(v, dv) + np.outer(dv, v)) + (c_pen / h) * np.outer(v, v)
        return M, St, Wl

    Mp, Sp, _ = mats(p)
    Mq, Sq, Wq = mats(q)
    free = slice(1, n + p - 1)
    Mpf, Spf = Mp[free, free], Sp[free, free]
    # u_x rows (iy, ix): x-degree p (free), y-degree q; tangential on the walls y = 0, 1
    Axx = sigma * np.kron(Mq, Mpf) + nu * (np.kron(Mq, Spf) + np.kron(Sq, Mpf) + np.kron(Wq, Mpf))
    # u_y rows (iy, ix): x-degree q, y-degree p (free); tangential on the walls x = 0, 1
    Ayy = sigma * np.kron(Mpf, Mq) + nu * (np.kron(Mpf, Sq) + np.kron(Spf, Mq) + np.kron(Mpf, Wq))
    ux, uy = slice(0, S.n_ux), slice(S.n_ux, S.n_u)
    for blk, A in ((K[ux, ux], Axx), (K[uy, uy], Ayy)):
        assert np.abs(blk - A).max() <= 1e-12 * np.abs(A).max()
    assert np.abs(K[ux, uy]).max() == 0.0 and np.abs(K[uy, ux]).max() == 0.0


# ---------------------------------------------------------------- multigrid --

@pytest.mark.parametrize("p", [2, 3])
def test_prolongation_preserves_functions(p):
    nc = 3
    P = o2.prolongation(p, nc)
    Sc, Sf = o2.Stokes2D(p, nc, 1, 1), o2.Stokes2D(p, 2 * nc, 1, 1)
    rng = np.random.default_rng(5)
    Uc = rng.standard_normal(Sc.ndof)
    Uf = P @ Uc
    x = rng.uniform(0, 1, 30)
    y = rng.uniform(0, 1, 30)

    def fields(S, U):
        n = S.n
        Vpx, Vqx = bs.basis_values(S.tp, p, x), bs.basis_values(S.tq, p - 1, x)
        Vpy, Vqy = bs.basis_values(S.tp, p, y), bs.basis_values(S.tq, p - 1, y)
        cx = np.zeros((n + p - 1, n + p)); cx[:, 1:-1] = U[: S.n_ux].reshape(n + p - 1, n + p - 2)
        cy = np.zeros((n + p, n + p - 1)); cy[1:-1, :] = U[S.n_ux: S.n_u].reshape(n + p - 2, n + p - 1)
        pp = U[S.n_u: S.n_u + S.n_p].reshape(n + p - 1, n + p - 1)
        return (np.einsum('ki,kj,ji->k', Vpx, Vqy, cx), np.einsum('ki,kj,ji->k', Vqx, Vpy, cy),
                np.einsum('ki,kj,ji->k', Vqx, Vqy, pp))

    for a, b in zip(fields(Sc, Uc), fields(Sf, Uf)):
        assert np.allclose(a, b, atol=1e-13)
    assert Uf[-1] == Uc[-1]


@pytest.mark.parametrize("p", [2, 3])
def test_galerkin_equals_reassembly_with_fine_penalty(p):
    # for constant-coefficient Stokes on the identity map, R K P is the same bilinear
    # form on the coarse space, i.e. re-assembly with the fine-mesh Nitsche penalty
    nf = 8
    Sf = o2.Stokes2D(p, nf, 3.0, 0.7)
    P = o2.prolongation(p, nf // 2)
    Kc = (P.T @ Sf.K @ P).toarray()
    Sc = o2.Stokes2D(p, nf // 2, 3.0, 0.7, h_pen=1.0 / nf)
    assert np.allclose(Kc, Sc.K.toarray(), atol=1e-11 * np.abs(Kc).max())


@pytest.mark.parametrize("p,n", [(2, 8), (3, 8)])
def test_patch_histograms_and_interior_dims(p, n):
    from collections import Counter
    S = o2.Stokes2D(p, n, 1, 1)
    L = o2.Level(p, n, S.K, S.m, S)
    L.build_patches()
    h = Counter((P.n_v, P.n_q) for P in L.patches)
    assert len(L.patches) == (n + p - 2) ** 2
    # interior subdomain: dim V_i = 4, dim Q_i = 4 - 1 (zero mean), dim Psi_i = 1 (Sec. 5.2)
    if p == 2:
        assert h == Counter({(4, 4): (n - 2) ** 2, (7, 6): 4 * (n - 2), (12, 9): 4})
    else:
        assert h == Counter({(4, 4): (n - 3) ** 2, (7, 6): 4 * (n - 3), (10, 8): 4 * (n - 3),
                             (12, 9): 4, (17, 12): 8, (24, 16): 4})


def test_same_colour_patches_do_not_couple():
    p, n = 2, 9
    S = o2.Stokes2D(p, n, 1, 1)
    L = o2.Level(p, n, S.K, S.m, S)
    L.build_patches()
    K = S.K.tocsr()
    by_c = {}
    for P in L.patches:
        by_c.setdefault(P.colour, []).append(P)
    assert len(by_c) == (p + 1) ** 2
    for c, ps in by_c.items():
        for i in range(len(ps)):
            for j in range(i + 1, len(ps)):
                assert not set(ps[i].dofs) & set(ps[j].dofs)
                assert abs(K[ps[i].dofs][:, ps[j].dofs]).max() == 0.0


def test_one_patch_sweep_is_exact_solve():
    # p=2 on one element: the single interior streamfunction support is the whole domain
    S = o2.Stokes2D(2, 1, 1.0, 1.0)
    L = o2.Level(2, 1, S.K, S.m, S)
    L.build_patches()
    assert len(L.patches) == 1
    F = S.load_vector(inputs.grf_forcing(2, 1, seed=3))
    U = np.zeros(S.ndof)
    L.sweep_multiplicative(U, F)
    Ux = spla.spsolve(S.K.tocsc(), F)
    assert np.allclose(U, Ux, atol=1e-13)


@pytest.mark.parametrize("p,sm,eta", [(2, "mult", 0.5), (3, "mult", 0.5), (2, "add", 0.3)])
def test_vcycles_converge_to_direct_solve(p, sm, eta):
    n = 8
    H = o2.Hierarchy(p, n, 3, 1.0, 1.0, smoother=sm, eta=eta, nu1=2, nu2=2)
    F = H.fine.load_vector(inputs.grf_forcing(p, n, seed=11))
    Ux = spla.spsolve(H.levels[-1].K.tocsc(), F)
    U = np.zeros_like(F)
    k, hist = H.solve(U, F, 1e-14, 80)
    assert np.abs(U - Ux).max() <= 1e-12 * np.abs(Ux).max()


def test_single_grid_vcycle_is_direct_solve():
    H = o2.Hierarchy(2, 4, 1, 1.0, 1.0)
    F = H.fine.load_vector(inputs.grf_forcing(2, 4, seed=5))
    U = np.ones_like(F)
    H.vcycle(U, F)
    assert np.allclose(U, spla.spsolve(H.fine.K.tocsc(), F), atol=1e-13)


@pytest.mark.parametrize("sm,eta", [("mult", 0.5), ("add", 0.5), ("add", 0.3)])
def test_divergence_free_invariant(sm, eta):
    # Sec. 5.3: from a divergence-free guess every iterate is pointwise divergence-free,
    # for any number of sweeps, levels and cycles (also while additive diverges in p)
    p, n = 2, 16
    H = o2.Hierarchy(p, n, 4, 1.0, 1.0, smoother=sm, eta=eta, nu1=1, nu2=2)
    S = H.fine
    psi, pr = inputs.random_divfree_guess(p, n, seed=9)
    U = S.curl(psi)
    U[S.n_u: S.n_u + S.n_p] = pr
    F = S.load_vector(inputs.grf_forcing(p, n, seed=10))
    for _ in range(3):
        H.vcycle(U, F)
        assert S.div_inf(U) <= 1e-12 * max(1.0, np.abs(U[: S.n_u]).max())
        H.smooth(n_l := H.n_levels - 1, U, F)
        assert S.div_inf(U) <= 1e-12 * max(1.0, np.abs(U[: S.n_u]).max())


@pytest.mark.parametrize("n,n_whole", [(1, 1), (2, 4)])
def test_additive_sweep_scales_by_eta(n, n_whole):
    # eq. ASM: U += eta * sum_i E_i^T K_i^{-1} E_i r.  For p = 2 on one element the single
    # interior streamfunction support is the whole domain, and on two elements all four are,
    # so one additive sweep from zero is n_whole * eta * the direct solve (velocity and
    # pressure; the multiplier is not a subdomain unknown and stays 0).  A dropped, squared or
    # misplaced eta, or a sum that skips a subdomain, fails this.
    S = o2.Stokes2D(2, n, 1.0, 1.0)
    L = o2.Level(2, n, S.K, S.m, S)
    L.build_patches()
    assert len(L.patches) == n_whole
    F = S.load_vector(inputs.grf_forcing(2, n, seed=31))
    Ux = spla.spsolve(S.K.tocsc(), F)
    assert abs(Ux[-1]) <= 1e-12 * np.abs(Ux).max()     # lambda = 0 for a velocity-only load
    for eta in (0.5, 0.3):
        U = np.zeros(S.ndof)
        L.sweep_additive(U, F, eta)
        assert np.allclose(U, n_whole * eta * Ux, rtol=0, atol=1e-12 * np.abs(Ux).max())


@pytest.mark.parametrize("p,n_l", [(2, 1), (3, 1), (3, 2)])
def test_table1_smallest_meshes_take_one_cycle(p, n_l):
    # The n_l = 1 row of Table 1 (and n_l = 2 for p = 3) is not compared with the paper's
    # counts (3 / 2 and 6 / 6 at n_l = 1; 12 / 14 at n_l = 2, p = 3): on 2^n_l elements with
    # p + 1 >= 2^n_l some interior streamfunction support (p + 1 elements wide, clipped to
    # the domain) is the whole domain, so under Sec. 5.2's subdomains that patch's solve in
    # the first pre-smoothing sweep is exact up to the pressure mean (later patches then see
    # a zero residual), and the exact coarse solve of Algorithm 1 restores the mean: one
    # V(1,2) cycle, whatever the guess.  The oracle must show exactly that.
    n = 2 ** n_l
    S = o2.Stokes2D(p, n, 1.0, 1.0)
    L = o2.Level(p, n, S.K, S.m, S)
    L.build_patches()
    assert any(len(P.dofs) == S.ndof - 1 for P in L.patches)
    for sigma in (1.0, 1000.0):
        H = o2.Hierarchy(p, n, n_l + 1, sigma, 1.0, smoother="mult", nu1=1, nu2=2)
        psi, pr = inputs.random_divfree_guess(p, n, seed=n_l)
        U = H.fine.curl(psi)
        U[H.fine.n_u: H.fine.n_u + H.fine.n_p] = pr
        F = H.fine.load_vector(inputs.manufactured_forcing(p, n, sigma, 1.0))
        k, hist = H.solve(U, F, 1e-6, 10)
        assert k == 1 and hist[-1] <= 1e-12 * hist[0], (k, hist)


def test_paper_table1_cycle_counts_loosely():
    # protocol of Sec. 6: V(1,2), multiplicative, random divergence-free guess, 1e6 reduction,
    # coarsest mesh one element.  The paper leaves ordering, guess and norm open, so only
    # +-2 cycles are asked (p = 2).  Row n_l = 1 is pinned separately: there the method is
    # exact in one cycle (test_table1_smallest_meshes_take_one_cycle).
    tab = _table("table1")
    for row in tab[1:4]:
        nl, da1, da1000 = row[0], row[2], row[3]
        n = 2 ** nl
        for sigma, want in ((1.0, da1), (1000.0, da1000)):
            H = o2.Hierarchy(2, n, nl + 1, sigma, 1.0, smoother="mult", nu1=1, nu2=2)
            S = H.fine
            psi, pr = inputs.random_divfree_guess(2, n, seed=nl)
            U = S.curl(psi)
            U[S.n_u: S.n_u + S.n_p] = pr
            F = S.load_vector(inputs.manufactured_forcing(2, n, sigma, 1.0))
            k, _ = H.solve(U, F, 1e-6, 40)
            assert abs(k - want) <= 2, (nl, sigma, k, want)


def test_mesh_independent_contraction():
    rates = []
    for n, L in ((16, 3), (32, 4)):
        H = o2.Hierarchy(2, n, L, 1.0, 1.0, nu1=2, nu2=2)
        F = H.fine.load_vector(inputs.grf_forcing(2, n, seed=21))
        U = np.zeros_like(F)
        k, hist = H.solve(U, F, 1e-8, 40)
        rates.append((hist[-1] / hist[0]) ** (1.0 / k))
    # V(2,2) contraction stays well below one and grows only slowly with the mesh
    # (the paper's Tables 1-7 report mesh-independent cycle counts)
    assert max(rates) < 0.35
    assert abs(rates[0] - rates[1]) < 0.1


# ----------------------------------------------- W-cycle and full multigrid --
# Sec. 5's opening paragraph: the method also applies inside a W-cycle or a full
# multigrid (nested iteration) framework.

@pytest.mark.parametrize("p", [2, 3])
def test_w_cycle_on_two_grids_is_the_v_cycle(p):
    # with two grids the coarse correction is an exact solve; repeating it from its own
    # result changes nothing (a second correction added on top would double it)
    n = 8
    F = o2.Hierarchy(p, n, 2, 1.0, 1.0).fine.load_vector(inputs.grf_forcing(p, n, seed=21))
    HV = o2.Hierarchy(p, n, 2, 1.0, 1.0, gamma=1)
    HW = o2.Hierarchy(p, n, 2, 1.0, 1.0, gamma=2)
    UV, UW = np.zeros_like(F), np.zeros_like(F)
    HV.vcycle(UV, F)
    HW.vcycle(UW, F)
    assert np.abs(UV - UW).max() <= 1e-13 * np.abs(UV).max()


def test_many_coarse_cycles_tend_to_the_exact_two_grid_cycle():
    # gamma coarse cycles per level, each continuing from the last, converge to the exact
    # coarse correction: three grids with large gamma = two grids (same coarse operator
    # K_1 = P^T K_2 P) to round-off
    p, n = 2, 8
    H3 = o2.Hierarchy(p, n, 3, 1.0, 1.0, gamma=30)
    H2 = o2.Hierarchy(p, n, 2, 1.0, 1.0)
    assert np.abs((H3.levels[1].K - H2.levels[0].K).toarray()).max() <= 1e-12
    F = H2.fine.load_vector(inputs.grf_forcing(p, n, seed=22))
    U3, U2 = np.zeros_like(F), np.zeros_like(F)
    H3.vcycle(U3, F)
    H2.vcycle(U2, F)
    assert np.abs(U3 - U2).max() <= 1e-11 * np.abs(U2).max()
    # and gamma = 2 is a different, better-converging cycle than gamma = 1 there
    HV = o2.Hierarchy(p, n, 3, 1.0, 1.0, gamma=1)
    UV = np.zeros_like(F)
    HV.vcycle(UV, F)
    Ux = spla.spsolve(H2.fine.K.tocsc(), F)
    HW = o2.Hierarchy(p, n, 3, 1.0, 1.0, gamma=2)
    UW = np.zeros_like(F)
    HW.vcycle(UW, F)
    assert np.linalg.norm(UW - Ux) < np.linalg.norm(UV - Ux)


@pytest.mark.parametrize("p", [2, 3])
def test_fmg_is_exact_on_prolongated_solutions(p):
    # if U* = P_2 P_1 P_0 u_0 then every restricted right-hand side is K_l of the matching
    # prolongation (Galerkin operators), the coarsest solve recovers u_0 and every cycle
    # starts from an exact solution, so FMG returns U* to round-off
    n = 16
    H = o2.Hierarchy(p, n, 4, 1.0, 1.0)
    rng = np.random.default_rng(5)
    u = rng.uniform(-1, 1, H.levels[0].K.shape[0])
    for l in range(1, 4):
        u = H.P[l - 1] @ u
    F = H.levels[-1].K @ u
    U = H.fmg(F)
    assert np.abs(U - u).max() <= 1e-11 * np.abs(u).max()


def test_fmg_on_one_grid_is_the_direct_solve():
    H = o2.Hierarchy(2, 4, 1, 1.0, 1.0)
    F = H.fine.load_vector(inputs.grf_forcing(2, 4, seed=23))
    assert np.allclose(H.fmg(F), spla.spsolve(H.fine.K.tocsc(), F), atol=1e-13)


@pytest.mark.parametrize("p,gamma,fmg", [(2, 2, False), (3, 2, False), (2, 1, True), (3, 2, True)])
def test_w_and_fmg_solves_converge_to_direct_solve(p, gamma, fmg):
    n = 8
    H = o2.Hierarchy(p, n, 3, 1.0, 1.0, gamma=gamma)
    F = H.fine.load_vector(inputs.grf_forcing(p, n, seed=24))
    Ux = spla.spsolve(H.levels[-1].K.tocsc(), F)
    U = np.zeros_like(F)
    k, hist = H.solve(U, F, 1e-14, 80, fmg=fmg)
    assert np.abs(U - Ux).max() <= 1e-12 * np.abs(Ux).max()
    assert all(b < a for a, b in zip(hist[:3], hist[1:4]))


def test_fmg_first_step_beats_one_v_cycle_from_zero():
    # nested iteration starts the finest cycle from the interpolated coarse solution: on a
    # smooth forcing its first residual is far below that of one V-cycle from zero
    p, n = 2, 32
    H = o2.Hierarchy(p, n, 4, 1.0, 1.0)
    F = H.fine.load_vector(inputs.manufactured_forcing(p, n, 1.0, 1.0))
    UV = np.zeros_like(F)
    H.vcycle(UV, F)
    UF = H.fmg(F)
    rv = np.linalg.norm(F - H.fine.K @ UV)
    rf = np.linalg.norm(F - H.fine.K @ UF)
    assert rf < 0.5 * rv, (rf, rv)
