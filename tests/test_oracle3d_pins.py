"""Pins for the 3D (unit cube) oracle: the paper's Table 4 space dimensions, exactness of
the 3D discrete complex, the curl and divergence checked on function values, the
manufactured solution of Sec. 6.3 converging at the expected rate, knot-insertion
prolongation preserving functions, R K P = re-assembly, the paper's interior patch
dimensions, colour independence, direct-solve limits and the divergence-free invariant."""
import os
from collections import Counter

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bspline as bs
from oracle import stokes3d as o3
from paper_1705_09282_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


def _table(name):
    rows, cur = {}, None
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("table"):
            cur = line
            rows[cur] = []
            continue
        rows[cur].append([int(v) for v in line.split()])
    return rows[name]


def _eval(S, U, pts):
    """(u_x, u_y, u_z, p) of coefficient vector U at points pts (k, 3) = (x, y, z), from
    basis values only (no difference matrices)."""
    p, q, n = S.p, S.q, S.n
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    V = {d: [bs.basis_values(S.tp if d == p else S.tq, d, c) for c in (x, y, z)] for d in (p, q)}
    out = []
    for c in range(3):
        A = S._full_u(U, c)                               # [z, y, x]
        dg = [q, q, q]
        dg[c] = p
        out.append(np.einsum("ki,kj,kl,lji->k", V[dg[0]][0], V[dg[1]][1], V[dg[2]][2], A))
    P = U[S.n_u: S.n_u + S.n_p].reshape(S.nq, S.nq, S.nq)
    out.append(np.einsum("ki,kj,kl,lji->k", V[q][0], V[q][1], V[q][2], P))
    return out


@pytest.mark.parametrize("p", [2, 3])
def test_paper_table4_dof_column(p):
    # Table 4 "DOFs" = 3 (2^n_l + p - 1)(2^n_l + p)^2: the unconstrained vector-potential
    # space S^{q,p,p} x S^{p,q,p} x S^{p,p,q} on the oracle's knot vectors
    for row in _table("table4"):
        nl = row[0]
        n = 2 ** nl
        S = o3.Stokes3D(p, n, 1.0, 1.0, assemble=False)
        dim = 3 * bs.n_basis(S.tq, p - 1) * bs.n_basis(S.tp, p) ** 2
        assert dim == (row[1] if p == 2 else row[4])


@pytest.mark.parametrize("p,n", [(2, 3), (3, 2)])
def test_discrete_complex_exact(p, n):
    S = o3.Stokes3D(p, n, 1.0, 1.0)
    n_phi = S.ni ** 3                                  # scalar potentials vanishing on the boundary
    # Euler characteristic of Phi_0 -> Psi_0 -> V_0 -> Q_0/R
    assert n_phi - S.n_psi() + S.n_u - (S.n_p - 1) == 0
    C = np.stack([S.curl(e)[: S.n_u] for e in np.eye(S.n_psi())], axis=1)
    assert np.linalg.matrix_rank(C) == S.n_psi() - n_phi
    Bt = S.K[S.n_u: S.n_u + S.n_p, : S.n_u].toarray()
    assert np.linalg.matrix_rank(Bt) == S.n_p - 1
    assert np.abs(Bt @ C).max() <= 1e-12 * np.abs(C).max()
    # dim ker(div) = dim range(curl): curl is onto the divergence-free velocities
    assert S.n_u - (S.n_p - 1) == S.n_psi() - n_phi


def test_curl_is_the_curl():
    p, n = 2, 3
    S = o3.Stokes3D(p, n, 1.0, 1.0)
    rng = np.random.default_rng(2)
    psi = rng.uniform(-1, 1, S.n_psi())
    U = S.curl(psi)
    pts = rng.uniform(0, 1, (25, 3))
    ux, uy, uz, _ = _eval(S, U, pts)
    # psi as functions: family x in S^{q,p,p}, y in S^{p,q,p}, z in S^{p,p,q}
    q, ni, nq = p - 1, S.ni, S.nq
    blk = nq * ni * ni
    px = np.zeros((n + p, n + p, n + q)); px[1:-1, 1:-1, :] = psi[:blk].reshape(ni, ni, nq)
    py = np.zeros((n + p, n + q, n + p)); py[1:-1, :, 1:-1] = psi[blk:2 * blk].reshape(ni, nq, ni)
    pz = np.zeros((n + q, n + p, n + p)); pz[:, 1:-1, 1:-1] = psi[2 * blk:].reshape(nq, ni, ni)
    x, y, z = pts.T
    Vp = [bs.basis_values(S.tp, p, c) for c in (x, y, z)]
    Dp = [bs.basis_derivs(S.tp, p, c) for c in (x, y, z)]
    Vq = [bs.basis_values(S.tq, q, c) for c in (x, y, z)]
    ev = lambda A, a, b, c: np.einsum("ki,kj,kl,lji->k", a, b, c, A)
    dpz_dy = ev(pz, Vp[0], Dp[1], Vq[2]); dpy_dz = ev(py, Vp[0], Vq[1], Dp[2])
    dpx_dz = ev(px, Vq[0], Vp[1], Dp[2]); dpz_dx = ev(pz, Dp[0], Vp[1], Vq[2])
    dpy_dx = ev(py, Dp[0], Vq[1], Vp[2]); dpx_dy = ev(px, Vq[0], Dp[1], Vp[2])
    assert np.allclose(ux, dpz_dy - dpy_dz, atol=1e-11)
    assert np.allclose(uy, dpx_dz - dpz_dx, atol=1e-11)
    assert np.allclose(uz, dpy_dx - dpx_dy, atol=1e-11)


def test_divergence_pairing_is_b():
    # q^T (B^T u) = int (div u_h) q_h by a finer, higher-order quadrature on values
    p, n = 2, 3
    S = o3.Stokes3D(p, n, 1.0, 1.0)
    rng = np.random.default_rng(7)
    U = np.zeros(S.ndof)
    U[: S.n_u] = rng.standard_normal(S.n_u)
    qv = rng.standard_normal(S.n_p)
    lhs = qv @ (S.K[S.n_u: S.n_u + S.n_p, : S.n_u] @ U[: S.n_u])
    g, w = bs.gauss_legendre(p + 3)
    m = 2 * n
    x = np.concatenate([(e + g) / m for e in range(m)])
    wx = np.concatenate([w / m for _ in range(m)])
    Vq = bs.basis_values(S.tq, p - 1, x)
    divh = np.einsum("ai,bj,ck,kji->cba", Vq, Vq, Vq, S.div_coeffs(U))   # [z, y, x] grid
    qh = np.einsum("ai,bj,ck,kji->cba", Vq, Vq, Vq, qv.reshape(S.nq, S.nq, S.nq))
    W = np.einsum("a,b,c->abc", wx, wx, wx)
    rhs = np.sum(W * divh * qh)
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))


def test_manufactured_forcing_is_consistent():
    # the closed-form f of the cube's solution: sigma u - nu Lap u + grad p, checked
    # against central differences of the closed-form u and p
    sigma, nu, h = 2.0, 0.5, 1e-3
    f = inputs.manufactured_forcing_3d(2, 1, sigma, nu)
    x = inputs.quad_points_1d(2, 1)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    terms = inputs._poly_terms_3d()
    u = lambda X, Y, Z: [inputs._eval_terms(t, X, Y, Z) for t in terms]
    pr = lambda X, Y, Z: np.sin(np.pi * X) * np.sin(np.pi * Y)
    u0 = u(X, Y, Z)
    for c in range(3):
        lap = sum((u(*(v + h * e for v, e in zip((X, Y, Z), d)))[c] - 2 * u0[c]
                   + u(*(v - h * e for v, e in zip((X, Y, Z), d)))[c]) / h ** 2 for d in np.eye(3))
        dp = (pr(*(v + h * e for v, e in zip((X, Y, Z), np.eye(3)[c])))
              - pr(*(v - h * e for v, e in zip((X, Y, Z), np.eye(3)[c])))) / (2 * h)
        assert np.allclose(f[c], sigma * u0[c] - nu * lap + dp, atol=1e-4)
    # u is divergence-free and vanishes on the boundary (no-slip)
    div = sum((u(*(v + h * e for v, e in zip((X, Y, Z), np.eye(3)[c])))[c]
               - u(*(v - h * e for v, e in zip((X, Y, Z), np.eye(3)[c])))[c]) / (2 * h) for c in range(3))
    assert np.abs(div).max() < 1e-6          # O(h^2) central-difference error only
    b = np.array([0.0, 1.0])
    for c in range(3):
        for pts in (np.meshgrid(b, x, x, indexing="ij"), np.meshgrid(x, b, x, indexing="ij"),
                    np.meshgrid(x, x, b, indexing="ij")):
            assert np.abs(u(pts[2], pts[1], pts[0])[c]).max() < 1e-15


@pytest.mark.parametrize("p", [2, 3])
def test_manufactured_convergence_rate(p):
    # velocity L2 error ~ h^p; zero-mean pressure; pointwise divergence-free solution
    sigma, nu = 1.0, 1.0
    errs = []
    for n in (4, 8):
        S = o3.Stokes3D(p, n, sigma, nu)
        U = spla.spsolve(S.K.tocsc(), S.load_vector(inputs.manufactured_forcing_3d(p, n, sigma, nu)))
        x, w = o3.quad_points_1d(p, n)
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        uh = _eval(S, U, pts)
        ue = inputs.manufactured_solution_3d(p, n)
        W = np.einsum("a,b,c->abc", w, w, w).ravel()
        ev = np.sqrt(sum(np.sum(W * (uh[c] - ue[c].ravel()) ** 2) for c in range(3)))
        ep = np.sqrt(np.sum(W * (uh[3] - ue[3].ravel()) ** 2))
        errs.append((ev, ep, abs(np.sum(W * uh[3])), S.div_inf(U)))
    rate = np.log2(errs[0][0] / errs[1][0])
    assert p - 0.5 <= rate <= p + 1.0, (rate, errs)
    assert errs[1][1] < 0.1
    assert errs[1][2] < 1e-12
    assert errs[1][3] < 1e-10


@pytest.mark.parametrize("p", [2, 3])
def test_prolongation_preserves_functions(p):
    nc = 2
    P = o3.prolongation3d(p, nc)
    Sc, Sf = o3.Stokes3D(p, nc, 1, 1, assemble=False), o3.Stokes3D(p, 2 * nc, 1, 1, assemble=False)
    rng = np.random.default_rng(5)
    Uc = rng.standard_normal(Sc.ndof)
    Uf = P @ Uc
    pts = rng.uniform(0, 1, (30, 3))
    for a, b in zip(_eval(Sc, Uc, pts), _eval(Sf, Uf, pts)):
        assert np.allclose(a, b, atol=1e-13)
    assert Uf[-1] == Uc[-1]


@pytest.mark.parametrize("p", [2, 3])
def test_galerkin_equals_reassembly_with_fine_penalty(p):
    nf = 4
    Sf = o3.Stokes3D(p, nf, 3.0, 0.7)
    P = o3.prolongation3d(p, nf // 2)
    Kc = (P.T @ Sf.K @ P).toarray()
    Sc = o3.Stokes3D(p, nf // 2, 3.0, 0.7, h_pen=1.0 / nf)
    assert np.allclose(Kc, Sc.K.toarray(), atol=1e-11 * np.abs(Kc).max())


def test_patch_counts_interior_dims_and_colours():
    p, n = 2, 8
    H = o3.Hierarchy3D(p, n, 2, 1.0, 1.0)
    L = H.levels[-1]
    h = Counter((P.n_v, P.n_q) for P in L.patches)
    assert len(L.patches) == 3 * (n + p - 1) * (n + p - 2) ** 2
    # interior subdomain: dim V_i = 4, dim Q_i = 4 (3 after the mean), dim Psi_i = 1 (Sec. 5.2)
    assert h[(4, 4)] == 3 * (n - 1) * (n - 2) ** 2
    assert all(nv >= 4 and nq >= 4 for nv, nq in h)
    assert len({P.colour for P in L.patches}) == 3 * p * (p + 1) ** 2
    # patches of one colour share no DOF and do not couple through K
    K = L.K.tocsr()
    by_c = {}
    for P in L.patches:
        by_c.setdefault(P.colour, []).append(P)
    for ps in by_c.values():
        d = np.concatenate([P.dofs for P in ps])
        assert len(np.unique(d)) == len(d)
        for i in range(len(ps)):
            others = np.concatenate([ps[j].dofs for j in range(len(ps)) if j != i]) if len(ps) > 1 else []
            if len(others):
                assert abs(K[ps[i].dofs][:, others]).max() == 0.0


def test_local_velocity_space_is_one_curl():
    # dim Psi_i = 1 for an interior subdomain: the patch's divergence-free local velocities
    # are the multiples of the curl of its own vector-potential function
    p, n = 2, 6
    H = o3.Hierarchy3D(p, n, 2, 1.0, 1.0)
    S = H.fine
    L = H.levels[-1]
    P = next(P for P in L.patches if (P.n_v, P.n_q) == (4, 4) and P.fam == 1)
    Bt = S.K[S.n_u: S.n_u + S.n_p, :S.n_u].toarray()[:, P.dofs[:P.n_v]]
    kern = np.linalg.svd(Bt)[2][np.linalg.matrix_rank(Bt):]
    assert kern.shape[0] == 1
    # the family-y function with indices (i, j, k)
    e = np.zeros(S.n_psi())
    blk = S.nq * S.ni * S.ni
    e[blk + ((P.k - 1) * S.nq + P.j) * S.ni + (P.i - 1)] = 1.0
    c = S.curl(e)[: S.n_u]
    assert set(np.nonzero(np.abs(c) > 1e-14)[0]) == set(P.dofs[:P.n_v])
    v = c[P.dofs[:P.n_v]]
    assert abs(abs(kern[0] @ v) - np.linalg.norm(v)) < 1e-12 * np.linalg.norm(v)


@pytest.mark.parametrize("p,n", [(2, 4), (3, 4)])
def test_vcycles_converge_to_direct_solve(p, n):
    H = o3.Hierarchy3D(p, n, 2, 1.0, 1.0)
    F = H.fine.load_vector(inputs.manufactured_forcing_3d(p, n, 1.0, 1.0))
    Ux = spla.spsolve(H.levels[-1].K.tocsc(), F)
    U = np.zeros_like(F)
    H.solve(U, F, 1e-14, 80)
    assert np.abs(U - Ux).max() <= 1e-11 * np.abs(Ux).max()


def test_patch_covering_domain_is_exact():
    # p = 3, n = 2: every vector-potential support is the whole cube, so one patch
    # solve is a direct solve
    H = o3.Hierarchy3D(3, 2, 2, 1.0, 1.0)
    F = H.fine.load_vector(inputs.manufactured_forcing_3d(3, 2, 1.0, 1.0))
    U = np.zeros_like(F)
    L = H.levels[-1]
    P = L.patches[0]
    U[P.dofs] = 0.0
    L.sweep_multiplicative(U, F)
    assert np.allclose(U, spla.spsolve(L.K.tocsc(), F), atol=1e-12)


def test_divergence_free_invariant():
    p, n = 2, 8
    H = o3.Hierarchy3D(p, n, 3, 1.0, 1.0, nu1=1, nu2=2)
    S = H.fine
    psi, pr = inputs.random_divfree_guess_3d(p, n, seed=9)
    U = S.curl(psi)
    U[S.n_u: S.n_u + S.n_p] = pr
    F = S.load_vector(inputs.manufactured_forcing_3d(p, n, 1.0, 1.0))
    scale = np.abs(U[: S.n_u]).max()
    for _ in range(2):
        H.vcycle(U, F)
        assert S.div_inf(U) <= 1e-12 * max(1.0, scale)


def test_paper_table4_cycle_counts_loosely():
    # Table 4 protocol (V(1,2), multiplicative, random divergence-free guess, 1e6 reduction,
    # coarsest mesh one element).  Only n_l = 1 is a pin against the paper: on two elements
    # per direction some vector-potential support is the whole cube, so one cycle is exact
    # and the paper's 1 follows.  For n_l = 2, 3 the oracle needs 3-6 cycles where the table
    # prints 1-2 under every reading of Sec. 5.2 tried (oracle/paper_tables.py); those bounds
    # are the oracle's own counts, kept as a regression check, not a parity claim.
    tab = {r[0]: r for r in _table("table4")}
    for nl, bound in ((1, 1), (2, 4), (3, 6)):
        n = 2 ** nl
        for sigma in (1.0, 1000.0):
            H = o3.Hierarchy3D(2, n, nl + 1, sigma, 1.0, nu1=1, nu2=2)
            S = H.fine
            psi, pr = inputs.random_divfree_guess_3d(2, n, seed=nl)
            U = S.curl(psi)
            U[S.n_u: S.n_u + S.n_p] = pr
            F = S.load_vector(inputs.manufactured_forcing_3d(2, n, sigma, 1.0))
            k, _ = H.solve(U, F, 1e-6, 40)
            assert k <= bound, (nl, sigma, k)
            if nl == 1:
                assert k == tab[1][2]


def test_oseen_manufactured_convergence_3d():
    # generalized Oseen with beta = the (scaled) manufactured velocity: rate ~ h^2 for p = 2,
    # divergence-free discrete solution, and a non-symmetric operator
    p, sigma, nu = 2, 1.0, 0.1
    errs = []
    for n in (4, 8):
        beta = inputs.oseen_advection_3d(p, n, 1.0)
        S = o3.Stokes3D(p, n, sigma, nu, beta=beta)
        U = spla.spsolve(S.K.tocsc(), S.load_vector(inputs.oseen_forcing_3d(p, n, sigma, nu, beta)))
        x, w = o3.quad_points_1d(p, n)
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        uh = _eval(S, U, np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1))
        ue = inputs.manufactured_solution_3d(p, n)
        W = np.einsum("a,b,c->abc", w, w, w).ravel()
        errs.append(np.sqrt(sum(np.sum(W * (uh[c] - ue[c].ravel()) ** 2) for c in range(3))))
        assert S.div_inf(U) < 1e-10
    rate = np.log2(errs[0] / errs[1])
    assert 1.5 <= rate <= 3.0, (rate, errs)
    K = S.K.toarray()
    assert np.abs(K - K.T).max() > 1e-6 * np.abs(K).max()


@pytest.mark.parametrize("p,n", [(2, 3), (3, 2)])
def test_oseen_advection_blocks_exact_3d(p, n):
    # The 3D advection term (beta . grad u_c, v_c), per velocity component, against an
    # independent evaluation: scipy's B-splines on the same open uniform knots, 1D integrals by
    # 12-point Gauss-Legendre per element (exact here), beta = (c1 + a1 y, c2 + a2 z, c3 + a3 x),
    # for which each block is a sum of three-factor Kronecker products (z slowest, x fastest).
    from scipy.interpolate import BSpline
    c1, a1, c2, a2, c3, a3 = 0.7, -1.3, -0.4, 2.1, 0.25, 0.9
    x = inputs.quad_points_1d(p, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    beta = np.stack([c1 + a1 * Y, c2 + a2 * Z, c3 + a3 * X])
    K = (o3.Stokes3D(p, n, 1.0, 1.0, beta=beta).K - o3.Stokes3D(p, n, 1.0, 1.0).K).toarray()
    S = o3.Stokes3D(p, n, 1.0, 1.0, assemble=False)
    q = p - 1
    gx, gw = np.polynomial.legendre.leggauss(12)

    def integral(d, derivative_j, weight):
        # M[i, j] = int_0^1 weight(s) N^d_i(s) (N^d_j)^(derivative_j)(s) ds
        t = np.concatenate([np.zeros(d + 1), np.arange(1, n) / n, np.ones(d + 1)])
        m = n + d
        M = np.zeros((m, m))
        for e in range(n):
            s = (e + 0.5 * (gx + 1)) / n
            w = 0.5 * gw / n * weight(s)
            B = np.nan_to_num(np.array([BSpline(t, np.eye(m)[i], d, extrapolate=False)(s) for i in range(m)]))
            Bd = B if not derivative_j else np.nan_to_num(np.array(
                [BSpline(t, np.eye(m)[j], d, extrapolate=False).derivative(derivative_j)(s) for j in range(m)]))
            M += (B * w) @ Bd.T
        return M

    one = lambda s: np.ones_like(s)   # noqa: E731
    lin = lambda s: s                 # noqa: E731
    kron3 = lambda Mz, My, Mx: np.kron(Mz, np.kron(My, Mx))   # noqa: E731
    free = slice(1, n + p - 1)
    for c in range(3):
        deg = [q, q, q]
        deg[c] = p
        M = [integral(deg[a], 0, one) for a in range(3)]
        Ml = [integral(deg[a], 0, lin) for a in range(3)]
        D = [integral(deg[a], 1, one) for a in range(3)]
        cut = lambda A, a: A[free, free] if a == c else A   # noqa: E731
        Mc = [cut(M[a], a) for a in range(3)]
        W = [cut(c0 * M[a] + s0 * Ml[a], a) for a, (c0, s0) in enumerate(((c3, a3), (c1, a1), (c2, a2)))]
        Dc = [cut(D[a], a) for a in range(3)]
        # b1(y) d/dx + b2(z) d/dy + b3(x) d/dz; W[a] is the weight that depends on axis a
        A = kron3(Mc[2], W[1], Dc[0]) + kron3(W[2], Dc[1], Mc[0]) + kron3(Dc[2], Mc[1], W[0])
        blk = slice(c * S.n_uc, (c + 1) * S.n_uc)
        assert np.abs(K[blk, blk] - A).max() <= 1e-13 * np.abs(A).max(), c
        K[blk, blk] = 0.0
    assert np.abs(K).max() <= 1e-15 * np.abs(A).max()


@pytest.mark.parametrize("p,n", [(2, 3), (3, 2)])
def test_load_vector_exact_3d(p, n):
    # The 3D load vector for f = (a + b y z, c + d x, e + g x y) at the Gauss points against
    # products of 1D moments int s^k N_i(s) ds of scipy's B-splines (12-point Gauss-Legendre per
    # element, exact); component c's own axis runs over its interior indices; pressure and
    # multiplier rows are zero.
    from scipy.interpolate import BSpline
    a, b, c, d, e, g = 0.3, -1.7, 0.9, 2.4, -0.6, 1.1
    x = inputs.quad_points_1d(p, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = np.stack([a + b * Y * Z, c + d * X, e + g * X * Y])
    S = o3.Stokes3D(p, n, 1.0, 1.0)
    F = S.load_vector(f)
    q = p - 1
    gx, gw = np.polynomial.legendre.leggauss(12)

    def moments(deg, k):
        t = np.concatenate([np.zeros(deg + 1), np.arange(1, n) / n, np.ones(deg + 1)])
        m = np.zeros(n + deg)
        for el in range(n):
            s_ = (el + 0.5 * (gx + 1)) / n
            w = 0.5 * gw / n * s_ ** k
            for i in range(n + deg):
                m[i] += np.dot(w, np.nan_to_num(BSpline(t, np.eye(n + deg)[i], deg, extrapolate=False)(s_)))
        return m

    free = slice(1, n + p - 1)
    kron3 = lambda mz, my, mx: np.kron(mz, np.kron(my, mx))   # noqa: E731
    mp0, mq0, mq1 = moments(p, 0)[free], moments(q, 0), moments(q, 1)
    Fx = a * kron3(mq0, mq0, mp0) + b * kron3(mq1, mq1, mp0)          # u_x: x-degree p
    Fy = c * kron3(mq0, mp0, mq0) + d * kron3(mq0, mp0, mq1)          # u_y: y-degree p
    Fz = e * kron3(mp0, mq0, mq0) + g * kron3(mp0, mq1, mq1)          # u_z: z-degree p
    expect = np.concatenate([Fx, Fy, Fz])
    assert np.abs(F[: S.n_u] - expect).max() <= 1e-14 * np.abs(expect).max()
    assert np.abs(F[S.n_u:]).max() == 0.0


@pytest.mark.parametrize("p,n,sigma,nu", [(2, 3, 1.7, 0.3), (3, 2, 0.2, 2.5)])
def test_velocity_blocks_with_nitsche_terms_exact_3d(p, n, sigma, nu):
    # Each 3D velocity block of a_h (Sec. 3.3): sigma mass + nu stiffness + the Nitsche wall terms
    # on the four faces where the component is tangential (C_I = 4(p-1), h = 1/n), as sums of
    # three-factor Kronecker products of 1D matrices from scipy's B-splines (mass and stiffness by
    # 12-point Gauss-Legendre per element, wall terms by point values and derivatives at 0 and 1);
    # no coupling between velocity components on the cube.
    from scipy.interpolate import BSpline
    S = o3.Stokes3D(p, n, sigma, nu)
    K = S.K.toarray()
    q = p - 1
    gx, gw = np.polynomial.legendre.leggauss(12)
    c_pen, h = 4.0 * (p - 1), 1.0 / n

    def mats(deg):
        t = np.concatenate([np.zeros(deg + 1), np.arange(1, n) / n, np.ones(deg + 1)])
        B = [BSpline(t, np.eye(n + deg)[i], deg) for i in range(n + deg)]
        m = len(B)
        M, St, Wl = np.zeros((m, m)), np.zeros((m, m)), np.zeros((m, m))
        for e in range(n):
            s_ = (e + 0.5 * (gx + 1)) / n
            w = 0.5 * gw / n
            V = np.array([b(s_) for b in B])
            D = np.array([b.derivative()(s_) for b in B])
            M += (V * w) @ V.T
            St += (D * w) @ D.T
        for s0, sign in ((0.0, -1.0), (1.0, 1.0)):
            v = np.array([float(b(s0)) for b in B])
            dv = np.array([float(b.derivative()(s0)) for b in B])
            Wl += -sign * (np.outer(v, dv) + np.outer(dv, v)) + (c_pen / h) * np.outer(v, v)
        return M, St, Wl

    free = slice(1, n + p - 1)
    Mp, Sp, _ = mats(p)
    Mq, Sq, Wq = mats(q)
    kron3 = lambda Az, Ay, Ax: np.kron(Az, np.kron(Ay, Ax))   # noqa: E731
    for c in range(3):
        M = [Mq, Mq, Mq]; St = [Sq, Sq, Sq]; W = [Wq, Wq, Wq]
        M[c], St[c], W[c] = Mp[free, free], Sp[free, free], None
        A = sigma * kron3(M[2], M[1], M[0])
        A = A + nu * (kron3(M[2], M[1], St[0]) + kron3(M[2], St[1], M[0]) + kron3(St[2], M[1], M[0]))
        for a in range(3):                 # walls normal to axis a, where component c is tangential
            if a == c:
                continue
            F = list(M)
            F[a] = W[a]
            A = A + nu * kron3(F[2], F[1], F[0])
        blk = slice(c * S.n_uc, (c + 1) * S.n_uc)
        assert np.abs(K[blk, blk] - A).max() <= 1e-12 * np.abs(A).max(), c
        for c2 in range(3):
            if c2 != c:
                assert np.abs(K[blk, c2 * S.n_uc:(c2 + 1) * S.n_uc]).max() == 0.0


def test_oseen_forcing_matches_closed_form_derivatives():
    # beta . grad u from the polynomial terms against central differences
    p, n, h = 2, 1, 1e-4
    beta = inputs.oseen_advection_3d(p, n, 1.0)
    f0 = inputs.manufactured_forcing_3d(p, n, 1.0, 1.0)
    f1 = inputs.oseen_forcing_3d(p, n, 1.0, 1.0, beta)
    x = inputs.quad_points_1d(p, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = lambda X, Y, Z: [inputs._eval_terms(t, X, Y, Z) for t in inputs._poly_terms_3d()]
    for c in range(3):
        grad = [(u(*(v + h * e for v, e in zip((X, Y, Z), d)))[c] - u(*(v - h * e for v, e in zip((X, Y, Z), d)))[c])
                / (2 * h) for d in np.eye(3)]
        adv = beta[0] * grad[0] + beta[1] * grad[1] + beta[2] * grad[2]
        assert np.allclose(f1[c] - f0[c], adv, atol=1e-7)
    # beta is divergence-free, zero on the boundary, max |beta| = 1
    assert np.sqrt((beta ** 2).sum(axis=0)).max() <= 1.0 + 1e-12


# ---- W-cycle and full multigrid (Sec. 5 opening paragraph) ------------------------------

def test_w_cycle_on_two_grids_is_the_v_cycle_3d():
    p, n = 2, 4
    HV = o3.Hierarchy3D(p, n, 2, 1.0, 1.0, gamma=1)
    HW = o3.Hierarchy3D(p, n, 2, 1.0, 1.0, gamma=2)
    F = HV.fine.load_vector(inputs.manufactured_forcing_3d(p, n, 1.0, 1.0))
    UV, UW = np.zeros_like(F), np.zeros_like(F)
    HV.vcycle(UV, F)
    HW.vcycle(UW, F)
    assert np.abs(UV - UW).max() <= 1e-13 * np.abs(UV).max()


def test_fmg_is_exact_on_prolongated_solutions_3d():
    p, n = 2, 8
    H = o3.Hierarchy3D(p, n, 3, 1.0, 1.0)
    rng = np.random.default_rng(6)
    u = rng.uniform(-1, 1, H.levels[0].K.shape[0])
    for l in range(1, 3):
        u = H.P[l - 1] @ u
    F = H.levels[-1].K @ u
    U = H.fmg(F)
    assert np.abs(U - u).max() <= 1e-11 * np.abs(u).max()


def test_w_and_fmg_solves_converge_to_direct_solve_3d():
    p, n = 2, 8
    H = o3.Hierarchy3D(p, n, 3, 1.0, 1.0, gamma=2)
    F = H.fine.load_vector(inputs.manufactured_forcing_3d(p, n, 1.0, 1.0))
    Ux = spla.spsolve(H.levels[-1].K.tocsc(), F)
    U = np.zeros_like(F)
    H.solve(U, F, 1e-13, 60, fmg=True)
    assert np.abs(U - Ux).max() <= 1e-10 * np.abs(Ux).max()
