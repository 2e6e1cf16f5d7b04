"""Univariate B-splines for the oracle: knots, Cox-de Boor evaluation, knot insertion.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package;
only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.

Everything here is written for clarity, in FP64, following the paper:
  * open knot vectors, first/last knot repeated p+1 times, domain (0,1)  -- Sec. 4.2
  * maximally smooth B-splines on uniform knot vectors                    -- Sec. 6 preamble
  * Cox-de Boor recursion for the basis                                   -- Sec. 4.2
  * knot insertion transformation matrix T (N_i = sum_j T_ij N~_j)        -- Sec. 4.4
    built here with Boehm's single-knot insertion (a textbook algorithm;
    the paper defers the construction to its references).
"""
import numpy as np


def uniform_open_knots(degree, n_elem):
    """Open uniform knot vector on [0,1] with n_elem elements (Sec. 4.2, Sec. 6)."""
    inner = [k / n_elem for k in range(1, n_elem)]
    return np.array([0.0] * (degree + 1) + inner + [1.0] * (degree + 1))


def n_basis(knots, degree):
    return len(knots) - degree - 1


def basis_values(knots, degree, x):
    """All B-spline values N_{i,degree}(x) for the points x.  Returns (len(x), n).

    Straight Cox-de Boor recursion (Sec. 4.2) with 0/0 := 0.  The degree-0
    functions use half-open spans [xi_i, xi_{i+1}); the right end x = 1 is
    attributed to the last non-degenerate span so that the basis stays a
    partition of unity on the closed interval.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = knots
    m = len(t) - 1  # number of degree-0 functions
    N = np.zeros((len(x), m))
    for i in range(m):
        N[:, i] = ((t[i] <= x) & (x < t[i + 1])).astype(np.float64)
    # close the right end: x = 1 belongs to the last non-degenerate span
    k_end = m - 1
    while t[k_end + 1] <= t[k_end]:
        k_end -= 1
    N[x == t[-1], :] = 0.0
    N[x == t[-1], k_end] = 1.0
    for q in range(1, degree + 1):
        Nn = np.zeros((len(x), m - q))
        for i in range(m - q):
            left = np.zeros(len(x))
            right = np.zeros(len(x))
            d1 = t[i + q] - t[i]
            d2 = t[i + q + 1] - t[i + 1]
            if d1 > 0:
                left = (x - t[i]) / d1 * N[:, i]
            if d2 > 0:
                right = (t[i + q + 1] - x) / d2 * N[:, i + 1]
            Nn[:, i] = left + right
        N = Nn
    return N


def basis_derivs(knots, degree, x):
    """First derivatives of all degree-`degree` B-splines at x (Sec. 4.3: the
    derivative of a degree-p B-spline is a combination of degree p-1 B-splines
    on the same knot vector)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    t = knots
    n = n_basis(t, degree)
    if degree == 0:
        return np.zeros((len(x), n))
    Nl = basis_values(t, degree - 1, x)  # functions on the same knots, n+1 of them
    d = np.zeros((len(x), n))
    for i in range(n):
        a = t[i + degree] - t[i]
        b = t[i + degree + 1] - t[i + 1]
        if a > 0:
            d[:, i] += degree / a * Nl[:, i]
        if b > 0:
            d[:, i] -= degree / b * Nl[:, i + 1]
    return d


def support_elements(knots, degree, i, n_elem):
    """Closed element-index interval [lo, hi] of the support of N_{i,degree} on a
    uniform open knot vector with n_elem elements."""
    # knots t_k = 0 for k<=degree, (k-degree)/n_elem inside, 1 after; element e spans
    # [e/n, (e+1)/n].  supp N_i = [t_i, t_{i+degree+1}].
    lo_x = knots[i]
    hi_x = knots[i + degree + 1]
    lo = int(round(lo_x * n_elem))
    hi = int(round(hi_x * n_elem)) - 1
    return lo, hi


def integrals(knots, degree):
    """int_0^1 N_{i,degree} = (xi_{i+p+1} - xi_i)/(p+1) (standard B-spline identity)."""
    n = n_basis(knots, degree)
    return np.array([(knots[i + degree + 1] - knots[i]) / (degree + 1) for i in range(n)])


def boehm_insert(knots, degree, xbar):
    """Insert one knot xbar.  Returns (new_knots, T1) with T1 of shape (n_new, n_old) so
    that new control points = T1 @ old control points (Boehm's algorithm)."""
    t = knots
    n = n_basis(t, degree)
    # span k with t_k <= xbar < t_{k+1}
    k = None
    for j in range(len(t) - 1):
        if t[j] <= xbar < t[j + 1]:
            k = j
    assert k is not None
    T1 = np.zeros((n + 1, n))
    for i in range(n + 1):
        if i <= k - degree:
            T1[i, i] = 1.0
        elif i >= k + 1:
            T1[i, i - 1] = 1.0
        else:
            a = (xbar - t[i]) / (t[i + degree] - t[i])
            T1[i, i] = a
            T1[i, i - 1] = 1.0 - a
    new_t = np.concatenate([t[: k + 1], [xbar], t[k + 1:]])
    return new_t, T1


def refinement_matrix(knots, degree, new_knots_inserted):
    """Prolongation of coefficients (fine x coarse) for inserting the given knots
    one at a time.  In the notation of Sec. 4.4 this is T transposed:
    u~_j = sum_i T_ij u_i."""
    t = np.array(knots, dtype=np.float64)
    P = np.eye(n_basis(t, degree))
    for xb in new_knots_inserted:
        t, T1 = boehm_insert(t, degree, xb)
        P = T1 @ P
    return t, P


def dyadic_prolongation(degree, n_coarse):
    """1D prolongation for midpoint refinement of a uniform open knot vector
    (n_coarse -> 2 n_coarse elements), shape (2 n_coarse + degree, n_coarse + degree)."""
    t = uniform_open_knots(degree, n_coarse)
    mids = [(k + 0.5) / n_coarse for k in range(n_coarse)]
    tf, P = refinement_matrix(t, degree, mids)
    assert np.allclose(tf, uniform_open_knots(degree, 2 * n_coarse))
    return P


def gauss_legendre(npts):
    """Gauss-Legendre nodes/weights on [0,1] (library routine)."""
    g, w = np.polynomial.legendre.leggauss(npts)
    return (g + 1.0) / 2.0, w / 2.0
