"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds none of the method's arithmetic: it only draws random numbers
and evaluates closed-form forcing / advection fields at given points.  Both the
library's tests and the oracle's tests take their inputs from here, so the two
sides see bit-identical right-hand sides.

Point layout used everywhere: each of the n elements per direction carries
G = p + 2 Gauss-Legendre points; a field sampled "at the quadrature points" is an
array (2, n*G, n*G) indexed [component, y point, x point], points element-major.
"""
import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014), counter-based, on numpy uint64."""

    def __init__(self, seed):
        self.state = np.uint64(seed) & _MASK

    def next_u64(self, count):
        with np.errstate(over="ignore"):
            k = np.arange(1, count + 1, dtype=np.uint64)
            z = self.state + k * np.uint64(0x9E3779B97F4A7C15)
            self.state = self.state + np.uint64(count) * np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, count):
        """Uniform doubles in [0,1) from the top 53 bits."""
        return (self.next_u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, count):
        """Standard normals by Box-Muller."""
        m = (count + 1) // 2
        u1 = 1.0 - self.uniform(m)          # (0,1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:count]


def quad_points_1d(p, n):
    """Abscissae of the (p+2)-point Gauss-Legendre rule in each of n uniform elements."""
    g, _ = np.polynomial.legendre.leggauss(p + 2)
    g = (g + 1.0) / 2.0
    return np.concatenate([(e + g) / n for e in range(n)])


def manufactured_forcing(p, n, sigma, nu):
    """f = sigma u - nu Lap u + grad p for psi = sin^2(pi x) sin^2(pi y),
    u = (d psi/dy, -d psi/dx), p = sin(pi x) sin(pi y) - 4/pi^2 (closed form)."""
    x = quad_points_1d(p, n)
    X, Y = np.meshgrid(x, x)
    pi = np.pi
    ux = pi * np.sin(pi * X) ** 2 * np.sin(2 * pi * Y)
    uy = -pi * np.sin(2 * pi * X) * np.sin(pi * Y) ** 2
    lap_ux = 2 * pi ** 3 * np.sin(2 * pi * Y) * (2 * np.cos(2 * pi * X) - 1)
    lap_uy = -2 * pi ** 3 * np.sin(2 * pi * X) * (2 * np.cos(2 * pi * Y) - 1)
    fx = sigma * ux - nu * lap_ux + pi * np.cos(pi * X) * np.sin(pi * Y)
    fy = sigma * uy - nu * lap_uy + pi * np.sin(pi * X) * np.cos(pi * Y)
    return np.ascontiguousarray(np.stack([fx, fy]))


def manufactured_solution(p, n):
    """(u_x, u_y, p) of the manufactured solution at the quadrature points."""
    x = quad_points_1d(p, n)
    X, Y = np.meshgrid(x, x)
    pi = np.pi
    ux = pi * np.sin(pi * X) ** 2 * np.sin(2 * pi * Y)
    uy = -pi * np.sin(2 * pi * X) * np.sin(pi * Y) ** 2
    pr = np.sin(pi * X) * np.sin(pi * Y) - 4.0 / pi ** 2
    return ux, uy, pr


def grf_grid(xs, ys, seed, length=0.1, n_features=512):
    """Two independent unit-variance Gaussian random fields with squared-exponential
    covariance exp(-r^2 / (2 length^2)), by random Fourier features
    f(x, y) = sqrt(2/M) sum_k cos(w_k . (x, y) + b_k), on the tensor grid ys x xs
    (result (2, len(ys), len(xs))).  The sum is evaluated as Re(E_y^T diag(e^{i b}) E_x)
    with E_x[k, j] = exp(i w_kx x_j); the same seed gives the same fields on any grid."""
    rng = SplitMix64(seed)
    xs, ys = np.asarray(xs, dtype=np.float64), np.asarray(ys, dtype=np.float64)
    out = []
    for _ in range(2):
        w = rng.normal(2 * n_features).reshape(n_features, 2) / length
        b = 2 * np.pi * rng.uniform(n_features)
        ex = np.exp(1j * np.outer(w[:, 0], xs))          # (M, nx)
        ey = np.exp(1j * np.outer(w[:, 1], ys))          # (M, ny)
        f = np.real((ey * np.exp(1j * b)[:, None]).T @ ex)
        out.append(f * np.sqrt(2.0 / n_features))
    return np.ascontiguousarray(np.stack(out))


def grf_forcing(p, n, seed, length=0.1, n_features=512):
    """The GRF forcing at the quadrature points, layout (2, n*G, n*G)."""
    x = quad_points_1d(p, n)
    return grf_grid(x, x, seed, length, n_features)


def streamfunction_grid(p, n):
    """Sample points of the warm-start network's input grid: the (n+p) Greville abscissae
    (knot averages) of the degree-p open uniform knot vector on n elements, per direction."""
    t = np.concatenate([np.zeros(p + 1), np.arange(1, n) / n, np.ones(p + 1)])
    return np.array([t[i + 1: i + p + 1].mean() for i in range(n + p)])


def warm_start_input(p, n, seed, sigma, nu):
    """Network input (3, n+p, n+p) float32: the GRF forcing (same seed as grf_forcing) at the
    streamfunction grid, and log10(sigma/nu) broadcast."""
    g = streamfunction_grid(p, n)
    f = grf_grid(g, g, seed)
    lg = np.full((1, len(g), len(g)), np.log10(sigma / nu))
    return np.ascontiguousarray(np.concatenate([f, lg]).astype(np.float32))


def warm_start_scale(sigma, nu):
    """Output scale of the warm-start network: the streamfunction of a unit forcing with
    wavenumber ~10 (the GRF length 0.1) is about 1 / (k (sigma + nu k^2)); the network
    predicts psi / scale."""
    return 1.0 / (10.0 * (sigma + 100.0 * nu))


def warm_start_pressure_scale():
    """Output scale of the network's pressure channel: the pressure balances the gradient
    part of a unit-variance forcing of length 0.1, so it is of size ~0.1 whatever sigma/nu."""
    return 0.1


def batch_problems(count, seed0, sizes=(64, 96, 128), log_ratio=(-2.0, 4.0)):
    """(n, sigma, nu, seed) for `count` independent problems: sizes round-robin, nu = 1,
    sigma/nu log-uniform in 10^log_ratio, forcing seeds seed0 + i."""
    rng = SplitMix64(seed0)
    u = rng.uniform(count)
    out = []
    for i in range(count):
        ratio = 10.0 ** (log_ratio[0] + (log_ratio[1] - log_ratio[0]) * u[i])
        out.append((sizes[i % len(sizes)], ratio, 1.0, seed0 + i))
    return out


def oseen_advection(p, n, max_speed=1.0):
    """beta = curl of sin^2(pi x) sin^2(pi y), scaled so that max |beta| = max_speed
    (divergence-free, zero on the boundary)."""
    x = quad_points_1d(p, n)
    X, Y = np.meshgrid(x, x)
    pi = np.pi
    bx = pi * np.sin(pi * X) ** 2 * np.sin(2 * pi * Y)
    by = -pi * np.sin(2 * pi * X) * np.sin(pi * Y) ** 2
    # max of |curl psi| over the square, from a fine sampling of the closed form
    s = np.linspace(0, 1, 2001)
    S, T = np.meshgrid(s, s)
    vmax = np.sqrt((pi * np.sin(pi * S) ** 2 * np.sin(2 * pi * T)) ** 2
                   + (pi * np.sin(2 * pi * S) * np.sin(pi * T) ** 2) ** 2).max()
    return np.ascontiguousarray(np.stack([bx, by]) * (max_speed / vmax))


def random_divfree_guess(p, n, seed):
    """Random streamfunction coefficients on the (n+p-2)^2 interior, U(-1,1), and random
    pressure coefficients on the (n+p-1)^2 pressure space, U(-1,1)."""
    rng = SplitMix64(seed)
    psi = 2.0 * rng.uniform((n + p - 2) ** 2) - 1.0
    pr = 2.0 * rng.uniform((n + p - 1) ** 2) - 1.0
    return psi, pr


def random_vector(count, seed):
    """Standard normal vector (for parity tests of single operators)."""
    return SplitMix64(seed).normal(count)


# ---- 3D (unit cube) ------------------------------------------------------------------

def _poly_terms_3d():
    """The cube's manufactured velocity u = curl psi for psi = (a(x) b(y) b(z), 0,
    b(x) b(y) a(z)), a(t) = t(t-1), b(t) = t^2 (t-1)^2, as sums of separable products
    c * fx(x) fy(y) fz(z) per component (numpy polynomials)."""
    P = np.polynomial.Polynomial
    a = P([0.0, -1.0, 1.0])
    b = P([0.0, 0.0, 1.0, -2.0, 1.0])
    db = b.deriv()
    ux = [(1.0, b, db, a)]
    uy = [(1.0, a, b, db), (-1.0, db, b, a)]
    uz = [(-1.0, a, db, b)]
    return [ux, uy, uz]


def _eval_terms(terms, X, Y, Z, lap=False):
    out = np.zeros_like(X)
    for c, fx, fy, fz in terms:
        if lap:
            out += c * (fx.deriv(2)(X) * fy(Y) * fz(Z) + fx(X) * fy.deriv(2)(Y) * fz(Z)
                        + fx(X) * fy(Y) * fz.deriv(2)(Z))
        else:
            out += c * fx(X) * fy(Y) * fz(Z)
    return out


def manufactured_solution_3d(p, n):
    """(u_x, u_y, u_z, p) of the cube's manufactured solution at the quadrature points,
    arrays [z, y, x]; p = sin(pi x) sin(pi y) - 4/pi^2 (zero mean)."""
    x = quad_points_1d(p, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    us = [_eval_terms(t, X, Y, Z) for t in _poly_terms_3d()]
    pr = np.sin(np.pi * X) * np.sin(np.pi * Y) - 4.0 / np.pi ** 2
    return us[0], us[1], us[2], pr


def manufactured_forcing_3d(p, n, sigma, nu):
    """f = sigma u - nu Lap u + grad p for the cube's manufactured solution, at the
    quadrature points, layout (3, nG, nG, nG) [component, z, y, x]."""
    x = quad_points_1d(p, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    pi = np.pi
    grad = [pi * np.cos(pi * X) * np.sin(pi * Y), pi * np.sin(pi * X) * np.cos(pi * Y), np.zeros_like(X)]
    f = [sigma * _eval_terms(t, X, Y, Z) - nu * _eval_terms(t, X, Y, Z, lap=True) + g
         for t, g in zip(_poly_terms_3d(), grad)]
    return np.ascontiguousarray(np.stack(f))


def random_divfree_guess_3d(p, n, seed):
    """Random vector-potential coefficients, U(-1,1), on the constrained space
    (three families of (n+p-1)(n+p-2)^2 each) and random pressure coefficients on the
    (n+p-1)^3 pressure space, U(-1,1)."""
    rng = SplitMix64(seed)
    psi = 2.0 * rng.uniform(3 * (n + p - 1) * (n + p - 2) ** 2) - 1.0
    pr = 2.0 * rng.uniform((n + p - 1) ** 3) - 1.0
    return psi, pr


def oseen_advection_3d(p, n, max_speed=1.0):
    """beta = the cube's manufactured velocity (divergence-free, zero on the boundary),
    scaled so that max |beta| = max_speed; layout (3, nG, nG, nG) [component, z, y, x]."""
    x = quad_points_1d(p, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    terms = _poly_terms_3d()
    b = np.stack([_eval_terms(t, X, Y, Z) for t in terms])
    s = np.linspace(0, 1, 81)
    S3 = np.meshgrid(s, s, s, indexing="ij")
    vmax = np.sqrt(sum(_eval_terms(t, S3[2], S3[1], S3[0]) ** 2 for t in terms)).max()
    return np.ascontiguousarray(b * (max_speed / vmax))


def oseen_forcing_3d(p, n, sigma, nu, beta):
    """f = sigma u - nu Lap u + beta . grad u + grad p for the cube's manufactured solution,
    beta given at the quadrature points (3, nG, nG, nG)."""
    x = quad_points_1d(p, n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = manufactured_forcing_3d(p, n, sigma, nu)
    for c, terms in enumerate(_poly_terms_3d()):
        for coef, fx, fy, fz in terms:
            f[c] += coef * (beta[0] * fx.deriv()(X) * fy(Y) * fz(Z) + beta[1] * fx(X) * fy.deriv()(Y) * fz(Z)
                            + beta[2] * fx(X) * fy(Y) * fz.deriv()(Z))
    return np.ascontiguousarray(f)


# ---- quarter annulus (Sec. 6.2's domain: r_i = 0.075, r_o = 0.225) ------------------------
# Manufactured solution given directly in physical coordinates: u = curl psi with the
# polynomial psi = c (x y g1 g2)^2, g1 = x^2 + y^2 - r_i^2, g2 = r_o^2 - x^2 - y^2, which
# vanishes with its gradient on all four walls (so u = 0 there and div u = 0), and the
# zero-mean pressure p = x y - (r_i^2 + r_o^2) / (2 pi).  Fields are evaluated at given
# physical points (x, y arrays of any shape).

ANNULUS_RI, ANNULUS_RO = 0.075, 0.225


def _pmul(a, b):
    out = np.zeros((a.shape[0] + b.shape[0] - 1, a.shape[1] + b.shape[1] - 1))
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            if a[i, j] != 0.0:
                out[i: i + b.shape[0], j: j + b.shape[1]] += a[i, j] * b
    return out


def _annulus_psi_coeffs(r_i, r_o):
    """Coefficients c[i, j] of x^i y^j of psi, scaled so that max |u| is about 1."""
    xy = np.zeros((2, 2)); xy[1, 1] = 1.0
    g1 = np.zeros((3, 3)); g1[2, 0] = g1[0, 2] = 1.0; g1[0, 0] = -r_i * r_i
    g2 = np.zeros((3, 3)); g2[2, 0] = g2[0, 2] = -1.0; g2[0, 0] = r_o * r_o
    b = _pmul(_pmul(xy, g1), g2)
    c = _pmul(b, b)
    return c / (r_o ** 12) * 8.0


def _pder(c, axis, k=1):
    from numpy.polynomial import polynomial as P
    return P.polyder(c, m=k, axis=axis)


def _pval(c, x, y):
    from numpy.polynomial import polynomial as P
    return P.polyval2d(x, y, c)


def annulus_solution(x, y, r_i=ANNULUS_RI, r_o=ANNULUS_RO):
    """(u (2, ...), p (...)) of the manufactured quarter-annulus solution at (x, y)."""
    c = _annulus_psi_coeffs(r_i, r_o)
    u = np.stack([_pval(_pder(c, 1), x, y), -_pval(_pder(c, 0), x, y)])
    p = x * y - (r_i * r_i + r_o * r_o) / (2.0 * np.pi)
    return u, p


def annulus_forcing(x, y, sigma, nu, r_i=ANNULUS_RI, r_o=ANNULUS_RO):
    """f = sigma u - nu lap u + grad p (generalized Stokes, Sec. 3.1) at (x, y): (2, ...)."""
    c = _annulus_psi_coeffs(r_i, r_o)
    ux, uy = _pder(c, 1), -_pder(c, 0)
    fx = sigma * _pval(ux, x, y) - nu * (_pval(_pder(ux, 0, 2), x, y) + _pval(_pder(ux, 1, 2), x, y)) + y
    fy = sigma * _pval(uy, x, y) - nu * (_pval(_pder(uy, 0, 2), x, y) + _pval(_pder(uy, 1, 2), x, y)) + x
    return np.stack([fx, fy])


# ---- hollow cylinder section (the quarter annulus extruded by a depth of 0.1) ---------------
# u = g(z) (d psi/dy, -d psi/dx, 0) with the quarter-annulus psi above and g(z) =
# 16 (z (d - z))^2 / d^4, which vanishes on all six walls and is divergence-free;
# p = x y - (r_i^2 + r_o^2) / (2 pi) (zero mean over the section).

CYLINDER_DEPTH = 0.1


def _cyl_g(z, d):
    h = (z * (d - z)) ** 2
    h2 = 2 * (d - z) ** 2 - 8 * z * (d - z) + 2 * z ** 2
    return 16.0 * h / d ** 4, 16.0 * h2 / d ** 4


def cylinder_solution(x, y, z, r_i=ANNULUS_RI, r_o=ANNULUS_RO, depth=CYLINDER_DEPTH):
    """(u (3, ...), p (...)) of the manufactured hollow-cylinder solution at (x, y, z)."""
    c = _annulus_psi_coeffs(r_i, r_o)
    g, _ = _cyl_g(z, depth)
    u = np.stack([g * _pval(_pder(c, 1), x, y), -g * _pval(_pder(c, 0), x, y), 0.0 * x])
    p = x * y - (r_i * r_i + r_o * r_o) / (2.0 * np.pi)
    return u, p


def cylinder_forcing(x, y, z, sigma, nu, r_i=ANNULUS_RI, r_o=ANNULUS_RO, depth=CYLINDER_DEPTH):
    """f = sigma u - nu lap u + grad p (generalized Stokes, Sec. 3.1) at (x, y, z): (3, ...)."""
    c = _annulus_psi_coeffs(r_i, r_o)
    g, g2 = _cyl_g(z, depth)
    comps = []
    for a, sgn in ((_pder(c, 1), 1.0), (_pder(c, 0), -1.0)):
        val = _pval(a, x, y)
        lap = _pval(_pder(a, 0, 2), x, y) + _pval(_pder(a, 1, 2), x, y)
        comps.append(sgn * (sigma * g * val - nu * (g * lap + g2 * val)))
    return np.stack([comps[0] + y, comps[1] + x, 0.0 * x])
