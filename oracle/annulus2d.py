"""Generalized Stokes on a mapped 2D domain: isogeometric compatible B-splines defined
through push-forwards of the parametric spaces (Sec. 4.3), on the quarter annulus of
Sec. 6.2 (inner radius 0.075, outer radius 0.225, quadratic rational Bezier map).

TEST INFRASTRUCTURE ONLY (the oracle).  Only tests/, __graft_entry__.smoke() and
bench.py's CPU legs may import it; the product path never does.

What it follows:
  * physical spaces by push-forward (Sec. 4.3): psi = psi_hat o F^-1,
    v = (1/det J) J v_hat o F^-1 (contravariant Piola), q = (1/det J) q_hat o F^-1;
    so div v = (1/det J) div_hat v_hat and the discrete complex is kept
  * weak form of Sec. 3.1 / 3.3 on the physical domain, integrated over the parametric
    square with (p+2)-point Gauss rules (the same points as on the unit square)
  * Nitsche terms on all four walls for the tangential velocity, the normal component
    removed strongly (v_hat . n_hat = 0 is v . n = 0 under the Piola map)

Readings where the paper is silent:
  * parametric directions: xi (first) is radial, eta (second) is angular; the arc is the
    rational quadratic Bezier curve with control points (1,0), (1,1), (0,1) and weights
    (1, sqrt(2)/2, 1), scaled by r(xi) = r_i + (r_o - r_i) xi;
  * Nitsche length h at a wall point = the element's height normal to the wall,
    det J / (|tangent| n); on the unit square it is 1/n as in Sec. 6;
  * load vector l(v) = int f . v dx = int (J^T f) . v_hat dxi, with f sampled at the
    images of the parametric quadrature points.
"""
import numpy as np
import scipy.sparse as sp

from . import bspline as bs
from .stokes2d import Stokes2D, n_quad


class QuarterAnnulus:
    """F(xi, eta) = r(xi) C(eta): C the rational quadratic quarter circle."""

    def __init__(self, r_i=0.075, r_o=0.225):
        self.r_i, self.r_o = float(r_i), float(r_o)

    def _arc(self, t):
        s = np.sqrt(0.5)
        P0, P1, P2 = np.array([1.0, 0.0]), np.array([1.0, 1.0]), np.array([0.0, 1.0])
        t = np.asarray(t, dtype=float)
        b0, b1, b2 = (1 - t) ** 2, 2 * t * (1 - t), t * t
        d0, d1, d2 = -2 * (1 - t), 2 - 4 * t, 2 * t
        N = b0[..., None] * P0 + (s * b1)[..., None] * P1 + b2[..., None] * P2
        dN = d0[..., None] * P0 + (s * d1)[..., None] * P1 + d2[..., None] * P2
        ddN = 2 * P0 - 4 * s * P1 + 2 * P2
        W = b0 + s * b1 + b2
        dW = d0 + s * d1 + d2
        ddW = 2 - 4 * s + 2
        W_, dW_ = W[..., None], dW[..., None]
        C = N / W_
        A = dN * W_ - N * dW_                              # C' = A / W^2
        dC = A / W_ ** 2
        dA = ddN * W_ - N * ddW                            # derivative of A (the dN dW terms cancel)
        ddC = dA / W_ ** 2 - 2 * A * dW_ / W_ ** 3
        return C, dC, ddC

    def eval(self, xi, eta):
        """X (..., 2); DF (..., 2, 2) with DF[..., i, k] = dX_i / dxi_k; dDF (..., 2, 2, 2)
        with dDF[..., i, k, l] = d^2 X_i / dxi_k dxi_l."""
        xi, eta = np.broadcast_arrays(np.asarray(xi, float), np.asarray(eta, float))
        dr = self.r_o - self.r_i
        r = self.r_i + dr * xi
        C, dC, ddC = self._arc(eta)
        X = r[..., None] * C
        DF = np.stack([dr * C, r[..., None] * dC], axis=-1)
        dDF = np.zeros(xi.shape + (2, 2, 2))
        dDF[..., :, 0, 1] = dr * dC
        dDF[..., :, 1, 0] = dr * dC
        dDF[..., :, 1, 1] = r[..., None] * ddC
        return X, DF, dDF


class IdentityMap:
    """The unit square itself (F = identity): the mapped assembly must reproduce Stokes2D."""

    def eval(self, xi, eta):
        xi, eta = np.broadcast_arrays(np.asarray(xi, float), np.asarray(eta, float))
        X = np.stack([xi, eta], axis=-1)
        DF = np.zeros(xi.shape + (2, 2))
        DF[..., 0, 0] = DF[..., 1, 1] = 1.0
        return X, DF, np.zeros(xi.shape + (2, 2, 2))


def _piola(N, dN, c, DF, dDF):
    """Physical value (..., 2) and gradient (..., 2, 2) [i, j] = d v_i / d x_j of the pushed-
    forward velocity basis v = N a_c / det J, a_c = column c of DF; N and dN (..., 2) are the
    parametric value and parametric gradient."""
    J = DF[..., 0, 0] * DF[..., 1, 1] - DF[..., 0, 1] * DF[..., 1, 0]
    a = DF[..., :, c]
    # dJ/dxi_k = det[d a_0 / dxi_k, a_1] + det[a_0, d a_1 / dxi_k]
    dJ = np.stack([dDF[..., 0, 0, k] * DF[..., 1, 1] - dDF[..., 1, 0, k] * DF[..., 0, 1]
                   + DF[..., 0, 0] * dDF[..., 1, 1, k] - DF[..., 1, 0] * dDF[..., 0, 1, k] for k in (0, 1)], -1)
    v = (N / J)[..., None] * a
    G = np.zeros(v.shape + (2,))                                 # [i, k] = d v_i / d xi_k
    for k in (0, 1):
        da = dDF[..., :, c, k]
        G[..., :, k] = ((dN[..., k] / J)[..., None] * a + (N / J)[..., None] * da
                        - (N * dJ[..., k] / J ** 2)[..., None] * a)
    inv = np.linalg.inv(DF)                                      # [k, j] = d xi_k / d x_j
    return v, np.einsum('...ik,...kj->...ij', G, inv), J


class MappedStokes2D(Stokes2D):
    """Generalized Stokes (sigma u - nu lap u + grad p = f, div u = 0, no slip) on the image
    of the unit square under `geom`, discretized by the pushed-forward compatible
    B-splines; DOF layout identical to Stokes2D (the parametric coefficients)."""

    def __init__(self, p, n, sigma, nu, geom, c_pen=None):
        self.geom = geom
        super().__init__(p, n, sigma, nu, c_pen=c_pen)

    def _points(self):
        n, G = self.n, n_quad(self.p)
        g, w = bs.gauss_legendre(G)
        xs = ((np.arange(n)[:, None] + g[None, :]) / n).ravel()   # element-major
        ws = np.tile(w / n, n)
        return xs, ws

    def quad_points_xy(self):
        """Physical images of the quadrature points, (2, nG, nG) [component, eta point, xi point]."""
        xs, _ = self._points()
        X, _, _ = self.geom.eval(xs[None, :], xs[:, None])
        return np.moveaxis(X, -1, 0)

    def _local(self, ex, ey, xi, eta):
        """Local free velocity functions of element (ex, ey) at points (xi, eta) (1D arrays of
        equal length): list of (gid, value (m, 2), grad (m, 2, 2), divhat (m,)) and pressure
        list of (gid, qhat (m,)), plus det J (m,)."""
        p, q = self.p, self.q
        _, DF, dDF = self.geom.eval(xi, eta)
        Vpx = bs.basis_values(self.tp, p, xi); Dpx = bs.basis_derivs(self.tp, p, xi)
        Vqx = bs.basis_values(self.tq, q, xi); Dqx = bs.basis_derivs(self.tq, q, xi)
        Vpy = bs.basis_values(self.tp, p, eta); Dpy = bs.basis_derivs(self.tp, p, eta)
        Vqy = bs.basis_values(self.tq, q, eta); Dqy = bs.basis_derivs(self.tq, q, eta)
        vel, pre = [], []
        J = None
        for kx in range(p + 1):                         # u_x: degree p in xi, q in eta
            for ky in range(q + 1):
                g = self.gid_ux(ex + kx, ey + ky)
                if g < 0:
                    continue
                N = Vpx[:, ex + kx] * Vqy[:, ey + ky]
                dN = np.stack([Dpx[:, ex + kx] * Vqy[:, ey + ky], Vpx[:, ex + kx] * Dqy[:, ey + ky]], -1)
                v, gv, J = _piola(N, dN, 0, DF, dDF)
                vel.append((g, v, gv, dN[:, 0]))
        for kx in range(q + 1):                         # u_y: degree q in xi, p in eta
            for ky in range(p + 1):
                g = self.gid_uy(ex + kx, ey + ky)
                if g < 0:
                    continue
                N = Vqx[:, ex + kx] * Vpy[:, ey + ky]
                dN = np.stack([Dqx[:, ex + kx] * Vpy[:, ey + ky], Vqx[:, ex + kx] * Dpy[:, ey + ky]], -1)
                v, gv, J = _piola(N, dN, 1, DF, dDF)
                vel.append((g, v, gv, dN[:, 1]))
        for kx in range(q + 1):
            for ky in range(q + 1):
                pre.append((self.gid_p(ex + kx, ey + ky), Vqx[:, ex + kx] * Vqy[:, ey + ky]))
        if J is None:
            J = DF[:, 0, 0] * DF[:, 1, 1] - DF[:, 0, 1] * DF[:, 1, 0]
        return vel, pre, J, DF

    def _assemble(self):
        p, q, n = self.p, self.q, self.n
        G = n_quad(p)
        g1, w1 = bs.gauss_legendre(G)
        sig, nu = self.sigma, self.nu
        rows, cols, vals = [], [], []

        def put(r, c, v):
            rows.append(r); cols.append(c); vals.append(v)

        # volume terms: sigma (u,v) + nu (grad u, grad v) - (div v, p) + (div u, q)
        for ey in range(n):
            for ex in range(n):
                xi = np.repeat((ex + g1) / n, G)         # (gx, gy) pairs, xi slow
                eta = np.tile((ey + g1) / n, G)
                wt = np.repeat(w1, G) * np.tile(w1, G) / (n * n)
                vel, pre, J, _ = self._local(ex, ey, xi, eta)
                gv = np.array([t[0] for t in vel])
                V = np.array([t[1] for t in vel])        # (a, m, 2)
                GV = np.array([t[2] for t in vel])       # (a, m, 2, 2)
                DV = np.array([t[3] for t in vel])       # (a, m)
                gq = np.array([t[0] for t in pre])
                QH = np.array([t[1] for t in pre])       # (b, m)
                M = sig * np.einsum('ami,bmi,m->ab', V, V, wt * J) + nu * np.einsum('amij,bmij,m->ab', GV, GV, wt * J)
                # b(v, q) = int div v q dx = int divhat vhat qhat / det J dxi
                Bl = np.einsum('am,bm,m->ab', DV, QH, wt / J)
                put(np.repeat(gv, len(gv)), np.tile(gv, len(gv)), M.ravel())
                put(np.repeat(gv, len(gq)), np.tile(gq, len(gv)), -Bl.ravel())
                put(np.repeat(gq, len(gv)), np.tile(gv, len(gq)), Bl.T.ravel())
        # Nitsche terms on the four walls (Sec. 3.3):
        #   - int nu (grad u n).v - int nu (grad v n).u + int C_I nu / h u.v   ds
        pen_c = self.c_pen * nu
        for wall in range(4):
            fixed_xi = wall < 2
            side = wall % 2                              # 0: at 0, 1: at 1
            for e in range(n):
                t = (e + g1) / n
                wt = w1 / n
                if fixed_xi:
                    xi, eta = np.full(G, float(side)), t
                    ex, ey = (0 if side == 0 else n - 1), e
                else:
                    xi, eta = t, np.full(G, float(side))
                    ex, ey = e, (0 if side == 0 else n - 1)
                vel, _, J, DF = self._local(ex, ey, xi, eta)
                inv = np.linalg.inv(DF)
                k = 0 if fixed_xi else 1                 # parametric direction normal to the wall
                grad_k = inv[:, k, :]                    # gradient of xi_k in x
                nvec = (1.0 if side == 1 else -1.0) * grad_k / np.linalg.norm(grad_k, axis=-1)[:, None]
                tang = DF[:, :, 1 - k]                   # tangent along the wall
                tl = np.linalg.norm(tang, axis=-1)
                ds = wt * tl
                h = J / (tl * n)
                gv = np.array([t[0] for t in vel])
                V = np.array([t[1] for t in vel])
                DN = np.einsum('amij,mj->ami', np.array([t[2] for t in vel]), nvec)   # (grad v) n
                M = (-nu * np.einsum('bmi,ami,m->ab', DN, V, ds) - nu * np.einsum('ami,bmi,m->ab', DN, V, ds)
                     + np.einsum('ami,bmi,m->ab', V, V, ds * pen_c / h))
                put(np.repeat(gv, len(gv)), np.tile(gv, len(gv)), M.ravel())
        # mean constraint: m_j = int q_j dx = int qhat_j dxi (unchanged by the map)
        mq = bs.integrals(self.tq, q)
        m = np.zeros(self.ndof)
        for iy in range(n + q):
            for ix in range(n + q):
                m[self.gid_p(ix, iy)] = mq[ix] * mq[iy]
        self.m = m
        idx = np.nonzero(m)[0]
        lam = self.gid_lambda
        R = np.concatenate(rows + [idx, np.full(len(idx), lam)])
        C = np.concatenate(cols + [np.full(len(idx), lam), idx])
        V = np.concatenate(vals + [m[idx], m[idx]])
        self.K = sp.coo_matrix((V, (R, C)), shape=(self.ndof, self.ndof)).tocsr()
        self.K.sum_duplicates()

    def load_vector(self, f):
        """F = (l(v), 0, 0), l(v) = int f . v dx = int (J^T f) . v_hat dxi; f at the images of
        the quadrature points, (2, nG, nG) [component, eta point, xi point]."""
        n, G, p, q = self.n, n_quad(self.p), self.p, self.q
        xs, ws = self._points()
        _, DF, _ = self.geom.eval(xs[None, :], xs[:, None])
        f = np.asarray(f, dtype=float)
        fh = np.einsum('abic,iab->cab', DF, f)           # (J^T f)_c at [eta, xi]
        W = ws[:, None] * ws[None, :]
        Vpx = bs.basis_values(self.tp, p, xs); Vqx = bs.basis_values(self.tq, q, xs)
        F = np.zeros(self.ndof)
        # u_x: component 0 of J^T f against N_p(xi) N_q(eta)
        A = Vqx.T @ (W * fh[0]) @ Vpx                    # [iy, ix]
        for iy in range(n + q):
            for ix in range(1, n + p - 1):
                F[self.gid_ux(ix, iy)] = A[iy, ix]
        B = Vpx.T @ (W * fh[1]) @ Vqx
        for iy in range(1, n + p - 1):
            for ix in range(n + q):
                F[self.gid_uy(ix, iy)] = B[iy, ix]
        return F

    def velocity_at(self, U, xi, eta):
        """Physical velocity (m, 2) of the discrete field U at parametric points."""
        p, q = self.p, self.q
        X, DF, _ = self.geom.eval(xi, eta)
        Vpx = bs.basis_values(self.tp, p, xi); Vqx = bs.basis_values(self.tq, q, xi)
        Vpy = bs.basis_values(self.tp, p, eta); Vqy = bs.basis_values(self.tq, q, eta)
        n = self.n
        ux = np.zeros((n + q, n + p)); ux[:, 1:-1] = U[: self.n_ux].reshape(n + q, n + p - 2)
        uy = np.zeros((n + p, n + q)); uy[1:-1, :] = U[self.n_ux: self.n_u].reshape(n + p - 2, n + q)
        vx = np.einsum('mi,ji,mj->m', Vpx, ux, Vqy)
        vy = np.einsum('mi,ji,mj->m', Vqx, uy, Vpy)
        J = DF[:, 0, 0] * DF[:, 1, 1] - DF[:, 0, 1] * DF[:, 1, 0]
        return (vx / J)[:, None] * DF[:, :, 0] + (vy / J)[:, None] * DF[:, :, 1], X
