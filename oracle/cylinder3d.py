"""Generalized Stokes on a mapped 3D domain: compatible B-splines pushed forward from the
parametric cube (Sec. 4.3), on the hollow cylinder section of Sec. 6.4 (the Sec. 6.2
quarter annulus extruded in z by a depth of 0.1).

TEST INFRASTRUCTURE ONLY (the oracle).  Only tests/, __graft_entry__.smoke() and
bench.py's CPU legs may import it; the product path never does.

What it follows:
  * 3D push-forwards of Sec. 4.3: velocity by det(J) J^-1 (contravariant Piola,
    v = J v_hat / det J), pressure by det(J) (q = q_hat / det J), so div v =
    div_hat v_hat / det J and the discrete complex is kept
  * the weak form of Sec. 3.1 / 3.3 on the physical domain, integrated over the parametric
    cube with (p+2)-point Gauss rules per direction
  * Nitsche terms on the six faces for the tangential velocity; the normal component is
    removed strongly as on the cube (the Piola map keeps v . n = 0)

Readings where the paper is silent:
  * map: (x, y) = the quarter-annulus map of oracle/annulus2d.py in (xi, eta), z = d zeta;
  * Nitsche length h at a face point = the element's height normal to the face,
    det J / (|t1 x t2| n) with t1, t2 the face's tangent columns of J (1/n on the cube);
  * load vector l(v) = int f . v dx = int (J^T f) . v_hat dxi, f sampled at the images of
    the parametric quadrature points.
"""
import numpy as np
import scipy.sparse as sp

from . import bspline as bs
from .annulus2d import QuarterAnnulus
from .stokes3d import Stokes3D


class HollowCylinder:
    """F(xi, eta, zeta) = (r(xi) C(eta), d zeta)."""

    def __init__(self, r_i=0.075, r_o=0.225, depth=0.1):
        self.plane = QuarterAnnulus(r_i, r_o)
        self.d = float(depth)

    def eval(self, xi, eta, zeta):
        """X (..., 3); DF (..., 3, 3) [i, k] = dX_i / dxi_k; dDF (..., 3, 3, 3) [i, k, l] =
        d^2 X_i / dxi_k dxi_l."""
        xi, eta, zeta = np.broadcast_arrays(np.asarray(xi, float), np.asarray(eta, float), np.asarray(zeta, float))
        X2, DF2, dDF2 = self.plane.eval(xi, eta)
        X = np.concatenate([X2, (self.d * zeta)[..., None]], axis=-1)
        DF = np.zeros(xi.shape + (3, 3))
        DF[..., :2, :2] = DF2
        DF[..., 2, 2] = self.d
        dDF = np.zeros(xi.shape + (3, 3, 3))
        dDF[..., :2, :2, :2] = dDF2
        return X, DF, dDF


class IdentityMap3:
    """The unit cube itself: the mapped assembly must reproduce Stokes3D."""

    def eval(self, xi, eta, zeta):
        xi, eta, zeta = np.broadcast_arrays(np.asarray(xi, float), np.asarray(eta, float), np.asarray(zeta, float))
        X = np.stack([xi, eta, zeta], axis=-1)
        DF = np.zeros(xi.shape + (3, 3))
        DF[..., 0, 0] = DF[..., 1, 1] = DF[..., 2, 2] = 1.0
        return X, DF, np.zeros(xi.shape + (3, 3, 3))


def _piola3(N, dN, c, DF, dDF):
    """Value (..., 3), physical gradient (..., 3, 3) [i, j] = d v_i / d x_j and det J of the
    pushed-forward basis v = N a_c / det J (a_c = column c of DF); N, dN (..., 3) parametric.
    d(det J)/dxi_k by Jacobi's formula, det J tr(J^-1 dJ/dxi_k)."""
    J = np.linalg.det(DF)
    inv = np.linalg.inv(DF)                                   # [k, j] = d xi_k / d x_j
    dJ = np.stack([J * np.einsum("...ij,...ji->...", inv, dDF[..., :, :, k]) for k in range(3)], -1)
    a = DF[..., :, c]
    v = (N / J)[..., None] * a
    G = np.zeros(v.shape + (3,))                              # [i, k] = d v_i / d xi_k
    for k in range(3):
        G[..., :, k] = ((dN[..., k] / J)[..., None] * a + (N / J)[..., None] * dDF[..., :, c, k]
                        - (N * dJ[..., k] / J ** 2)[..., None] * a)
    return v, np.einsum("...ik,...kj->...ij", G, inv), J


class MappedStokes3D(Stokes3D):
    """Generalized Stokes on the image of the unit cube under `geom`, discretized by the
    pushed-forward compatible B-splines; DOF layout identical to Stokes3D."""

    def __init__(self, p, n, sigma, nu, geom, c_pen=None):
        self.geom = geom
        super().__init__(p, n, sigma, nu, c_pen=c_pen)

    def _points(self):
        n, G = self.n, self.p + 2
        g, w = bs.gauss_legendre(G)
        xs = ((np.arange(n)[:, None] + g[None, :]) / n).ravel()       # element-major
        return xs, np.tile(w / n, n)

    def quad_points_xyz(self):
        """Physical images of the quadrature points, (3, nG, nG, nG) [component, z, y, x]."""
        xs, _ = self._points()
        X, _, _ = self.geom.eval(xs[None, None, :], xs[None, :, None], xs[:, None, None])
        return np.moveaxis(X, -1, 0)

    def _basis(self, deg, t):
        knots = self.tp if deg == self.p else self.tq
        return bs.basis_values(knots, deg, t), bs.basis_derivs(knots, deg, t)

    def _local(self, e, pts):
        """Free velocity functions of element e = (ex, ey, ez) at points pts = (xi, eta, zeta)
        (1D arrays of one length m): arrays of global ids, values (a, m, 3), physical
        gradients (a, m, 3, 3), parametric divergences (a, m); pressure ids and values
        (b, m); det J (m,) and DF (m, 3, 3)."""
        p, q = self.p, self.q
        _, DF, dDF = self.geom.eval(*pts)
        tab = {(d, ax): self._basis(d, pts[ax]) for d in (p, q) for ax in range(3)}
        degs = [(p, q, q), (q, p, q), (q, q, p)]
        gid, V, GV, DV = [], [], [], []
        J = np.linalg.det(DF)
        for c in range(3):
            dg = degs[c]
            for kz in range(dg[2] + 1):
                for ky in range(dg[1] + 1):
                    for kx in range(dg[0] + 1):
                        ijk = (e[0] + kx, e[1] + ky, e[2] + kz)
                        g = self.gid_u(c, *ijk)
                        if g < 0:
                            continue
                        vals = [tab[(dg[ax], ax)][0][:, ijk[ax]] for ax in range(3)]
                        ders = [tab[(dg[ax], ax)][1][:, ijk[ax]] for ax in range(3)]
                        N = vals[0] * vals[1] * vals[2]
                        dN = np.stack([ders[0] * vals[1] * vals[2], vals[0] * ders[1] * vals[2],
                                       vals[0] * vals[1] * ders[2]], -1)
                        v, gv, _ = _piola3(N, dN, c, DF, dDF)
                        gid.append(g); V.append(v); GV.append(gv); DV.append(dN[:, c])
        pid, QH = [], []
        for kz in range(q + 1):
            for ky in range(q + 1):
                for kx in range(q + 1):
                    ijk = (e[0] + kx, e[1] + ky, e[2] + kz)
                    pid.append(self.gid_p(*ijk))
                    QH.append(tab[(q, 0)][0][:, ijk[0]] * tab[(q, 1)][0][:, ijk[1]] * tab[(q, 2)][0][:, ijk[2]])
        return (np.array(gid), np.array(V), np.array(GV), np.array(DV), np.array(pid), np.array(QH), J, DF)

    def _assemble(self):
        p, q, n = self.p, self.q, self.n
        G = p + 2
        g1, w1 = bs.gauss_legendre(G)
        sig, nu = self.sigma, self.nu
        rows, cols, vals = [], [], []

        def put(ri, ci, M):
            rows.append(np.repeat(ri, len(ci))); cols.append(np.tile(ci, len(ri))); vals.append(M.ravel())

        # volume terms: sigma (u,v) + nu (grad u, grad v) - (div v, p) + (div u, q)
        Z, Y, X_ = np.meshgrid(g1, g1, g1, indexing="ij")
        WZ, WY, WX = np.meshgrid(w1, w1, w1, indexing="ij")
        wt = (WZ * WY * WX).ravel() / n ** 3
        for ez in range(n):
            for ey in range(n):
                for ex in range(n):
                    pts = ((ex + X_.ravel()) / n, (ey + Y.ravel()) / n, (ez + Z.ravel()) / n)
                    gv, V, GV, DV, gq, QH, J, _ = self._local((ex, ey, ez), pts)
                    M = (sig * np.einsum("ami,bmi,m->ab", V, V, wt * J)
                         + nu * np.einsum("amij,bmij,m->ab", GV, GV, wt * J))
                    # b(v, q) = int div v q dx = int divhat vhat qhat / det J dxi
                    Bl = np.einsum("am,bm,m->ab", DV, QH, wt / J)
                    put(gv, gv, M)
                    put(gv, gq, -Bl)
                    put(gq, gv, Bl.T)
        self._nitsche(put, g1, w1)
        # mean constraint: m_j = int q_j dx = int qhat_j dxi (unchanged by the map)
        mq = bs.integrals(self.tq, q)
        m = np.zeros(self.ndof)
        for k in range(n + q):
            for j in range(n + q):
                for i in range(n + q):
                    m[self.gid_p(i, j, k)] = mq[i] * mq[j] * mq[k]
        self.m = m
        idx = np.nonzero(m)[0]
        lam = self.ndof - 1
        R = np.concatenate(rows + [idx, np.full(len(idx), lam)])
        C = np.concatenate(cols + [np.full(len(idx), lam), idx])
        Vv = np.concatenate(vals + [m[idx], m[idx]])
        self.K = sp.coo_matrix((Vv, (R, C)), shape=(self.ndof, self.ndof)).tocsr()
        self.K.sum_duplicates()

    def _nitsche(self, put, g1, w1):
        """-int nu (grad u n).v - int nu (grad v n).u + int C_I nu / h u.v on the six faces
        (Sec. 3.3), h = det J / (|t1 x t2| n)."""
        n, nu = self.n, self.nu
        G = len(g1)
        pen_c = self.c_pen * nu
        A, B = np.meshgrid(g1, g1, indexing="ij")
        WA, WB = np.meshgrid(w1, w1, indexing="ij")
        wt = (WA * WB).ravel() / n ** 2
        for k in range(3):
            a1, a2 = [ax for ax in range(3) if ax != k]
            for side in (0, 1):
                for e1 in range(n):
                    for e2 in range(n):
                        e = [0, 0, 0]
                        e[k] = 0 if side == 0 else n - 1
                        e[a1], e[a2] = e1, e2
                        pts = [None, None, None]
                        pts[k] = np.full(G * G, float(side))
                        pts[a1] = (e1 + A.ravel()) / n
                        pts[a2] = (e2 + B.ravel()) / n
                        gv, V, GV, _, _, _, J, DF = self._local(tuple(e), tuple(pts))
                        inv = np.linalg.inv(DF)
                        nv = inv[:, k, :]                                  # gradient of xi_k
                        nv = (1.0 if side == 1 else -1.0) * nv / np.linalg.norm(nv, axis=-1)[:, None]
                        area = np.linalg.norm(np.cross(DF[:, :, a1], DF[:, :, a2]), axis=-1)
                        ds = wt * area
                        h = J / (area * n)
                        DN = np.einsum("amij,mj->ami", GV, nv)                # (grad v) n
                        M = (-nu * np.einsum("bmi,ami,m->ab", DN, V, ds) - nu * np.einsum("ami,bmi,m->ab", DN, V, ds)
                             + np.einsum("ami,bmi,m->ab", V, V, ds * pen_c / h))
                        put(gv, gv, M)

    def load_vector(self, f):
        """F = (l(v), 0, 0), l(v) = int (J^T f) . v_hat dxi; f: the physical field at the images
        of the quadrature points, (3, nG, nG, nG) [component, z, y, x]."""
        p, q, n = self.p, self.q, self.n
        xs, ws = self._points()
        _, DF, _ = self.geom.eval(xs[None, None, :], xs[None, :, None], xs[:, None, None])
        fh = np.einsum("zyxic,izyx->czyx", DF, np.asarray(f, dtype=float))
        W = ws[:, None, None] * ws[None, :, None] * ws[None, None, :]
        V = {d: bs.basis_values(self.tp if d == p else self.tq, d, xs) for d in (p, q)}
        degs = [(p, q, q), (q, p, q), (q, q, p)]
        F = np.zeros(self.ndof)
        for c in range(3):
            dx, dy, dz = degs[c]
            A = np.einsum("zyx,zk,yj,xi->kji", W * fh[c], V[dz], V[dy], V[dx])
            for (i, j, k) in self._full_indices(c):
                g = self.gid_u(c, i, j, k)
                if g >= 0:
                    F[g] = A[k, j, i]
        return F

    def velocity_at(self, U, xi, eta, zeta):
        """Physical velocity (m, 3) of U at parametric points, and the points' images."""
        p, q = self.p, self.q
        X, DF, _ = self.geom.eval(xi, eta, zeta)
        V = {(d, ax): bs.basis_values(self.tp if d == p else self.tq, d, t)
             for d in (p, q) for ax, t in enumerate((xi, eta, zeta))}
        degs = [(p, q, q), (q, p, q), (q, q, p)]
        uh = np.zeros((len(xi), 3))
        for c in range(3):
            full = self._full_u(U, c)                                      # [z, y, x]
            dx, dy, dz = degs[c]
            comp = np.einsum("kji,mk,mj,mi->m", full, V[(dz, 2)], V[(dy, 1)], V[(dx, 0)])
            uh += (comp / np.linalg.det(DF))[:, None] * DF[:, :, c]
        return uh, X
