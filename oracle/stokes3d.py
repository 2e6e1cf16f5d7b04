"""3D isogeometric compatible B-spline discretization of the generalized Stokes problem on
the unit cube and the paper's V-cycle with vector-potential-support Schwarz patches,
written plainly in FP64.

TEST INFRASTRUCTURE ONLY (the oracle).  Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg may import it; the product path never does.

Follows (3D versions of the 2D oracle's steps):
  * spaces: velocity S^{p,q,q} x S^{q,p,q} x S^{q,q,p}, pressure S^{q,q,q} (q = p-1),
    v.n = 0 strongly, mean(p) = 0 by a Lagrange multiplier                       -- Sec. 4.3
  * weak form with Nitsche no-slip on the tangential components, C_I = 4(p-1)    -- Sec. 3.1-3.3, Sec. 6
  * K_l = R K P with tensor-product knot-insertion prolongations                -- Sec. 5.1
  * subdomains = supports of vector-potential basis functions
    Psi = S^{q,p,p} x S^{p,q,p} x S^{p,p,q} with psi x n = 0 on the boundary     -- Sec. 5.2
  * generalized Oseen: + (beta . grad u, v) componentwise; coarse levels = R K P   -- Sec. 3.1, Sec. 5.1
  * Algorithm 1 with the multiplicative Schwarz smoother (eq. MSM), exact
    coarsest solve (the paper's 3D results use the multiplicative smoother only)  -- Sec. 5.1-5.2, Sec. 6.3
Readings: local pressure bordered with m (zero-mean local pressure); multiplicative order
family-major (x, y, z), inside a family colour = (i mod s_x, j mod s_y, k mod s_z) with
strides p along the family's own axis and p+1 across, lexicographic (z, y, x) inside a
colour; (p+2)-point Gauss quadrature per direction.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import bspline as bs


def quad_points_1d(p, n):
    g, w = bs.gauss_legendre(p + 2)
    return np.concatenate([(e + g) / n for e in range(n)]), np.concatenate([w / n for _ in range(n)])


class Stokes3D:
    """Layout of U: [u_x (z, y, x interior), u_y (z, y interior, x), u_z (z interior, y, x),
    p (z, y, x), lambda], x fastest; interior = indices 1..n+p-2 of the degree-p direction."""

    def __init__(self, p, n, sigma, nu, c_pen=None, h_pen=None, assemble=True, beta=None):
        """beta: advection at the quadrature points, (3, nG, nG, nG) [component, z, y, x], for
        the generalized Oseen problem (Sec. 3.1), or None for generalized Stokes."""
        self.beta = beta
        self.p, self.q, self.n = p, p - 1, n
        self.sigma, self.nu = float(sigma), float(nu)
        self.c_pen = 4.0 * (p - 1) if c_pen is None else float(c_pen)
        self.h_pen = 1.0 / n if h_pen is None else float(h_pen)
        self.tp = bs.uniform_open_knots(p, n)
        self.tq = bs.uniform_open_knots(p - 1, n)
        q = p - 1
        self.ni, self.nq = n + p - 2, n + q          # interior degree-p count, degree-q count
        self.n_uc = self.ni * self.nq * self.nq        # one velocity component
        self.n_u = 3 * self.n_uc
        self.n_p = self.nq ** 3
        self.ndof = self.n_u + self.n_p + 1
        if assemble:
            self._assemble()

    # numbering: component c in {0,1,2}; indices (i, j, k) = (x, y, z) 1D basis indices
    def gid_u(self, c, i, j, k):
        idx = [i, j, k]
        if idx[c] < 1 or idx[c] > self.ni:
            return -1
        dims = [self.nq, self.nq, self.nq]
        dims[c] = self.ni
        loc = [i, j, k]
        loc[c] -= 1
        return c * self.n_uc + (loc[2] * dims[1] + loc[1]) * dims[0] + loc[0]

    def gid_p(self, i, j, k):
        return self.n_u + (k * self.nq + j) * self.nq + i

    def _full_indices(self, c):
        """(i, j, k) over the full tensor basis of component c, z slowest, x fastest."""
        dims = [self.nq, self.nq, self.nq]
        dims[c] = self.n + self.p
        return [(i, j, k) for k in range(dims[2]) for j in range(dims[1]) for i in range(dims[0])]

    def _tables(self, knots, degree, x):
        n, G = self.n, self.p + 2
        V = bs.basis_values(knots, degree, x)
        D = bs.basis_derivs(knots, degree, x)
        val = np.zeros((n, degree + 1, G))
        der = np.zeros((n, degree + 1, G))
        for e in range(n):
            for k in range(degree + 1):
                val[e, k] = V[e * G:(e + 1) * G, e + k]
                der[e, k] = D[e * G:(e + 1) * G, e + k]
        return val, der

    def _assemble(self):
        p, q, n = self.p, self.q, self.n
        G = p + 2
        x, _ = quad_points_1d(p, n)
        g, w = bs.gauss_legendre(G)
        W3 = np.einsum("a,b,c->abc", w, w, w) / n ** 3                  # (gz, gy, gx)
        T = {p: self._tables(self.tp, p, x), q: self._tables(self.tq, q, x)}
        self._T = T
        rows, cols, vals = [], [], []
        degs = [(p, q, q), (q, p, q), (q, q, p)]                       # (x, y, z) degrees per component

        def comp_tables(c):
            dx_, dy_, dz_ = degs[c]
            (vx, gx_), (vy, gy_), (vz, gz_) = T[dx_], T[dy_], T[dz_]
            # (ez, ey, ex, local(kz,ky,kx), gz, gy, gx)
            val = np.einsum("zkc,yjb,xia->zyxkjicba", vz, vy, vx)
            ddx = np.einsum("zkc,yjb,xia->zyxkjicba", vz, vy, gx_)
            ddy = np.einsum("zkc,yjb,xia->zyxkjicba", vz, gy_, vx)
            ddz = np.einsum("zkc,yjb,xia->zyxkjicba", gz_, vy, vx)
            s = val.shape
            shp = (s[0], s[1], s[2], s[3] * s[4] * s[5], s[6], s[7], s[8])
            return [a.reshape(shp) for a in (val, ddx, ddy, ddz)]

        def ids(c):
            dx_, dy_, dz_ = degs[c]
            out = np.zeros((n, n, n, (dx_ + 1) * (dy_ + 1) * (dz_ + 1)), dtype=np.int64)
            for ez in range(n):
                for ey in range(n):
                    for ex in range(n):
                        m = 0
                        for kz in range(dz_ + 1):
                            for ky in range(dy_ + 1):
                                for kx in range(dx_ + 1):
                                    out[ez, ey, ex, m] = self.gid_u(c, ex + kx, ey + ky, ez + kz)
                                    m += 1
            return out

        pv = np.einsum("zkc,yjb,xia->zyxkjicba", T[q][0], T[q][0], T[q][0])
        s = pv.shape
        pv = pv.reshape(s[0], s[1], s[2], s[3] * s[4] * s[5], s[6], s[7], s[8])
        pid = np.zeros((n, n, n, (q + 1) ** 3), dtype=np.int64)
        for ez in range(n):
            for ey in range(n):
                for ex in range(n):
                    m = 0
                    for kz in range(q + 1):
                        for ky in range(q + 1):
                            for kx in range(q + 1):
                                pid[ez, ey, ex, m] = self.gid_p(ex + kx, ey + ky, ez + kz)
                                m += 1

        def add(ri, ci, M):
            R = np.broadcast_to(ri[..., :, None], M.shape)
            C = np.broadcast_to(ci[..., None, :], M.shape)
            mask = (R >= 0) & (C >= 0)
            rows.append(R[mask]); cols.append(C[mask]); vals.append(M[mask])

        sig, nu = self.sigma, self.nu
        self._ct, self._cid = [], []
        for c in range(3):
            v, dx, dy, dz = comp_tables(c)
            idc = ids(c)
            self._ct.append(v); self._cid.append(idc)
            M = sig * np.einsum("zyxaghk,zyxbghk,ghk->zyxab", v, v, W3)
            for d in (dx, dy, dz):
                M += nu * np.einsum("zyxaghk,zyxbghk,ghk->zyxab", d, d, W3)
            if self.beta is not None:
                # Oseen: + int v_c (beta . grad u_c), componentwise (Sec. 3.1)
                bq = [np.asarray(self.beta[a]).reshape(n, G, n, G, n, G).transpose(0, 2, 4, 1, 3, 5) for a in range(3)]
                adv = bq[0][:, :, :, None] * dx + bq[1][:, :, :, None] * dy + bq[2][:, :, :, None] * dz
                M += np.einsum("zyxaghk,zyxbghk,ghk->zyxab", v, adv, W3)
            add(idc, idc, M)
            dv = (dx, dy, dz)[c]                                        # d u_c / d x_c
            Bl = np.einsum("zyxaghk,zyxbghk,ghk->zyxab", dv, pv, W3)
            add(idc, pid, -Bl)
            add(pid, idc, np.swapaxes(Bl, -1, -2))
        self._W3 = W3

        # Nitsche for each tangential component on each wall (Sec. 3.3):
        #   - int nu v.d_n u - int nu d_n v . u + int C_I nu / h v.u  over the wall faces.
        # On the face normal to axis a the integrand of component c is a product of 1D
        # functions, so the face integral is (1D wall factor along a) x (1D mass along the
        # two in-face axes); the 1D masses are computed by the same Gauss rule.
        pen = self.c_pen * nu / self.h_pen
        ends = np.array([0.0, 1.0])
        xx, ww = quad_points_1d(p, n)
        M1, F1 = {}, {}
        for d, t in ((p, self.tp), (q, self.tq)):
            V = bs.basis_values(t, d, xx)
            M1[d] = V.T @ (ww[:, None] * V)
            ve, ge = bs.basis_values(t, d, ends), bs.basis_derivs(t, d, ends)
            F1[d] = sum(-nu * s_ * (np.outer(ve[w_], ge[w_]) + np.outer(ge[w_], ve[w_]))
                        + pen * np.outer(ve[w_], ve[w_]) for w_, s_ in ((0, -1.0), (1, 1.0)))
        for c in range(3):
            keep = np.array([self.gid_u(c, *idx) for idx in self._full_indices(c)])
            sel = np.nonzero(keep >= 0)[0]
            for a in range(3):
                if a == c:
                    continue
                fac = [M1[degs[c][ax]] if ax != a else F1[degs[c][ax]] for ax in range(3)]
                Kf = sp.kron(sp.kron(sp.csr_matrix(fac[2]), sp.csr_matrix(fac[1])), sp.csr_matrix(fac[0])).tocsr()
                Kf = Kf[sel][:, sel].tocoo()
                rows.append(keep[sel][Kf.row]); cols.append(keep[sel][Kf.col]); vals.append(Kf.data)
        mq = bs.integrals(self.tq, q)
        m = np.zeros(self.ndof)
        for k in range(n + q):
            for j in range(n + q):
                for i in range(n + q):
                    m[self.gid_p(i, j, k)] = mq[i] * mq[j] * mq[k]
        self.m = m
        idx = np.nonzero(m)[0]
        lam = self.ndof - 1
        rows.append(idx); cols.append(np.full(len(idx), lam)); vals.append(m[idx])
        rows.append(np.full(len(idx), lam)); cols.append(idx); vals.append(m[idx])
        R = np.concatenate(rows); C = np.concatenate(cols); V = np.concatenate(vals)
        self.K = sp.coo_matrix((V, (R, C)), shape=(self.ndof, self.ndof)).tocsr()
        self.K.sum_duplicates()

    def load_vector(self, f):
        """f: (3, nG, nG, nG) at the quadrature points, indexed [component, z, y, x]."""
        n, G = self.n, self.p + 2
        F = np.zeros(self.ndof)
        for c in range(3):
            fc = np.asarray(f[c]).reshape(n, G, n, G, n, G).transpose(0, 2, 4, 1, 3, 5)
            loc = np.einsum("zyxaghk,zyxghk,ghk->zyxa", self._ct[c], fc, self._W3)
            mask = self._cid[c] >= 0
            np.add.at(F, self._cid[c][mask], loc[mask])
        return F

    # ---- discrete complex --------------------------------------------------------------
    def _diff1d(self, knots, degree):
        nb = bs.n_basis(knots, degree)
        Dm = np.zeros((nb - 1, nb))
        for k in range(1, nb):
            h = knots[k + degree] - knots[k]
            Dm[k - 1, k] = degree / h
            Dm[k - 1, k - 1] = -degree / h
        return Dm

    def _full_u(self, U, c):
        """component c of U as a full 3D array [z, y, x] with zero boundary normals."""
        n, p, q = self.n, self.p, self.q
        shape = [n + q, n + q, n + q]
        shape[2 - c] = n + p
        A = np.zeros(shape)
        inner = [slice(None)] * 3
        inner[2 - c] = slice(1, -1)
        dims = [n + q, n + q, n + q]
        dims[2 - c] = n + p - 2
        A[tuple(inner)] = U[c * self.n_uc:(c + 1) * self.n_uc].reshape(dims)
        return A

    def div_coeffs(self, U):
        Dm = self._diff1d(self.tp, self.p)
        ux, uy, uz = (self._full_u(U, c) for c in range(3))
        return (np.einsum("ai,zyi->zya", Dm, ux) + np.einsum("aj,zjx->zax", Dm, uy)
                + np.einsum("ak,kyx->ayx", Dm, uz))

    def div_inf(self, U):
        return float(np.max(np.abs(self.div_coeffs(U))))

    def n_psi(self):
        return 3 * self.nq * self.ni * self.ni

    def curl(self, psi):
        """u = curl psi for psi on the constrained vector-potential space, given as the
        concatenation of its three families (family x: (z in 1..ni, y in 1..ni, x in 0..nq-1))."""
        n, p, q, ni, nq = self.n, self.p, self.q, self.ni, self.nq
        Dm = self._diff1d(self.tp, p)
        blk = nq * ni * ni
        # full arrays [z, y, x]: psi_x degree (q, p, p), psi_y (p, q, p), psi_z (p, p, q)
        px = np.zeros((n + p, n + p, n + q)); px[1:-1, 1:-1, :] = psi[:blk].reshape(ni, ni, nq)
        py = np.zeros((n + p, n + q, n + p)); py[1:-1, :, 1:-1] = psi[blk:2 * blk].reshape(ni, nq, ni)
        pz = np.zeros((n + q, n + p, n + p)); pz[:, 1:-1, 1:-1] = psi[2 * blk:].reshape(nq, ni, ni)
        # u_x = d psi_z/dy - d psi_y/dz ; u_y = d psi_x/dz - d psi_z/dx ; u_z = d psi_y/dx - d psi_x/dy
        ux = np.einsum("aj,zjx->zax", Dm, pz) - np.einsum("ak,kyx->ayx", Dm, py)
        uy = np.einsum("ak,kyx->ayx", Dm, px) - np.einsum("ai,zyi->zya", Dm, pz)
        uz = np.einsum("ai,zyi->zya", Dm, py) - np.einsum("aj,zjx->zax", Dm, px)
        U = np.zeros(self.ndof)
        U[:self.n_uc] = ux[:, :, 1:-1].ravel()
        U[self.n_uc:2 * self.n_uc] = uy[:, 1:-1, :].ravel()
        U[2 * self.n_uc:3 * self.n_uc] = uz[1:-1, :, :].ravel()
        return U


def prolongation3d(p, n_coarse):
    q = p - 1
    Pp = bs.dyadic_prolongation(p, n_coarse)
    Pq = bs.dyadic_prolongation(q, n_coarse)
    Pf = sp.csr_matrix(Pp[1:-1, 1:-1])
    Q = sp.csr_matrix(Pq)
    P_ux = sp.kron(sp.kron(Q, Q), Pf)          # rows (z, y, x), x fastest
    P_uy = sp.kron(sp.kron(Q, Pf), Q)
    P_uz = sp.kron(sp.kron(Pf, Q), Q)
    P_p = sp.kron(sp.kron(Q, Q), Q)
    return sp.block_diag([P_ux, P_uy, P_uz, P_p, sp.identity(1)]).tocsr()


class Patch3D:
    __slots__ = ("fam", "i", "j", "k", "colour", "dofs", "n_v", "n_q", "lu", "Krows")


class Level3D:
    def __init__(self, p, n, K, m, layout):
        self.p, self.n, self.K, self.m, self.layout = p, n, K, m, layout

    def build_patches(self, patch_set="interior", local_pressure="border"):
        """Subdomains = supports of the vector-potential basis functions (Sec. 5.2).

        patch_set "interior" takes the functions of the constrained space (tangential
        trace zero); "all" adds the supports of the constrained (boundary) ones as well.
        local_pressure "border" (zero integral mean by a bordered row), "pin" (the first
        local pressure function dropped) or "lstsq" (minimum-norm least squares): readings
        of the Sec. 5.2 footnote on the local pressure space's zero-average constraint."""
        p, q, n, Lo = self.p, self.p - 1, self.n, self.layout
        ni, nq = n + p - 2, n + q
        self.local_pressure = local_pressure

        def sup(i, d):
            return max(0, i - d), min(n - 1, i)

        def inside(a, box):
            return box[0] <= a[0] and a[1] <= box[1]

        patches = []
        fam_deg = [(q, p, p), (p, q, p), (p, p, q)]
        strides_all = [(p, p + 1, p + 1), (p + 1, p, p + 1), (p + 1, p + 1, p)]
        ncol_fam = p * (p + 1) ** 2
        for fam in range(3):
            dg = fam_deg[fam]
            if patch_set == "interior":
                rng = [range(nq) if dg[a] == q else range(1, ni + 1) for a in range(3)]
            else:
                rng = [range(nq) if dg[a] == q else range(0, n + p) for a in range(3)]
            st = strides_all[fam]
            for k in rng[2]:
                for j in rng[1]:
                    for i in rng[0]:
                        box = [sup(i, dg[0]), sup(j, dg[1]), sup(k, dg[2])]
                        vd, qd = [], []
                        for c in range(3):
                            degc = [q, q, q]
                            degc[c] = p
                            near = [range(max(0, v - p - 1), min(n + p, v + p + 2)) for v in (i, j, k)]
                            for kk in near[2]:
                                for jj in near[1]:
                                    for ii in near[0]:
                                        g = Lo.gid_u(c, ii, jj, kk)
                                        if g < 0 or ii >= n + degc[0] or jj >= n + degc[1] or kk >= n + degc[2]:
                                            continue
                                        if all(inside(sup(v, degc[a]), box[a]) for a, v in enumerate((ii, jj, kk))):
                                            vd.append(g)
                        near = [range(max(0, v - p - 1), min(nq, v + p + 2)) for v in (i, j, k)]
                        for kk in near[2]:
                            for jj in near[1]:
                                for ii in near[0]:
                                    if all(inside(sup(v, q), box[a]) for a, v in enumerate((ii, jj, kk))):
                                        qd.append(Lo.gid_p(ii, jj, kk))
                        if not vd and not qd:
                            continue
                        P = Patch3D()
                        P.fam, P.i, P.j, P.k = fam, i, j, k
                        P.colour = fam * ncol_fam + ((k % st[2]) * st[1] + (j % st[1])) * st[0] + (i % st[0])
                        P.dofs = np.array(sorted(vd) + sorted(qd), dtype=np.int64)
                        P.n_v, P.n_q = len(vd), len(qd)
                        patches.append(P)
        K = self.K.tocsr()
        for P in patches:
            d = P.dofs
            nl = len(d)
            Kl = K[d][:, d].toarray()
            if local_pressure == "border":
                Kb = np.zeros((nl + 1, nl + 1))
                Kb[:nl, :nl] = Kl
                Kb[nl, :nl] = self.m[d]
                Kb[:nl, nl] = self.m[d]
                P.lu = sla.lu_factor(Kb)
            elif local_pressure == "pin":
                keep = [t for t in range(nl) if not (P.n_q > 0 and t == P.n_v)]
                P.lu = (np.array(keep), np.linalg.pinv(Kl[np.ix_(keep, keep)]))
            else:
                P.lu = np.linalg.pinv(Kl)
            P.Krows = K[d]
        self.patches = patches
        self.colour_order = sorted(range(len(patches)), key=lambda t: patches[t].colour)

    def sweep_multiplicative(self, U, F):
        for t in self.colour_order:
            P = self.patches[t]
            r = F[P.dofs] - P.Krows @ U
            lp = getattr(self, "local_pressure", "border")
            if lp == "border":
                U[P.dofs] += sla.lu_solve(P.lu, np.concatenate([r, [0.0]]))[:-1]
            elif lp == "pin":
                keep, Ki = P.lu
                U[P.dofs[keep]] += Ki @ r[keep]
            else:
                U[P.dofs] += P.lu @ r


class Hierarchy3D:
    def __init__(self, p, n_fine, n_levels, sigma, nu, nu1=2, nu2=2, beta=None, gamma=1, fine=None,
                 patch_set="interior", local_pressure="border"):
        """fine: a prebuilt finest-level discretization (e.g. on a mapped domain) in place of
        the unit cube's; the coarse levels are its Galerkin products either way.
        patch_set / local_pressure: alternative readings of Sec. 5.2 (Level3D.build_patches);
        the defaults are the readings used throughout."""
        self.p, self.n_levels, self.nu1, self.nu2 = p, n_levels, nu1, nu2
        self.gamma = gamma
        if fine is None:
            fine = Stokes3D(p, n_fine, sigma, nu, beta=beta)
        self.fine = fine
        levels, Ps = [None] * n_levels, [None] * n_levels
        K, m = fine.K, fine.m
        levels[-1] = Level3D(p, n_fine, K, m, fine)
        n = n_fine
        for l in range(n_levels - 2, -1, -1):
            nc = n // 2
            P = prolongation3d(p, nc)
            Ps[l] = P
            K = (P.T @ K @ P).tocsr()
            m = P.T @ m
            levels[l] = Level3D(p, nc, K, m, Stokes3D(p, nc, sigma, nu, assemble=False))
            n = nc
        self.levels, self.P = levels, Ps
        for l in range(1, n_levels):
            levels[l].build_patches(patch_set, local_pressure)
        self.coarse_lu = sla.lu_factor(levels[0].K.toarray())

    def mgv(self, l, U, F):
        """Algorithm 1 in place on U; gamma = 2 takes the coarse correction from two cycles
        on level l-1, the second starting from the first (W-cycle, Sec. 5 opening paragraph)."""
        if l == 0:
            U[:] = sla.lu_solve(self.coarse_lu, F)
            return
        lev = self.levels[l]
        for _ in range(self.nu1):
            self.smooth(l, U, F)
        G = self.P[l - 1].T @ (F - lev.K @ U)
        dU = np.zeros(self.levels[l - 1].K.shape[0])
        for _ in range(self.gamma):
            self.mgv(l - 1, dU, G)
        U += self.P[l - 1] @ dU
        for _ in range(self.nu2):
            self.smooth(l, U, F)

    def smooth(self, l, U, F):
        self.levels[l].sweep_multiplicative(U, F)

    def vcycle(self, U, F):
        self.mgv(self.n_levels - 1, U, F)

    def fmg(self, F):
        """Full multigrid (nested iteration, Sec. 5 opening paragraph): F restricted to every
        level, the coarsest solved exactly, then on each finer level one cycle from the
        prolongated coarser solution.  Returns the finest level's approximation of K^{-1} F."""
        L = self.n_levels
        Fs = [None] * L
        Fs[-1] = np.asarray(F, dtype=float)
        for l in range(L - 1, 0, -1):
            Fs[l - 1] = self.P[l - 1].T @ Fs[l]
        U = sla.lu_solve(self.coarse_lu, Fs[0])
        for l in range(1, L):
            U = self.P[l - 1] @ U
            self.mgv(l, U, Fs[l])
        return U

    def solve(self, U, F, rtol, max_cycles, fmg=False):
        """Cycles to rtol; with fmg the first step is U += fmg(F - K U), counted as one cycle."""
        K = self.levels[-1].K
        r0 = np.linalg.norm(F - K @ U)
        hist = [r0]
        if r0 == 0.0:
            return 0, hist
        for k in range(1, max_cycles + 1):
            if fmg and k == 1:
                U += self.fmg(F - K @ U)
            else:
                self.vcycle(U, F)
            hist.append(np.linalg.norm(F - K @ U))
            if hist[-1] <= rtol * r0:
                return k, hist
        return max_cycles, hist
