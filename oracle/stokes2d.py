"""2D isogeometric compatible (divergence-conforming) B-spline discretization of the
generalized Stokes / Oseen problem on the unit square, and the paper's geometric
multigrid V-cycle with overlapping Schwarz smoothers, written plainly in FP64.

TEST INFRASTRUCTURE ONLY (the oracle).  Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg may import it; the product path never does.

What it follows, step by step:
  * weak form a(v,u) - b(v,p) + b(u,q) = l(v), generalized Stokes / Oseen    -- Sec. 3.1
  * Nitsche weak no-slip, strong no-penetration, penalty C_I nu / h           -- Sec. 3.3
  * block matrix K = [A -B; B^T 0] (+ a Lagrange multiplier for mean(p)=0)    -- Sec. 3.4, Sec. 4.3
  * 2D compatible spaces: psi in S^{p,p}, v in S^{p,p-1} x S^{p-1,p},
    q in S^{p-1,p-1}; psi = 0 and v.n = 0 on the boundary                     -- Sec. 4.3
  * C_I = 4(p-1), p = streamfunction degree, maximal smoothness, uniform knots -- Sec. 6 preamble
  * prolongation by knot insertion, R = P^T, K_l = R K_{l+1} P                 -- Sec. 5.1
  * Algorithm 1 (MGV), exact coarsest solve                                    -- Sec. 5.1, Algorithm 1
  * W-cycle (gamma = 2 coarse cycles per level) and full multigrid (nested
    iteration), the settings Sec. 5's opening paragraph names besides the V-cycle
  * subdomains = supports of streamfunction basis functions; local spaces are
    the basis functions supported inside; additive (eq. ASM) and
    multiplicative (eq. MSM) Schwarz smoothers                                  -- Sec. 5.2

Readings where the paper is silent:
  * local pressure null space: the local system is bordered with
    m_j = int N^q_j over the patch pressure functions (zero-mean local pressure);
  * multiplicative order: colour-major, colour of patch (a,b) =
    (b mod (p+1))*(p+1) + (a mod (p+1)), lexicographic (b, then a) inside a colour;
  * quadrature: (p+2)-point Gauss-Legendre per direction for every term (exact for
    the polynomial Stokes terms; also used for f and the advection field);
  * residual norm: Euclidean norm of the whole residual (u, p, lambda).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import bspline as bs


def n_quad(p):
    """Gauss points per direction per element."""
    return p + 2


def quad_points_1d(p, n):
    """1D quadrature abscissae (n*G,) and weights (n*G,) on [0,1], element-major."""
    g, w = bs.gauss_legendre(n_quad(p))
    x = np.concatenate([(e + g) / n for e in range(n)])
    wt = np.concatenate([w / n for e in range(n)])
    return x, wt


class Stokes2D:
    """Fine-level (or any re-assembled level) operator of Sec. 3.4 in 2D.

    DOF layout of U (and F, residuals):
      [u_x (iy in 0..n+p-2) x (ix in 1..n+p-2), x fastest;
       u_y (iy in 1..n+p-2) x (ix in 0..n+p-2), x fastest;
       p   (iy in 0..n+p-2) x (ix in 0..n+p-2), x fastest;
       lambda]
    """

    def __init__(self, p, n, sigma, nu, c_pen=None, h_pen=None, beta=None):
        assert p >= 2
        self.p, self.n = p, n
        self.sigma, self.nu = float(sigma), float(nu)
        self.c_pen = 4.0 * (p - 1) if c_pen is None else float(c_pen)
        self.h_pen = 1.0 / n if h_pen is None else float(h_pen)
        self.beta = beta
        q = p - 1
        self.q = q
        self.tp = bs.uniform_open_knots(p, n)
        self.tq = bs.uniform_open_knots(q, n)
        self.np_, self.nq_ = n + p, n + q          # 1D basis counts
        # free DOF counts
        self.nx_ux, self.ny_ux = n + p - 2, n + q
        self.nx_uy, self.ny_uy = n + q, n + p - 2
        self.n_ux = self.nx_ux * self.ny_ux
        self.n_uy = self.nx_uy * self.ny_uy
        self.n_u = self.n_ux + self.n_uy
        self.n_p = (n + q) ** 2
        self.ndof = self.n_u + self.n_p + 1
        self._assemble()

    # ---- global numbering -------------------------------------------------
    def gid_ux(self, ix, iy):
        """ix = degree-p index in x (free: 1..n+p-2), iy = degree-(p-1) index in y."""
        if ix < 1 or ix > self.n + self.p - 2:
            return -1
        return iy * self.nx_ux + (ix - 1)

    def gid_uy(self, ix, iy):
        if iy < 1 or iy > self.n + self.p - 2:
            return -1
        return self.n_ux + (iy - 1) * self.nx_uy + ix

    def gid_p(self, ix, iy):
        return self.n_u + iy * (self.n + self.q) + ix

    @property
    def gid_lambda(self):
        return self.ndof - 1

    # ---- assembly -----------------------------------------------------------
    def _tables(self, knots, degree, x):
        """Per-element local basis values/derivatives at the element's quad points:
        (n, degree+1, G) arrays; local function k on element e is global e+k."""
        n, G = self.n, n_quad(self.p)
        V = bs.basis_values(knots, degree, x)
        D = bs.basis_derivs(knots, degree, x)
        val = np.zeros((n, degree + 1, G))
        der = np.zeros((n, degree + 1, G))
        for e in range(n):
            rows = slice(e * G, (e + 1) * G)
            for k in range(degree + 1):
                val[e, k] = V[rows, e + k]
                der[e, k] = D[rows, e + k]
        return val, der

    def _assemble(self):
        p, q, n = self.p, self.q, self.n
        G = n_quad(p)
        x, _ = quad_points_1d(p, n)
        g, w = bs.gauss_legendre(G)
        W2 = np.outer(w, w) / (n * n)                       # (gy, gx) weights incl. Jacobian
        Vp, Dp = self._tables(self.tp, p, x)               # degree p
        Vq, Dq = self._tables(self.tq, q, x)               # degree p-1
        self._Vp, self._Vq = Vp, Vq

        # local functions per element, values and gradients at (gy, gx):
        # arrays shaped (ey, ex, local, gy, gx)
        def tensor(vx, dx, vy, dy):
            # vx: (n, kx, G), vy: (n, ky, G)  ->  local index = ky*(kx_count) + kx
            val = np.einsum('yjg,xih->yxjigh', vy, vx)
            gx_ = np.einsum('yjg,xih->yxjigh', vy, dx)
            gy_ = np.einsum('yjg,xih->yxjigh', dy, vx)
            s = val.shape
            shp = (s[0], s[1], s[2] * s[3], s[4], s[5])
            return val.reshape(shp), gx_.reshape(shp), gy_.reshape(shp)

        ux_v, ux_dx, ux_dy = tensor(Vp, Dp, Vq, Dq)        # u_x: degree p in x, p-1 in y
        uy_v, uy_dx, uy_dy = tensor(Vq, Dq, Vp, Dp)        # u_y: degree p-1 in x, p in y
        pq_v, _, _ = tensor(Vq, Dq, Vq, Dq)                # pressure

        # global ids of local functions, (ey, ex, local)
        def ids(kx_count, ky_count, fn):
            out = np.zeros((n, n, kx_count * ky_count), dtype=np.int64)
            for ey in range(n):
                for ex in range(n):
                    for ky in range(ky_count):
                        for kx in range(kx_count):
                            out[ey, ex, ky * kx_count + kx] = fn(ex + kx, ey + ky)
            return out

        id_ux = ids(p + 1, q + 1, self.gid_ux)
        id_uy = ids(q + 1, p + 1, self.gid_uy)
        id_p = ids(q + 1, q + 1, self.gid_p)

        rows, cols, vals = [], [], []

        def add(ri, ci, M):
            # ri: (ey,ex,a), ci: (ey,ex,b), M: (ey,ex,a,b)
            R = np.broadcast_to(ri[:, :, :, None], M.shape)
            C = np.broadcast_to(ci[:, :, None, :], M.shape)
            mask = (R >= 0) & (C >= 0)
            rows.append(R[mask]); cols.append(C[mask]); vals.append(M[mask])

        sig, nu = self.sigma, self.nu
        # a(v,u): sigma (v,u) + nu (grad v, grad u), componentwise (Sec. 3.1)
        for (v, dx, dy, idv) in ((ux_v, ux_dx, ux_dy, id_ux), (uy_v, uy_dx, uy_dy, id_uy)):
            M = sig * np.einsum('yxagh,yxbgh,gh->yxab', v, v, W2)
            M += nu * np.einsum('yxagh,yxbgh,gh->yxab', dx, dx, W2)
            M += nu * np.einsum('yxagh,yxbgh,gh->yxab', dy, dy, W2)
            add(idv, idv, M)
        # Oseen: + int v . (beta . grad u)   (Sec. 3.1, generalized Oseen)
        if self.beta is not None:
            bx = np.asarray(self.beta[0]).reshape(n, G, n, G).transpose(0, 2, 1, 3)
            by = np.asarray(self.beta[1]).reshape(n, G, n, G).transpose(0, 2, 1, 3)
            for (v, dx, dy, idv) in ((ux_v, ux_dx, ux_dy, id_ux), (uy_v, uy_dx, uy_dy, id_uy)):
                adv = bx[:, :, None] * dx + by[:, :, None] * dy      # beta . grad (trial)
                M = np.einsum('yxagh,yxbgh,gh->yxab', v, adv, W2)
                add(idv, idv, M)
        # b(v,p) = int (div v) p ; K has -B in the (u,p) block and B^T in (p,u)
        for (dv, idv) in ((ux_dx, id_ux), (uy_dy, id_uy)):
            Bl = np.einsum('yxagh,yxbgh,gh->yxab', dv, pq_v, W2)
            add(idv, id_p, -Bl)
            add(id_p, idv, np.swapaxes(Bl, 2, 3))

        # Nitsche wall terms (Sec. 3.3) for the tangential component on each wall:
        #   - int nu v.d_n u - int nu d_n v . u + int C_I nu / h v.u
        pen = self.c_pen * nu / self.h_pen
        w1 = w / n
        tq_ = self.tq
        y01 = np.array([0.0, 1.0])
        Vq01 = bs.basis_values(tq_, q, y01)      # (2, n+q)
        Dq01 = bs.basis_derivs(tq_, q, y01)
        nx_sign = {0: -1.0, 1: +1.0}             # outward normal component at the wall
        for wall in (0, 1):
            s = nx_sign[wall]
            # u_x on y = wall (tangential): d_n = s * d_y
            for ex in range(n):
                e_wall = 0 if wall == 0 else n - 1
                ky_list = range(e_wall, e_wall + q + 1)
                for kx in range(p + 1):
                    for kx2 in range(p + 1):
                        fx = np.sum(w1 * Vp[ex, kx] * Vp[ex, kx2])
                        for iy in ky_list:
                            for iy2 in ky_list:
                                a_, b_ = Vq01[wall, iy], Vq01[wall, iy2]
                                da, db = Dq01[wall, iy], Dq01[wall, iy2]
                                val = fx * (-nu * s * (a_ * db + da * b_) + pen * a_ * b_)
                                r = self.gid_ux(ex + kx, iy)
                                c = self.gid_ux(ex + kx2, iy2)
                                if r >= 0 and c >= 0 and val != 0.0:
                                    rows.append(np.array([r])); cols.append(np.array([c]))
                                    vals.append(np.array([val]))
            # u_y on x = wall: d_n = s * d_x
            for ey in range(n):
                e_wall = 0 if wall == 0 else n - 1
                kx_list = range(e_wall, e_wall + q + 1)
                for ky in range(p + 1):
                    for ky2 in range(p + 1):
                        fy = np.sum(w1 * Vp[ey, ky] * Vp[ey, ky2])
                        for ix in kx_list:
                            for ix2 in kx_list:
                                a_, b_ = Vq01[wall, ix], Vq01[wall, ix2]
                                da, db = Dq01[wall, ix], Dq01[wall, ix2]
                                val = fy * (-nu * s * (a_ * db + da * b_) + pen * a_ * b_)
                                r = self.gid_uy(ix, ey + ky)
                                c = self.gid_uy(ix2, ey + ky2)
                                if r >= 0 and c >= 0 and val != 0.0:
                                    rows.append(np.array([r])); cols.append(np.array([c]))
                                    vals.append(np.array([val]))

        # mean constraint via Lagrange multiplier: m_j = int N^q_j  (Sec. 4.3 footnote)
        mq = bs.integrals(self.tq, q)
        m = np.zeros(self.ndof)
        for iy in range(n + q):
            for ix in range(n + q):
                m[self.gid_p(ix, iy)] = mq[ix] * mq[iy]
        self.m = m
        idx = np.nonzero(m)[0]
        lam = self.gid_lambda
        rows.append(idx); cols.append(np.full(len(idx), lam)); vals.append(m[idx])
        rows.append(np.full(len(idx), lam)); cols.append(idx); vals.append(m[idx])

        R = np.concatenate(rows); C = np.concatenate(cols); V = np.concatenate(vals)
        self.K = sp.coo_matrix((V, (R, C)), shape=(self.ndof, self.ndof)).tocsr()
        self.K.sum_duplicates()

        # keep what the load vector needs
        self._ux_v, self._uy_v, self._id_ux, self._id_uy, self._W2 = ux_v, uy_v, id_ux, id_uy, W2

    def load_vector(self, f):
        """F = (l(v), 0, 0) with l(v) = int v . f (Sec. 3.1); f given at the quadrature
        points as an array (2, n*G, n*G) indexed [component, y point, x point]."""
        n, G = self.n, n_quad(self.p)
        F = np.zeros(self.ndof)
        for comp, (v, idv) in enumerate(((self._ux_v, self._id_ux), (self._uy_v, self._id_uy))):
            fc = np.asarray(f[comp]).reshape(n, G, n, G).transpose(0, 2, 1, 3)   # (ey,ex,gy,gx)
            loc = np.einsum('yxagh,yxgh,gh->yxa', v, fc, self._W2)
            mask = idv >= 0
            np.add.at(F, idv[mask], loc[mask])
        return F

    # ---- discrete complex (Sec. 4.3) ------------------------------------------
    def _diff1d(self, knots, degree):
        """(n_{degree-1} x n_degree) map from degree-p coefficients to the coefficients of
        the derivative in the degree-(p-1) basis (derivative formula, Sec. 4.3)."""
        nb = bs.n_basis(knots, degree)
        Dm = np.zeros((nb - 1, nb))
        for k in range(1, nb):
            h = knots[k + degree] - knots[k]
            Dm[k - 1, k] = degree / h
            Dm[k - 1, k - 1] = -degree / h
        return Dm

    def div_coeffs(self, U):
        """Coefficients of div u in the full pressure spline space S^{p-1,p-1}."""
        p, q, n = self.p, self.q, self.n
        Dm = self._diff1d(self.tp, p)                       # (n+q, n+p)
        ux = np.zeros((n + q, n + p))                        # (iy, ix) incl. zero boundary
        ux[:, 1:-1] = U[: self.n_ux].reshape(n + q, n + p - 2)
        uy = np.zeros((n + p, n + q))
        uy[1:-1, :] = U[self.n_ux: self.n_u].reshape(n + p - 2, n + q)
        return ux @ Dm.T + Dm @ uy

    def div_inf(self, U):
        return float(np.max(np.abs(self.div_coeffs(U))))

    def curl(self, psi):
        """u = curl psi = (d psi/dy, -d psi/dx) for psi given on the interior
        (n+p-2)^2 streamfunction coefficients (psi = 0 on the boundary)."""
        p, n = self.p, self.n
        Dm = self._diff1d(self.tp, p)
        P = np.zeros((n + p, n + p))
        P[1:-1, 1:-1] = np.asarray(psi).reshape(n + p - 2, n + p - 2)
        ux = Dm @ P                  # (iy', ix): d/dy
        uy = -(P @ Dm.T)             # (iy, ix'): -d/dx
        U = np.zeros(self.ndof)
        U[: self.n_ux] = ux[:, 1:-1].ravel()
        U[self.n_ux: self.n_u] = uy[1:-1, :].ravel()
        return U

    def n_psi_interior(self):
        return (self.n + self.p - 2) ** 2


# --------------------------------------------------------------------------------
# Multigrid hierarchy (Sec. 5.1, 5.2)
# --------------------------------------------------------------------------------

def prolongation(p, n_coarse):
    """Group-variable prolongation P_l (fine x coarse) restricted to free DOFs (Sec. 5.1):
    block diag(P^v, P^q, 1) with tensor products of 1D knot-insertion matrices."""
    q = p - 1
    Pp = bs.dyadic_prolongation(p, n_coarse)       # (2nc+p, nc+p)
    Pq = bs.dyadic_prolongation(q, n_coarse)       # (2nc+q, nc+q)
    Pp_free = Pp[1:-1, 1:-1]
    assert np.all(Pp[0, 1:-1] == 0) and np.all(Pp[-1, 1:-1] == 0)
    P_ux = sp.kron(sp.csr_matrix(Pq), sp.csr_matrix(Pp_free))   # rows (iy, ix) x fastest
    P_uy = sp.kron(sp.csr_matrix(Pp_free), sp.csr_matrix(Pq))
    P_p = sp.kron(sp.csr_matrix(Pq), sp.csr_matrix(Pq))
    one = sp.identity(1)
    return sp.block_diag([P_ux, P_uy, P_p, one]).tocsr()


class Patch:
    __slots__ = ("a", "b", "colour", "dofs", "n_v", "n_q", "lu", "Krows")


class Level:
    """One grid of the hierarchy: operator K_l, patches, colouring."""

    def __init__(self, p, n, K, m, layout):
        self.p, self.n, self.K, self.m = p, n, K, m
        self.layout = layout           # a Stokes2D-like object for numbering (no operator use)
        self.patches = None
        self.colour_order = None

    def build_patches(self, patch_set="interior", local_pressure="border"):
        """Subdomains = supports of streamfunction basis functions (Sec. 5.2); local spaces
        = velocity / pressure basis functions supported inside.

        patch_set: "interior" takes the supports of the basis functions of Psi_h, which
        vanish on the boundary (Sec. 4.3 defines Psi_h with psi = 0 on the boundary), the
        reading used everywhere else; "all" adds the supports of the boundary streamfunction
        basis functions, so that the subdomains are the supports of all (n+p)^2 functions
        that the tables' DOF column counts.
        local_pressure: how the local pressure space's constant-like null direction is
        removed (Sec. 5.2 footnote: the local pressures satisfy a zero-average constraint).
        "border": bordered local system with m_j = int N^q_j (zero integral mean);
        "pin": the first local pressure function is dropped (its coefficient held fixed);
        "lstsq": the unbordered singular local system solved in the least-squares sense
        with the minimum-norm solution (the pseudo-inverse)."""
        p, q, n, L = self.p, self.p - 1, self.n, self.layout
        self.local_pressure = local_pressure

        def sup(i, deg):
            return max(0, i - deg), min(n - 1, i)

        def inside(s, box):
            return box[0] <= s[0] and s[1] <= box[1]

        def near(c, lo, hi):
            # candidate basis indices: any basis supported inside the patch has its
            # index within p+1 of the patch index (supports have at most p+1 elements)
            return range(max(lo, c - p - 1), min(hi, c + p + 2))

        lo_psi, hi_psi = (1, n + p - 1) if patch_set == "interior" else (0, n + p)
        patches = []
        for b in range(lo_psi, hi_psi):
            for a in range(lo_psi, hi_psi):
                bx, by = sup(a, p), sup(b, p)
                vd, qd = [], []
                for iy in near(b, 0, n + q):
                    for ix in near(a, 1, n + p - 1):
                        if inside(sup(ix, p), bx) and inside(sup(iy, q), by):
                            vd.append(L.gid_ux(ix, iy))
                for iy in near(b, 1, n + p - 1):
                    for ix in near(a, 0, n + q):
                        if inside(sup(ix, q), bx) and inside(sup(iy, p), by):
                            vd.append(L.gid_uy(ix, iy))
                for iy in near(b, 0, n + q):
                    for ix in near(a, 0, n + q):
                        if inside(sup(ix, q), bx) and inside(sup(iy, q), by):
                            qd.append(L.gid_p(ix, iy))
                if not vd and not qd:
                    continue
                P = Patch()
                P.a, P.b = a, b
                P.colour = (b % (p + 1)) * (p + 1) + (a % (p + 1))
                P.dofs = np.array(vd + qd, dtype=np.int64)
                P.n_v, P.n_q = len(vd), len(qd)
                patches.append(P)
        K = self.K.tocsr()
        for P in patches:
            d = P.dofs
            Kl = K[d][:, d].toarray()
            nl = len(d)
            if local_pressure == "border":
                Kb = np.zeros((nl + 1, nl + 1))
                Kb[:nl, :nl] = Kl
                Kb[nl, :nl] = self.m[d]
                Kb[:nl, nl] = self.m[d]
                P.lu = sla.lu_factor(Kb)
            elif local_pressure == "pin":
                keep = [k for k in range(nl) if not (P.n_q > 0 and k == P.n_v)]
                P.lu = (np.array(keep), np.linalg.pinv(Kl[np.ix_(keep, keep)]))
            else:
                P.lu = np.linalg.pinv(Kl)
            P.Krows = K[d]
        self.patches = patches
        # colour-major, lexicographic (b, a) inside a colour (list is already b-major)
        self.colour_order = sorted(range(len(patches)), key=lambda i: patches[i].colour)

    def local_correction(self, P, r_local):
        lp = getattr(self, "local_pressure", "border")
        if lp == "border":
            rhs = np.concatenate([r_local, [0.0]])
            return sla.lu_solve(P.lu, rhs)[:-1]
        if lp == "pin":
            keep, Ki = P.lu
            out = np.zeros_like(r_local)
            out[keep] = Ki @ r_local[keep]
            return out
        return P.lu @ r_local

    def sweep_multiplicative(self, U, F):
        """One application of eq. MSM: patches solved one after another, each from the
        current iterate's local residual, updates applied immediately."""
        for i in self.colour_order:
            P = self.patches[i]
            r = F[P.dofs] - P.Krows @ U
            U[P.dofs] += self.local_correction(P, r)

    def sweep_additive(self, U, F, eta):
        """One application of eq. ASM: all local problems from one residual, summed,
        scaled by eta."""
        r = F - self.K @ U
        dU = np.zeros_like(U)
        for P in self.patches:
            dU[P.dofs] += self.local_correction(P, r[P.dofs])
        U += eta * dU


class Hierarchy:
    """Nested levels l = 0 (coarsest) .. L-1 (finest) with Galerkin coarse operators."""

    def __init__(self, p, n_fine, n_levels, sigma, nu, c_pen=None, beta=None,
                 smoother="mult", eta=0.5, nu1=2, nu2=2, gamma=1, fine=None,
                 patch_set="interior", local_pressure="border"):
        """fine: a prebuilt finest-level discretization (e.g. on a mapped domain) in place
        of the unit square's; the coarse levels are its Galerkin products either way.
        patch_set / local_pressure: alternative readings of Sec. 5.2's subdomains and local
        pressure spaces (Level.build_patches); the defaults are the readings used throughout."""
        self.p, self.n_levels = p, n_levels
        self.smoother, self.eta, self.nu1, self.nu2 = smoother, eta, nu1, nu2
        self.gamma = gamma
        assert n_fine % (1 << (n_levels - 1)) == 0
        if fine is None:
            fine = Stokes2D(p, n_fine, sigma, nu, c_pen=c_pen, beta=beta)
        self.fine = fine
        levels = [None] * n_levels
        Ps = [None] * n_levels
        K, m = fine.K, fine.m
        levels[-1] = Level(p, n_fine, K, m, fine)
        n = n_fine
        for l in range(n_levels - 2, -1, -1):
            nc = n // 2
            P = prolongation(p, nc)
            Ps[l] = P                                # P_l : level l -> l+1
            K = (P.T @ K @ P).tocsr()                # K_l = R_{l+1} K_{l+1} P_l
            m = P.T @ m
            layout = _Layout(p, nc)
            levels[l] = Level(p, nc, K, m, layout)
            n = nc
        self.levels, self.P = levels, Ps
        for l in range(1, n_levels):
            levels[l].build_patches(patch_set, local_pressure)
        self.coarse_lu = sla.lu_factor(levels[0].K.toarray())

    def smooth(self, l, U, F):
        lev = self.levels[l]
        if self.smoother == "mult":
            lev.sweep_multiplicative(U, F)
        else:
            lev.sweep_additive(U, F, self.eta)

    def mgv(self, l, U, F):
        """Algorithm 1, applied in place to U.  With gamma = 1 this is the V-cycle of
        Algorithm 1.  With gamma = 2 (the W-cycle that Sec. 5's opening paragraph names as
        another setting for the method) the coarse correction dU comes from two cycles on
        level l-1 for the same coarse right-hand side G, the second starting from the
        first's result."""
        if l == 0:
            U[:] = sla.lu_solve(self.coarse_lu, F)
            return
        K = self.levels[l].K
        for _ in range(self.nu1):
            self.smooth(l, U, F)
        G = self.P[l - 1].T @ (F - K @ U)
        dU = np.zeros(self.levels[l - 1].K.shape[0])
        for _ in range(self.gamma):
            self.mgv(l - 1, dU, G)
        U += self.P[l - 1] @ dU
        for _ in range(self.nu2):
            self.smooth(l, U, F)

    def vcycle(self, U, F):
        self.mgv(self.n_levels - 1, U, F)

    def fmg(self, F):
        """Full multigrid (nested iteration), the other setting that Sec. 5's opening
        paragraph names: F restricted to every level (F_{l-1} = P_{l-1}^T F_l), the coarsest
        problem solved exactly, then on each finer level l the prolongated solution of level
        l-1 taken as the initial guess of one cycle (mgv) for F_l.  Returns the finest
        level's approximation of K^{-1} F."""
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

    def residual(self, U, F):
        return F - self.levels[-1].K @ U

    def solve(self, U, F, rtol, max_cycles, fmg=False):
        """Cycles until ||F - K U||_2 <= rtol ||F - K U_0||_2 (Sec. 6 protocol with the
        relative tolerance as a parameter).  With fmg the first step is U += fmg(F - K U)
        (one full-multigrid pass on the residual equation), counted as one cycle.
        Returns (cycles, history)."""
        r0 = np.linalg.norm(self.residual(U, F))
        hist = [r0]
        if r0 == 0.0:
            return 0, hist
        for k in range(1, max_cycles + 1):
            if fmg and k == 1:
                U += self.fmg(self.residual(U, F))
            else:
                self.vcycle(U, F)
            rk = np.linalg.norm(self.residual(U, F))
            hist.append(rk)
            if rk <= rtol * r0:
                return k, hist
        return max_cycles, hist


class _Layout(Stokes2D):
    """Numbering only (no assembly) for coarse levels, whose operators are Galerkin
    products rather than re-assembled matrices."""

    def __init__(self, p, n):  # noqa: D401 - numbering only
        self.p, self.n, self.q = p, n, p - 1
        q = p - 1
        self.tp = bs.uniform_open_knots(p, n)
        self.tq = bs.uniform_open_knots(q, n)
        self.nx_ux, self.ny_ux = n + p - 2, n + q
        self.nx_uy, self.ny_uy = n + q, n + p - 2
        self.n_ux = self.nx_ux * self.ny_ux
        self.n_uy = self.nx_uy * self.ny_uy
        self.n_u = self.n_ux + self.n_uy
        self.n_p = (n + q) ** 2
        self.ndof = self.n_u + self.n_p + 1
