"""CPU checks of the 3D (unit cube) host set-up against the 3D oracle's independent
assembly: level operators (re-assembled coarse levels = R K P), the row records the
kernels evaluate, the knot-insertion prolongations and the vector-potential patch
tables with their colours.  No GPU is needed."""
import numpy as np
import pytest

from oracle import stokes3d as o3


@pytest.mark.parametrize("p,n,L,sigma,nu", [(2, 8, 3, 1.0, 1.0), (3, 4, 2, 100.0, 0.3), (2, 4, 2, 1e-4, 1.0)])
def test_level_operators_match_oracle_galerkin(p, n, L, sigma, nu):
    from paper_1705_09282_gb300.solver import host_level_matrix
    H = o3.Hierarchy3D(p, n, L, sigma, nu)
    for lev in range(L):
        Kg = host_level_matrix(p, n, L, sigma, nu, lev, dim=3)
        Ko = H.levels[lev].K.toarray()
        assert Kg.shape == Ko.shape
        assert np.abs(Kg - Ko).max() <= 1e-12 * np.abs(Ko).max(), lev


@pytest.mark.parametrize("p,n,L", [(2, 4, 2), (3, 2, 2)])
def test_kernel_row_records_reproduce_operator(p, n, L):
    # the row evaluation the 3D kernels run (class records, clamped neighbours), executed
    # on the host, against the oracle's operators (fine level: assembly; coarse levels:
    # re-assembly with the fine penalty = R K P); n = 10 has interior classes
    from paper_1705_09282_gb300.solver import host_operator_rows
    for lev in range(L):
        nl = n >> (L - 1 - lev)
        Ko = o3.Stokes3D(p, nl, 2.0, 0.5, h_pen=1.0 / n).K.toarray()
        Kr = host_operator_rows(p, n, L, 2.0, 0.5, lev, dim=3)
        assert np.abs(Kr - Ko).max() <= 1e-12 * np.abs(Ko).max(), lev


@pytest.mark.parametrize("p", [2, 3])
def test_prolongations_match_oracle(p):
    from paper_1705_09282_gb300.solver import host_prolongation
    n, L = 8, 3
    for lev in range(1, L):
        Pg = host_prolongation(p, n, L, lev, dim=3)
        Po = o3.prolongation3d(p, n >> (L - lev)).toarray()
        assert Pg.shape == Po.shape
        assert np.abs(Pg - Po).max() <= 1e-13


@pytest.mark.parametrize("p,n", [(2, 8), (3, 4), (2, 4)])
def test_patch_tables_match_oracle(p, n):
    from paper_1705_09282_gb300.solver import host_patches
    col, dofs = host_patches(p, n, 2, 1, dim=3)
    H = o3.Hierarchy3D(p, n, 2, 1.0, 1.0)
    lev = H.levels[-1]
    want = sorted((P.colour, tuple(sorted(P.dofs))) for P in lev.patches)
    got = [(int(c), tuple(sorted(int(g) for g in d if g >= 0))) for c, d in zip(col, dofs)]
    assert [c for c, _ in got] == sorted(c for c, _ in got)
    assert sorted(got) == want
    assert len(set(c for c, _ in got)) == 3 * p * (p + 1) ** 2


def test_unsupported_3d_choices_rejected():
    import ctypes
    from paper_1705_09282_gb300 import _lib
    L = _lib.lib()
    h = ctypes.c_void_p()
    pr = _lib.make_problem(2, 8, 2, 1.0, 1.0, smoother="add", dim=3)
    assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -2
    pr = _lib.make_problem(2, 6, 3, 1.0, 1.0, dim=3)            # 6 not divisible by 4
    assert L.igamg_create(ctypes.byref(pr), None, ctypes.byref(h)) == -1


@pytest.mark.parametrize("p,n,L", [(2, 10, 2), (2, 16, 3), (3, 12, 2)])
def test_kernel_row_records_apply_operator(p, n, L):
    # K_l V through the kernels' row evaluation against the oracle's K_l V for random V,
    # on levels large enough to hold the translation-invariant interior classes
    from paper_1705_09282_gb300.solver import host_operator_apply
    rng = np.random.default_rng(3)
    for lev in range(L):
        nl = n >> (L - 1 - lev)
        Ko = o3.Stokes3D(p, nl, 2.0, 0.5, h_pen=1.0 / n).K
        for _ in range(2):
            V = rng.standard_normal(Ko.shape[0])
            want = Ko @ V
            got = host_operator_apply(p, n, L, 2.0, 0.5, lev, V, dim=3)
            assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), lev


@pytest.mark.parametrize("p,n,L", [(2, 4, 2), (2, 8, 3), (3, 4, 2)])
def test_oseen_operators_match_oracle_galerkin(p, n, L):
    # 3D generalized Oseen: fine operator with the advection block, coarse levels R K P;
    # the library's per-row records reproduce the oracle on every level
    from paper_1705_09282_gb300 import inputs
    from paper_1705_09282_gb300.solver import host_level_matrix, host_operator_apply
    beta = inputs.oseen_advection_3d(p, n, 0.5)
    sigma, nu = 1.0, 0.01
    H = o3.Hierarchy3D(p, n, L, sigma, nu, beta=beta)
    rng = np.random.default_rng(8)
    for lev in range(L):
        Ko = H.levels[lev].K.toarray()
        scale = np.abs(Ko).max()
        Kg = host_level_matrix(p, n, L, sigma, nu, lev, beta=beta, dim=3)
        assert np.abs(Kg - Ko).max() <= 1e-12 * scale, (lev, np.abs(Kg - Ko).max() / scale)
        V = rng.standard_normal(Ko.shape[0])
        KV = host_operator_apply(p, n, L, sigma, nu, lev, V, beta=beta, dim=3)
        assert np.abs(KV - Ko @ V).max() <= 1e-12 * np.abs(Ko @ V).max(), lev
    K = H.levels[-1].K.toarray()
    assert np.abs(K - K.T).max() > 1e-6 * np.abs(K).max()


# ---- hollow cylinder section (Sec. 4.3 push-forwards, Sec. 6.4) ----------------------------

@pytest.mark.parametrize("p,n,L,sigma,nu", [(2, 4, 3, 1.3, 0.7), (3, 2, 2, 1.0, 1.0), (2, 4, 2, 1e3, 1.0)])
def test_cylinder_operators_match_oracle(p, n, L, sigma, nu):
    # host assembly on the mapped cube (extra record box for u_x - u_y) and whole-row
    # Galerkin coarse levels, entry by entry and through the kernels' row evaluation
    from oracle import cylinder3d as C
    from paper_1705_09282_gb300.solver import host_level_matrix, host_operator_apply, host_operator_rows
    fine = C.MappedStokes3D(p, n, sigma, nu, C.HollowCylinder())
    H = o3.Hierarchy3D(p, n, L, sigma, nu, fine=fine)
    rng = np.random.default_rng(4)
    for lev in range(L):
        Ko = H.levels[lev].K
        scale = abs(Ko).max()
        Kd = Ko.toarray()
        assert np.abs(host_level_matrix(p, n, L, sigma, nu, lev, dim=3, geometry=2) - Kd).max() <= 1e-13 * scale, lev
        assert np.abs(host_operator_rows(p, n, L, sigma, nu, lev, dim=3, geometry=2) - Kd).max() <= 1e-13 * scale, lev
        V = rng.standard_normal(Ko.shape[0])
        got = host_operator_apply(p, n, L, sigma, nu, lev, V, dim=3, geometry=2)
        assert np.abs(got - Ko @ V).max() <= 1e-12 * np.abs(Ko @ V).max(), lev
