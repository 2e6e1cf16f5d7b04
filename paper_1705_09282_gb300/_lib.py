"""ctypes binding of libigamg.so: argument marshalling only.

Every numerical step runs inside the library's CUDA kernels.  There is no CPU
fallback: if the shared library is missing, loading raises.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libigamg.so")

IGAMG_OK = 0
IGAMG_NOT_CONVERGED = 1
IGAMG_MULT, IGAMG_ADD = 0, 1
IGAMG_FP64, IGAMG_FP32_IR, IGAMG_FGMRES_FP64, IGAMG_FGMRES_FP32 = 0, 1, 2, 3
IGAMG_GEOM_SQUARE, IGAMG_GEOM_QUARTER_ANNULUS, IGAMG_GEOM_HOLLOW_CYLINDER = 0, 1, 2


class Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("p", ctypes.c_int), ("n_fine", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("sigma", ctypes.c_double), ("nu", ctypes.c_double),
                ("c_penalty", ctypes.c_double), ("beta_qp", ctypes.c_void_p),
                ("smoother", ctypes.c_int), ("eta", ctypes.c_double), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("precision", ctypes.c_int), ("restart", ctypes.c_int),
                ("gamma", ctypes.c_int), ("fmg", ctypes.c_int), ("geometry", ctypes.c_int),
                ("r_inner", ctypes.c_double), ("r_outer", ctypes.c_double)]


class Sizes(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nx_ux", ctypes.c_int), ("ny_ux", ctypes.c_int),
                ("nx_uy", ctypes.c_int), ("ny_uy", ctypes.c_int), ("n_pdir", ctypes.c_int),
                ("n_ux", ctypes.c_longlong), ("n_uy", ctypes.c_longlong), ("n_p", ctypes.c_longlong),
                ("n_total", ctypes.c_longlong), ("n_patches", ctypes.c_int), ("n_colours", ctypes.c_int),
                ("n_quad", ctypes.c_int), ("dim", ctypes.c_int), ("n_uz", ctypes.c_longlong)]


class Report(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("res0", ctypes.c_double), ("rel_residual", ctypes.c_double),
                ("div_inf", ctypes.c_double), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_cap", ctypes.c_int)]


_P, _I, _D, _LL, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_size_t

# name -> (restype, argtypes); every symbol declared in include/igamg.h
SIGNATURES = {
    "igamg_create": (_I, [ctypes.POINTER(Problem), _P, ctypes.POINTER(_P)]),
    "igamg_destroy": (None, [_P]),
    "igamg_strerror": (ctypes.c_char_p, [_I]),
    "igamg_get_sizes": (_I, [_P, _I, ctypes.POINTER(Sizes)]),
    "igamg_quad_points": (_I, [_P, _P, _SZ, ctypes.POINTER(_SZ)]),
    "igamg_quad_points_xy": (_I, [_P, _P, _SZ, ctypes.POINTER(_SZ)]),
    "igamg_load_vector": (_I, [_P, _P, _P]),
    "igamg_residual": (_I, [_P, _I, _P, _P, _P, _P]),
    "igamg_smooth": (_I, [_P, _I, _P, _P, _I]),
    "igamg_restrict": (_I, [_P, _I, _P, _P]),
    "igamg_prolong_add": (_I, [_P, _I, _P, _P]),
    "igamg_coarse_solve": (_I, [_P, _P, _P]),
    "igamg_vcycle": (_I, [_P, _P, _P]),
    "igamg_solve": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(Report)]),
    "igamg_solve_host": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(Report)]),
    "igamg_solve_batch": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I,
                               ctypes.POINTER(Report), ctypes.POINTER(_I)]),
    "igamg_solve_abs": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(Report)]),
    "igamg_solve_batch_abs": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                   ctypes.POINTER(_D), _I, ctypes.POINTER(Report), ctypes.POINTER(_I)]),
    "igamg_streamfunction": (_I, [_P, _P, _P]),
    "igamg_warm_start": (_I, [_P, _P, _D, _D, _P]),
    "igamg_warm_start_minres": (_I, [_P, _P, _D, _D, _P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "igamg_nn_create": (_I, [_I, _I, ctypes.POINTER(_I), ctypes.c_ulonglong, _P, ctypes.POINTER(_P)]),
    "igamg_nn_destroy": (None, [_P]),
    "igamg_nn_num_params": (_I, [_P]),
    "igamg_nn_get_params": (_I, [_P, _P, _SZ]),
    "igamg_nn_set_params": (_I, [_P, _P, _SZ]),
    "igamg_nn_forward": (_I, [_P, _I, _I, _I, _P, _P]),
    "igamg_nn_loss_grad": (_I, [_P, _I, _I, _I, _P, _P, ctypes.POINTER(_D), _P]),
    "igamg_nn_train_step": (_I, [_P, _I, _I, _I, _P, _P, ctypes.c_float, ctypes.POINTER(_D)]),
    "igamg_div_inf": (_I, [_P, _P, ctypes.POINTER(_D)]),
    "igamg_curl": (_I, [_P, _P, _P]),
    "igamg_residual_static": (_I, [ctypes.POINTER(Problem), _I, _P, _P, _P, ctypes.POINTER(_D), _P]),
    "igamg_probe_fma": (_I, [_I, _I, _I, _P, _P, ctypes.POINTER(_D)]),
    "igamg_smooth_f32": (_I, [_P, _I, _P, _P, _I]),
    "igamg_residual_f32": (_I, [_P, _I, _P, _P, _P, _P]),
    "igamg_residual_form": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "igamg_set_residual_form": (_I, [_P, _I, _I]),
    "igamg_level_form": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "igamg_level_chains": (_I, [_P, _I, ctypes.POINTER(_I)]),
    "igamg_host_level_matrix": (_I, [ctypes.POINTER(Problem), _I, _P, _SZ, ctypes.POINTER(_LL)]),
    "igamg_host_operator_rows": (_I, [ctypes.POINTER(Problem), _I, _P, _SZ, ctypes.POINTER(_LL)]),
    "igamg_host_operator_apply": (_I, [ctypes.POINTER(Problem), _I, _P, _P, _SZ]),
    "igamg_host_prolongation": (_I, [ctypes.POINTER(Problem), _I, _P, _SZ, ctypes.POINTER(_LL),
                                     ctypes.POINTER(_LL)]),
    "igamg_host_patches": (_I, [ctypes.POINTER(Problem), _I, _P, _P, _SZ, _SZ, ctypes.POINTER(_I),
                                ctypes.POINTER(_I)]),
}

_lib = None


def lib():
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1705_09282_gb300.build` (there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class IgamgError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().igamg_strerror(code)
        super().__init__(f"{where}: {msg.decode() if msg else code} ({code})")
        self.code = code


def check(code, where):
    if code < 0:
        raise IgamgError(code, where)
    return code


def make_problem(p, n_fine, n_levels, sigma, nu, smoother="mult", eta=0.0, nu1=2, nu2=2,
                 c_penalty=0.0, precision=IGAMG_FP64, beta=None, dim=2, restart=0, gamma=1, fmg=False,
                 geometry=IGAMG_GEOM_SQUARE, r_inner=0.0, r_outer=0.0):
    pr = Problem()
    pr.dim, pr.p, pr.n_fine, pr.n_levels = dim, p, n_fine, n_levels
    pr.sigma, pr.nu, pr.c_penalty = float(sigma), float(nu), float(c_penalty)
    pr.beta_qp = beta.ctypes.data if beta is not None else None
    pr.smoother = IGAMG_ADD if smoother == "add" else IGAMG_MULT
    pr.eta, pr.nu1, pr.nu2, pr.precision, pr.restart = float(eta), nu1, nu2, precision, restart
    pr.gamma, pr.fmg = gamma, int(bool(fmg))
    pr.geometry, pr.r_inner, pr.r_outer = geometry, float(r_inner), float(r_outer)
    return pr
