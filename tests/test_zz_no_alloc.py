"""The residual entry point that allocates no device memory (igamg_residual_static).

It serves callers that cannot call cudaMalloc -- programs whose device memory belongs
to their own pool or arena -- by keeping its scratch in a fixed array the library
declares in device memory.  This file is collected last so that a run stopping at the
first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

from paper_1705_09282_gb300 import inputs

pytestmark = pytest.mark.gpu


def _static(pr, level, U, F, R, norm, stream):
    from paper_1705_09282_gb300 import _lib
    return _lib.lib().igamg_residual_static(ctypes.byref(pr), level, ctypes.c_void_p(U.data_ptr()),
                                            ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                                            ctypes.byref(norm) if norm is not None else None, stream)


def _torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


# (p, n_fine, grids, sigma, nu): small hierarchies, and for each degree one whose finest
# level needs about 92 % of the static array (p = 2: 2176^2; p = 3: 1792^2)
CASES = [(2, 64, 4, 3.0, 0.5), (3, 64, 4, 0.2, 2.0), (2, 2176, 8, 1.0, 1.0), (3, 1792, 9, 1.0, 1.0)]


@pytest.mark.parametrize("p,n,L,sigma,nu", CASES)
def test_static_scratch_residual_matches_handle_residual_twice(p, n, L, sigma, nu):
    torch = _torch_cuda()
    from paper_1705_09282_gb300 import _lib
    from paper_1705_09282_gb300.solver import Solver

    S = Solver(p, n, L, sigma, nu)
    pr = _lib.make_problem(p, n, L, sigma, nu)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # fine level twice in a row (the second call must not see the first one's scratch),
    # then a coarse level
    for call, level in enumerate((L - 1, L - 1, 1)):
        nd = S.ndof(level)
        U = torch.tensor(inputs.random_vector(nd, seed=31 + call), device="cuda")
        F = torch.tensor(inputs.random_vector(nd, seed=41 + call), device="cuda")
        R_ref, nrm_ref = S.residual(U, F, level=level, norm=True)
        R = torch.full((nd,), float("nan"), dtype=torch.float64, device="cuda")
        nrm = ctypes.c_double()
        assert _static(pr, level, U, F, R, nrm, stream) == 0
        a, b = R.cpu().numpy(), R_ref.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
        assert abs(nrm.value - nrm_ref) <= 1e-13 * nrm_ref
    S.close()


def test_static_scratch_refuses_levels_beyond_its_limit():
    torch = _torch_cuda()
    from paper_1705_09282_gb300 import _lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    U = torch.zeros(8, dtype=torch.float64, device="cuda")
    # refused before any GPU work (the buffers are far too small for the level)
    for p, n in ((2, 2272), (3, 1920)):
        big = _lib.make_problem(p, n, 1, 1.0, 1.0)
        assert _static(big, 0, U, U, U, None, stream) == -1          # IGAMG_EINVAL
