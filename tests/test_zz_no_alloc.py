"""The residual entry point that allocates no device memory (igamg_residual_static).

It serves callers that cannot call cudaMalloc -- programs whose device memory belongs
to their own pool or arena, or that run where allocation is not allowed -- by keeping
its scratch in a fixed array the library declares in device memory.  This file is
collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

from paper_1705_09282_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_static_scratch_residual_matches_handle_residual_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_09282_gb300 import _lib
    from paper_1705_09282_gb300.solver import Solver

    p, n, L, sigma, nu = 2, 64, 4, 3.0, 0.5
    S = Solver(p, n, L, sigma, nu)
    pr = _lib.make_problem(p, n, L, sigma, nu)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, level in enumerate((L - 1, L - 1)):
        nd = S.ndof(level)
        U = torch.tensor(inputs.random_vector(nd, seed=31 + call), device="cuda")
        F = torch.tensor(inputs.random_vector(nd, seed=41 + call), device="cuda")
        R_ref, nrm_ref = S.residual(U, F, level=level, norm=True)
        R = torch.full((nd,), float("nan"), dtype=torch.float64, device="cuda")
        nrm = ctypes.c_double()
        rc = _lib.lib().igamg_residual_static(ctypes.byref(pr), level, ctypes.c_void_p(U.data_ptr()),
                                              ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                                              ctypes.byref(nrm), stream)
        assert rc == 0
        a, b = R.cpu().numpy(), R_ref.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
        assert abs(nrm.value - nrm_ref) <= 1e-13 * nrm_ref
    # a level too large for the static array is refused before any GPU work
    big = _lib.make_problem(3, 2048, 1 + 7, 1.0, 1.0)
    rc = _lib.lib().igamg_residual_static(ctypes.byref(big), 7, ctypes.c_void_p(U.data_ptr()),
                                          ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                                          None, stream)
    assert rc == -1
    S.close()
