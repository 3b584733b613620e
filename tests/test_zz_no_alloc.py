"""gm_residual_noalloc through the C ABI, against gm_residual.

The allocation-free entry point serves callers that may not allocate device
memory while it runs; it must give the same residual vector and scaled norm as
gm_residual.  Two calls in a row with different seeded increments check that
the shared scratch array left by one call does not leak into the next.  This
file is collected last so a failure here cannot hide the other GPU tests."""
import ctypes

import numpy as np
import pytest

import workloads as W

from gpu_common import cuda, need_gpu, rel, solver_for, torch

pytestmark = pytest.mark.gpu


def test_residual_noalloc_matches_residual_twice():
    need_gpu()
    prob = W.tiny_faulted(17, 16, 6, seed=5, h=(0.4, 0.3, 0.5))
    s = solver_for(prob)
    s.timestep(1.3)
    lib = s._L
    fixed = np.asarray(prob.fixed, bool)
    for seed in (101, 202):
        du, dp = W.random_vectors(s.N, seed, scale_u=1e-6, scale_p=1e5)
        du = np.where(fixed[0:3], 0.0, du)
        dp = np.where(fixed[3], 0.0, dp)
        du_t, dp_t = cuda(du), cuda(dp)
        b_ref = torch.empty((4, s.N), dtype=torch.float64, device="cuda")
        r_ref = ctypes.c_double()
        assert lib.gm_residual(s.h, ctypes.c_void_p(du_t.data_ptr()), ctypes.c_void_p(dp_t.data_ptr()),
                               ctypes.c_void_p(b_ref.data_ptr()), ctypes.byref(r_ref), None) == 0
        b_na = torch.full((4, s.N), np.nan, dtype=torch.float64, device="cuda")
        r_na = ctypes.c_double()
        rc = lib.gm_residual_noalloc(s.h, ctypes.c_void_p(du_t.data_ptr()), ctypes.c_void_p(dp_t.data_ptr()),
                                     ctypes.c_void_p(b_na.data_ptr()), ctypes.byref(r_na), None)
        assert rc == 0, lib.gm_last_error(s.h)
        b1, b2 = b_ref.cpu().numpy(), b_na.cpu().numpy()
        assert rel(b2, b1) < 1e-12
        assert abs(r_na.value - r_ref.value) <= 1e-12 * r_ref.value
        assert r_ref.value > 0


def test_residual_noalloc_rejects_grids_beyond_its_scratch():
    """257^3 nodes exceed the fixed scratch limit of 2^24 nodes: the call must
    return GM_EINVAL (-1) with a message naming the limit, before any GPU
    work, and leave the output untouched."""
    need_gpu()
    import paper_2410_17133_gb300 as gm
    n = 256
    s = gm.Solver(0)
    s.mesh(n, n, n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    s.materials(np.full(n ** 3, 20e9), 1e-15, 0.25, 0.8, 50e9, 1e-3)
    s.bind()
    assert s.N == (n + 1) ** 3 > 1 << 24
    du = torch.zeros((3, s.N), dtype=torch.float64, device="cuda")
    dp = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    b = torch.full((4, s.N), 7.0, dtype=torch.float64, device="cuda")
    r = ctypes.c_double(-1.0)
    rc = s._L.gm_residual_noalloc(s.h, ctypes.c_void_p(du.data_ptr()), ctypes.c_void_p(dp.data_ptr()),
                                  ctypes.c_void_p(b.data_ptr()), ctypes.byref(r), None)
    assert rc == -1
    assert b"16777216" in s._L.gm_last_error(s.h)
    assert torch.all(b == 7.0) and r.value == -1.0
    s.close()
