"""The allocation-free load-vector entry point (for callers that cannot call
cudaMalloc, e.g. while capturing a CUDA graph or under a memory manager that owns
the device) must reproduce the context path's load vector, call after call.

This file is collected last on purpose; it must pass alone and after the others."""
import ctypes

import numpy as np
import pytest

from paper_1503_08509_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_static_load_vector_matches_context_path_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_08509_gb300 import _lib, api, build
    build.build()
    lib = _lib.load()
    for pos_np, Q_np, L, n in [(*workloads.uniform_pm(1000, seed=1), 1.0, 16),
                               (*workloads.rock_salt(16, jitter=1e-3, seed=2), 1.0, 16),
                               (*workloads.uniform_pm(300, seed=13), 2.5, 9)]:
        eng = api.FEP3M(L, n)
        pos = torch.tensor(pos_np, device="cuda")
        Q = torch.tensor(Q_np, device="cuda")
        eng.set_particles(pos, Q)
        eng.compute(forces=False)
        ref = eng.mesh()["b"]
        scale = np.abs(ref).max()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for _ in range(2):
            b = torch.full((27 * n ** 3,), float("nan"), dtype=torch.float64, device="cuda")
            st = lib.fep3m_load_vector_static(L, n, len(Q_np), ctypes.c_void_p(pos.data_ptr()),
                                              ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(b.data_ptr()), stream)
            assert st == _lib.FEP3M_OK
            torch.cuda.synchronize()
            assert np.abs(b.cpu().numpy() - ref).max() <= 1e-12 * scale
        eng.close()
    # sizes beyond the static maximum are rejected before any work
    too_big = lib.fep3m_load_vector_static(1.0, 65, 1, ctypes.c_void_p(pos.data_ptr()),
                                           ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(b.data_ptr()), None)
    assert too_big == _lib.FEP3M_EINVAL
    # so are host buffers (the call takes device memory of the current device only)
    host_b = np.empty(27 * 16 ** 3)
    on_host = lib.fep3m_load_vector_static(1.0, 16, 1, ctypes.c_void_p(pos.data_ptr()),
                                           ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(host_b.ctypes.data), None)
    assert on_host == _lib.FEP3M_EINVAL
