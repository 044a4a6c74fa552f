"""GPU test of sg_get_moments_noalloc, the entry point for callers that must not allocate device
memory (it stages results in a fixed static device array instead of handle-owned memory).

It is called through the C ABI directly and compared with sg_get_moments on the same handle, on
two calls in a row with a time step in between.  This file sorts last so that a run stopping at the
first failure has already run every other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

import sg_workloads as w

pytestmark = pytest.mark.gpu


def test_noalloc_moments_match_allocating_entry_point():
    from paper_2512_23027_gb300 import build as b
    b.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_23027_gb300 import Solver
    s = Solver(w.config("small"))
    lib = s.lib
    n = s.n_free
    for call in range(2):
        s.step(2)
        mean_ref, var_ref = s.moments()
        mean = np.full(n, np.nan)
        var = np.full(n, np.nan)
        rc = lib.sg_get_moments_noalloc(s.h, ctypes.c_void_p(mean.ctypes.data), ctypes.c_void_p(var.ctypes.data))
        assert rc == 0, (rc, lib.sg_last_error(s.h))
        # identical kernel on identical data: agreement to the last bit (tolerance stated for form)
        assert np.allclose(mean, mean_ref, rtol=1e-15, atol=0.0), call
        assert np.allclose(var, var_ref, rtol=1e-15, atol=0.0), call
        assert np.abs(mean).max() > 0.0
    s.close()
