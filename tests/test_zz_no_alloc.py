"""ocean_tridiag_batched_static: the batched tridiagonal solve for callers that cannot
allocate device memory (for example code inside a host framework whose allocator owns
the device's free memory, or a runtime with a fixed memory budget).  It must give the same solution as
ocean_tridiag_batched, call after call, and refuse requests larger than its static
scratch before launching anything.

Collected last on purpose (the file name sorts after every other test module)."""
import ctypes

import numpy as np
import pytest

from paper_2309_06662_gb300 import ocean

TOL = {ocean.OCEAN_FP64: 1e-14, ocean.OCEAN_MIXED: 1e-6}


def _system(rng, n, nsys):
    a = -rng.uniform(0, 1, (n, nsys))
    c = -rng.uniform(0, 1, (n, nsys))
    b = 1 + np.abs(a) + np.abs(c) + rng.uniform(0, 1, (n, nsys))
    d = rng.standard_normal((n, nsys))
    return a, b, c, d


def _call(fn, tensors, x, n, nsys, precision, stream):
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in tensors]
    return fn(*ptrs, ctypes.c_void_p(x.data_ptr()), n, nsys, precision, ctypes.c_void_p(stream))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [ocean.OCEAN_FP64, ocean.OCEAN_MIXED])
def test_static_variant_matches_allocating_solve_twice(precision):
    import torch
    L = ocean.load()
    dt = torch.float64 if precision == ocean.OCEAN_FP64 else torch.float32
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(11 + precision)
    for n, nsys in ((48, 1500), (7, 333)):          # two calls in a row, different shapes
        sysm = [torch.tensor(t, dtype=dt, device="cuda") for t in _system(rng, n, nsys)]
        x_ref = torch.empty((n, nsys), dtype=dt, device="cuda")
        x_new = torch.full((n, nsys), float("nan"), dtype=dt, device="cuda")
        assert _call(L.ocean_tridiag_batched, sysm, x_ref, n, nsys, precision, stream) == 0
        assert _call(L.ocean_tridiag_batched_static, sysm, x_new, n, nsys, precision,
                     stream) == 0, L.ocean_last_error(None)
        torch.cuda.synchronize()
        ref = x_ref.double().cpu().numpy()
        new = x_new.double().cpu().numpy()
        assert np.all(np.isfinite(new))
        assert np.max(np.abs(new - ref)) <= TOL[precision] * max(1.0, np.max(np.abs(ref)))


def test_static_variant_rejects_oversize_before_launching():
    # fake, never-dereferenced pointers: the size check returns before any CUDA call
    L = ocean.load()
    fake = [ctypes.c_void_p(4096 * (q + 1)) for q in range(5)]
    words = 1 << 21
    for precision, cap in ((ocean.OCEAN_FP64, words), (ocean.OCEAN_MIXED, 2 * words)):
        n = 64
        nsys = cap // n + 1
        rc = L.ocean_tridiag_batched_static(*fake, n, nsys, precision, None)
        assert rc == -1
        assert b"exceeds the static scratch" in L.ocean_last_error(None)
    assert L.ocean_tridiag_batched_static(*fake, 0, 10, ocean.OCEAN_FP64, None) == -1
