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


@pytest.mark.gpu
def test_static_variant_inside_a_captured_cuda_graph():
    # the use the entry point exists for: after one eager call (which looks up its
    # scratch array), a call captured into a CUDA graph and replayed on new inputs copied
    # into the captured buffers solves each new system
    import torch
    L = ocean.load()
    precision, dt = ocean.OCEAN_FP64, torch.float64
    rng = np.random.default_rng(29)
    n, nsys = 40, 700
    sysm = [torch.tensor(t, dtype=dt, device="cuda") for t in _system(rng, n, nsys)]
    x = torch.empty((n, nsys), dtype=dt, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert _call(L.ocean_tridiag_batched_static, sysm, x, n, nsys, precision,
                     s.cuda_stream) == 0
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        rc = _call(L.ocean_tridiag_batched_static, sysm, x, n, nsys, precision, s.cuda_stream)
    assert rc == 0, L.ocean_last_error(None)
    for _ in range(2):
        new = [torch.tensor(t, dtype=dt, device="cuda") for t in _system(rng, n, nsys)]
        for dst, src in zip(sysm, new):
            dst.copy_(src)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        ref = torch.empty_like(x)
        assert _call(L.ocean_tridiag_batched, new, ref, n, nsys, precision,
                     torch.cuda.current_stream().cuda_stream) == 0
        torch.cuda.synchronize()
        err = (x - ref).abs().max().item()
        assert err <= 1e-14 * max(1.0, ref.abs().max().item()), err
