"""relearn_morton_order_noalloc serves callers that cannot allocate device memory
(for example code running under another framework's allocator, or a real-time
loop that must not wait on cudaMalloc): it must give exactly the order that the
context-based path (relearn_build_octree, reported by relearn_get_tree) gives,
and it must not change the device's free memory.

Collected last on purpose, and written to pass both alone in a fresh process and
after every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _call(L, stream, x, y, z, codes, perm, box=None):
    lo = hi = None
    if box is not None:
        lo = box[0].ctypes.data_as(ctypes.c_void_p)
        hi = box[1].ctypes.data_as(ctypes.c_void_p)
    return L.relearn_morton_order_noalloc(x.numel(), _ptr(x), _ptr(y), _ptr(z), lo, hi,
                                          _ptr(codes), _ptr(perm), stream)


def test_noalloc_morton_order_matches_context_path_on_two_calls():
    import torch

    import oracle
    from paper_2509_26193_gb300 import build, relearn as R, workloads
    build.build()
    oracle.build()
    L = R.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    # two calls in a row; the second is smaller, so anything left over in the shared
    # scratch from the first call would show up as a wrong order. The third call gives
    # a clamped, anisotropic box (positions outside it clamp to the edge cells).
    box = (np.array([100, 100, 100], np.float32), np.array([900, 800, 950], np.float32))
    cases = [(workloads.gaussian_clusters(n=300000, clusters=8, side=3000, std=150, seed=101),
              None),
             (workloads.uniform_cube(n=70001, seed=102), None),
             (workloads.uniform_cube(n=5000, side=1000, seed=44), box)]
    for net, bx in cases:
        x, y, z = d(net.x), d(net.y), d(net.z)
        codes = torch.full((net.n,), -1, dtype=torch.int32, device="cuda")
        perm = torch.full((net.n,), -1, dtype=torch.int32, device="cuda")
        assert _call(L, stream, x, y, z, codes, perm, bx) == R.OK
        torch.cuda.synchronize()
        ctx = R.relearn_create(net.n, 16)
        try:
            R.relearn_build_octree(ctx, x, y, z, None, *(bx if bx else (None, None)))
            want = R.relearn_get_tree(ctx)["perm"]
        finally:
            ctx.close()
        assert np.array_equal(perm.cpu().numpy(), want)
        oc, _, _ = oracle.morton(net.x, net.y, net.z, *(bx if bx else (None, None)))
        assert np.array_equal(codes.cpu().numpy().view(np.uint32), oc[want])


def test_noalloc_call_leaves_free_device_memory_unchanged():
    import torch

    from paper_2509_26193_gb300 import build, relearn as R, workloads
    build.build()
    L = R.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    net = workloads.uniform_cube(n=1 << 20, seed=103)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, y, z = d(net.x), d(net.y), d(net.z)
    codes = torch.empty(net.n, dtype=torch.int32, device="cuda")
    perm = torch.empty(net.n, dtype=torch.int32, device="cuda")
    # the first call on a device may make the driver load the library's kernels (and
    # place the static scratch array with them); later calls must allocate nothing
    assert _call(L, stream, x, y, z, codes, perm) == R.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _call(L, stream, x, y, z, codes, perm) == R.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    # sizes above the stated maximum are refused before any GPU work; the buffers are
    # full size, so a refusal that came too late would give a wrong status, not a fault
    n_big = (1 << 20) + 1
    xb, yb, zb = (torch.zeros(n_big, dtype=torch.float32, device="cuda") for _ in range(3))
    cb = torch.empty(n_big, dtype=torch.int32, device="cuda")
    pb = torch.empty(n_big, dtype=torch.int32, device="cuda")
    assert _call(L, stream, xb, yb, zb, cb, pb) == R.ERR_CAPACITY
    torch.cuda.synchronize()
