"""relearn_morton_order_noalloc serves callers that cannot allocate device memory
(for example code running under another framework's allocator, or a real-time
loop that must not wait on cudaMalloc): it must give exactly the order that the
context-based path (relearn_build_octree, reported by relearn_get_tree) gives.

Collected last on purpose, and written to pass both alone in a fresh process and
after every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_morton_order_matches_context_path_on_two_calls():
    import torch

    import oracle
    from paper_2509_26193_gb300 import build, relearn as R, workloads
    build.build()
    oracle.build()
    L = R.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two calls in a row; the second is smaller, so anything left over in the shared
    # scratch from the first call would show up as a wrong order
    nets = [workloads.gaussian_clusters(n=300000, clusters=8, side=3000, std=150, seed=101),
            workloads.uniform_cube(n=70001, seed=102)]
    for net in nets:
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        x, y, z = d(net.x), d(net.y), d(net.z)
        codes = torch.full((net.n,), -1, dtype=torch.int32, device="cuda")
        perm = torch.full((net.n,), -1, dtype=torch.int32, device="cuda")
        st = L.relearn_morton_order_noalloc(net.n, _ptr(x), _ptr(y), _ptr(z), None, None,
                                            _ptr(codes), _ptr(perm), stream)
        assert st == R.OK
        torch.cuda.synchronize()
        ctx = R.relearn_create(net.n, 16)
        try:
            R.relearn_build_octree(ctx, x, y, z)
            want = R.relearn_get_tree(ctx)["perm"]
        finally:
            ctx.close()
        assert np.array_equal(perm.cpu().numpy(), want)
        oc, _, _ = oracle.morton(net.x, net.y, net.z)
        assert np.array_equal(codes.cpu().numpy().view(np.uint32), oc[want])
    # sizes above the stated maximum are refused before any GPU work
    n_big = (1 << 20) + 1
    st = L.relearn_morton_order_noalloc(n_big, _ptr(x), _ptr(y), _ptr(z), None, None,
                                        _ptr(codes), _ptr(perm), stream)
    assert st == R.ERR_CAPACITY
