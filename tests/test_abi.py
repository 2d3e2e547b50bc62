"""The C-ABI library builds, loads without a GPU, exports every function that
include/relearn.h declares, and rejects bad host arguments before touching CUDA."""
import ctypes

import pytest

from paper_2509_26193_gb300 import build, relearn


@pytest.fixture(scope="module")
def L():
    build.build()
    return relearn.lib()


def test_every_declared_symbol_is_exported(L):
    names = relearn.header_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(relearn._SIGS)


def test_host_argument_errors_need_no_gpu(L):
    h = ctypes.c_void_p()
    assert L.relearn_create(None, 0, 10, 10, 0) == relearn.ERR_INVALID_ARG
    assert L.relearn_create(ctypes.byref(h), 0, 0, 10, 0) == relearn.ERR_INVALID_ARG
    assert L.relearn_create(ctypes.byref(h), 0, 10, 0, 0) == relearn.ERR_INVALID_ARG
    assert L.relearn_create(ctypes.byref(h), 0, 10, 10, -1) == relearn.ERR_INVALID_ARG
    assert not h.value
    assert L.relearn_build_octree(None, 1, None, None, None, None, None, None,
                                  None) == relearn.ERR_INVALID_ARG
    p = relearn.params(1.0, 0.3, 1, 0)
    assert L.relearn_update_connectivity(None, ctypes.byref(p), None, None, None, None,
                                         None) == relearn.ERR_INVALID_ARG
    assert L.relearn_delete_synapses(None, ctypes.byref(p), None, None, None, None, None,
                                     None) == relearn.ERR_INVALID_ARG
    assert L.relearn_deliver_spikes(None, None, None, None) == relearn.ERR_INVALID_ARG
    cnt = ctypes.c_int64()
    assert L.relearn_get_synapses(None, 0, ctypes.byref(cnt), None, None,
                                  None) == relearn.ERR_INVALID_ARG
    assert L.relearn_philox4x32_10(None, None, None, -1, None) == relearn.ERR_INVALID_ARG
    assert L.relearn_philox4x32_10(None, None, None, 0, None) == relearn.OK
    # the batched, typed, differentiable and rate entry points, the testing hook
    assert L.relearn_create_batched(None, 0, 10, 10, 0, 2) == relearn.ERR_INVALID_ARG
    assert L.relearn_build_octree_batch(None, 2, None, None, None, None, None,
                                        None) == relearn.ERR_INVALID_ARG
    assert L.relearn_update_connectivity_typed(None, ctypes.byref(p), None, None, None, None,
                                               None, None) == relearn.ERR_INVALID_ARG
    assert L.relearn_mean_length(None, ctypes.byref(p), None, None, None, None,
                                 None) == relearn.ERR_INVALID_ARG
    assert L.relearn_mean_length_backward(None, None, None, None, None, None, None, None,
                                          None) == relearn.ERR_INVALID_ARG
    assert L.relearn_deliver_rates(None, None, 1, 0, None, None) == relearn.ERR_INVALID_ARG
    assert L.relearn_debug_stall_scan(None, 0) == relearn.ERR_INVALID_ARG
    ops = ctypes.c_int64()
    assert L.relearn_peak_probe(1, 0, None, 1, ctypes.byref(ops), None) == relearn.ERR_INVALID_ARG
    assert L.relearn_peak_probe(1, 1, None, 1, ctypes.byref(ops), None) == relearn.ERR_INVALID_ARG
    assert L.relearn_morton_order_noalloc(0, None, None, None, None, None, None, None,
                                          None) == relearn.ERR_INVALID_ARG
    msg = ctypes.c_char_p()
    assert L.relearn_last_error(None, ctypes.byref(msg)) == relearn.ERR_INVALID_ARG
    assert L.relearn_destroy(None) == relearn.OK


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(relearn, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(relearn, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        relearn.lib()
