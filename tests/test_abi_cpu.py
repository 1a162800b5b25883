"""The C ABI library builds for sm_103a, loads, and exports every function
include/km.h declares.  No compute call is made (there is no GPU here); a
context cannot be created without an sm_103a device and says so."""
import ctypes

import pytest

import paper_2405_12052_gb300 as km


@pytest.fixture(scope="module")
def libkm():
    km.build()
    return km.lib()


def test_header_declares_the_abi():
    names = km.header_symbols()
    for must in ("km_create", "km_set_points", "km_set_init", "km_step", "km_run",
                 "km_get_labels", "km_get_centroids", "km_get_counts", "km_destroy",
                 "km_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(libkm):
    missing = [s for s in km.header_symbols() if not hasattr(libkm, s)]
    assert not missing, missing


def test_version_string(libkm):
    assert b"sm_103a" in libkm.km_version()


def test_create_without_gpu_fails_loudly(libkm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(km.KMError) as ei:
        km.KMeans(1000, 3, 4)
    assert ei.value.status == -3  # KM_ECUDA: no CPU fallback


def test_bad_arguments_rejected_before_any_device_call(libkm):
    h = ctypes.c_void_p()
    assert libkm.km_create(ctypes.byref(h), 10, 2, 11, None) == -1  # K > N
    assert libkm.km_create(ctypes.byref(h), 0, 2, 1, None) == -1
    assert libkm.km_create(ctypes.byref(h), 10, 0, 1, None) == -1
    assert libkm.km_create(None, 10, 2, 3, None) == -1
