"""The C-ABI library loads, exports every function include/esom.h declares,
and rejects invalid arguments before touching a device (CPU only: nothing
here launches a kernel)."""
import ctypes

import pytest

from paper_2201_00701_gb300 import binding as B


@pytest.fixture(scope="module")
def lib():
    return B.load(build_if_missing=True)


def test_exports_every_declared_function(lib):
    names = B.declared_functions()
    assert {"esom_create", "esom_set_landmarks", "esom_project", "esom_knn",
            "esom_destroy", "esom_last_error"} <= set(names)
    for name in names:
        assert hasattr(lib, name), f"{name} declared in esom.h but not exported"


def test_binding_names_match_abi():
    for name in B.declared_functions():
        if name == "esom_status_string":
            continue
        assert hasattr(B, name), f"binding lacks {name}"


def test_status_strings(lib):
    assert B.status_string(0) == "ESOM_OK"
    assert B.status_string(B.ESOM_EALIGN) == "ESOM_EALIGN"
    assert B.status_string(B.ESOM_EDEVICE) == "ESOM_EDEVICE"


@pytest.mark.parametrize("d,L,k,expect", [
    (15, 100, 10, B.ESOM_EALIGN),        # d not a multiple of 4
    (0, 100, 10, B.ESOM_EINVAL),
    (68, 100, 10, B.ESOM_EINVAL),        # above the largest compiled d
    (16, 0, 1, B.ESOM_EINVAL),
    (16, 100, 1, B.ESOM_EINVAL),         # k < 2
    (16, 10, 11, B.ESOM_EINVAL),         # k > L
    (16, 100, 33, B.ESOM_EUNSUPPORTED),  # above the largest compiled k
])
def test_create_rejects_before_device(lib, d, L, k, expect):
    st, h = B.esom_create(d, L, k)
    assert st == expect and h is None
    assert B.esom_last_error()


def test_null_handle_calls(lib):
    assert B.esom_destroy(None) == 0
    assert B.esom_project(None, 0, 0, 0, 1.0, 1.0) == B.ESOM_EINVAL
    assert B.esom_knn(None, 0, 0, 0, None) == B.ESOM_EINVAL
    assert B.esom_set_landmarks(None, 0, 0) == B.ESOM_EINVAL
    assert B.esom_device_status(None) == B.ESOM_EINVAL
    assert B.esom_landmark_version(None) == 0
    st, _ = B.esom_get_config(None)
    assert st == B.ESOM_EINVAL
    assert B.esom_project_host(None, 0, 0, 0, 1.0, 1.0) == B.ESOM_EINVAL
    assert B.esom_set_screening(None, B.ESOM_SCREEN_TF32) == B.ESOM_EINVAL
    assert B.esom_set_split(None, True) == B.ESOM_EINVAL
    assert B.esom_set_centering(None, True) == B.ESOM_EINVAL
    assert B.esom_tune(None, 0, 1, 0, 1.0, 1.0)[0] == B.ESOM_EINVAL
    assert B.esom_knn_variant(None, B.ESOM_KNN_BASE, 0, 0, 0, None) == B.ESOM_EINVAL
    assert B.esom_project_knn(None, B.ESOM_PROJ_TABLE, 0, 0, 0, 0, 0, 1.0, 1.0) == B.ESOM_EINVAL
    assert B.esom_test_stall(None, 10_000) == B.ESOM_EINVAL
    assert B.esom_selftest_drcp(0, 0, 0, 0) == B.ESOM_OK       # n = 0: nothing to do
    assert B.esom_selftest_drcp(0, 5, 0, 0) == B.ESOM_EINVAL
    assert B.esom_selftest_drcp(0, -1, 0, 0) == B.ESOM_EINVAL


def test_header_declares_c_linkage():
    text = open(B.HEADER).read()
    assert 'extern "C"' in text
    assert "torch" not in text.lower().replace("torch's", "")
