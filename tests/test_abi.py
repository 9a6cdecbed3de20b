"""Host-side checks of the C ABI: the library loads, exports every function
include/kstap.h declares, and rejects bad parameters before touching a GPU."""
import os
import re

import numpy as np
import pytest

import paper_1604_03622_b300 as K
from paper_1604_03622_b300 import build as kbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(kstap_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    kbuild.build()
    L = K.lib()
    names = declared_functions()
    assert "kstap_create" in names and "kstap_detect" in names
    for n in names:
        assert hasattr(L, n), n


def test_create_rejects_unsupported_parameters_without_gpu():
    bad = [
        K.make_params(4, 16, 1, 3, 4, 7, 1, 2, 10.0),    # p != 3
        K.make_params(3, 10, 1, 3, 4, 7, 1, 2, 10.0),    # q not in {8,12,16,24,32}
        K.make_params(3, 48, 1, 3, 4, 7, 1, 2, 10.0),    # q > 32
        K.make_params(3, 16, 3, 3, 4, 7, 1, 2, 10.0),    # r_a > 2
        K.make_params(3, 16, 2, 3, 4, 7, 1, 2, 10.0, precision="fp16x3"),   # r_a = 2: FP32 bank
        K.make_params(3, 16, 2, 3, 4, 7, 1, 2, 10.0, filter="classical"),   # r_a = 2: Kron filter
        K.make_params(3, 8, 1, 8, 3, 4, 1, 2, 10.0),     # r_b >= q (Sec. 5)
        K.make_params(3, 16, 1, 9, 4, 7, 1, 2, 10.0),    # r_b > 8
        K.make_params(3, 12, 1, 12, 4, 7, 1, 2, 10.0),   # r_b >= q
        K.make_params(3, 16, 1, 5, 4, 7, 1, 2, 10.0, precision="fp16x3"),   # r_b > 4: FP32 bank
        K.make_params(6, 16, 1, 5, 4, 7, 1, 2, 10.0),    # r_b > 4: p = 3
        K.make_params(3, 16, 1, 3, 1, 7, 2, 2, 10.0),    # guard > ring
        K.make_params(3, 16, 1, 3, 0, 0, 0, 0, 10.0),    # empty ring
        K.make_params(3, 16, 1, 3, 12, 24, 1, 1, 10.0),  # box > 1024
        K.make_params(3, 16, 1, 3, 4, 7, 1, 2, 10.0, filter="classical",
                      precision="fp16x3"),                # classical filter: FP32 route only
        K.make_params(6, 32, 2, 3, 4, 7, 1, 2, 10.0),    # stacked passes: q <= 16
        K.make_params(6, 16, 3, 3, 4, 7, 1, 2, 10.0),    # stacked passes: r_a <= 2
        K.make_params(6, 16, 2, 3, 4, 7, 1, 2, 10.0, precision="fp16x3"),
        K.make_params(6, 16, 2, 3, 4, 7, 1, 2, 10.0, filter="classical"),
    ]
    dummy = np.zeros(64, np.complex64)   # never dereferenced: validation fails first
    for prm in bad:
        with pytest.raises(K.KstapError, match="EINVAL"):
            K.kstap_create(prm, _Fake(dummy), _Fake(dummy), 8)
        assert K.kstap_last_error(None) != ""


def test_domain_accepted_by_validation_without_gpu():
    """q in {8, 12, 16, 24, 32} and 1 <= r_b <= min(q - 1, 8) pass the checks
    that run before any device work: the workspace size is defined for them."""
    for q in (8, 12, 16, 24, 32):
        for r_b in range(1, min(q - 1, 8) + 1):
            prm = K.make_params(3, q, 1, r_b, 4, 7, 1, 2, 10.0)
            assert K.kstap_workspace_bytes(prm, 40, 40 + q) > 0, (q, r_b)
    for q in (12, 24):
        for prec in ("fp16x3", "bf16x3"):
            prm = K.make_params(3, q, 1, 4, 4, 7, 1, 2, 10.0, precision=prec)
            assert K.kstap_workspace_bytes(prm, 40, 40 + q) > 0, (q, prec)


def test_noalloc_and_change_map_reject_without_gpu():
    import ctypes
    dummy = np.zeros(64, np.complex64)
    fac = K.make_factors(_Fake(dummy), _Fake(dummy), _Fake(dummy))
    prm = K.make_params(6, 8, 2, 2, 4, 7, 1, 2, 10.0)    # stacked passes: context path only
    with pytest.raises(K.KstapError, match="EINVAL"):
        K.kstap_fit_project_noalloc(prm, _Fake(dummy), 20, 40, fac)
    t = np.zeros(8, np.float32)
    for ncell, V, Kp in ((4, 0, 2), (4, 2, 0), (-1, 2, 2)):
        st = K.lib().kstap_change_map(t.ctypes.data, ncell, V, Kp, None, None, None)
        assert K.STATUS[st] == "KSTAP_EINVAL"
    # no cells: nothing to do, nothing launched
    assert K.lib().kstap_change_map(None, 0, 2, 2, None, None, None) == K.KSTAP_OK


def test_workspace_size_formula():
    prm = K.make_params(3, 16, 1, 3, 4, 7, 1, 2, 10.0)
    H, W = 1024, 1024
    b = K.kstap_workspace_bytes(prm, H + 8, W + 14 + 15)
    per_cell = (45 + 9 + 9) * 8                       # M, block sums, a
    lag_store = H * 16 * 9 * (W + 15) * 16            # exact lag sums, float-float
    expect = per_cell * H * W + lag_store
    assert expect <= b <= expect + 4096
    assert K.kstap_workspace_bytes(prm, 5, 5) == 0


class _Fake:
    """Stands in for a device tensor: only data_ptr() is read."""

    def __init__(self, arr):
        self.arr = arr

    def data_ptr(self):
        return self.arr.ctypes.data
