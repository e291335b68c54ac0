"""Host-side tests of the C ABI: the library loads, exports every declared
symbol, and its host logic (size policy, argument validation, status codes)
behaves as documented. No kernel is launched."""
import ctypes
import os
import re

import pytest
import torch

from paper_1902_00176_gb300 import gfc

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gfc.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gfc_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(gfc_lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(gfc_lib, n), n
    assert set(names) == set(gfc._SIGNATURES), "binding and header disagree"


def _smooth(n):
    for f in (2, 3, 5, 7):
        while n % f == 0:
            n //= f
    return n == 1


@pytest.mark.parametrize("H,W,pad", [(64, 96, 4), (801, 1200, 4), (1024, 1536, 4), (256, 256, 4), (16, 16, 4),
                                     (2, 2, 1), (127, 2048, 4), (999, 4000, 3), (500, 700, 0), (300, 1000, 4),
                                     (40, 129, 4), (40, 128, 4), (2040, 2050, 4), (123, 2051, 4)])
def test_padded_size_policy(gfc_lib, H, W, pad):
    """M: the smallest even 7-smooth size >= H + 2p. N: the smallest compiled row
    length >= W + 2p when W + 2p lies in (136, max length], else as M."""
    M, N = gfc.padded_size(H, W, pad)
    p = 4 if pad <= 0 else pad
    rows = gfc.row_lengths()
    need = H + 2 * p
    assert M % 2 == 0 and _smooth(M) and M >= need
    assert not any(m % 2 == 0 and _smooth(m) for m in range(need, M))
    need = W + 2 * p
    assert N % 2 == 0 and _smooth(N) and N >= need
    if 136 < need <= rows[-1]:
        assert N in rows and not any(need <= r < N for r in rows)
    else:
        assert not any(m % 2 == 0 and _smooth(m) for m in range(need, N))


def test_row_lengths_are_even_smooth_and_ascending(gfc_lib):
    rows = gfc.row_lengths()
    assert rows == sorted(set(rows)) and len(rows) >= 25
    assert all(r % 2 == 0 and _smooth(r) for r in rows)
    assert {108, 270, 1250, 1568} <= set(rows) and rows[-1] >= 2048 + 8
    # consecutive lengths above the policy's lower end are within 15% of each other
    big = [r for r in rows if r >= 140]
    assert all(b / a <= 1.15 for a, b in zip(big, big[1:]))


def test_padded_sizes_of_the_paper_workloads(gfc_lib):
    assert gfc.padded_size(64, 96) == (72, 108)
    assert gfc.padded_size(801, 1200) == (810, 1250)
    assert gfc.padded_size(1024, 1536) == (1050, 1568)
    assert gfc.padded_size(256, 256) == (270, 270)


def test_padded_size_rejects_bad_arguments(gfc_lib):
    with pytest.raises(gfc.GFCError) as e:
        gfc.padded_size(1, 10)
    assert e.value.status == 1
    with pytest.raises(gfc.GFCError) as e:
        gfc.padded_size(5000, 10)
    assert e.value.status == 2
    M = ctypes.c_int()
    assert gfc_lib.gfc_padded_size(10, 10, 4, 7, ctypes.byref(M), ctypes.byref(M)) == 1
    assert b"policy" in gfc_lib.gfc_last_error()


def test_status_strings_and_null_arguments(gfc_lib):
    assert gfc_lib.gfc_status_string(0) == b"GFC_OK"
    assert gfc_lib.gfc_status_string(5) == b"GFC_ERR_TIMEOUT"
    assert gfc_lib.gfc_solve_from_gradient(None, None, None, None) == 1
    assert gfc_lib.gfc_solve_from_laplacian(None, None, None) == 1
    assert gfc_lib.gfc_backward(None, None, None, None) == 1
    assert gfc_lib.gfc_plan_sync(None) == 1
    assert gfc_lib.gfc_destroy(None) == 0
    h = ctypes.c_void_p()
    assert gfc_lib.gfc_plan_create(ctypes.byref(h), 1, 10, 1, 1, 0) == 1
    assert gfc_lib.gfc_plan_create(ctypes.byref(h), 10, 10, 0, 1, 0) == 1
    assert gfc_lib.gfc_plan_create(ctypes.byref(h), 10, 10, 1, 1, 9) == 1
    assert h.value is None


def test_fft_entry_validates_before_launch(gfc_lib):
    fake = ctypes.c_void_p(1 << 20)
    assert gfc_lib.gfc_fft_c2c(11, 1, -1, fake, fake, None) == 2      # 11 is not 7-smooth
    assert gfc_lib.gfc_fft_c2c(8192, 1, -1, fake, fake, None) == 2    # too long
    assert gfc_lib.gfc_fft_c2c(8, 1, 0, fake, fake, None) == 1        # bad direction
    assert gfc_lib.gfc_fft_c2c(8, 0, -1, fake, fake, None) == 0       # nothing to do


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_plan_create_without_gpu_reports_cuda_error(gfc_lib):
    h = ctypes.c_void_p()
    st = gfc_lib.gfc_plan_create(ctypes.byref(h), 64, 96, 1, 1, 0)
    assert st in (3, 4)
    assert gfc_lib.gfc_last_error() != b""


def test_exact_size_policy(gfc_lib):
    # Algorithm A's own size: image plus the pad on both sides, any factors
    assert gfc.padded_size(801, 1200, exact=True) == (809, 1208)
    assert gfc.padded_size(23, 29, exact=True) == (31, 37)
    assert gfc.padded_size(10, 17, pad=2, exact=True) == (14, 21)
    with pytest.raises(gfc.GFCError):
        gfc.padded_size(2041, 10, exact=True)  # Bluestein length would exceed the engine's 4096
