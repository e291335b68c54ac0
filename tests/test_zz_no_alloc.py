"""The allocation-free entry point gives the same answer as the plan-based one.

``gfc_solve_from_gradient_noalloc`` exists for callers that are not allowed
to allocate device memory (plug-ins inside an application that owns all GPU
memory, pipelines with a fixed memory budget, latency-bound loops that cannot
afford cudaMalloc's implicit device synchronisation). It works out of one
static device array owned by the library, which every call reuses. This file
is collected last so that, if it fails, a run stopping at the first failure
has already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle.gfc_oracle as O
from paper_1902_00176_gb300 import gfc, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
REL_F32, MAXABS_F32 = 1e-5, 1e-4


def _noalloc(lib, gx, gy, out):
    B, C, H, W = gx.shape
    st = lib.gfc_solve_from_gradient_noalloc(H, W, B * C, gx.data_ptr(), gy.data_ptr(), out.data_ptr(),
                                             ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream))
    assert st == 0, lib.gfc_last_error()
    return out


@pytest.mark.parametrize("B,H,W", [(3, 64, 96), (2, 801, 1200)])
def test_noalloc_matches_plan_entry_on_two_calls_in_a_row(gfc_lib, B, H, W):
    plan = gfc.Plan(H, W, 1, B, device=DEV)
    for call, seed in enumerate((11, 12)):  # two calls in a row, different inputs
        gx, gy = synth.perturbed_gradient_batch(batch=B, H=H, W=W, seed=seed * 1000)
        tx = torch.from_numpy(gx).to(DEV)
        ty = torch.from_numpy(gy).to(DEV)
        ref = plan.solve_from_gradient(tx, ty).double().cpu().numpy()
        out = torch.full_like(tx, float("nan"))
        got = _noalloc(gfc_lib, tx, ty, out)
        torch.cuda.synchronize()
        got = got.double().cpu().numpy()
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= REL_F32, (call, rel)
        assert np.abs(got - ref).max() <= MAXABS_F32, call
    plan.close()


def test_noalloc_python_wrapper_matches_oracle(gfc_lib):
    """Through gfc.solve_noalloc (with its input checks) against the FP64 oracle."""
    _, gx, gy = synth.gradient_removal_image(seed=0, H=64, W=96)
    tx = torch.from_numpy(gx).to(DEV).view(1, 1, 64, 96)
    ty = torch.from_numpy(gy).to(DEV).view(1, 1, 64, 96)
    out = torch.full_like(tx, float("nan"))
    gfc.solve_noalloc(tx, ty, out)
    torch.cuda.synchronize()
    M, N = gfc.padded_size(64, 96)
    ref = O.solve_from_gradient(gx.astype(np.float64), gy.astype(np.float64), M, N, 4)
    got = out.double().cpu().numpy()[0, 0]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= REL_F32
    assert np.abs(got - ref).max() <= MAXABS_F32
    with pytest.raises(ValueError):
        gfc.solve_noalloc(tx, ty, out.double())
    with pytest.raises(ValueError):
        gfc.solve_noalloc(tx, ty.cpu(), out)


def test_noalloc_near_the_static_limit_matches_plan_entry(gfc_lib):
    """A padded size close to the 2^21-element limit (2000 x 2000 -> 2016 x 2016,
    M x ldS = 2016 x 1012), routed to the generic passes by the plan as well."""
    H = W = 2000
    M, N = gfc.padded_size(H, W)
    ldS = (N // 2 + 1 + 3) // 4 * 4
    assert M * ldS <= 1 << 21 and M * ldS > 0.9 * (1 << 21)
    gx, gy = synth.perturbed_gradient_batch(batch=1, H=H, W=W, seed=31000)
    tx = torch.from_numpy(gx).to(DEV)
    ty = torch.from_numpy(gy).to(DEV)
    plan = gfc.Plan(H, W, 1, 1, device=DEV)
    ref = plan.solve_from_gradient(tx, ty).double().cpu().numpy()
    plan.close()
    for _ in range(2):
        out = torch.full_like(tx, float("nan"))
        got = _noalloc(gfc_lib, tx, ty, out)
        torch.cuda.synchronize()
        got = got.double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= REL_F32
        assert np.abs(got - ref).max() <= MAXABS_F32


def test_noalloc_rejects_sizes_beyond_its_static_scratch(gfc_lib):
    # buffers that really hold the declared 2040 x 2100 field, so the call stays
    # memory-safe whatever the static limit is
    H, W = 2040, 2100
    x = torch.zeros((1, 1, H, W), device=DEV)
    y = torch.zeros_like(x)
    o = torch.zeros_like(x)
    st = gfc_lib.gfc_solve_from_gradient_noalloc(H, W, 1, x.data_ptr(), y.data_ptr(), o.data_ptr(), None)
    assert st == 2
    assert b"static scratch" in gfc_lib.gfc_last_error()
    torch.cuda.synchronize()
    assert not bool(o.any())  # nothing was launched
