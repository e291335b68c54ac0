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


def test_noalloc_rejects_sizes_beyond_its_static_scratch(gfc_lib):
    x = torch.zeros((1, 1, 16, 16), device=DEV)
    st = gfc_lib.gfc_solve_from_gradient_noalloc(2040, 2100, 1, x.data_ptr(), x.data_ptr() + 1024,
                                                 x.data_ptr() + 2048, None)
    assert st == 2
    assert b"static scratch" in gfc_lib.gfc_last_error()
