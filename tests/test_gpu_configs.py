"""Parity with the FP64 oracle for the workloads the benchmark times, in the
launch configurations it times them.

* the differentiable merging layer: 32 x 64 x 256x256 gradient fields in BF16
  storage (270 x 270 torus, the short-row kernels that run 4 blocks per SM),
  forward, hand-written adjoint and the autograd layer (Sec. 4);
* Poisson blending, 16 x 3 x 1024x1536 (1050 x 1568 torus) in FP32 and with
  FP16 storage (Sec. 3.2.1), every channel of sampled items checked.

16-bit storage is checked against the oracle run on the dequantised 16-bit
inputs (relative L2 <= 2e-3: input quantisation is not counted, output
rounding is); FP32 at relative L2 <= 1e-5 and max-abs <= 1e-4 on data of a
[0, 1] range.
"""
import numpy as np
import pytest
import torch

import oracle.gfc_oracle as O
from paper_1902_00176_gb300 import gfc, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
REL_F32, MAXABS_F32, REL_16 = 1e-5, 1e-4, 2e-3


@pytest.fixture(autouse=True)
def _lib(gfc_lib):
    yield


def _rel(got, ref):
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def _np(t):
    return t.double().cpu().numpy()


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(dtype)


# ---------------------------------------------------------------- layer, BF16 270x270

@pytest.mark.parametrize("C,B", [(3, 2), (8, 1)])
def test_layer_bf16_forward_backward_autograd_match_oracle(C, B):
    """Forward, adjoint and the autograd layer on the 270 x 270 torus in BF16 storage."""
    H = W = 256
    fx, fy = synth.feature_gradients(batch=B, C=C, H=H, W=W, seed=4100 + C)
    tx, ty = _dev(fx, torch.bfloat16), _dev(fy, torch.bfloat16)
    gout = _dev(synth.upstream_gradient((B, C, H, W), seed=4600 + C), torch.bfloat16)
    p = gfc.Plan(H, W, C, B, torch.bfloat16, device=DEV)
    assert (p.M, p.N) == (270, 270)
    out = _np(p.solve_from_gradient(tx, ty))
    ref = O.solve_from_gradient_batch(_np(tx), _np(ty), p.M, p.N, p.pad)
    for b in range(B):
        for c in range(C):
            assert _rel(out[b, c], ref[b, c]) <= REL_16, (b, c)
    bx, by = p.backward(gout)
    rx, ry = O.backward_batch(_np(gout), p.M, p.N, p.pad)
    for b in range(B):
        for c in range(C):
            assert _rel(_np(bx[b, c]), rx[b, c]) <= REL_16, (b, c)
            assert _rel(_np(by[b, c]), ry[b, c]) <= REL_16, (b, c)
    # the autograd layer: forward through GFCFunction, backward through gfc_backward
    lx = tx.clone().requires_grad_(True)
    ly = ty.clone().requires_grad_(True)
    y = gfc.gfc_layer(lx, ly)
    y.backward(gout)
    assert y.dtype == torch.bfloat16 and lx.grad.dtype == torch.bfloat16
    assert _rel(_np(y.detach()), ref) <= REL_16
    assert _rel(_np(lx.grad), rx) <= REL_16 and _rel(_np(ly.grad), ry) <= REL_16
    p.close()


def test_layer_bf16_full_size_sampled_fields_match_oracle():
    """32 x 64 x 256x256 BF16 in one call each way, as the benchmark times it;
    three (item, channel) fields checked in full against the oracle."""
    B, C, H, W = 32, 64, 256, 256
    fx, fy = synth.feature_gradients(batch=B, C=C, H=H, W=W)
    tx, ty = _dev(fx, torch.bfloat16), _dev(fy, torch.bfloat16)
    del fx, fy
    gout = torch.randn((B, C, H, W), generator=torch.Generator(device=DEV).manual_seed(7), device=DEV)
    gout = gout.to(torch.bfloat16)
    p = gfc.Plan(H, W, C, B, torch.bfloat16, device=DEV)
    out = p.solve_from_gradient(tx, ty)
    bx, by = p.backward(gout)
    torch.cuda.synchronize()
    for b, c in ((0, 0), (17, 33), (31, 63)):
        ref = O.solve_from_gradient(_np(tx[b, c]), _np(ty[b, c]), p.M, p.N, p.pad)
        assert _rel(_np(out[b, c]), ref) <= REL_16, (b, c)
        rx, ry = O.backward(_np(gout[b, c]), p.M, p.N, p.pad)
        assert _rel(_np(bx[b, c]), rx) <= REL_16, (b, c)
        assert _rel(_np(by[b, c]), ry) <= REL_16, (b, c)
    p.close()


# ---------------------------------------------------------------- blending, 1050x1568

@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
def test_blend_full_batch_sampled_items_all_channels_match_oracle(dtype):
    """16 x 3 x 1024x1536 in one call, as the benchmark times it; every channel of
    items 0 and 15 checked in full against the oracle."""
    B, C, H, W = 16, 3, 1024, 1536
    gx, gy, _ = synth.poisson_blend_batch(batch=B, C=C, H=H, W=W)
    tx, ty = _dev(gx, dtype), _dev(gy, dtype)
    del gx, gy
    p = gfc.Plan(H, W, C, B, dtype, device=DEV)
    assert (p.M, p.N) == (1050, 1568)
    out = p.solve_from_gradient(tx, ty)
    torch.cuda.synchronize()
    for b in (0, 15):
        for c in range(C):
            ref = O.solve_from_gradient(_np(tx[b, c]), _np(ty[b, c]), p.M, p.N, p.pad)
            got = _np(out[b, c])
            if dtype == torch.float32:
                assert _rel(got, ref) <= REL_F32, (b, c, _rel(got, ref))
                assert np.abs(got - ref).max() <= MAXABS_F32, (b, c)
            else:
                assert _rel(got, ref) <= REL_16, (b, c, _rel(got, ref))
    p.close()
