"""The one-launch solve for small tori against the FP64 oracle and against the
three-launch path of the same plan.

Where a field's row-major spectrum fits the shared memory of a thread-block
cluster (short rows), a plain solve from gradients runs as one kernel: every
CTA of the field's cluster transforms its bands of rows, keeps them in shared
memory, folds all bands' sums (read from the other CTAs through distributed
shared memory) into its carries and u[0,0], solves its bands and writes the
output. The cases cover the 270 x 270 and 72 x 108 tori in FP32 and 16-bit
storage, one field (clusters spread to cover the SMs) and many, image heights
that leave a band with no image row, and short row lengths of the compiled
family. The library takes the fused solve for launches whose CTAs are all
resident at once (latency-bound batches); GFC_FUSED_SMALL=1 takes it whenever
it applies, GFC_UNFUSED_SMALL=1 forces the three-launch path on the same plan.
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


def _launches(p, fn):
    p.set_profiling(True)
    p.profile(reset=True)
    out = fn()
    pr = p.profile(reset=True)
    p.set_profiling(False)
    return out, [int(x) for x in pr["launches"]]


# (H, W, dtype, fields): the 270 x 270 torus of 256 x 256 feature maps in BF16,
# FP16 and FP32; the 72 x 108 torus of a 64 x 96 image (one field, and five);
# 63 x 100 (72 x 108 torus, a band clipped at the torus end); 256 x 256 with
# many fields; row-family lengths 252, 320 and 400 (FP32)
CASES = [(256, 256, torch.bfloat16, 6), (256, 256, torch.float16, 3), (256, 256, torch.float32, 2),
         (64, 96, torch.float32, 1), (64, 96, torch.float32, 5), (63, 100, torch.float32, 3),
         (256, 256, torch.float32, 64), (240, 244, torch.float32, 2), (300, 308, torch.float32, 2),
         (380, 388, torch.float32, 1)]


@pytest.mark.parametrize("H,W,dt,B", CASES)
def test_fused_small_matches_oracle_and_three_launch_path(H, W, dt, B, monkeypatch):
    monkeypatch.setenv("GFC_FUSED_SMALL", "1")
    gx, gy = synth.perturbed_gradient_batch(batch=B, H=H, W=W, seed=12000 + H + B)
    tx = torch.from_numpy(gx).to(DEV).to(dt)
    ty = torch.from_numpy(gy).to(DEV).to(dt)
    p = gfc.Plan(H, W, 1, B, dtype=dt, device=DEV)
    out, launches = _launches(p, lambda: p.solve_from_gradient(tx, ty))
    assert sum(launches) == 1, (p.M, p.N, launches)  # the fused solve ran
    a = _np(out)
    # the same inputs (dequantised for 16-bit storage) through the FP64 oracle
    x64, y64 = _np(tx), _np(ty)
    for f in range(B) if B <= 6 else (0, B // 2, B - 1):
        ref = O.solve_from_gradient(x64[f, 0], y64[f, 0], p.M, p.N, p.pad)
        if dt == torch.float32:
            assert _rel(a[f, 0], ref) <= REL_F32, (f, _rel(a[f, 0], ref))
            assert np.abs(a[f, 0] - ref).max() <= MAXABS_F32, f
        else:
            assert _rel(a[f, 0], ref) <= REL_16, (f, _rel(a[f, 0], ref))
    # deterministic, and the three-launch path of the same plan agrees
    assert torch.equal(out, p.solve_from_gradient(tx, ty))
    monkeypatch.delenv("GFC_FUSED_SMALL")
    monkeypatch.setenv("GFC_UNFUSED_SMALL", "1")
    b, launches3 = _launches(p, lambda: p.solve_from_gradient(tx, ty))
    monkeypatch.delenv("GFC_UNFUSED_SMALL")
    assert sum(launches3) >= 3, launches3
    # the same arithmetic in the same order (the carries' recurrences and the
    # u[0,0] sum follow the carry sweep's), so the same bits
    assert torch.equal(out, b), _rel(a, _np(b))
    p.close()


def test_fused_small_chunked_streams_and_layer_shape(monkeypatch):
    """The layer's shape (4 x 64 channels of 256 x 256, BF16) split into chunks on
    several streams, against one chunk: the last chunk's 16 fields spread over
    clusters of a different size, and the result does not change."""
    monkeypatch.setenv("GFC_FUSED_SMALL", "1")
    B, C, H, W = 4, 64, 256, 256
    fx, fy = synth.feature_gradients(batch=B, C=C, H=H, W=W, seed=12500)
    gx = torch.from_numpy(fx).to(DEV).to(torch.bfloat16)
    gy = torch.from_numpy(fy).to(DEV).to(torch.bfloat16)
    one = gfc.Plan(H, W, C, B, dtype=torch.bfloat16, device=DEV)
    split = gfc.Plan(H, W, C, B, dtype=torch.bfloat16, device=DEV, chunk=48, streams=3)
    a = one.solve_from_gradient(gx, gy)
    b = split.solve_from_gradient(gx, gy)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    ref = O.solve_from_gradient(_np(gx)[3, 63], _np(gy)[3, 63], one.M, one.N, one.pad)
    assert _rel(_np(a)[3, 63], ref) <= REL_16
    one.close()
    split.close()


def test_fused_small_taken_for_latency_bound_launches_only():
    """The default takes the fused solve where each CTA of a field's cluster holds
    one band (tori of at most 8 bands) and the launch is latency-bound: one and
    64 fields of 64 x 96 (72 x 108 torus, 4 bands) run as one launch; 76 fields
    (every CTA slot of the GPU) and a 270 x 270 torus (19 bands, 3 per CTA)
    run the three launches, which measured faster there."""
    def launches(H, W, B, dt=torch.float32):
        x = torch.zeros((B, 1, H, W), device=DEV, dtype=dt)
        p = gfc.Plan(H, W, 1, B, dtype=dt, device=DEV)
        _, n = _launches(p, lambda: p.solve_from_gradient(x, x))
        p.close()
        return sum(n)
    assert launches(64, 96, 1) == 1
    assert launches(64, 96, 64) == 1
    assert launches(64, 96, 76) >= 3
    assert launches(256, 256, 1, torch.bfloat16) >= 3
    assert launches(256, 256, 2048, torch.bfloat16) >= 3
