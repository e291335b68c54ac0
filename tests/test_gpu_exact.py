"""EXACT size policy (Algorithm A's own padded size, M = H + 2p, N = W + 2p):
parity of the Bluestein/Stockham row DFTs and the recursive column solve with
the oracle run on the same torus, and of the recursive column solve with the
column DFTs (GFC_EXACT_COLUMN_DFT) on the same plan.

The tolerance is the solver's: relative L2 <= 1e-5 in FP32 on image-like
inputs, 2e-3 for 16-bit storage against the oracle on the dequantised inputs.
"""
import numpy as np
import pytest
import torch

import oracle.gfc_oracle as O
from paper_1902_00176_gb300 import gfc, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
REL_F32, REL_16 = 1e-5, 2e-3


@pytest.fixture(autouse=True)
def _lib(gfc_lib):
    yield


def _rel(got, ref):
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV).to(dtype)


def _np(t):
    return t.double().cpu().numpy()


# (H, W): 72x104 (N = 8 x 13 runs Bluestein), 31x37 (both prime), 18x25 (odd,
# 7-smooth: direct), 809x1208 (the paper's 801x1200 image: 809 prime, 1208 = 8 x 151)
@pytest.mark.parametrize("H,W,B", [(64, 96, 2), (23, 29, 3), (10, 17, 2), (801, 1200, 1)])
def test_exact_solve_matches_oracle(H, W, B):
    gx, gy = synth.perturbed_gradient_batch(B, H, W, seed=7000)
    p = gfc.Plan(H, W, 1, B, device=DEV, exact=True)
    assert (p.M, p.N) == (H + 8, W + 8)
    out = _np(p.solve_from_gradient(_dev(gx), _dev(gy)))
    for b in range(B):
        ref = O.solve_from_gradient(gx[b, 0].astype(np.float64), gy[b, 0].astype(np.float64), p.M, p.N, p.pad)
        err = _rel(out[b, 0], ref)
        assert err <= REL_F32, (b, err)
    p.close()


def test_exact_recovers_conservative_image():
    rng = np.random.default_rng(7100)
    img, c = synth.constant_border_image(rng, 41, 53)
    gx, gy = synth.forward_gradient(img)
    p = gfc.Plan(41, 53, device=DEV, exact=True)  # 49 x 61: 7^2 direct, 61 prime
    out = _np(p.solve_from_gradient(_dev(gx[None, None]), _dev(gy[None, None])))[0, 0]
    np.testing.assert_allclose(out, img - c, atol=1e-5)
    p.close()


def test_exact_laplacian_and_bf16():
    gx, gy = synth.perturbed_gradient_batch(2, 30, 44, seed=7200)
    lap = gx + gy  # any field serves as a Laplacian
    p = gfc.Plan(30, 44, 1, 2, device=DEV, exact=True)
    out = _np(p.solve_from_laplacian(_dev(lap)))
    for b in range(2):
        ref = O.solve_from_laplacian(lap[b, 0].astype(np.float64), p.M, p.N, p.pad)
        assert _rel(out[b, 0], ref) <= REL_F32
    p.close()
    q = gfc.Plan(30, 44, 1, 2, dtype=torch.bfloat16, device=DEV, exact=True)
    dx, dy = _dev(gx, torch.bfloat16), _dev(gy, torch.bfloat16)
    out = _np(q.solve_from_gradient(dx, dy))
    xq, yq = _np(dx), _np(dy)
    for b in range(2):
        ref = O.solve_from_gradient(xq[b, 0], yq[b, 0], q.M, q.N, q.pad)
        assert _rel(out[b, 0], ref) <= REL_16
    q.close()


def test_exact_edited_solve_matches_two_step():
    img, gx, gy, edges = synth.edit_batch(2, 1, 45, 70, seed=7300)
    p = gfc.Plan(45, 70, 1, 2, device=DEV, exact=True)
    dx, dy, de = _dev(gx), _dev(gy), _dev(edges)
    tx, ty = p.gradient_threshold(dx, dy, 0.2)
    assert torch.equal(p.solve_edited(dx, dy, "threshold", frac=0.2), p.solve_from_gradient(tx, ty))
    mx, my = p.gradient_merge(dx, dy, de, 0.5)
    assert torch.equal(p.solve_edited(dx, dy, "merge", alpha=0.5, edges=de), p.solve_from_gradient(mx, my))
    p.close()


def test_exact_against_smooth_sizes():
    """EXACT and SMOOTH solve the same least-squares problem on tori a few pixels
    apart; the gap is reported, not gated (both are checked against the oracle)."""
    gx, gy = synth.perturbed_gradient_batch(1, 801, 1200, seed=7400)
    pe = gfc.Plan(801, 1200, device=DEV, exact=True)
    ps = gfc.Plan(801, 1200, device=DEV)
    oe = _np(pe.solve_from_gradient(_dev(gx), _dev(gy)))
    os_ = _np(ps.solve_from_gradient(_dev(gx), _dev(gy)))
    gap = _rel(oe - oe.mean(), os_ - os_.mean())
    print(f"EXACT {pe.M}x{pe.N} vs SMOOTH {ps.M}x{ps.N}: relative L2 gap {gap:.3e}")
    assert np.isfinite(gap)
    pe.close()
    ps.close()


def _torch_fp32_adjoint(gout, M, N, p):
    """The adjoint in plain PyTorch FP32 (rfft2 / irfft2 on the same torus): the
    FP32 baseline error for white-noise upstream gradients."""
    H, W = gout.shape
    G = torch.from_numpy(O.green_spectrum(M, N)[:, : N // 2 + 1]).float().to(DEV)
    z = torch.zeros((M, N), device=DEV)
    g = torch.from_numpy(np.ascontiguousarray(gout)).float().to(DEV)
    z[p:p + H, p:p + W] = g
    z[0, 0] -= g.sum()
    w = torch.fft.irfft2(torch.fft.rfft2(z) * G, s=(M, N))
    gx = (w - torch.roll(w, -1, -1))[p:p + H, p:p + W]
    gy = (w - torch.roll(w, -1, -2))[p:p + H, p:p + W]
    return gx.double().cpu().numpy(), gy.double().cpu().numpy()


# 72x104 (Bluestein along rows), 31x37 (both prime), 18x25 (direct), 809x1208
@pytest.mark.parametrize("H,W,B", [(64, 96, 2), (23, 29, 3), (10, 17, 1), (801, 1200, 1)])
def test_exact_backward_matches_oracle(H, W, B):
    """The adjoint on Algorithm A's own torus against the oracle's transpose,
    bounded like the other white-noise adjoint checks."""
    gout = synth.upstream_gradient((B, 1, H, W), seed=7500 + H)
    p = gfc.Plan(H, W, 1, B, device=DEV, exact=True)
    bx, by = p.backward(_dev(gout))
    bx, by = _np(bx), _np(by)
    for b in range(B):
        g0 = gout[b, 0].astype(np.float64)
        rx, ry = O.backward(g0, p.M, p.N, p.pad)
        tx, ty = _torch_fp32_adjoint(gout[b, 0], p.M, p.N, p.pad)
        assert _rel(bx[b, 0], rx) <= max(REL_F32, 3.0 * _rel(tx, rx)), (b, _rel(bx[b, 0], rx), _rel(tx, rx))
        assert _rel(by[b, 0], ry) <= max(REL_F32, 3.0 * _rel(ty, ry)), (b, _rel(by[b, 0], ry), _rel(ty, ry))
    p.close()


def test_exact_backward_is_the_transpose_and_bf16():
    """<solve(gx, gy), g> = <(gx, gy), backward(g)> on the EXACT torus (the
    forward is linear), and BF16 storage against the oracle on the dequantised
    upstream gradient."""
    H, W = 30, 44
    gx, gy = synth.perturbed_gradient_batch(1, H, W, seed=7600)
    g = synth.upstream_gradient((1, 1, H, W), seed=7601)
    p = gfc.Plan(H, W, device=DEV, exact=True)
    y = _np(p.solve_from_gradient(_dev(gx), _dev(gy)))
    bx, by = p.backward(_dev(g))
    lhs = float((y * g).sum())
    rhs = float((gx * _np(bx)).sum() + (gy * _np(by)).sum())
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs) + 1.0), (lhs, rhs)
    p.close()
    q = gfc.Plan(H, W, dtype=torch.bfloat16, device=DEV, exact=True)
    dg = _dev(g, torch.bfloat16)
    qx, qy = q.backward(dg)
    rx, ry = O.backward(_np(dg)[0, 0], q.M, q.N, q.pad)
    assert _rel(_np(qx)[0, 0], rx) <= REL_16 and _rel(_np(qy)[0, 0], ry) <= REL_16
    q.close()


@pytest.mark.parametrize("H,W,B", [(801, 1200, 3), (23, 29, 3), (64, 96, 2)])
def test_exact_recursive_columns_match_column_dfts(H, W, B, monkeypatch):
    """The column direction by the recursive column solve (in place on the
    row-major pair tori, column 0 exactly in FP64) against the Bluestein column
    DFTs with the Green multiply, for the solve and the adjoint; odd B leaves
    the last pair torus half empty."""
    gx, gy = synth.perturbed_gradient_batch(B, H, W, seed=7300)
    g = (gx + 0.5 * gy).astype(np.float32)  # an image-like upstream gradient
    p = gfc.Plan(H, W, 1, B, device=DEV, exact=True)
    a = _np(p.solve_from_gradient(_dev(gx), _dev(gy)))
    ax, ay = (_np(t) for t in p.backward(_dev(g)))
    monkeypatch.setenv("GFC_EXACT_COLUMN_DFT", "1")
    b = _np(p.solve_from_gradient(_dev(gx), _dev(gy)))
    bx, by = (_np(t) for t in p.backward(_dev(g)))
    monkeypatch.delenv("GFC_EXACT_COLUMN_DFT")
    assert _rel(a, b) <= 2e-6, _rel(a, b)
    ref = O.solve_from_gradient(gx[B - 1, 0].astype(np.float64), gy[B - 1, 0].astype(np.float64), p.M, p.N, p.pad)
    assert _rel(a[B - 1, 0], ref) <= REL_F32
    # the adjoint against the FP64 oracle: its output is large and dominated by
    # the lowest Green bins, so both column methods are held to 3x the error of a
    # plain torch FP32 evaluation, like every large adjoint
    rx, ry = O.backward(g[0, 0].astype(np.float64), p.M, p.N, p.pad)
    tx, ty = _torch_fp32_adjoint(g[0, 0], p.M, p.N, p.pad)
    bar_x, bar_y = max(REL_F32, 3.0 * _rel(tx, rx)), max(REL_F32, 3.0 * _rel(ty, ry))
    for ox, oy in ((ax, ay), (bx, by)):
        assert _rel(ox[0, 0], rx) <= bar_x and _rel(oy[0, 0], ry) <= bar_y, (_rel(ox[0, 0], rx), bar_x,
                                                                           _rel(oy[0, 0], ry), bar_y)
    p.close()


@pytest.mark.parametrize("H,W,B", [(801, 1200, 3), (37, 1195, 2)])
def test_exact_register_rows_match_generic_rows(H, W, B, monkeypatch):
    """Rows whose Bluestein length is 2430 (n = 1208 and 1203 here) run on the
    register schedule 45 x 54; the shared-memory engine on the same plan
    (GFC_EXACT_GENERIC_ROWS) agrees within FP32 rounding for the solve, and
    both adjoints are held to the oracle with the bar of a large FP32 adjoint."""
    gx, gy = synth.perturbed_gradient_batch(B, H, W, seed=7600)
    g = (gx + 0.5 * gy).astype(np.float32)
    p = gfc.Plan(H, W, 1, B, device=DEV, exact=True)
    assert p.N == W + 8
    a = _np(p.solve_from_gradient(_dev(gx), _dev(gy)))
    ax, ay = (_np(t) for t in p.backward(_dev(g)))
    monkeypatch.setenv("GFC_EXACT_GENERIC_ROWS", "1")
    b = _np(p.solve_from_gradient(_dev(gx), _dev(gy)))
    bx, by = (_np(t) for t in p.backward(_dev(g)))
    monkeypatch.delenv("GFC_EXACT_GENERIC_ROWS")
    assert _rel(a, b) <= 5e-6, _rel(a, b)  # two FP32 evaluations of the same transforms
    for f in range(B):
        ref = O.solve_from_gradient(gx[f, 0].astype(np.float64), gy[f, 0].astype(np.float64), p.M, p.N, p.pad)
        assert _rel(a[f, 0], ref) <= REL_F32 and _rel(b[f, 0], ref) <= REL_F32, (f, _rel(a[f, 0], ref),
                                                                                 _rel(b[f, 0], ref))
    rx, ry = O.backward(g[0, 0].astype(np.float64), p.M, p.N, p.pad)
    tx, ty = _torch_fp32_adjoint(g[0, 0], p.M, p.N, p.pad)
    bar_x, bar_y = max(REL_F32, 3.0 * _rel(tx, rx)), max(REL_F32, 3.0 * _rel(ty, ry))
    for ox, oy in ((ax, ay), (bx, by)):
        assert _rel(ox[0, 0], rx) <= bar_x and _rel(oy[0, 0], ry) <= bar_y, (_rel(ox[0, 0], rx), bar_x,
                                                                           _rel(oy[0, 0], ry), bar_y)
    p.close()
