"""Parity of the editing kernels (through the C ABI) with the editing oracle.

Integer outcomes are compared exactly: the keep/drop decisions of the gradient
threshold are taken in FP32 on both sides, so the thresholded gradients must
match bit for bit. Floating-point results use the solver's tolerances:
relative L2 <= 1e-5 in FP32, <= 2e-3 for 16-bit storage against the oracle run
on the dequantised inputs.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1902_00176_gb300 import gfc, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
REL_F32, REL_16 = 1e-5, 2e-3
DT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}


@pytest.fixture(autouse=True)
def _lib(gfc_lib):
    yield


def _rel(got, ref):
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV).to(dtype)


def _np(t):
    return t.double().cpu().numpy()


def _deq(a, dtype):
    """The values a 16-bit (or FP32) tensor of ``a`` holds, as float64."""
    return _np(_dev(a, dtype))


# ---- statistics and colour correction (Eq. 25) ------------------------------------

@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("shape", [(3, 2, 64, 96), (2, 1, 801, 1200), (1, 3, 17, 5)])
def test_field_stats(shape, dt):
    img = synth.edit_batch(shape[0], shape[1], shape[2], shape[3], seed=5100)[0]
    x = _dev(img, DT[dt])
    p = gfc.Plan(shape[2], shape[3], C=shape[1], batch=shape[0], dtype=DT[dt], device=DEV)
    m, s = p.field_stats(x)
    m2, s2 = p.field_stats(x)
    torch.cuda.synchronize()
    assert torch.equal(m, m2) and torch.equal(s, s2)  # fixed reduction order
    rm, rs = oracle.field_stats_batch(_np(x))
    m, s = _np(m), _np(s)
    assert np.abs(m - rm).max() <= 1e-6 * (np.abs(rm).max() + rs.max())
    assert np.abs(s - rs).max() <= 1e-5 * rs.max()
    p.close()


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_color_correct_unit(dt):
    # a field with its own offset and contrast, corrected to another image's statistics
    img = synth.edit_batch(2, 3, 40, 56, seed=5200)[0]
    rng = np.random.default_rng(5201)
    X = (3.0 * synth.edit_batch(2, 3, 40, 56, seed=5202)[0] - 1.0 + rng.uniform(-0.5, 0.5, (2, 3, 1, 1)))
    p = gfc.Plan(40, 56, C=3, batch=2, dtype=DT[dt], device=DEV)
    ref_mean, ref_std = p.field_stats(_dev(img, DT[dt]))
    x = _dev(X, DT[dt])
    xin = _np(x)
    p.color_correct(x, ref_mean, ref_std)
    imq = _deq(img, DT[dt])
    want = np.stack([oracle.color_correct(a, b) for a, b in zip(xin.reshape(-1, 40, 56), imq.reshape(-1, 40, 56))])
    err = _rel(_np(x).reshape(want.shape), want)
    assert err <= (REL_F32 if dt == "f32" else REL_16), err
    p.close()


def test_color_correct_constant_field():
    p = gfc.Plan(16, 24, C=2, batch=1, device=DEV)
    x = torch.full((1, 2, 16, 24), 0.75, device=DEV)
    ref_mean = torch.tensor([[0.2, -3.0]], device=DEV)
    ref_std = torch.tensor([[0.1, 2.0]], device=DEV)
    p.color_correct(x, ref_mean, ref_std)
    got = x.cpu()
    assert torch.all(got[0, 0] == 0.2) and torch.all(got[0, 1] == -3.0)
    p.close()


@pytest.mark.parametrize("H,W,C,B", [(64, 96, 3, 2), (801, 1200, 1, 1)])
def test_threshold_solve_correct_pipeline(H, W, C, B):
    """The editing flow of Sec. 3.2.3: threshold at 10%, solve (Eq. 23), correct (Eq. 25)."""
    img, gx, gy, _ = synth.edit_batch(B, C, H, W, seed=5300)
    p = gfc.Plan(H, W, C=C, batch=B, device=DEV)
    tx, ty = p.gradient_threshold(_dev(gx), _dev(gy), 0.1)
    out = p.solve_from_gradient(tx, ty)
    m, s = p.field_stats(_dev(img))
    p.color_correct(out, m, s)
    ox, oy = oracle.gradient_threshold_batch(gx, gy, 0.1)
    ref = np.empty((B, C, H, W))
    for b in range(B):
        for c in range(C):
            ic = oracle.solve_from_gradient(ox[b, c].astype(np.float64), oy[b, c].astype(np.float64), p.M, p.N, p.pad)
            ref[b, c] = oracle.color_correct(ic, img[b, c])
    assert np.array_equal(_np(tx), ox) and np.array_equal(_np(ty), oy)
    err = _rel(_np(out), ref)
    assert err <= REL_F32, err
    p.close()


# ---- thresholding -------------------------------------------------------------------

@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("frac,ref", [(0.1, 0.0), (0.3, 0.0), (0.5, 0.0), (0.3, 1.0), (0.0, 0.0), (1.0, 0.0)])
def test_threshold_bit_exact(frac, ref, dt):
    _, gx, gy, _ = synth.edit_batch(2, 2, 72, 100, seed=5400)
    p = gfc.Plan(72, 100, C=2, batch=2, dtype=DT[dt], device=DEV)
    dx, dy = _dev(gx, DT[dt]), _dev(gy, DT[dt])
    ox, oy = p.gradient_threshold(dx, dy, frac, ref)
    wx, wy = oracle.gradient_threshold_batch(_np(dx).astype(np.float32), _np(dy).astype(np.float32), frac,
                                             ref if ref > 0 else None)
    assert np.array_equal(_np(ox), wx) and np.array_equal(_np(oy), wy)
    # in place gives the same
    p.gradient_threshold(dx, dy, frac, ref, gx_out=dx, gy_out=dy)
    assert torch.equal(dx, ox) and torch.equal(dy, oy)
    p.close()


def test_threshold_full_size():
    _, gx, gy, _ = synth.edit_batch(1, 3, 801, 1200, seed=5500)
    p = gfc.Plan(801, 1200, C=3, batch=1, device=DEV)
    ox, oy = p.gradient_threshold(_dev(gx), _dev(gy), 0.3)
    wx, wy = oracle.gradient_threshold_batch(gx, gy, 0.3)
    assert np.array_equal(_np(ox), wx) and np.array_equal(_np(oy), wy)
    kept = float((wx != 0).mean())
    assert 0.0 < kept < 1.0
    p.close()


# ---- gradient-domain merging (Eq. 26) -------------------------------------------------

@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("alpha", [0.0, 0.25, 0.5, 1.0])
def test_merge(alpha, dt):
    _, gx, gy, edges = synth.edit_batch(2, 2, 64, 80, seed=5600)
    p = gfc.Plan(64, 80, C=2, batch=2, dtype=DT[dt], device=DEV)
    dx, dy, de = _dev(gx, DT[dt]), _dev(gy, DT[dt]), _dev(edges, DT[dt])
    ox, oy = p.gradient_merge(dx, dy, de, alpha)
    wx, wy = oracle.gradient_merge_batch(_np(dx), _np(dy), _np(de), alpha)
    if alpha == 0.0:
        assert torch.equal(ox, dx) and torch.equal(oy, dy)
    tol = REL_F32 if dt == "f32" else REL_16
    ex, ey = _rel(_np(ox), wx), _rel(_np(oy), wy)
    assert ex <= tol and ey <= tol, (ex, ey)
    # no orientation where |E| = 0 (the replicate border): exactly 0
    zero = (wx == 0) & (wy == 0)
    assert not _np(ox)[zero].any() and not _np(oy)[zero].any()
    p.close()


def test_merge_then_solve_full_size():
    img, gx, gy, edges = synth.edit_batch(1, 1, 801, 1200, seed=5700)
    p = gfc.Plan(801, 1200, C=1, batch=1, device=DEV)
    mx, my = p.gradient_merge(_dev(gx), _dev(gy), _dev(edges), 0.5)
    out = p.solve_from_gradient(mx, my)
    m, s = p.field_stats(_dev(img))
    p.color_correct(out, m, s)
    wx, wy = oracle.gradient_merge(gx[0, 0], gy[0, 0], edges[0, 0], 0.5)
    ref = oracle.color_correct(oracle.solve_from_gradient(wx, wy, p.M, p.N, p.pad), img[0, 0])
    err = _rel(_np(out)[0, 0], ref)
    assert err <= REL_F32, err
    p.close()


# ---- boundary-preserving offset (Sec. 2.3.2) ------------------------------------------

@pytest.mark.parametrize("H,W,ring", [(70, 102, 3), (807, 1206, 3), (20, 30, 1), (33, 47, 5)])
def test_boundary_offset(H, W, ring):
    B = 2 if H < 100 else 1
    img, gx, gy = synth.ring_padded_batch(B, 1, H, W, ring=ring, seed=5800)
    p = gfc.Plan(H, W, C=1, batch=B, device=DEV)
    out = p.solve_from_gradient(_dev(gx), _dev(gy))
    inner = p.boundary_offset(out, ring)
    again = p.boundary_offset(out, ring)
    assert torch.equal(inner, again)
    for b in range(B):
        u = oracle.solve_from_gradient(gx[b, 0].astype(np.float64), gy[b, 0].astype(np.float64), p.M, p.N, p.pad)
        ref = oracle.boundary_offset(u, ring)
        err = _rel(_np(inner)[b, 0], ref)
        assert err <= REL_F32, err
    p.close()


def test_boundary_offset_bf16_and_errors():
    img, gx, gy = synth.ring_padded_batch(2, 2, 40, 52, ring=3, seed=5900)
    p = gfc.Plan(40, 52, C=2, batch=2, dtype=torch.bfloat16, device=DEV)
    dx, dy = _dev(gx, torch.bfloat16), _dev(gy, torch.bfloat16)
    out = p.solve_from_gradient(dx, dy)
    inner = p.boundary_offset(out, 3)
    xq, yq = _np(dx), _np(dy)
    for b in range(2):
        for c in range(2):
            u = oracle.solve_from_gradient(xq[b, c], yq[b, c], p.M, p.N, p.pad)
            ref = oracle.boundary_offset(u, 3)
            # two 16-bit roundings: of the solved field (relative to its own
            # size, before the ring offset) and of the result
            tol = REL_16 * (1.0 + np.linalg.norm(u[3:-3, 3:-3]) / np.linalg.norm(ref))
            err = _rel(_np(inner)[b, c], ref)
            assert err <= tol, (err, tol)
    for bad in (0, 20, 26):
        with pytest.raises((gfc.GFCError, ValueError, RuntimeError)):
            p.boundary_offset(out, bad)
    p.close()


def test_edit_calls_reject_ragged_plans():
    rp = gfc.RaggedPlan([(1, 32, 48), (2, 40, 40)], device=DEV)
    st = gfc.lib().gfc_field_stats(rp._h, None, None, None)
    assert st == 2  # GFC_ERR_UNSUPPORTED
    rp.close()


# ---- edits fused into the solve's first pass -----------------------------------------

@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("H,W,C,B", [(64, 96, 2, 2), (40, 56, 1, 3), (801, 1200, 1, 2)])
def test_solve_edited_matches_two_step(H, W, C, B, dt):
    """The fused edit gives the same bits as the standalone edit followed by a solve,
    on the register-resident path (64x96, 801x1200) and the generic one (40x56)."""
    img, gx, gy, edges = synth.edit_batch(B, C, H, W, seed=6100)
    p = gfc.Plan(H, W, C=C, batch=B, dtype=DT[dt], device=DEV)
    dx, dy, de = _dev(gx, DT[dt]), _dev(gy, DT[dt]), _dev(edges, DT[dt])
    for frac, ref in ((0.1, 0.0), (0.3, 1.0)):
        tx, ty = p.gradient_threshold(dx, dy, frac, ref)
        two = p.solve_from_gradient(tx, ty)
        one = p.solve_edited(dx, dy, "threshold", frac=frac, ref=ref)
        assert torch.equal(one, two), (frac, ref)
    mx, my = p.gradient_merge(dx, dy, de, 0.5)
    two = p.solve_from_gradient(mx, my)
    one = p.solve_edited(dx, dy, "merge", alpha=0.5, edges=de)
    assert torch.equal(one, two)
    plain = p.solve_from_gradient(dx, dy)
    assert torch.equal(p.solve_edited(dx, dy, "none"), plain)
    p.close()


def test_solve_edited_against_oracle():
    img, gx, gy, edges = synth.edit_batch(2, 1, 64, 96, seed=6200)
    p = gfc.Plan(64, 96, C=1, batch=2, device=DEV)
    out_t = p.solve_edited(_dev(gx), _dev(gy), "threshold", frac=0.3)
    out_m = p.solve_edited(_dev(gx), _dev(gy), "merge", alpha=0.5, edges=_dev(edges))
    tx, ty = oracle.gradient_threshold_batch(gx, gy, 0.3)
    for b in range(2):
        ref = oracle.solve_from_gradient(tx[b, 0].astype(np.float64), ty[b, 0].astype(np.float64), p.M, p.N, p.pad)
        assert _rel(_np(out_t)[b, 0], ref) <= REL_F32
        mx, my = oracle.gradient_merge(gx[b, 0], gy[b, 0], edges[b, 0], 0.5)
        ref = oracle.solve_from_gradient(mx, my, p.M, p.N, p.pad)
        assert _rel(_np(out_m)[b, 0], ref) <= REL_F32
    p.close()


def test_solve_edited_rejects_bad_edits():
    p = gfc.Plan(32, 48, device=DEV)
    x = torch.zeros((1, 1, 32, 48), device=DEV)
    with pytest.raises(gfc.GFCError):
        p.solve_edited(x, x.clone(), "merge", alpha=1.5, edges=x.clone())
    e = gfc._Edit(7, 0.1, 0.0, 0.5, None)
    out = torch.empty_like(x)
    st = gfc.lib().gfc_solve_edited(p._h, x.data_ptr(), x.data_ptr(), gfc.ctypes.byref(e), out.data_ptr())
    assert st == 1  # GFC_ERR_INVALID_ARG
    e = gfc._Edit(2, 0.0, 0.0, 0.5, None)  # merge without an edge map
    st = gfc.lib().gfc_solve_edited(p._h, x.data_ptr(), x.data_ptr(), gfc.ctypes.byref(e), out.data_ptr())
    assert st == 1
    p.close()


# ---- the editing flow in one call: edit, solve, colour-correct (Eq. 25 fused) ---------

@pytest.mark.parametrize("edit", ["none", "threshold", "merge"])
@pytest.mark.parametrize("H,W,C,B,dt", [(801, 1200, 1, 3, "f32"), (64, 96, 3, 2, "f32"), (256, 256, 2, 2, "bf16")])
def test_solve_corrected_matches_two_step_and_oracle(H, W, C, B, dt, edit):
    """gfc_solve_corrected (statistics taken as the last pass stores the field) against
    the solve followed by gfc_color_correct, and against the oracle's flow."""
    img, gx, gy, edges = synth.edit_batch(B, C, H, W, seed=6300)
    p = gfc.Plan(H, W, C=C, batch=B, dtype=DT[dt], device=DEV)
    dx, dy, de = _dev(gx, DT[dt]), _dev(gy, DT[dt]), _dev(edges, DT[dt])
    m, s = p.field_stats(_dev(img, DT[dt]))
    kw = {"none": {}, "threshold": dict(frac=0.1), "merge": dict(alpha=0.5, edges=de)}[edit]
    one = p.solve_corrected(dx, dy, m, s, edit=edit, **kw)
    two = p.solve_edited(dx, dy, edit, **kw)
    p.color_correct(two, m, s)
    tol = REL_F32 if dt == "f32" else REL_16
    assert _rel(_np(one), _np(two)) <= (1e-6 if dt == "f32" else tol)
    again = p.solve_corrected(dx, dy, m, s, edit=edit, **kw)
    assert torch.equal(one, again)  # fixed reduction order
    if dt != "f32" and edit == "merge":
        p.close()  # 16-bit merge rounds the merged gradient to storage first: two-step parity only
        return
    mm, ss = _np(m), _np(s)
    X, Y, E = _np(dx), _np(dy), _np(de)
    for b in range(B):
        for c in range(C):
            ex, ey = X[b, c], Y[b, c]
            if edit == "threshold":
                ex, ey, _ = oracle.gradient_threshold(ex.astype(np.float32), ey.astype(np.float32), 0.1)
            elif edit == "merge":
                ex, ey = oracle.gradient_merge(ex, ey, E[b, c], 0.5)
            ic = oracle.solve_from_gradient(np.asarray(ex, np.float64), np.asarray(ey, np.float64), p.M, p.N, p.pad)
            ref = oracle.color_correct_with(ic, mm.reshape(B, C)[b, c], ss.reshape(B, C)[b, c])
            got = _np(one)[b, c]
            if dt == "f32":
                assert _rel(got, ref) <= REL_F32 and np.abs(got - ref).max() <= 1e-4, (b, c, _rel(got, ref))
            else:
                # rounded to 16 bits twice, by the solve's store and after the correction's
                # gain g = ref_std / std(I_c): the first rounding reaches the result
                # scaled by g (the bound used for every twice-rounded 16-bit result)
                g = ss.reshape(B, C)[b, c] / max(float(np.std(ic)), 1e-300)
                tol = REL_16 * (1.0 + g * np.linalg.norm(ic - ic.mean()) / np.linalg.norm(ref))
                assert _rel(got, ref) <= tol, (b, c, _rel(got, ref), tol)
    p.close()


@pytest.mark.parametrize("kw", [dict(H=40, W=56), dict(H=801, W=1200, column_fft=True)])
def test_solve_corrected_on_other_plans_is_the_two_step_flow(kw):
    """Plans without the recursive column solve (generic sizes, column-FFT plans) run
    the solve and then gfc_color_correct: the same bits as the two calls."""
    B, C = 2, 1
    img, gx, gy, _ = synth.edit_batch(B, C, kw["H"], kw["W"], seed=6400)
    p = gfc.Plan(C=C, batch=B, device=DEV, **kw)
    dx, dy = _dev(gx), _dev(gy)
    m, s = p.field_stats(_dev(img))
    one = p.solve_corrected(dx, dy, m, s, edit="threshold", frac=0.2)
    two = p.solve_edited(dx, dy, "threshold", frac=0.2)
    p.color_correct(two, m, s)
    assert torch.equal(one, two)
    p.close()


def test_solve_corrected_rejects_bad_arguments():
    p = gfc.Plan(32, 48, device=DEV)
    x = torch.zeros((1, 1, 32, 48), device=DEV)
    m = torch.zeros((1, 1), device=DEV)
    e = gfc._Edit(0, 0.0, 0.0, 0.5, None)
    st = gfc.lib().gfc_solve_corrected(p._h, x.data_ptr(), x.data_ptr(), gfc.ctypes.byref(e), None, m.data_ptr(),
                                       torch.empty_like(x).data_ptr())
    assert st == 1
    with pytest.raises(gfc.GFCError):
        p.solve_corrected(x, x.clone(), m, m, edit="merge", alpha=2.0, edges=x.clone())
    p.close()
