"""The recursive (tridiagonal) column solve against the FP64 oracle and against
the column-FFT path of the same operator.

After the row transforms, column l of Eq. 23's Green multiply is the inverse of
the cyclic tridiagonal operator S + S^-1 - b_l along the torus rows; the plan's
default applies it by causal and anticausal first-order recursions over bands
of rows, with carries swept around the cycle and column 0 solved exactly. The
sizes below cover every register-resident torus, bands that end before the
torus does (tail rows), a band clipped at the torus end, 16-bit storage, the
Laplacian entry and the edited solves.
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


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(dtype)


# (H, W): 801x1200 (bands reach the torus end), 795x1199 (6 tail rows after the
# last band), 1024x1536, 256x256, 64x96, 60x100 (72x108 torus, a clipped band)
SIZES = [(801, 1200), (795, 1199), (1024, 1536), (256, 256), (64, 96), (60, 100), (802, 1242)]


@pytest.mark.parametrize("H,W", SIZES)
def test_recursive_column_solve_matches_oracle_and_column_fft(H, W):
    B = 2
    gx, gy = synth.perturbed_gradient_batch(batch=B, H=H, W=W, seed=7100 + H)
    tx, ty = _dev(gx), _dev(gy)
    rec = gfc.Plan(H, W, 1, B, device=DEV)
    fft = gfc.Plan(H, W, 1, B, device=DEV, column_fft=True)
    assert (rec.M, rec.N) == (fft.M, fft.N)
    a = _np(rec.solve_from_gradient(tx, ty))
    b = _np(fft.solve_from_gradient(tx, ty))
    for f in range(B):
        ref = O.solve_from_gradient(gx[f, 0].astype(np.float64), gy[f, 0].astype(np.float64), rec.M, rec.N,
                                    rec.pad)
        assert _rel(a[f, 0], ref) <= REL_F32, (f, _rel(a[f, 0], ref))
        assert np.abs(a[f, 0] - ref).max() <= MAXABS_F32, f
    assert _rel(a, b) <= 2e-6, _rel(a, b)
    a2 = _np(rec.solve_from_gradient(tx, ty))
    assert np.array_equal(a, a2)  # deterministic
    rec.close()
    fft.close()


@pytest.mark.parametrize("H,W", [(801, 1200), (256, 256), (64, 96), (795, 1199)])
def test_recursive_column_solve_laplacian_entry(H, W):
    rng = np.random.default_rng(H * 11 + W)
    lap = (rng.standard_normal((2, 1, H, W)) * 0.01).astype(np.float32)
    p = gfc.Plan(H, W, 1, 2, device=DEV)
    out = _np(p.solve_from_laplacian(_dev(lap)))
    for f in range(2):
        ref = O.solve_from_laplacian(lap[f, 0].astype(np.float64), p.M, p.N, p.pad)
        # white-noise Laplacian: the FP32 conditioning limit of white inputs (|G| ~ (M/2pi)^2
        # amplifies round-off in the lowest bins); the column-FFT path is the same-math bar
        q = gfc.Plan(H, W, 1, 2, device=DEV, column_fft=True)
        alt = _np(q.solve_from_laplacian(_dev(lap)))[f, 0]
        q.close()
        assert _rel(out[f, 0], ref) <= max(REL_F32, 3.0 * _rel(alt, ref)), (_rel(out[f, 0], ref), _rel(alt, ref))
    p.close()


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("H,W", [(801, 1200), (256, 256)])
def test_recursive_column_solve_16bit_storage(dtype, H, W):
    gx, gy = synth.perturbed_gradient_batch(batch=1, H=H, W=W, seed=7300)
    tx, ty = _dev(gx, dtype), _dev(gy, dtype)
    p = gfc.Plan(H, W, 1, 1, dtype, device=DEV)
    out = _np(p.solve_from_gradient(tx, ty))[0, 0]
    ref = O.solve_from_gradient(_np(tx)[0, 0], _np(ty)[0, 0], p.M, p.N, p.pad)
    assert _rel(out, ref) <= REL_16
    p.close()


@pytest.mark.parametrize("edit", ["threshold", "merge"])
def test_recursive_column_solve_edited(edit):
    H, W, B = 801, 1200, 2
    img, gx, gy, edges = synth.edit_batch(B, 1, H, W, seed=7400)
    tx, ty, te = _dev(gx), _dev(gy), _dev(edges)
    rec = gfc.Plan(H, W, 1, B, device=DEV)
    fft = gfc.Plan(H, W, 1, B, device=DEV, column_fft=True)
    kw = dict(frac=0.1) if edit == "threshold" else dict(alpha=0.5, edges=te)
    a = _np(rec.solve_edited(tx, ty, edit, **kw))
    b = _np(fft.solve_edited(tx, ty, edit, **kw))
    assert _rel(a, b) <= 2e-6
    rec.close()
    fft.close()


def test_unknown_column_solver_is_rejected():
    import ctypes

    o = gfc._Opts(64, 96, 1, 1, 0, 4, 0, 0, None, 0, 7)
    h = ctypes.c_void_p()
    assert gfc.lib().gfc_plan_create_ex(ctypes.byref(h), ctypes.byref(o)) == 1


def _torch_fp32_adjoint(gout, M, N, p):
    """The adjoint in plain PyTorch FP32 (rfft2 / irfft2): the FP32 baseline error."""
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


def _random_sizes(n=10, seed=9100):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(128, 2049)), int(rng.integers(128, 2049))) for _ in range(n)]


@pytest.mark.parametrize("H,W", _random_sizes())
def test_random_sizes_on_the_row_length_family(H, W, monkeypatch):
    """Ten seeded sizes in [128, 2048]: the row length comes from the compiled family
    (register-resident row passes, recursive column solve); the result matches the
    oracle on the plan's torus and the generic passes on the same torus."""
    gx, gy = synth.ragged_item_gradients((1, H, W), item=H % 97, seed=9200)
    tx, ty = _dev(gx[None]), _dev(gy[None])
    p = gfc.Plan(H, W, 1, 1, device=DEV)
    assert p.N in gfc.row_lengths()
    out = _np(p.solve_from_gradient(tx, ty))[0, 0]
    ref = O.solve_from_gradient(gx[0].astype(np.float64), gy[0].astype(np.float64), p.M, p.N, p.pad)
    assert _rel(out, ref) <= REL_F32, _rel(out, ref)
    assert np.abs(out - ref).max() <= MAXABS_F32
    monkeypatch.setenv("GFC_FORCE_GENERIC", "1")
    q = gfc.Plan(H, W, 1, 1, device=DEV)
    monkeypatch.delenv("GFC_FORCE_GENERIC")
    assert (q.M, q.N) == (p.M, p.N)
    assert _rel(out, _np(q.solve_from_gradient(tx, ty))[0, 0]) <= 2e-6
    # the Laplacian entry and the adjoint (generic fallback) on the same plan
    lap = (gx[0] - np.pad(gx[0], ((0, 0), (1, 0)))[:, :-1]) + (gy[0] - np.pad(gy[0], ((1, 0), (0, 0)))[:-1, :])
    lo = _np(p.solve_from_laplacian(_dev(lap[None, None])))[0, 0]
    assert _rel(lo, O.solve_from_laplacian(lap.astype(np.float64), p.M, p.N, p.pad)) <= REL_F32
    # the adjoint (generic passes) of a gradient-shaped upstream field: its output is
    # large and dominated by the lowest bins, the FP32 conditioning limit documented
    # for white inputs; the bar is 3x the error of a plain torch FP32 evaluation
    bx, by = p.backward(_dev(gx[None]))
    rx, ry = O.backward(gx[0].astype(np.float64), p.M, p.N, p.pad)
    tx_, ty_ = _torch_fp32_adjoint(gx[0], p.M, p.N, p.pad)
    assert _rel(_np(bx)[0, 0], rx) <= max(REL_F32, 3.0 * _rel(tx_, rx))
    assert _rel(_np(by)[0, 0], ry) <= max(REL_F32, 3.0 * _rel(ty_, ry))
    p.close()
    q.close()


# (H, W, dtype): the benchmark torus; 800 rows, whose last band holds no row of
# grad_out (only the divergence's extra row); tail rows; 16-bit storage
ADJ_CASES = [(801, 1200, torch.float32), (800, 1200, torch.float32), (795, 1199, torch.float32),
             (256, 256, torch.bfloat16), (64, 96, torch.float16), (60, 100, torch.float32)]


@pytest.mark.parametrize("H,W,dt", ADJ_CASES)
def test_recursive_adjoint_matches_oracle_and_column_fft_adjoint(H, W, dt):
    """The adjoint by the recursive column solve (half-band recursions, the
    -(sum grad_out) e_00 term carried through the sweep and column 0) against
    the FP64 oracle's adjoint and the column-FFT adjoint of the same torus."""
    B = 2
    rng = np.random.default_rng(9300 + H)
    img = np.stack([synth.gaussian_image(rng, H, W, 16, max(2.0, H / 30), max(4.0, H / 4)) for _ in range(B)])
    gout = (img - 0.3)[:, None].astype(np.float32)  # an image-like upstream gradient with a non-zero sum
    tg = _dev(gout, dt)
    rec = gfc.Plan(H, W, 1, B, dtype=dt, device=DEV)
    fft = gfc.Plan(H, W, 1, B, dtype=dt, device=DEV, column_fft=True)
    ax, ay = rec.backward(tg)
    bx, by = fft.backward(tg)
    g64 = _np(tg)
    for f in range(B):
        rx, ry = O.backward(g64[f, 0], rec.M, rec.N, rec.pad)
        if dt == torch.float32:
            # the output of an image-like upstream field is large and dominated by the
            # lowest Green bins: the bar is the FP32 conditioning limit used for every
            # large adjoint (3x the error of a plain torch FP32 evaluation)
            tx_, ty_ = _torch_fp32_adjoint(g64[f, 0].astype(np.float32), rec.M, rec.N, rec.pad)
            tolx, toly = max(REL_F32, 3.0 * _rel(tx_, rx)), max(REL_F32, 3.0 * _rel(ty_, ry))
        else:
            tolx = toly = REL_16
        ex, ey = _rel(_np(ax)[f, 0], rx), _rel(_np(ay)[f, 0], ry)
        assert ex <= tolx, (f, ex, tolx)
        assert ey <= toly, (f, ey, toly)
        # the column-FFT adjoint of the same torus is held to the same bar
        assert _rel(_np(bx)[f, 0], rx) <= tolx and _rel(_np(by)[f, 0], ry) <= toly
    rec.close()
    fft.close()


def test_recursive_adjoint_dot_product_identity():
    """<solve(gx, gy), g> = <gx, adj_x(g)> + <gy, adj_y(g)> on the recursive plan."""
    H, W, B = 801, 1200, 2
    rng = np.random.default_rng(9400)
    gx = _dev(rng.standard_normal((B, 1, H, W)).astype(np.float32))
    gy = _dev(rng.standard_normal((B, 1, H, W)).astype(np.float32))
    g = _dev(rng.standard_normal((B, 1, H, W)).astype(np.float32))
    p = gfc.Plan(H, W, 1, B, device=DEV)
    y = p.solve_from_gradient(gx, gy)
    bx, by = p.backward(g)
    lhs = float((y.double() * g.double()).sum())
    rhs = float((gx.double() * bx.double()).sum() + (gy.double() * by.double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * (abs(lhs) + abs(rhs) + 1.0), (lhs, rhs)
    p.close()


def test_l2_resident_split_is_bitwise_equal_to_one_chunk(monkeypatch):
    """A split whose spectrum hand-off fits the L2 budget (evict-first gradients,
    evict-last spectrum, the inverse row pass dropping the spectrum lines it has
    read) gives the same bits as one chunk and as the same split without the
    policies, call after call; the Laplacian entry and the corrected solve run
    the same passes."""
    B, H, W = 16, 801, 1200
    gx, gy = synth.perturbed_gradient_batch(batch=B, H=H, W=W, seed=9500)
    tx, ty = _dev(gx), _dev(gy)
    one = gfc.Plan(H, W, 1, B, device=DEV)  # 16 fields x 5.7 MB: above the budget
    res = gfc.Plan(H, W, 1, B, device=DEV, chunk=3, streams=4)
    monkeypatch.setenv("GFC_NO_L2RES", "1")
    off = gfc.Plan(H, W, 1, B, device=DEV, chunk=3, streams=4)
    monkeypatch.delenv("GFC_NO_L2RES")
    assert res.l2_resident and not one.l2_resident and not off.l2_resident
    a = one.solve_from_gradient(tx, ty)
    assert torch.equal(a, off.solve_from_gradient(tx, ty))
    for _ in range(3):
        assert torch.equal(a, res.solve_from_gradient(tx, ty))
    lap = torch.roll(tx, 1, -1) - tx
    assert torch.equal(one.solve_from_laplacian(lap), res.solve_from_laplacian(lap))
    ref = O.solve_from_gradient(gx[5, 0].astype(np.float64), gy[5, 0].astype(np.float64), res.M, res.N, res.pad)
    assert _rel(_np(a)[5, 0], ref) <= REL_F32
    for p in (one, res, off):
        p.close()
