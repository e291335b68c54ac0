"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures on natural images (ECSSD, an 801x1200 photograph, stamp
images for Poisson blending). None of them ship here, so these generators
stand in for them: smooth images made of random Gaussians (natural-image-like
low-frequency structure), their forward-difference gradients, and the
non-conservative edits the paper applies to gradients (removal of a region,
additive rectangles, mixed source/target gradients inside a mask, Sec. 3.1.4
and Sec. 3.2.1).

This module holds no arithmetic of the solver itself (no divergence, no
transform, no Green's function); it only makes inputs. Both the CUDA path's
tests and the FP64 oracle consume what it produces. All randomness comes from
``numpy.random.default_rng(seed)``.

Gradient convention: ``gx[i, j] = I[i, j+1] - I[i, j]`` (forward difference
along the width), ``gy[i, j] = I[i+1, j] - I[i, j]`` (along the height), with
the last column of gx and the last row of gy set to 0 (replicate border).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_image",
    "forward_gradient",
    "constant_border_image",
    "gradient_removal_image",
    "perturbed_gradient_batch",
    "poisson_blend_batch",
    "ragged_items",
    "ragged_item_gradients",
    "feature_gradients",
    "upstream_gradient",
    "edit_batch",
    "ring_padded_batch",
]


def gaussian_image(rng, H, W, n_gauss, sigma_lo, sigma_hi, noise=0.0):
    """Sum of ``n_gauss`` isotropic Gaussians, plus U[0, noise] noise, min-max rescaled to [0, 1].

    Centres are uniform over the image, sigmas uniform in [sigma_lo, sigma_hi]
    pixels, amplitudes uniform in [0, 1]. Each Gaussian is separable, so the
    image is one small matrix product.
    """
    cy = rng.uniform(0, H, n_gauss)
    cx = rng.uniform(0, W, n_gauss)
    sig = rng.uniform(sigma_lo, sigma_hi, n_gauss)
    amp = rng.uniform(0.0, 1.0, n_gauss)
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[:, None]
    Ey = np.exp(-0.5 * ((yy - cy[None, :]) / sig[None, :]) ** 2) * amp[None, :]  # [H, n]
    Ex = np.exp(-0.5 * ((xx - cx[None, :]) / sig[None, :]) ** 2)  # [W, n]
    img = Ey @ Ex.T
    if noise > 0.0:
        img = img + rng.uniform(0.0, noise, (H, W))
    lo, hi = img.min(), img.max()
    return (img - lo) / (hi - lo) if hi > lo else np.zeros_like(img)


def forward_gradient(img):
    """Forward differences with a replicate border (last gx column, last gy row are 0)."""
    img = np.asarray(img, dtype=np.float64)
    gx = np.zeros_like(img)
    gy = np.zeros_like(img)
    gx[:, :-1] = img[:, 1:] - img[:, :-1]
    gy[:-1, :] = img[1:, :] - img[:-1, :]
    return gx, gy


def constant_border_image(rng, H, W, border=1):
    """A smooth image whose outer ``border`` pixels all equal one constant.

    Its forward-difference gradient, zero-extended, is exactly conservative on
    the padded torus, so a least-squares solver must return the image minus
    that constant.
    """
    img = gaussian_image(rng, H, W, 6, max(2.0, min(H, W) / 8), max(3.0, min(H, W) / 3))
    c = rng.uniform(0.0, 1.0)
    img[:border, :] = c
    img[-border:, :] = c
    img[:, :border] = c
    img[:, -border:] = c
    return img, c


def gradient_removal_image(seed=0, H=64, W=96, rect=(16, 24)):
    """One grayscale field: 8 Gaussians (sigma 4-20 px) + U[0,0.05] noise in [0,1],
    with its gradients zeroed inside a seeded ``rect`` rectangle (gradient removal).

    Returns ``(image, gx, gy)`` as float32 arrays of shape [H, W].
    """
    rng = np.random.default_rng(seed)
    img = gaussian_image(rng, H, W, 8, 4.0, 20.0, noise=0.05)
    gx, gy = forward_gradient(img)
    rh, rw = rect
    r0 = int(rng.integers(0, H - rh + 1))
    c0 = int(rng.integers(0, W - rw + 1))
    gx[r0:r0 + rh, c0:c0 + rw] = 0.0
    gy[r0:r0 + rh, c0:c0 + rw] = 0.0
    return img.astype(np.float32), gx.astype(np.float32), gy.astype(np.float32)


def _perturbed_field(rng, H, W, n_gauss, sigma_lo, sigma_hi, n_rect=5, amp=0.2):
    img = gaussian_image(rng, H, W, n_gauss, sigma_lo, sigma_hi)
    gx, gy = forward_gradient(img)
    for g in (gx, gy):
        for _ in range(n_rect):
            rh = int(rng.integers(max(1, H // 16), max(2, H // 4) + 1))
            rw = int(rng.integers(max(1, W // 16), max(2, W // 4) + 1))
            r0 = int(rng.integers(0, H - rh + 1))
            c0 = int(rng.integers(0, W - rw + 1))
            g[r0:r0 + rh, c0:c0 + rw] += rng.uniform(-amp, amp)
    return gx, gy


def perturbed_gradient_batch(batch=100, H=801, W=1200, seed=1000, items=None):
    """Batch of single-channel gradient fields [batch, 1, H, W] float32.

    Each field: 64 Gaussians (sigma 5-80 px) rescaled to [0, 1], its
    forward-difference gradient, then 5 seeded rectangles per component with
    one constant U[-0.2, 0.2] each (a non-conservative perturbation). Field
    ``b`` uses seed ``seed + b``. ``items`` selects a subset of field indices
    (the others are not generated).
    """
    idx = range(batch) if items is None else list(items)
    gx = np.empty((len(idx), 1, H, W), dtype=np.float32)
    gy = np.empty_like(gx)
    for n, b in enumerate(idx):
        rng = np.random.default_rng(seed + b)
        fx, fy = _perturbed_field(rng, H, W, 64, 5.0, 80.0)
        gx[n, 0] = fx
        gy[n, 0] = fy
    return gx, gy


def poisson_blend_batch(batch=16, C=3, H=1024, W=1536, patch=(300, 400), seed=2000, items=None):
    """Poisson blending inputs [batch, C, H, W] float32 (mixed gradients, Sec. 3.2.1).

    Target: per channel 8 Gaussians (sigma 64-320 px) + U[0,0.05] noise in [0,1].
    Source: a ``patch``-sized image made the same way (sigma 18-90 px), placed at
    a seeded offset fully inside the target, with a seeded inscribed ellipse
    mask (semi-axes U[0.6, 0.95] of the half-extents). Each forward edge takes
    the source gradient where its pixel lies inside the mask, else the target's.
    Returns ``(gx, gy, target)``.
    """
    idx = range(batch) if items is None else list(items)
    ph, pw = patch
    gx = np.empty((len(idx), C, H, W), dtype=np.float32)
    gy = np.empty_like(gx)
    tgt = np.empty_like(gx)
    for n, b in enumerate(idx):
        rng = np.random.default_rng(seed + b)
        r0 = int(rng.integers(0, H - ph + 1))
        c0 = int(rng.integers(0, W - pw + 1))
        ay = rng.uniform(0.6, 0.95) * ph / 2.0
        ax = rng.uniform(0.6, 0.95) * pw / 2.0
        yy = (np.arange(ph)[:, None] + 0.5 - ph / 2.0) / ay
        xx = (np.arange(pw)[None, :] + 0.5 - pw / 2.0) / ax
        mask = (yy * yy + xx * xx) <= 1.0
        for c in range(C):
            t = gaussian_image(rng, H, W, 8, 64.0, 320.0, noise=0.05)
            s = gaussian_image(rng, ph, pw, 8, 18.0, 90.0, noise=0.05)
            tx, ty = forward_gradient(t)
            sx, sy = forward_gradient(s)
            tx[r0:r0 + ph, c0:c0 + pw][mask] = sx[mask]
            ty[r0:r0 + ph, c0:c0 + pw][mask] = sy[mask]
            gx[n, c] = tx
            gy[n, c] = ty
            tgt[n, c] = t
    return gx, gy, tgt


def ragged_items(n_items=64, lo=128, hi=2048, seed=3000):
    """Seeded item shapes for a ragged batch: list of ``(C, H, W)``, C in {1, 3}, H, W ~ U{lo..hi}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_items):
        C = int(rng.choice([1, 3]))
        H = int(rng.integers(lo, hi + 1))
        W = int(rng.integers(lo, hi + 1))
        out.append((C, H, W))
    return out


def ragged_item_gradients(shape, item, seed=3000):
    """Gradients [C, H, W] float32 of one ragged item, built like ``perturbed_gradient_batch``
    with the Gaussian sigmas scaled by sqrt(H*W / (801*1200))."""
    C, H, W = shape
    s = float(np.sqrt(H * W / (801.0 * 1200.0)))
    gx = np.empty((C, H, W), dtype=np.float32)
    gy = np.empty_like(gx)
    for c in range(C):
        rng = np.random.default_rng(seed * 1000 + item * 3 + c)
        fx, fy = _perturbed_field(rng, H, W, 64, 5.0 * s, 80.0 * s)
        gx[c] = fx
        gy[c] = fy
    return gx, gy


def _box5(a):
    """5x5 box mean with zero boundary ('same' size), over the last two axes."""
    pad = np.zeros(a.shape[:-2] + (a.shape[-2] + 4, a.shape[-1] + 4), dtype=np.float32)
    pad[..., 2:-2, 2:-2] = a
    cs = np.cumsum(pad, axis=-1, dtype=np.float32)
    cs = np.concatenate([np.zeros_like(cs[..., :1]), cs], axis=-1)
    h = cs[..., 5:] - cs[..., :-5]
    cs = np.cumsum(h, axis=-2, dtype=np.float32)
    cs = np.concatenate([np.zeros_like(cs[..., :1, :]), cs], axis=-2)
    v = cs[..., 5:, :] - cs[..., :-5, :]
    return v / 25.0


def feature_gradients(batch=32, C=64, H=256, W=256, seed=4000, items=None):
    """Feature-map gradients [batch, C, H, W] float32: N(0,1) filtered by a 5x5 box blur.

    Stands in for CNN feature gradients for the differentiable merging layer
    (Sec. 4). ``items`` selects a subset of batch indices.
    """
    idx = range(batch) if items is None else list(items)
    gx = np.empty((len(idx), C, H, W), dtype=np.float32)
    gy = np.empty_like(gx)
    for n, b in enumerate(idx):
        rng = np.random.default_rng(seed + b)
        gx[n] = _box5(rng.standard_normal((C, H, W), dtype=np.float32))
        gy[n] = _box5(rng.standard_normal((C, H, W), dtype=np.float32))
    return gx, gy


def upstream_gradient(shape, seed=4500):
    """Random upstream gradient N(0,1) float32 of the given shape."""
    return np.random.default_rng(seed).standard_normal(shape, dtype=np.float32)


def edit_batch(batch=4, C=3, H=801, W=1200, seed=5000, items=None):
    """Images, gradients and an edge map for the editing steps of Sec. 3.2.

    Each channel: 64 Gaussians (sigma 5-80 px) plus U[0, 0.05] texture noise,
    rescaled to [0, 1]; its forward-difference gradient; and an edge-intensity
    map standing in for an edge detector's output (Sec. 3.2.4 uses SE or RCF):
    the gradient magnitude of a 5x5 box-blurred copy, rescaled to [0, 1].
    Returns float32 arrays ``(img, gx, gy, edges)`` of shape [n, C, H, W];
    batch item ``b`` uses seed ``seed + b``.
    """
    idx = range(batch) if items is None else list(items)
    img = np.empty((len(idx), C, H, W), dtype=np.float32)
    gx, gy, edges = np.empty_like(img), np.empty_like(img), np.empty_like(img)
    for n, b in enumerate(idx):
        rng = np.random.default_rng(seed + b)
        for c in range(C):
            im = gaussian_image(rng, H, W, 64, 5.0, 80.0, noise=0.05)
            fx, fy = forward_gradient(im)
            bx, by = forward_gradient(_box5(im.astype(np.float32)).astype(np.float64))
            e = np.sqrt(bx * bx + by * by)
            img[n, c], gx[n, c], gy[n, c] = im, fx, fy
            edges[n, c] = e / e.max() if e.max() > 0 else e
    return img, gx, gy, edges


def ring_padded_batch(batch=4, C=1, H=807, W=1206, ring=3, seed=6000, items=None):
    """Images padded by a ring of zeros (Sec. 2.3.2) and their edited gradients.

    The inner (H - 2 ring) x (W - 2 ring) block is a 64-Gaussian image in
    [0, 1]; the ring is 0. Its forward-difference gradient then gets the
    additive rectangles of ``perturbed_gradient_batch`` inside the inner block,
    so the field is not conservative. Returns float32 ``(img, gx, gy)`` of
    shape [n, C, H, W]; batch item ``b`` uses seed ``seed + b``.
    """
    idx = range(batch) if items is None else list(items)
    img = np.zeros((len(idx), C, H, W), dtype=np.float32)
    gx, gy = np.empty_like(img), np.empty_like(img)
    Hi, Wi = H - 2 * ring, W - 2 * ring
    for n, b in enumerate(idx):
        rng = np.random.default_rng(seed + b)
        for c in range(C):
            im = np.zeros((H, W))
            im[ring:H - ring, ring:W - ring] = gaussian_image(rng, Hi, Wi, 64, 5.0, 80.0)
            fx, fy = forward_gradient(im)
            for g in (fx, fy):
                for _ in range(5):
                    rh = int(rng.integers(max(1, Hi // 16), max(2, Hi // 4) + 1))
                    rw = int(rng.integers(max(1, Wi // 16), max(2, Wi // 4) + 1))
                    r0 = ring + int(rng.integers(0, Hi - rh + 1))
                    c0 = ring + int(rng.integers(0, Wi - rw + 1))
                    g[r0:r0 + rh, c0:c0 + rw] += rng.uniform(-0.2, 0.2)
            img[n, c], gx[n, c], gy[n, c] = im, fx, fy
    return img, gx, gy
