"""FP64 CPU oracle for the gradient-domain edits around GFC -- TEST INFRASTRUCTURE ONLY.

Like ``gfc_oracle``, this module is the plain reference the CUDA editing
kernels are checked against; only the test suite, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py`` may import it, and it shares no code with the
product path.

What it computes (Beaini et al., Sec. 2.3.2 and Sec. 3.2):

* Eq. 25 (Sec. 3.2.2), colour correction of a solved field ``Ic`` against the
  original image ``I``: ``(Ic - mean(Ic)) * std(I) / std(Ic) + mean(I)``, per
  field (per channel of an image). The paper does not say which standard
  deviation; only the ratio of two of them enters, so the population and the
  sample definitions give the same result. The population one is used.
  A constant ``Ic`` (``std(Ic) = 0``) has no contrast to rescale; it maps to
  the constant ``mean(I)``.
* Sec. 3.1.4 / Sec. 3.2.3, gradient thresholding: a pixel whose gradient
  magnitude ``|E| = sqrt(Ex^2 + Ey^2)`` is below ``frac`` times a reference
  magnitude gets ``E = 0``. The reference is the largest magnitude of the
  field, or a caller-given value (the "highest possible gradient" of an image
  of known range). The keep/drop decision is an integer outcome decided in
  floating point, so it is taken here in FP32, the paper's precision, with the
  operations ordered as stated in ``gradient_threshold``.
* Eq. 26 (Sec. 3.2.4), gradient-domain merging: ``|Ep| = |E|^(1-alpha) C^alpha``
  with the orientation of ``E`` kept, i.e. ``Ep = E |E|^(-alpha) C^alpha``
  where ``|E| > 0`` and ``Ep = 0`` where ``|E| = 0`` (no orientation).
* Sec. 2.3.2, boundary preservation: the image is padded by a ring of zeros
  (3 pixels in the paper) before its gradient is taken; after the solve, the
  constant ``c`` is the one that brings the ring closest to zero in the least
  squares sense, which is minus the ring's mean; the ring is then cropped.

Every function works on one field (a 2-D array); ``*_batch`` helpers loop over
the leading axes.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "field_stats",
    "color_correct",
    "gradient_threshold",
    "gradient_merge",
    "ring_mask",
    "boundary_offset",
    "field_stats_batch",
    "color_correct_batch",
    "gradient_threshold_batch",
    "gradient_merge_batch",
    "boundary_offset_batch",
]


def field_stats(a: np.ndarray):
    """Mean and population standard deviation of one field, in FP64."""
    x = np.asarray(a, dtype=np.float64)
    mean = x.mean()
    std = np.sqrt(np.mean((x - mean) ** 2))
    return float(mean), float(std)


def color_correct(Ic: np.ndarray, I_ref: np.ndarray) -> np.ndarray:
    """Eq. 25: rescale the solved field to the mean and contrast of the original."""
    mc, sc = field_stats(Ic)
    mi, si = field_stats(I_ref)
    return color_correct_with(Ic, mi, si, mc, sc)


def color_correct_with(Ic: np.ndarray, ref_mean: float, ref_std: float, mean_c=None, std_c=None) -> np.ndarray:
    """Eq. 25 with the original image's statistics given as numbers."""
    x = np.asarray(Ic, dtype=np.float64)
    if mean_c is None or std_c is None:
        mean_c, std_c = field_stats(x)
    if std_c == 0.0:
        return np.full_like(x, ref_mean)
    return (x - mean_c) * (ref_std / std_c) + ref_mean


def gradient_threshold(gx: np.ndarray, gy: np.ndarray, frac: float, ref: float | None = None):
    """Zero the gradient where its magnitude is below ``frac`` of the reference.

    The decision is taken in FP32: ``m2 = fl(fl(gx*gx) + fl(gy*gy))`` per pixel;
    the reference magnitude ``r`` is ``fl(sqrt(max m2))`` (correctly rounded)
    or the caller's ``ref``; ``t = fl(frac * r)``; a pixel is dropped when
    ``m2 < fl(t * t)``. Kept pixels are copied unchanged.
    """
    x = np.asarray(gx, dtype=np.float32)
    y = np.asarray(gy, dtype=np.float32)
    m2 = (x * x) + (y * y)  # each product and the sum rounded to FP32
    if ref is None or ref <= 0:
        r = np.sqrt(m2.max()) if m2.size else np.float32(0)
    else:
        r = np.float32(ref)
    t = np.float32(frac) * np.float32(r)
    t2 = np.float32(t * t)
    keep = ~(m2 < t2)
    return np.where(keep, x, np.float32(0)), np.where(keep, y, np.float32(0)), keep


def gradient_merge(gx: np.ndarray, gy: np.ndarray, C: np.ndarray, alpha: float):
    """Eq. 26: ``Ep = E |E|^(-alpha) C^alpha`` (orientation of E kept), in FP64."""
    x = np.asarray(gx, dtype=np.float64)
    y = np.asarray(gy, dtype=np.float64)
    c = np.asarray(C, dtype=np.float64)
    mag = np.sqrt(x * x + y * y)
    out_x = np.zeros_like(x)
    out_y = np.zeros_like(y)
    nz = mag > 0
    # |Ep| = |E|^(1-alpha) C^alpha; the unit vector E/|E| carries the orientation.
    mag_p = mag[nz] ** (1.0 - alpha) * c[nz] ** alpha
    out_x[nz] = x[nz] / mag[nz] * mag_p
    out_y[nz] = y[nz] / mag[nz] * mag_p
    return out_x, out_y


def ring_mask(H: int, W: int, ring: int) -> np.ndarray:
    """True on the ``ring`` outermost rows and columns of an H x W field."""
    m = np.ones((H, W), dtype=bool)
    m[ring:H - ring, ring:W - ring] = False
    return m


def boundary_offset(u: np.ndarray, ring: int) -> np.ndarray:
    """Sec. 2.3.2: subtract the least-squares constant over the ring, then crop it."""
    x = np.asarray(u, dtype=np.float64)
    H, W = x.shape
    c = -x[ring_mask(H, W, ring)].mean()
    return (x + c)[ring:H - ring, ring:W - ring]


def _fields(a: np.ndarray):
    a = np.asarray(a)
    return a.reshape((-1,) + a.shape[-2:])


def field_stats_batch(a):
    f = _fields(a)
    st = np.array([field_stats(x) for x in f])
    lead = np.asarray(a).shape[:-2]
    return st[:, 0].reshape(lead), st[:, 1].reshape(lead)


def color_correct_batch(Ic, I_ref):
    a, b = _fields(Ic), _fields(I_ref)
    return np.stack([color_correct(x, y) for x, y in zip(a, b)]).reshape(np.asarray(Ic).shape)


def gradient_threshold_batch(gx, gy, frac, ref=None):
    shape = np.asarray(gx).shape
    outs = [gradient_threshold(x, y, frac, ref) for x, y in zip(_fields(gx), _fields(gy))]
    ox = np.stack([o[0] for o in outs]).reshape(shape)
    oy = np.stack([o[1] for o in outs]).reshape(shape)
    return ox, oy


def gradient_merge_batch(gx, gy, C, alpha):
    shape = np.asarray(gx).shape
    outs = [gradient_merge(x, y, c, alpha) for x, y, c in zip(_fields(gx), _fields(gy), _fields(C))]
    return np.stack([o[0] for o in outs]).reshape(shape), np.stack([o[1] for o in outs]).reshape(shape)


def boundary_offset_batch(u, ring):
    a = np.asarray(u)
    inner = np.stack([boundary_offset(x, ring) for x in _fields(a)])
    return inner.reshape(a.shape[:-2] + inner.shape[-2:])
