"""FP64 CPU oracle for Green Function Convolution (GFC) -- TEST INFRASTRUCTURE ONLY.

This module is the slow, plain reference that the CUDA path is checked
against. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the product path (the C-ABI library and its
Python binding) never does, and shares no code, table or helper with it.

What it computes (Beaini et al., "Fast and Optimal Laplacian Solver for
Gradient-Domain Image Editing using Green Function Convolution"):

* Eq. 3: the Laplacian of a gradient field is its divergence, ``L = div E``.
  The discrete divergence used here is the negative adjoint of the forward
  difference (the reading of the unstated gradient scheme in Sec. 2.1):
  ``L[r,c] = Ex[r,c] - Ex[r,c-1] + Ey[r,c] - Ey[r-1,c]``.
* Sec. 2.3.2 / Algorithm A: everything lives on a zero-padded M x N domain,
  treated as a torus by the DFT. The image block sits at offset ``(p, p)``.
* Eq. 15-22 / Algorithm A: the Green spectrum is ``F(delta)/F(K)`` with the
  Dirac and the 3x3 Laplace kernel both centred at ``[1, 1]``. The phases
  cancel, leaving the real value ``1/lambda(k,l)`` with
  ``lambda = 2cos(2 pi k/M) + 2cos(2 pi l/N) - 4``. Algorithm A's kernel
  sign (positive Laplacian, -4 centre) is used; Eq. 15 prints the negated
  kernel, which would return ``-I``. The DC bin is 0/0 in Algorithm A; it is
  set to 0 here (any finite value gives the same output once the offset of
  Algorithm B is removed, because a divergence sums to zero on the torus).
* Eq. 23 / Algorithm B: ``I = Re(IDFT(DFT(L) o G))``, then ``I -= I[0,0]``,
  then crop ``[p:p+H, p:p+W]``.

The DFTs are written out as their definition: explicit DFT matrices built
from ``exp(-2 pi i ((k m) mod n) / n)`` with exact integer reduction, applied
with matrix products (a library primitive used as a step). No FFT algorithm,
blocking or reordering is used, so a reader can check every line against the
equations above.

Every function works on one field (a 2-D array); ``*_batch`` helpers loop.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "dft_matrix",
    "dft2",
    "idft2",
    "green_spectrum",
    "zero_extend",
    "divergence_torus",
    "solve_torus",
    "solve_from_gradient",
    "solve_from_laplacian",
    "backward",
    "solve_from_gradient_batch",
    "solve_from_laplacian_batch",
    "backward_batch",
]

_DFT_CACHE: dict = {}


def dft_matrix(n: int, sign: int = -1) -> np.ndarray:
    """The n x n DFT matrix ``F[k, m] = exp(sign * 2 pi i * ((k*m) mod n) / n)``.

    The exponent is reduced modulo n in exact integer arithmetic before the
    angle is formed, so every entry is a correctly rounded FP64 root of unity.
    (Eq. 17: the Fourier transform used by the convolution theorem.)
    """
    key = (n, sign)
    F = _DFT_CACHE.get(key)
    if F is None:
        k = np.arange(n, dtype=np.int64)
        m = np.outer(k, k) % n
        ang = (2.0 * np.pi / n) * m
        F = np.cos(ang) + 1j * sign * np.sin(ang)
        if len(_DFT_CACHE) > 16:
            _DFT_CACHE.clear()
        _DFT_CACHE[key] = F
    return F


def dft2(x: np.ndarray) -> np.ndarray:
    """Forward 2-D DFT ``X[k,l] = sum_{r,c} x[r,c] w_M^{kr} w_N^{lc}`` (Eq. 17)."""
    M, N = x.shape
    return dft_matrix(M, -1) @ np.asarray(x, dtype=np.complex128) @ dft_matrix(N, -1)


def idft2(X: np.ndarray) -> np.ndarray:
    """Inverse 2-D DFT with the 1/(MN) factor (Eq. 17, Eq. 23)."""
    M, N = X.shape
    return (dft_matrix(M, +1) @ np.asarray(X, dtype=np.complex128) @ dft_matrix(N, +1)) / (M * N)


def green_spectrum(M: int, N: int) -> np.ndarray:
    """Numerical Green spectrum on the M x N torus (Eq. 19-22, Algorithm A).

    ``G[k,l] = 1 / lambda(k,l)``, ``lambda = 2cos(2 pi k/M) + 2cos(2 pi l/N) - 4``
    (the DFT of Algorithm A's Laplace kernel, divided into the DFT of its
    Dirac; both sit at [1,1] so the phase factors cancel). ``G[0,0] = 0``.
    No 1/(MN) factor: that belongs to the inverse DFT.
    """
    k = np.arange(M, dtype=np.int64)[:, None]
    l = np.arange(N, dtype=np.int64)[None, :]
    lam = 2.0 * np.cos(2.0 * np.pi * k / M) + 2.0 * np.cos(2.0 * np.pi * l / N) - 4.0
    G = np.zeros((M, N), dtype=np.float64)
    nz = np.ones((M, N), dtype=bool)
    nz[0, 0] = False
    G[nz] = 1.0 / lam[nz]
    return G


def zero_extend(a: np.ndarray, M: int, N: int, p: int) -> np.ndarray:
    """Place an H x W block at offset (p, p) of an M x N zero field (Algorithm A's padding)."""
    H, W = a.shape
    if p < 1 or H + p + 1 > M or W + p + 1 > N:
        raise ValueError("padded domain too small: need p >= 1, M >= H+p+1, N >= W+p+1")
    out = np.zeros((M, N), dtype=np.float64)
    out[p:p + H, p:p + W] = np.asarray(a, dtype=np.float64)
    return out


def divergence_torus(Ex: np.ndarray, Ey: np.ndarray) -> np.ndarray:
    """Discrete divergence on the torus, ``L = Ex - Ex(., c-1) + Ey - Ey(r-1, .)`` (Eq. 3).

    x runs along columns (the image width), y along rows (the height).
    Indices wrap, as they do for the DFT.
    """
    return (Ex - np.roll(Ex, 1, axis=1)) + (Ey - np.roll(Ey, 1, axis=0))


def solve_torus(L: np.ndarray) -> np.ndarray:
    """``u = Re(IDFT(DFT(L) o G))`` on the torus (Eq. 23, before the offset)."""
    M, N = L.shape
    return np.real(idft2(dft2(L) * green_spectrum(M, N)))


def _offset_and_crop(u: np.ndarray, H: int, W: int, p: int) -> np.ndarray:
    """Algorithm B: subtract ``u[0,0]`` (the pad's corner), then crop the image block."""
    u = u - u[0, 0]
    return u[p:p + H, p:p + W]


def solve_from_gradient(gx: np.ndarray, gy: np.ndarray, M: int, N: int, p: int) -> np.ndarray:
    """GFC solve of one field from its (possibly non-conservative) gradient (Eq. 3, Eq. 23, Alg. B).

    gx is the forward difference along the width, gy along the height, both
    H x W; they are zero-extended into the padded torus (zero flux in the pad,
    Sec. 2.2), their divergence is taken, and the Poisson problem is solved.
    """
    H, W = gx.shape
    L = divergence_torus(zero_extend(gx, M, N, p), zero_extend(gy, M, N, p))
    return _offset_and_crop(solve_torus(L), H, W, p)


def solve_from_laplacian(lap: np.ndarray, M: int, N: int, p: int) -> np.ndarray:
    """GFC solve of one field from a given H x W Laplacian (Eq. 23, Alg. B).

    The Laplacian is zero-extended into the torus ("padded_L" of Algorithm B).
    Its mean is projected out by ``G[0,0] = 0``.
    """
    H, W = lap.shape
    L = zero_extend(lap, M, N, p)
    return _offset_and_crop(solve_torus(L), H, W, p)


def backward(gout: np.ndarray, M: int, N: int, p: int):
    """Adjoint of ``(gx, gy) -> solve_from_gradient(gx, gy)`` applied to ``gout``.

    The forward map is ``y = Crop(u) - u[0,0]`` with ``u = g (*) div(E)``.
    Its transpose, step by step:
      z = Crop^T(gout) - (sum gout) e_00      (transpose of crop minus offset)
      w = Re(IDFT(DFT(z) o G))                (G real and even: the
                                               convolution is self-adjoint)
      grad Ex = w - w(., c+1), grad Ey = w - w(r+1, .)   (transpose of div)
    and the gradients of gx, gy are the image-block crops of grad Ex, grad Ey.
    """
    H, W = gout.shape
    z = zero_extend(gout, M, N, p)
    z[0, 0] -= float(np.sum(np.asarray(gout, dtype=np.float64)))
    w = solve_torus(z)
    gEx = w - np.roll(w, -1, axis=1)
    gEy = w - np.roll(w, -1, axis=0)
    return gEx[p:p + H, p:p + W].copy(), gEy[p:p + H, p:p + W].copy()


def _fields(a: np.ndarray):
    a = np.asarray(a)
    return a.reshape((-1,) + a.shape[-2:])


def solve_from_gradient_batch(gx, gy, M, N, p):
    """Loop ``solve_from_gradient`` over every leading index of ``[..., H, W]`` arrays."""
    fx, fy = _fields(gx), _fields(gy)
    out = np.stack([solve_from_gradient(fx[i], fy[i], M, N, p) for i in range(fx.shape[0])])
    return out.reshape(np.shape(gx))


def solve_from_laplacian_batch(lap, M, N, p):
    """Loop ``solve_from_laplacian`` over every leading index."""
    f = _fields(lap)
    out = np.stack([solve_from_laplacian(f[i], M, N, p) for i in range(f.shape[0])])
    return out.reshape(np.shape(lap))


def backward_batch(gout, M, N, p):
    """Loop ``backward`` over every leading index; returns (grad_gx, grad_gy)."""
    f = _fields(gout)
    res = [backward(f[i], M, N, p) for i in range(f.shape[0])]
    gx = np.stack([r[0] for r in res]).reshape(np.shape(gout))
    gy = np.stack([r[1] for r in res]).reshape(np.shape(gout))
    return gx, gy
