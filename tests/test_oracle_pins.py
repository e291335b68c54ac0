"""Pins for the FP64 oracle: each test ties it to something other than itself.

Pins used (none re-types the oracle's own formula):
* a library routine on the same definition (numpy's FFT for the DFT matrices,
  numpy's FFT of Algorithm A's literal matrices for the Green spectrum);
* the least-squares characterisation of Sec. 2.2 (dense lstsq on the torus,
  and an optimality inequality against other candidates);
* closed forms and invariants (exact recovery of a conservative field, Eq. 4;
  Green's function identity, Eq. 16; the Laplacian of the result, Eq. 3);
* brute force on tiny inputs (direct circular convolution, Eq. 17; the
  explicit matrix transpose for the adjoint);
* the values printed in the paper (tests/golden/paper_kernels.txt).
The planted-mistake tests at the end show that a plausible error in the
oracle (wrong kernel sign, shifted stencil, dropped offset term, transposed
axis) fails at least one pin.
"""
import os

import numpy as np
import pytest

import oracle.gfc_oracle as O
from paper_1902_00176_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_kernels.txt")


def _read_golden():
    vals, mats = {}, {}
    with open(GOLDEN) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        parts = lines[i].split()
        if parts[0].startswith("laplace_"):
            mats[parts[0]] = np.array([[float(x) for x in lines[i + k].split()] for k in (1, 2, 3)])
            i += 4
        else:
            vals[parts[0]] = [float(x) for x in parts[1:]]
            i += 1
    return vals, mats


def _torus_diff_matrix(M, N):
    """Dense forward-difference operators on the M x N torus, built by loops."""
    n = M * N
    Dx = np.zeros((n, n))
    Dy = np.zeros((n, n))
    for r in range(M):
        for c in range(N):
            i = r * N + c
            Dx[i, r * N + (c + 1) % N] += 1.0
            Dx[i, i] -= 1.0
            Dy[i, ((r + 1) % M) * N + c] += 1.0
            Dy[i, i] -= 1.0
    return Dx, Dy


def _extend_by_loops(a, M, N, p):
    out = np.zeros((M, N))
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            out[p + i, p + j] = a[i, j]
    return out


# --------------------------------------------------------------------------
# DFT and Green spectrum
# --------------------------------------------------------------------------

@pytest.mark.parametrize("M,N", [(6, 7), (8, 12), (11, 13), (72, 108), (30, 1)])
def test_dft2_matches_library_fft(M, N):
    rng = np.random.default_rng(M * 100 + N)
    x = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    assert np.allclose(O.dft2(x), np.fft.fft2(x), rtol=0, atol=1e-11 * M * N)
    assert np.allclose(O.idft2(x), np.fft.ifft2(x), rtol=0, atol=1e-13 * M * N)


def test_dft_matrix_entries_are_roots_of_unity():
    F = O.dft_matrix(810, -1)
    assert np.abs(np.abs(F) - 1.0).max() < 1e-15
    # row 1 is the 810th root of unity raised to m: F[1,m]^810 == 1
    assert abs(F[1, 1] ** 810 - 1.0) < 1e-12


@pytest.mark.parametrize("M,N", [(12, 10), (14, 9), (72, 108), (24, 24)])
def test_green_closed_form_equals_algorithm_a_literally(M, N):
    vals, mats = _read_golden()
    dr, dc = int(vals["dirac_row"][0]), int(vals["dirac_col"][0])
    dirac = np.zeros((M, N))
    dirac[dr, dc] = 1.0
    lap = np.zeros((M, N))
    lap[0:3, 0:3] = mats["laplace_alg_a"]
    with np.errstate(divide="ignore", invalid="ignore"):
        alg_a = np.fft.fft2(dirac) / np.fft.fft2(lap)
    G = O.green_spectrum(M, N)
    off = np.ones((M, N), dtype=bool)
    off[0, 0] = False
    assert np.abs(alg_a[off] - G[off]).max() < 1e-10 * np.abs(G).max()
    assert not np.isfinite(alg_a[0, 0])  # Algorithm A's DC bin is 0/0
    assert G[0, 0] == 0.0


def test_green_function_identity_delta_minus_mean():
    """Eq. 16 on the torus: (5-point Laplacian of g) = delta_00 - 1/(MN)."""
    M, N = 15, 22
    g = np.real(O.idft2(O.green_spectrum(M, N)))
    _, mats = _read_golden()
    K = mats["laplace_alg_a"]
    lap = np.zeros_like(g)
    for a in range(3):
        for b in range(3):
            lap += K[a, b] * np.roll(np.roll(g, 1 - a, axis=0), 1 - b, axis=1)
    expect = -np.full((M, N), 1.0 / (M * N))
    expect[0, 0] += 1.0
    assert np.abs(lap - expect).max() < 1e-13


def test_eq15_sign_would_negate_the_image():
    """With Eq. 15's printed sign the conservative round trip returns -I, with Algorithm A's it returns I."""
    rng = np.random.default_rng(3)
    img, c = synth.constant_border_image(rng, 9, 11)
    gx, gy = synth.forward_gradient(img)
    M, N, p = 18, 20, 4
    out = O.solve_from_gradient(gx, gy, M, N, p)
    assert np.abs(out - (img - c)).max() < 1e-12
    _, mats = _read_golden()
    lap15 = np.zeros((M, N))
    lap15[0:3, 0:3] = mats["laplace_eq15"]
    dirac = np.zeros((M, N))
    dirac[1, 1] = 1.0
    with np.errstate(divide="ignore", invalid="ignore"):
        G15 = np.fft.fft2(dirac) / np.fft.fft2(lap15)
    G15[0, 0] = 0.0
    L = O.divergence_torus(O.zero_extend(gx, M, N, p), O.zero_extend(gy, M, N, p))
    u15 = np.real(np.fft.ifft2(np.fft.fft2(L) * G15))
    out15 = (u15 - u15[0, 0])[p:p + 9, p:p + 11]
    assert np.abs(out15 + (img - c)).max() < 1e-12


# --------------------------------------------------------------------------
# Least squares (Sec. 2.2) and exact recovery (Eq. 4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("H,W,p,M,N", [(5, 7, 2, 10, 12), (4, 6, 1, 7, 9), (6, 5, 4, 14, 13), (3, 8, 3, 10, 15)])
def test_solve_equals_dense_least_squares_on_torus(H, W, p, M, N):
    rng = np.random.default_rng(H * 1000 + W * 10 + p)
    gx = rng.standard_normal((H, W))
    gy = rng.standard_normal((H, W))
    Dx, Dy = _torus_diff_matrix(M, N)
    A = np.vstack([Dx, Dy])
    e = np.concatenate([_extend_by_loops(gx, M, N, p).ravel(), _extend_by_loops(gy, M, N, p).ravel()])
    u, *_ = np.linalg.lstsq(A, e, rcond=None)
    u = u.reshape(M, N)
    ref = (u - u[0, 0])[p:p + H, p:p + W]
    got = O.solve_from_gradient(gx, gy, M, N, p)
    assert np.abs(got - ref).max() < 1e-10


@pytest.mark.parametrize("H,W,p,M,N", [(9, 11, 4, 18, 20), (16, 24, 4, 24, 32), (64, 96, 4, 72, 108)])
def test_conservative_gradient_recovers_image(H, W, p, M, N):
    rng = np.random.default_rng(H + W)
    img, c = synth.constant_border_image(rng, H, W)
    gx, gy = synth.forward_gradient(img)
    out = O.solve_from_gradient(gx, gy, M, N, p)
    assert np.abs(out - (img - c)).max() < 1e-11


def test_laplacian_input_recovers_image():
    H, W, p, M, N = 12, 17, 4, 24, 28
    rng = np.random.default_rng(7)
    img, c = synth.constant_border_image(rng, H, W)
    field = np.full((M, N), c)
    field[p:p + H, p:p + W] = img
    # 5-point Laplacian by explicit neighbour sums (constant outside => zero there)
    lap_full = np.zeros_like(field)
    for r in range(M):
        for s in range(N):
            lap_full[r, s] = (field[(r + 1) % M, s] + field[r - 1, s] + field[r, (s + 1) % N]
                              + field[r, s - 1] - 4.0 * field[r, s])
    assert np.abs(lap_full).sum() - np.abs(lap_full[p:p + H, p:p + W]).sum() < 1e-12
    out = O.solve_from_laplacian(lap_full[p:p + H, p:p + W], M, N, p)
    assert np.abs(out - (img - c)).max() < 1e-11


def test_laplacian_of_solution_reproduces_divergence():
    """Eq. 3/16: the 5-point Laplacian of the torus solution equals L (sum L = 0 for a divergence)."""
    H, W, p, M, N = 20, 26, 4, 28, 36
    _, gx, gy = synth.gradient_removal_image(seed=5, H=H, W=W, rect=(6, 8))
    Ex = _extend_by_loops(gx.astype(np.float64), M, N, p)
    Ey = _extend_by_loops(gy.astype(np.float64), M, N, p)
    L = O.divergence_torus(Ex, Ey)
    assert abs(L.sum()) < 1e-12
    u = O.solve_torus(L)
    lap = (np.roll(u, 1, 0) + np.roll(u, -1, 0) + np.roll(u, 1, 1) + np.roll(u, -1, 1) - 4 * u)
    assert np.abs(lap - L).max() < 1e-12
    # divergence sign: at an interior pixel it is gx[i,j]-gx[i,j-1]+gy[i,j]-gy[i-1,j]
    i, j = 7, 9
    assert abs(L[p + i, p + j] - (gx[i, j] - gx[i, j - 1] + gy[i, j] - gy[i - 1, j])) < 1e-7


def test_direct_circular_convolution_with_green_function():
    """Eq. 4/17/23: u = L (*) g computed by the O((MN)^2) circular sum."""
    M, N = 7, 9
    rng = np.random.default_rng(11)
    L = rng.standard_normal((M, N))
    L -= L.mean()
    g = np.real(O.idft2(O.green_spectrum(M, N)))
    u_direct = np.zeros((M, N))
    for r in range(M):
        for c in range(N):
            s = 0.0
            for a in range(M):
                for b in range(N):
                    s += L[a, b] * g[(r - a) % M, (c - b) % N]
            u_direct[r, c] = s
    assert np.abs(O.solve_torus(L) - u_direct).max() < 1e-12


def _torus_gradient_error(u, Ex, Ey):
    ex = (np.roll(u, -1, axis=1) - u) - Ex
    ey = (np.roll(u, -1, axis=0) - u) - Ey
    return float(np.sum(ex * ex) + np.sum(ey * ey))


def test_least_error_against_other_candidates():
    """Sec. 2.2 / Sec. 3.1.4: GFC has the least torus gradient error of any field,
    in particular less than a Neumann DCT solve (Tanaka-style) extended into the pad."""
    import scipy.fft as sf

    H, W, p, M, N = 24, 30, 4, 32, 40
    img, gx, gy = synth.gradient_removal_image(seed=9, H=H, W=W, rect=(8, 10))
    gx = gx.astype(np.float64)
    gy = gy.astype(np.float64)
    Ex = _extend_by_loops(gx, M, N, p)
    Ey = _extend_by_loops(gy, M, N, p)
    L = O.divergence_torus(Ex, Ey)
    u = O.solve_torus(L)
    e_gfc = _torus_gradient_error(u, Ex, Ey)
    rng = np.random.default_rng(1)
    for _ in range(10):
        v = u + 1e-3 * rng.standard_normal(u.shape)
        assert _torus_gradient_error(v, Ex, Ey) > e_gfc
    # Neumann DCT solve on the image block (divergence with a reflecting border)
    div = gx.copy()
    div[:, 1:] -= gx[:, :-1]
    div += gy
    div[1:, :] -= gy[:-1, :]
    k = np.arange(H)[:, None]
    l = np.arange(W)[None, :]
    lam = 2 * np.cos(np.pi * k / H) + 2 * np.cos(np.pi * l / W) - 4
    lam[0, 0] = 1.0
    D = sf.dctn(div, type=2, norm="ortho") / lam
    D[0, 0] = 0.0
    v_img = sf.idctn(D, type=2, norm="ortho")
    v = np.pad(v_img, ((p, M - H - p), (p, N - W - p)), mode="edge")
    assert _torus_gradient_error(v, Ex, Ey) >= e_gfc - 1e-12


# --------------------------------------------------------------------------
# Adjoint
# --------------------------------------------------------------------------

def test_backward_is_transpose_of_forward_matrix():
    H, W, p, M, N = 4, 5, 2, 8, 10
    n = H * W
    A = np.zeros((n, 2 * n))
    for k in range(2 * n):
        e = np.zeros(2 * n)
        e[k] = 1.0
        A[:, k] = O.solve_from_gradient(e[:n].reshape(H, W), e[n:].reshape(H, W), M, N, p).ravel()
    rng = np.random.default_rng(2)
    gout = rng.standard_normal((H, W))
    gx, gy = O.backward(gout, M, N, p)
    ref = A.T @ gout.ravel()
    assert np.abs(np.concatenate([gx.ravel(), gy.ravel()]) - ref).max() < 1e-12


def test_backward_matches_central_finite_differences():
    H, W, p, M, N = 6, 7, 4, 16, 16
    rng = np.random.default_rng(4)
    gx0 = rng.standard_normal((H, W))
    gy0 = rng.standard_normal((H, W))
    gout = rng.standard_normal((H, W))
    bx, by = O.backward(gout, M, N, p)
    h = 1e-3
    for (i, j) in [(0, 0), (2, 3), (5, 6), (3, 0)]:
        for which, bref in ((0, bx), (1, by)):
            xp = [gx0.copy(), gy0.copy()]
            xm = [gx0.copy(), gy0.copy()]
            xp[which][i, j] += h
            xm[which][i, j] -= h
            fp = np.sum(gout * O.solve_from_gradient(xp[0], xp[1], M, N, p))
            fm = np.sum(gout * O.solve_from_gradient(xm[0], xm[1], M, N, p))
            assert abs((fp - fm) / (2 * h) - bref[i, j]) < 1e-9


# --------------------------------------------------------------------------
# Planted mistakes (in the oracle, on the CPU): each must fail a pin above
# --------------------------------------------------------------------------

def _ls_pin_error(solve):
    H, W, p, M, N = 5, 7, 2, 10, 12
    rng = np.random.default_rng(99)
    gx = rng.standard_normal((H, W))
    gy = rng.standard_normal((H, W))
    Dx, Dy = _torus_diff_matrix(M, N)
    e = np.concatenate([_extend_by_loops(gx, M, N, p).ravel(), _extend_by_loops(gy, M, N, p).ravel()])
    u, *_ = np.linalg.lstsq(np.vstack([Dx, Dy]), e, rcond=None)
    u = u.reshape(M, N)
    return np.abs(solve(gx, gy, M, N, p) - (u - u[0, 0])[p:p + H, p:p + W]).max()


def test_planted_mistakes_fail_the_least_squares_pin(monkeypatch):
    assert _ls_pin_error(O.solve_from_gradient) < 1e-10
    good_div, good_green = O.divergence_torus, O.green_spectrum

    monkeypatch.setattr(O, "divergence_torus", lambda Ex, Ey: (Ex - np.roll(Ex, -1, 1)) + (Ey - np.roll(Ey, -1, 0)))
    assert _ls_pin_error(O.solve_from_gradient) > 1e-3  # stencil on the wrong side
    monkeypatch.setattr(O, "divergence_torus", lambda Ex, Ey: (Ex - np.roll(Ex, 1, 0)) + (Ey - np.roll(Ey, 1, 1)))
    assert _ls_pin_error(O.solve_from_gradient) > 1e-3  # axes transposed
    monkeypatch.setattr(O, "divergence_torus", good_div)

    monkeypatch.setattr(O, "green_spectrum", lambda M, N: -good_green(M, N))
    assert _ls_pin_error(O.solve_from_gradient) > 1e-3  # Eq. 15's sign
    monkeypatch.setattr(O, "green_spectrum", lambda M, N: good_green(M, N) * 2.0)
    assert _ls_pin_error(O.solve_from_gradient) > 1e-3  # wrong normalisation
    monkeypatch.setattr(O, "green_spectrum", good_green)

    monkeypatch.setattr(O, "_offset_and_crop", lambda u, H, W, p: u[p:p + H, p:p + W])
    assert _ls_pin_error(O.solve_from_gradient) > 1e-6  # offset of Algorithm B dropped


def test_planted_adjoint_mistake_fails_transpose_pin(monkeypatch):
    good = O.backward

    def no_offset_term(gout, M, N, p):
        H, W = gout.shape
        w = O.solve_torus(O.zero_extend(gout, M, N, p))
        gEx = w - np.roll(w, -1, axis=1)
        gEy = w - np.roll(w, -1, axis=0)
        return gEx[p:p + H, p:p + W], gEy[p:p + H, p:p + W]

    H, W, p, M, N = 4, 5, 2, 8, 10
    n = H * W
    A = np.zeros((n, 2 * n))
    for k in range(2 * n):
        e = np.zeros(2 * n)
        e[k] = 1.0
        A[:, k] = O.solve_from_gradient(e[:n].reshape(H, W), e[n:].reshape(H, W), M, N, p).ravel()
    gout = np.random.default_rng(5).standard_normal((H, W))
    ref = A.T @ gout.ravel()
    gx, gy = good(gout, M, N, p)
    assert np.abs(np.concatenate([gx.ravel(), gy.ravel()]) - ref).max() < 1e-12
    gx, gy = no_offset_term(gout, M, N, p)
    assert np.abs(np.concatenate([gx.ravel(), gy.ravel()]) - ref).max() > 1e-4


# --------------------------------------------------------------------------
# Generators (host logic): seeded, shaped, and with the stated structure
# --------------------------------------------------------------------------

def test_generators_are_seeded_and_shaped():
    img, gx, gy = synth.gradient_removal_image(seed=0)
    assert gx.shape == (64, 96) and gx.dtype == np.float32
    assert 0.0 <= img.min() and img.max() <= 1.0
    img2, gx2, _ = synth.gradient_removal_image(seed=0)
    assert np.array_equal(gx, gx2)
    assert np.all(gx[:, -1] == 0) and np.all(gy[-1, :] == 0)
    # a 16x24 block of zeroed gradients exists
    z = (gx == 0) & (gy == 0)
    found = any(z[r:r + 16, c:c + 24].all() for r in range(64 - 15) for c in range(96 - 23))
    assert found
    bx, by = synth.perturbed_gradient_batch(batch=3, H=40, W=50)
    assert bx.shape == (3, 1, 40, 50)
    bx1, _ = synth.perturbed_gradient_batch(batch=3, H=40, W=50, items=[1])
    assert np.array_equal(bx1[0], bx[1])
