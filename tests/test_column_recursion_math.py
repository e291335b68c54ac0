"""The operator identity behind the recursive column solve, pinned on the CPU.

After the row DFT, column l of the Green multiply of Eq. 23 (G = 1/lambda,
lambda(k, l) = 2 cos(2 pi k/M) + 2 cos(2 pi l/N) - 4, numpy normalisation) is
the cyclic convolution along the torus rows whose DFT is 1/lambda(., l): the
inverse of the cyclic tridiagonal matrix T_l = S + S^-1 - b_l I with
b_l = 4 - 2 cos(2 pi l/N). With a + 1/a = b, a < 1,
  T^-1 = -a / (1 - a^2) [ (I - a S)^-1 + (I - a S^-1)^-1 - I ],
and (I - a S)^-1 = sum_{k<M} a^k S^k / (1 - a^M) on the cycle. These tests
check the identity against a dense inverse and against the oracle's own Green
spectrum, and that the recursion's band sweep reproduces the cyclic filter.
"""
import numpy as np
import pytest

import oracle.gfc_oracle as O


def _shift(M):
    S = np.zeros((M, M))
    for r in range(M):
        S[r, (r - 1) % M] = 1.0  # (S y)[r] = y[r - 1]
    return S


def _a(b):
    d = b - 2.0
    return 2.0 / (2.0 + d + np.sqrt(d * (4.0 + d)))


@pytest.mark.parametrize("M,N,l", [(12, 10, 1), (12, 10, 5), (9, 14, 3), (16, 16, 8), (810, 1250, 1)])
def test_tridiagonal_inverse_is_two_recursions(M, N, l):
    if M > 64:  # dense check on a smaller cycle with the same b
        M = 64
    S = _shift(M)
    b = 4.0 - 2.0 * np.cos(2 * np.pi * l / N)
    T = S + S.T - b * np.eye(M)
    a = _a(b)
    assert abs(a + 1.0 / a - b) < 1e-12 and 0 < a < 1
    I = np.eye(M)
    R = -a / (1 - a * a) * (np.linalg.inv(I - a * S) + np.linalg.inv(I - a * S.T) - I)
    assert np.abs(R - np.linalg.inv(T)).max() < 1e-10 * np.abs(np.linalg.inv(T)).max()
    # the cyclic causal filter in closed form
    C = sum(a ** k * np.linalg.matrix_power(S, k) for k in range(M)) / (1 - a ** M)
    assert np.abs(C - np.linalg.inv(I - a * S)).max() < 1e-10


@pytest.mark.parametrize("M,N", [(12, 10), (24, 24)])
def test_column_operator_is_the_oracles_green_column(M, N):
    """The column convolution with DFT 1/lambda(., l) (oracle Green spectrum times MN,
    the numpy normalisation of the oracle's inverse transform) equals T_l^-1, l >= 1."""
    G = O.green_spectrum(M, N)  # [M, N], 1/lambda with G[0,0] = 0
    S = _shift(M)
    for l in range(1, N // 2 + 1):
        col = np.fft.ifft(G[:, l]).real  # kernel of the cyclic convolution along rows
        K = np.array([[col[(r - c) % M] for c in range(M)] for r in range(M)])
        b = 4.0 - 2.0 * np.cos(2 * np.pi * l / N)
        T = S + S.T - b * np.eye(M)
        assert np.abs(K - np.linalg.inv(T)).max() < 1e-10, l


def test_band_sweep_reproduces_the_cyclic_filters():
    """Bands with zero carries, then the carries from one sweep around the cycle
    (the pad rows above band 0 and tail rows below the last band zero), give the
    same causal and anticausal filter outputs as the dense inverses."""
    rng = np.random.default_rng(0)
    M, p, band, G = 37, 4, 6, 5  # rows p .. p + 30 in 5 bands, 3 tail rows
    tail = M - p - band * G
    x = np.zeros(M, complex)
    x[p:p + band * G] = rng.standard_normal(band * G) + 1j * rng.standard_normal(band * G)
    a = _a(2.0 + 0.3)
    S = _shift(M)
    I = np.eye(M)
    y_ref = np.linalg.solve(I - a * S, x)
    yp_ref = np.linalg.solve(I - a * S.T, x)
    starts = [p + band * g for g in range(G)]
    e = [sum(a ** (band - 1 - i) * x[s + i] for i in range(band)) for s in starts]
    ep = [sum(a ** i * x[s + i] for i in range(band)) for s in starts]
    P, t = [], 0.0
    for g in range(G):
        P.append(t)
        t = e[g] + a ** band * t
    ylast = a ** tail * t / (1 - a ** M)
    assert abs(ylast - y_ref[M - 1]) < 1e-12
    cin = a ** p * ylast
    Q, t = [0.0] * G, 0.0
    for g in range(G - 1, -1, -1):
        Q[g] = t
        t = ep[g] + a ** band * t
    y0 = a ** p * t / (1 - a ** M)
    assert abs(y0 - yp_ref[0]) < 1e-12
    for g, s in enumerate(starts):
        c = P[g] + a ** (band * g) * cin  # y[s - 1]
        cp = Q[g] + a ** (tail + band * (G - 1 - g)) * y0  # y'[s + band]
        assert abs(c - y_ref[s - 1]) < 1e-12 and abs(cp - yp_ref[(s + band) % M]) < 1e-12
