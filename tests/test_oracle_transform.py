"""Pins for the oracle's radial rule and pixel -> polar Fourier -> Fourier--Bessel
transform, against closed forms and exact symmetries (no GPU)."""

import math

import numpy as np
import pytest

from oracle import quadrature as quad
from oracle import transform as tr
from workloads import render_blobs


@pytest.mark.parametrize("M", [4, 16, 32])
def test_radial_rule_exact_for_polynomials(M):
    # Section 3.1: int_0^K g(k) k dk with a Gauss-Jacobi(0,1) rule of M nodes is
    # exact for polynomials g of degree <= 2M-1.  int_0^K k^d k dk = K^(d+2)/(d+2).
    K = 0.5 * math.pi * 2 * M
    k, w = quad.radial_rule(M, K)
    assert np.all(np.diff(k) > 0) and k[0] > 0 and k[-1] < K
    assert abs(w.sum() - K * K / 2) < 1e-12 * K * K
    for d in range(0, 2 * M):
        exact = K ** (d + 2) / (d + 2)
        got = float(np.sum(w * k ** d))
        assert abs(got - exact) <= 1e-11 * exact, d


def test_radial_rule_not_exact_beyond_degree():
    # sanity: a wrong rule (e.g. Gauss-Legendre weights) would also fail the
    # exactness test above; here check degree 2M is NOT integrated exactly.
    M, K = 6, 10.0
    k, w = quad.radial_rule(M, K)
    d = 2 * M
    assert abs(np.sum(w * k ** d) - K ** (d + 2) / (d + 2)) > 1e-9 * K ** (d + 2)


def _gauss_image(n, c, s):
    return render_blobs(n, np.asarray([c], float), np.asarray([s], float), np.asarray([1.0]))


def test_polar_fourier_of_gaussian_matches_continuous_ft():
    # eq. (Ahat): FT of exp(-|x-c|^2/(2 s^2)) is 2 pi s^2 exp(-s^2 |k|^2/2) exp(-i k.c).
    # The trapezoid sum of eq. (Ahattrap) on a well-sampled, well-contained
    # Gaussian agrees spectrally.  An off-centre, asymmetric centre checks the
    # sign of the exponent, the axis order (first index = x) and the grid offset.
    n, M, two_Q = 32, 16, 96
    dx = 2.0 / n
    c, s = (0.11, -0.07), 2.0 * dx
    img = _gauss_image(n, c, s)
    K = quad.nyquist_K(n)
    k, _ = quad.radial_rule(M, K)
    Ah = tr.polar_fourier(img, k, two_Q)[0]
    psi = quad.polar_angles(two_Q)
    kx, ky = np.outer(k, np.cos(psi)), np.outer(k, np.sin(psi))
    exact = 2 * math.pi * s * s * np.exp(-0.5 * s * s * (kx ** 2 + ky ** 2)) * np.exp(-1j * (kx * c[0] + ky * c[1]))
    assert np.abs(Ah - exact).max() < 1e-8 * np.abs(exact).max()


def test_ring_coefficients_match_fft_library():
    rng = np.random.default_rng(0)
    Ah = rng.normal(size=(3, 5, 24)) + 1j * rng.normal(size=(3, 5, 24))
    a = tr.ring_coefficients(Ah)
    assert np.allclose(a, np.fft.fft(Ah, axis=-1) / 24, atol=1e-13)


def _bordered_random(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n))
    A[0, :] = 0.0
    A[:, 0] = 0.0
    return A


def test_quarter_turn_is_diagonal_phase():
    # eq. (rot-def): R_gamma A(x) = A(R_{-gamma} x).  For gamma = pi/2 on the grid
    # x_i = (i - n/2) dx this is the exact pixel permutation A'[i][j] = A[j][n-i]
    # when row 0 and column 0 are zero.  Section 3: rotation acts on the
    # Fourier--Bessel coefficients as a(k; q) -> exp(-i q gamma) a(k; q).
    n, M, two_Q = 16, 8, 48
    A = _bordered_random(n, 1)
    Ar = np.zeros_like(A)
    for i in range(1, n):
        for j in range(n):
            Ar[i, j] = A[j, n - i]
    K = quad.nyquist_K(n)
    k, _ = quad.radial_rule(M, K)
    a = tr.fourier_bessel(A, k, two_Q)[0]
    ar = tr.fourier_bessel(Ar, k, two_Q)[0]
    q = np.arange(two_Q)
    q = np.where(q >= two_Q // 2, q - two_Q, q)
    assert np.abs(ar - np.exp(-1j * q * math.pi / 2)[None, :] * a).max() < 1e-11 * np.abs(a).max()


def test_integer_shift_is_plane_wave_factor():
    # eq. (Tdeltahat)/(Fdk): translating by delta multiplies Ahat by exp(-i delta.k).
    n, M, two_Q = 16, 8, 48
    dx = 2.0 / n
    A = np.zeros((n, n))
    A[3:11, 4:12] = np.random.default_rng(2).normal(size=(8, 8))
    u, v = 2, -3
    As = np.roll(np.roll(A, u, axis=0), v, axis=1)  # zero border: roll == shift
    K = quad.nyquist_K(n)
    k, _ = quad.radial_rule(M, K)
    Ah = tr.polar_fourier(A, k, two_Q)[0]
    Ahs = tr.polar_fourier(As, k, two_Q)[0]
    psi = quad.polar_angles(two_Q)
    phase = np.exp(-1j * (u * dx * np.outer(k, np.cos(psi)) + v * dx * np.outer(k, np.sin(psi))))
    assert np.abs(Ahs - phase * Ah).max() < 1e-12 * np.abs(Ah).max()


def test_real_images_have_hermitian_ring_coefficients():
    # Ahat(-k) = conj Ahat(k) for real A, and psi_{p+Q} = psi_p + pi, so
    # a(k; -q) = (-1)^q conj a(k; q).
    n, M, two_Q = 16, 8, 48
    A = np.random.default_rng(3).normal(size=(n, n))
    K = quad.nyquist_K(n)
    k, _ = quad.radial_rule(M, K)
    a = tr.fourier_bessel(A, k, two_Q)[0]
    q = np.arange(two_Q)
    qs = np.where(q >= two_Q // 2, q - two_Q, q)
    lhs = a[:, (-qs) % two_Q]
    rhs = ((-1.0) ** np.abs(qs))[None, :] * np.conj(a)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(a).max()
