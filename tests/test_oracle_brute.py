"""Pins for O1, the brute-force bandlimited inner product (no GPU).

The strongest pin is Plancherel (eq. planch): for smooth, well-contained images
the bandlimited inner product of eq. (Xdg) equals (2 pi)^2 times the continuous
pixel-domain inner product <R_gamma T_delta A, B>, which for sums of isotropic
Gaussians is a closed form.  That fixes the sign of the shift, the direction of
the rotation, the conjugation, the quadrature weights and the prefactor.
"""

import math

import numpy as np
import pytest

from oracle import brute, quadrature as quad, transform as tr
from oracle.best import best_pose
from workloads import blob_params, render_blobs, shift_lattice


def _gauss_inner(blobsA, blobsB, delta, gamma):
    """Closed-form <R_gamma T_delta A, B> for isotropic Gaussian sums.

    T_delta moves a centre c to c + delta, R_gamma rotates it about the origin;
    int exp(-|x-c1|^2/2s1^2) exp(-|x-c2|^2/2s2^2) dx
        = 2 pi s1^2 s2^2/(s1^2+s2^2) exp(-|c1-c2|^2 / (2 (s1^2+s2^2))).
    """
    (ca, sa, aa), (cb, sb, ab) = blobsA, blobsB
    R = np.array([[math.cos(gamma), -math.sin(gamma)], [math.sin(gamma), math.cos(gamma)]])
    ct = (ca + delta) @ R.T
    s2 = sa[:, None] ** 2 + sb[None, :] ** 2
    d2 = np.sum((ct[:, None, :] - cb[None, :, :]) ** 2, axis=-1)
    return float(np.sum(aa[:, None] * ab[None, :] * 2 * math.pi * sa[:, None] ** 2 * sb[None, :] ** 2 / s2
                        * np.exp(-d2 / (2 * s2))))


def test_o1_matches_closed_form_gaussian_inner_products():
    n, M, two_Q = 32, 32, 128
    rng = np.random.default_rng(11)
    bA = blob_params(rng, n, 6, (2.0, 4.0), False)
    bB = blob_params(rng, n, 6, (2.0, 4.0), False)
    A, B = render_blobs(n, *bA), render_blobs(n, *bB)
    K = quad.nyquist_K(n)
    k, w = quad.radial_rule(M, K)
    Ah, Bh = tr.polar_fourier(np.stack([A, B]), k, two_Q)
    delta = brute.shift_vectors(shift_lattice(0.5, 2.0), n)
    X = brute.bandlimited_inner_products(Ah, Bh, k, w, delta)
    scale = np.abs(X).max()
    for s in [0, 7, 24, 31, 48]:
        for r in [0, 3, 40, 77, 127]:
            ref = (2 * math.pi) ** 2 * _gauss_inner(bA, bB, delta[s], math.pi * r / (two_Q // 2))
            assert abs(X[s, r] - ref) < 1e-5 * scale, (s, r, X[s, r], ref)


def _small_case(seed=5, n=16, M=8, two_Q=48):
    rng = np.random.default_rng(seed)
    A, B = rng.normal(size=(2, n, n))
    K = quad.nyquist_K(n)
    k, w = quad.radial_rule(M, K)
    Ah, Bh = tr.polar_fourier(np.stack([A, B]), k, two_Q)
    delta = brute.shift_vectors(shift_lattice(0.5, 1.5), n)
    return Ah, Bh, k, w, delta


def test_o1_imaginary_part_vanishes_for_real_images():
    Ah, Bh, k, w, delta = _small_case()
    X = brute.bandlimited_inner_products(Ah, Bh, k, w, delta, return_complex=True)
    assert np.abs(X.imag).max() < 1e-12 * np.abs(X.real).max()


def test_o1_rotating_template_on_grid_shifts_rotation_index():
    # R_{g0} B has Bhat(k, psi - g0): with g0 = r0 grid steps the scores move to r - r0.
    Ah, Bh, k, w, delta = _small_case()
    r0 = 7
    X = brute.bandlimited_inner_products(Ah, Bh, k, w, delta)
    Xr = brute.bandlimited_inner_products(Ah, np.roll(Bh, r0, axis=1), k, w, delta)
    assert np.allclose(Xr, np.roll(X, r0, axis=1), atol=1e-12 * np.abs(X).max())


def test_o1_zero_shift_is_fft_rotational_correlation():
    # delta = 0: X(0, r) = (pi/Q) sum_m w_m sum_p Ahat_mp conj(Bhat_{m,p+r}),
    # a circular cross-correlation over p, evaluated independently with FFTs.
    Ah, Bh, k, w, _ = _small_case()
    two_Q = Ah.shape[1]
    X = brute.bandlimited_inner_products(Ah, Bh, k, w, np.zeros((1, 2)))[0]
    corr = np.fft.ifft(np.conj(np.fft.fft(Ah, axis=1)) * np.fft.fft(Bh, axis=1), axis=1)  # sum_p conj(A_p) B_{p+r}
    ref = (np.pi / (two_Q // 2)) * np.sum(w[:, None] * np.conj(corr), axis=0).real
    assert np.allclose(X, ref, atol=1e-12 * np.abs(ref).max())


def test_o1_is_bilinear():
    Ah, Bh, k, w, delta = _small_case()
    Ah2, Bh2, *_ = _small_case(seed=9)
    X11 = brute.bandlimited_inner_products(Ah, Bh, k, w, delta)
    X21 = brute.bandlimited_inner_products(Ah2, Bh, k, w, delta)
    Xc = brute.bandlimited_inner_products(2.0 * Ah - 0.5 * Ah2, Bh, k, w, delta)
    assert np.allclose(Xc, 2.0 * X11 - 0.5 * X21, atol=1e-12 * np.abs(X11).max())


@pytest.mark.parametrize("r0,s_idx,tpl", [(9, 17, 1), (40, 3, 2), (0, 24, 0)])
def test_o1_recovers_planted_on_grid_pose(r0, s_idx, tpl):
    # Section 6 consistency check: the maximum over (template, rotation, shift)
    # is the true template at the true on-grid pose (noise-free image).
    n, M, two_Q = 32, 16, 96
    Q = two_Q // 2
    rng = np.random.default_rng(21)
    blobs = []
    for _ in range(3):   # unit-L2 templates (Section 6): Cauchy-Schwarz makes the true pose the maximum
        c, s, a = blob_params(rng, n, 8, (1.5, 4.0), False)
        nrm = math.sqrt((2.0 / n) ** 2 * np.sum(render_blobs(n, c, s, a) ** 2))
        blobs.append((c, s, a / nrm))
    shifts = shift_lattice(0.5, 2.0)
    theta = -math.pi * r0 / Q      # image = T_s R_theta B: best at gamma = -theta, delta = -s
    s_true = -shifts[s_idx]
    c, s, a = blobs[tpl]
    R = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
    img = render_blobs(n, c @ R.T + s_true * (2.0 / n), s, a)
    tpls = np.stack([render_blobs(n, *b) for b in blobs])
    K = quad.nyquist_K(n)
    k, w = quad.radial_rule(M, K)
    Ah = tr.polar_fourier(img, k, two_Q)[0]
    Bhs = tr.polar_fourier(tpls, k, two_Q)
    delta = brute.shift_vectors(shifts, n)
    X = np.stack([brute.bandlimited_inner_products(Ah, Bh, k, w, delta) for Bh in Bhs])
    t, r, si, _ = best_pose(X)
    assert (t, r, si) == (tpl, r0 % two_Q, s_idx)
