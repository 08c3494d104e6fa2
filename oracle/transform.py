"""Pixel images to polar Fourier samples and Fourier--Bessel coefficients
(oracle; test infrastructure only).

eq. (Ahattrap), Section 2.1:
    Ahat(k) = dx^2 sum_{i,j=0}^{n-1} A_ij exp(-i k . x_ij),  x_ij = (i dx - 1, j dx - 1),
with dx = 2/n; the first array index is x. The sum runs over i, j = 0..n-1 (the
index range the paper uses to define the pixel grid).

eq. (aqkcalc), Section 3.2: on each ring k_m,
    a(k_m; q) = (1 / 2Q) sum_{p} Ahat(k_m, psi_p) exp(-i q psi_p),
a length-2Q DFT. q is taken modulo 2Q and stored at index q mod 2Q, so index
t >= Q holds q = t - 2Q.
"""

from __future__ import annotations

import numpy as np

from .quadrature import polar_angles


def pixel_coords(n: int) -> np.ndarray:
    dx = 2.0 / n
    return np.arange(n, dtype=np.float64) * dx - 1.0


def polar_fourier(images: np.ndarray, k: np.ndarray, two_Q: int) -> np.ndarray:
    """Direct trapezoid sum of eq. (Ahattrap) on the polar grid (k_m, psi_p).

    images: [B, n, n] real. Returns complex128 [B, M, 2Q].
    The exponential factors per axis (exp(-i k_x x_i) and exp(-i k_y y_j)) are
    formed explicitly; the double sum is then two contractions.
    """
    images = np.asarray(images, dtype=np.float64)
    if images.ndim == 2:
        images = images[None]
    n = images.shape[-1]
    dx = 2.0 / n
    xs = pixel_coords(n)
    psi = polar_angles(two_Q)
    kx = np.outer(k, np.cos(psi))  # [M, 2Q]
    ky = np.outer(k, np.sin(psi))
    Ex = np.exp(-1j * kx[..., None] * xs)  # [M, 2Q, n]  over i (x)
    Ey = np.exp(-1j * ky[..., None] * xs)  # [M, 2Q, n]  over j (y)
    out = np.empty((images.shape[0], k.size, two_Q), dtype=np.complex128)
    for b in range(images.shape[0]):
        T = np.einsum("ij,mpj->mpi", images[b], Ey)       # sum over j
        out[b] = dx * dx * np.einsum("mpi,mpi->mp", Ex, T)  # sum over i
    return out


def ring_coefficients(Ahat: np.ndarray) -> np.ndarray:
    """eq. (aqkcalc): a(k_m; q) = (1/2Q) sum_p Ahat(k_m, psi_p) e^{-i q psi_p}.

    Written as the explicit DFT matrix product; output index t = q mod 2Q.
    """
    two_Q = Ahat.shape[-1]
    p = np.arange(two_Q)
    F = np.exp(-2j * np.pi * np.outer(p, p) / two_Q)  # [q, p]
    return np.einsum("qp,...mp->...mq", F, Ahat) / two_Q


def fourier_bessel(images: np.ndarray, k: np.ndarray, two_Q: int) -> np.ndarray:
    """Images [B, n, n] -> Fourier--Bessel coefficients a [B, M, 2Q] (complex128)."""
    return ring_coefficients(polar_fourier(images, k, two_Q))
