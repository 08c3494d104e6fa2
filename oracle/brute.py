"""O1: the discretized bandlimited inner product by brute force
(oracle; test infrastructure only).

eq. (Xdg), Section 2:
    X(delta, gamma) = int_{Omega_K} F(delta, k) Ahat(k) conj(R_{-gamma} Bhat(k)) dk,
    F(delta, k) = exp(-i delta . k)   (eq. Fdk),   R_{-gamma} Bhat(k, psi) = Bhat(k, psi + gamma).
The printed eq. (Xdg) drops the conjugate on the rotated template; it is restored
here (it is present in eq. bessel-inner and eq. Xtrunc).

Discretized with the radial rule of Section 3.1 and the uniform angular grid of
Section 3.2 (angular step pi/Q), on the rotation grid gamma_r = pi r / Q:
    X(s, r) = (pi / Q) sum_m w_m sum_p F(delta_s, k_m, psi_p) Ahat(k_m, psi_p)
                                      conj(Bhat(k_m, psi_{(p + r) mod 2Q})).
A is the image (translated by delta, then rotated by gamma); B is the template.
The real part is returned (the imaginary part vanishes for real images up to
rounding because the grid is symmetric under psi -> psi + pi).
"""

from __future__ import annotations

import numpy as np

from .quadrature import polar_angles


def shift_vectors(shifts_px: np.ndarray, n: int) -> np.ndarray:
    """Shifts in pixels -> delta in image units (delta = s_px * dx, dx = 2/n)."""
    return np.asarray(shifts_px, dtype=np.float64) * (2.0 / n)


def bandlimited_inner_products(Ahat: np.ndarray, Bhat: np.ndarray, k: np.ndarray, w: np.ndarray,
                               delta: np.ndarray, return_complex: bool = False) -> np.ndarray:
    """O1 for one image/template pair.

    Ahat, Bhat: [M, 2Q] polar Fourier samples. delta: [N, 2] shifts (image units).
    Returns X [N, 2Q] (rows: shift s, columns: rotation r).

    The double sum over (m, p) for every (s, r) is one contraction; the rotated
    template Bhat(k_m, psi_{p+r}) is formed explicitly as an index gather.
    """
    two_Q = Ahat.shape[-1]
    Q = two_Q // 2
    psi = polar_angles(two_Q)
    kx = np.outer(k, np.cos(psi))
    ky = np.outer(k, np.sin(psi))
    F = np.exp(-1j * (delta[:, 0, None, None] * kx + delta[:, 1, None, None] * ky))  # [N, M, 2Q]
    C = F * Ahat[None]
    pr = (np.arange(two_Q)[None, :] + np.arange(two_Q)[:, None]) % two_Q           # [r, p]
    Brot = Bhat[:, pr]                                                                # [M, r, p]
    X = (np.pi / Q) * np.einsum("m,smp,mrp->sr", w, C, np.conj(Brot))
    return X if return_complex else X.real


def bandlimited_inner_products_rot(Ahat: np.ndarray, Bhat: np.ndarray, k: np.ndarray, w: np.ndarray,
                                   delta: np.ndarray, gammas: np.ndarray) -> np.ndarray:
    """O1 at arbitrary rotation angles gammas [R] (radians): X [N, R].

    Off the grid psi_p the rotated template Bhat(k_m, psi_p + gamma) is the trigonometric
    interpolant of its ring samples with the frequencies q = -Q..Q-1 of the ring DFT
    (eq. aqkcalc): Bhat(k_m, psi) = sum_q b(k_m; q) exp(i q psi). On the grid this is Bhat at a
    grid angle exactly; it is the reading under which a finer rotation grid is the zero-padding
    of Step 2 (Section 3.2).
    """
    two_Q = Ahat.shape[-1]
    Q = two_Q // 2
    psi = polar_angles(two_Q)
    q = np.arange(two_Q)
    q = np.where(q >= Q, q - two_Q, q)
    b = (Bhat @ np.exp(-1j * np.outer(psi, q))) / two_Q                              # b(k_m; q), [M, q]
    ang = psi[None, :] + np.asarray(gammas, dtype=np.float64)[:, None]               # [r, p]
    Brot = np.einsum("mq,rpq->mrp", b, np.exp(1j * ang[:, :, None] * q[None, None, :]))
    kx = np.outer(k, np.cos(psi))
    ky = np.outer(k, np.sin(psi))
    F = np.exp(-1j * (delta[:, 0, None, None] * kx + delta[:, 1, None, None] * ky))  # [N, M, 2Q]
    C = F * Ahat[None]
    return ((np.pi / Q) * np.einsum("m,smp,mrp->sr", w, C, np.conj(Brot))).real
