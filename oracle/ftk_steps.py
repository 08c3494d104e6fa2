"""O2: the FTK algorithm step by step (oracle; test infrastructure only).

Section 4.5, eq. (fbk3), for one image a and one template b (Fourier--Bessel
coefficients on the radial nodes k_m, index q stored modulo 2Q):

  Step 1  Zhat_zeta(q) = 2 pi sum_m w_m conj(b(k_m; q)) a(k_m; q - l_zeta) G_zeta(k_m)
  Step 2  Z_zeta(gamma) = sum_q exp(-i q gamma) Zhat_zeta(q),     gamma_r = pi r / Q
          (or on a finer grid gamma_r = 2 pi r / R, R > 2Q: Step 2 zero-padded)
  Step 3  X(delta, gamma) = sum_zeta Y_zeta(delta) Z_zeta(gamma)

q runs over the 2Q values -Q..Q-1 and q - l is taken modulo 2Q (the ring DFT of
eq. aqkcalc is periodic in q). Step 2 is written as the explicit DFT matrix.
"""

from __future__ import annotations

import numpy as np

from .svd_plan import Plan, radial_factors, shift_factors


def signed_q(two_Q: int) -> np.ndarray:
    q = np.arange(two_Q)
    return np.where(q >= two_Q // 2, q - two_Q, q)


def ftk_scores(a: np.ndarray, b: np.ndarray, k: np.ndarray, w: np.ndarray, plan: Plan,
               delta: np.ndarray, return_complex: bool = False, n_rot: int | None = None) -> np.ndarray:
    """X^svd for one image (a: [M, 2Q]) against templates b ([NT, M, 2Q] or [M, 2Q]).

    Returns [NT, N, R] (or [N, R]): rows shift s, columns rotation r, gamma_r = 2 pi r / R
    (a CTF plan, Section 7.1, has n_tau N rows: defocus b, shift s at row b N + s).
    R = n_rot, default 2Q (the grid of Section 3.2); a larger R evaluates Step 2 on a finer
    rotation grid, which is the zero-padding of the length-2Q transform over q (Section 3.2).
    """
    single = b.ndim == 2
    if single:
        b = b[None]
    two_Q = a.shape[-1]
    R = two_Q if n_rot is None else int(n_rot)
    qs = signed_q(two_Q)
    gam = 2.0 * np.pi * np.arange(R) / R
    dft = np.exp(-1j * np.outer(qs, gam))                     # [q, r]
    G = dict(radial_factors(plan, k))                          # l -> [M, H_l]
    Y = dict(shift_factors(plan, delta))                       # l -> [N, H_l]
    n_rows = delta.shape[0] * max(1, len(plan.taus))           # (defocus, shift) rows for a CTF plan
    X = np.zeros((b.shape[0], n_rows, R), dtype=np.complex128)
    bq = np.conj(b[:, :, qs % two_Q])                          # conj b(k_m; q), [NT, M, q]
    for l in sorted(G):
        a_shift = a[:, (qs - l) % two_Q]                       # a(k_m; q - l), [M, q]
        # Step 1
        Zhat = 2.0 * np.pi * np.einsum("m,jmq,mq,mh->jhq", w, bq, a_shift, G[l])
        # Step 2
        Z = np.einsum("jhq,qr->jhr", Zhat, dft)
        # Step 3
        X += np.einsum("sh,jhr->jsr", Y[l], Z)
    out = X if return_complex else X.real
    return out[0] if single else out

