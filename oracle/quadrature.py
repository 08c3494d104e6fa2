"""Radial quadrature and polar grid (oracle; test infrastructure only).

Section 3.1: the k-integral on [0, K] with area element k dk is replaced by a
Gauss--Jacobi rule of type alpha = 0, beta = 1, giving nodes k_m in (0, K) and
weights w_m, m = 1..M, with  int_0^K g(k) k dk ~= sum_m g(k_m) w_m.

Section 3.2: the angular grid is psi_p = pi p / Q, p = 0..2Q-1 (the paper counts
p from 1 with psi_p = pi (p-1)/Q; the set is the same).
"""

from __future__ import annotations

import numpy as np
import scipy.special as sps


def radial_rule(M: int, K: float):
    """Gauss--Jacobi(0,1) nodes and weights mapped to [0, K] with weight k dk.

    With t in [-1, 1] and k = K (1 + t) / 2 one has k dk = (K^2 / 4)(1 + t) dt,
    so the Jacobi weight (1 - t)^0 (1 + t)^1 is exactly the area element.
    """
    t, v = sps.roots_jacobi(M, 0.0, 1.0)
    k = 0.5 * K * (1.0 + t)
    w = 0.25 * K * K * v
    return k.astype(np.float64), w.astype(np.float64)


def polar_angles(two_Q: int) -> np.ndarray:
    """psi_p = 2 pi p / (2Q), p = 0..2Q-1 (Section 3.2)."""
    return 2.0 * np.pi * np.arange(two_Q, dtype=np.float64) / two_Q


def nyquist_K(n: int) -> float:
    """K = pi / dx = (pi / 2) n (Remark r:nyq)."""
    return 0.5 * np.pi * n
