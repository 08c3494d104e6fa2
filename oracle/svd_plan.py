"""The FTK plan: operator SVD of the modal translation kernels
(oracle; test infrastructure only).

Section 4.5. For each Bessel order l the kernel J_l(delta k) on
[0, D] x [0, K] (weights delta d delta and k dk) has the operator SVD
    J_l(delta k) = sum_eta U_eta(delta; l) Sigma_eta(l) V_eta(k; l)      (eq. Jsvd).
The singular values depend only on K D = 2 pi W (Lemma 1 proof), so the SVD is
computed in the rescaled variables x = K delta in [0, 2 pi W] (weight x dx) and
y = k / K in [0, 1] (weight y dy); U(x) V(y) products are then evaluated at
x = K delta_s and y = k_m / K (the rescaling factors K and 1/K of U and V cancel
in their product, which is all the algorithm uses).

Remark r:svd is followed as written: J_l(x y) is projected, by tensor-product
Gauss--Jacobi quadrature, onto orthonormal Jacobi(alpha=0, beta=1) polynomial
bases in x and in y (orthonormal for x dx and y dy); the coefficient matrix is
decomposed with a dense SVD; singular functions are the basis sums with the
singular-vector entries as coefficients.

Truncation (eq. svdtrunc and the text after eq. svdobjective): keep every term
with Sigma_eta(l) > eps (the paper writes both ">" and ">=" for this rule; strict
is used). Orders are scanned over |l| <= 2 calH, where calH is the constant of
Theorem 1's proof, beyond which H_l = 0 is proven.

  Y_eta(delta; l) = U_eta(delta; l) exp(-i l (omega + pi/2)),
  G_eta(k; l)     = Sigma_eta(l) V_eta(k; l).

Alternative weight on k (the remark following Remark r:svd): with a spectral weight
rho(k) the L2 norm over the k disk becomes rho(k) k dk, and the SVD is that of
J_l(delta k) sqrt(rho(k)) in the plain weights; then V_eta = Vtilde_eta / sqrt(rho), so
that U Sigma V reconstructs J_l(delta k) itself, optimally in the rho-weighted norm.
The weight here is the Gaussian spectral decay rho(y) ∝ exp(-beta y^2), y = k / K,
normalized to unit mean over the disk (int_0^1 rho(y) y dy = 1/2), so beta = 0 is the
plain plan.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.special as sps


def theorem1_calH(W: float, eps: float) -> float:
    """calH_{eps,W} = max(pi e^2 W, log(2 pi W / eps)) + 3/2 (proof of Theorem 1)."""
    return max(math.pi * math.e ** 2 * W, math.log(2.0 * math.pi * W / eps)) + 1.5


def lemma1_bound(l: int, W: float, eps: float) -> float:
    """H_l <= max(0, pi e^2 W - |l|/2, log(2 pi W/eps) + 3/2 - |l|/2)   (eq. rank)."""
    return max(0.0, math.pi * math.e ** 2 * W - abs(l) / 2.0,
               math.log(2.0 * math.pi * W / eps) + 1.5 - abs(l) / 2.0)


def _orthonormal_jacobi01(deg: int, x: np.ndarray, X: float) -> np.ndarray:
    """Jacobi(0,1) polynomials 0..deg-1 orthonormal on [0, X] for weight x dx.

    With t = 2x/X - 1, x dx = (X^2/4)(1 + t) dt and int (1+t) P_a^{(0,1)}(t)^2 dt = 2/(a+1).
    Returns [deg, len(x)].
    """
    t = 2.0 * x / X - 1.0
    out = np.empty((deg, x.size))
    for a in range(deg):
        out[a] = sps.eval_jacobi(a, 0.0, 1.0, t) / math.sqrt(0.25 * X * X * 2.0 / (a + 1))
    return out


def spectral_weight(y: np.ndarray, decay: float) -> np.ndarray:
    """rho(y) = exp(-decay y^2) decay / (1 - exp(-decay)): unit mean over the disk for weight y dy."""
    y = np.asarray(y, float)
    if decay == 0.0:
        return np.ones_like(y)
    return np.exp(-decay * y * y) * (decay / -math.expm1(-decay))


def _gauss_jacobi01(nq: int, X: float):
    t, v = sps.roots_jacobi(nq, 0.0, 1.0)
    return 0.5 * X * (1.0 + t), 0.25 * X * X * v


@dataclasses.dataclass
class ModalSVD:
    l: int
    sigma: np.ndarray      # [H_l] retained singular values
    sigma_all: np.ndarray  # all computed singular values (descending)
    u: np.ndarray          # [nb, H_l] coefficients of U in the x basis
    v: np.ndarray          # [nb, H_l] coefficients of V in the y basis
    X: float               # 2 pi W
    nb: int
    decay: float = 0.0     # spectral weight rho(y) ∝ exp(-decay y^2); 0: plain weights

    def U(self, x: np.ndarray) -> np.ndarray:
        """U_eta(x; l) at rescaled shift magnitudes x = K delta: [len(x), H_l]."""
        return _orthonormal_jacobi01(self.nb, np.asarray(x, float), self.X).T @ self.u

    def V(self, y: np.ndarray) -> np.ndarray:
        """V_eta(y; l) at rescaled frequencies y = k / K: [len(y), H_l]."""
        y = np.asarray(y, float)
        vt = _orthonormal_jacobi01(self.nb, y, 1.0).T @ self.v
        return vt / np.sqrt(spectral_weight(y, self.decay))[:, None]


def modal_svd(l: int, W: float, eps: float, nb: int | None = None, nq: int | None = None,
              decay: float = 0.0) -> ModalSVD:
    """Operator SVD of J_l(x y) on [0, 2 pi W] x [0, 1] (Remark r:svd), in the k weight
    rho(y) y dy (spectral_weight; decay 0: y dy)."""
    X = 2.0 * math.pi * W
    if nb is None:
        nb = int(math.ceil(X)) + 40
    if nq is None:
        nq = nb + 24
    xq, wx = _gauss_jacobi01(nq, X)
    yq, wy = _gauss_jacobi01(nq, 1.0)
    Px = _orthonormal_jacobi01(nb, xq, X)      # [nb, nq]
    Py = _orthonormal_jacobi01(nb, yq, 1.0)
    Jm = sps.jv(l, np.outer(xq, yq)) * np.sqrt(spectral_weight(yq, decay))[None, :]   # [nq, nq]
    C = (Px * wx) @ Jm @ (Py * wy).T            # projection coefficients [nb, nb]
    u, s, vt = np.linalg.svd(C)
    H = int(np.sum(s > eps))
    return ModalSVD(l=l, sigma=s[:H].copy(), sigma_all=s, u=u[:, :H].copy(), v=vt[:H].T.copy(),
                    X=X, nb=nb, decay=float(decay))


@dataclasses.dataclass
class Plan:
    W: float
    eps: float
    K: float
    modes: dict            # l -> ModalSVD (only orders with H_l > 0)
    taus: tuple = ()       # CTF defocus values (Section 7.1); empty: translations only
    phase: float = 0.0     # CTF phase offset
    decay: float = 0.0     # spectral weight of the SVD (modal_svd); 0: plain weights

    @property
    def H(self) -> int:
        return sum(m.sigma.size for m in self.modes.values())

    def H_l(self, l: int) -> int:
        return self.modes[l].sigma.size if l in self.modes else 0

    def terms(self):
        """Flattened index zeta -> (l, eta, Sigma), in non-increasing Sigma order."""
        t = [(m.l, e, float(m.sigma[e])) for m in self.modes.values() for e in range(m.sigma.size)]
        t.sort(key=lambda z: (-z[2], abs(z[0]), -z[0], z[1]))
        return t


def build_plan(W: float, eps: float, K: float, nb: int | None = None, nq: int | None = None,
               decay: float = 0.0) -> Plan:
    L_scan = int(math.ceil(2.0 * theorem1_calH(W, eps)))
    modes = {}
    for l in range(-L_scan, L_scan + 1):
        m = modal_svd(l, W, eps, nb, nq, decay)
        if m.sigma.size > 0:
            modes[l] = m
    return Plan(W=W, eps=eps, K=K, modes=modes, decay=float(decay))


def radial_factors(plan: Plan, k: np.ndarray):
    """G_zeta(k_m) = Sigma V(k_m / K) per retained term: list of (l, [M, H_l])."""
    return [(l, m.V(k / plan.K) * m.sigma[None, :]) for l, m in sorted(plan.modes.items())]


def shift_factors(plan: Plan, delta: np.ndarray):
    """Y_zeta(delta_s) = U(K delta_s) exp(-i l (omega_s + pi/2)): list of (l, [N, H_l]).

    For a CTF plan the rows are the pairs (defocus b, shift s), row b N + s, with
    U(K delta_s, tau_b).
    """
    d = np.hypot(delta[:, 0], delta[:, 1])
    om = np.arctan2(delta[:, 1], delta[:, 0])
    out = []
    for l, m in sorted(plan.modes.items()):
        ph = np.exp(-1j * l * (om + 0.5 * np.pi))[:, None]
        if plan.taus:
            out.append((l, np.concatenate([m.U(plan.K * d, b) * ph for b in range(len(plan.taus))], axis=0)))
        else:
            out.append((l, m.U(plan.K * d) * ph))
    return out


# ---- CTF-filtered templates (Section 7.1) ------------------------------------------------
#
# Translating by delta and filtering the template by a radially symmetric contrast transfer
# function C(k; tau) multiplies the Fourier transform pointwise by F(delta, k) C(k; tau). Per
# order l the kernel J_l(delta k) C(k; tau) is factorized jointly in (delta, tau) and k:
#   J_l(x y) C(K y; tau_b) = sum_eta U_eta(x, tau_b) Sigma_eta V_eta(y),
# the operator SVD on {(x, tau_b)} x [0, 1] with weights x dx / n_tau and y dy (each defocus
# value weighted equally). Steps 1-3 are unchanged with the rows (tau_b, delta_s) in place
# of the shifts.


def ctf(k: np.ndarray, K: float, tau: float, phase: float) -> np.ndarray:
    """C(k; tau) = -sin(pi tau (k / K)^2 + phase): defocus tau in units of half phase turns at
    k = K (no spherical aberration), amplitude-contrast phase `phase`."""
    return -np.sin(np.pi * tau * (np.asarray(k, float) / K) ** 2 + phase)


@dataclasses.dataclass
class CtfModalSVD:
    l: int
    sigma: np.ndarray      # [H_l]
    sigma_all: np.ndarray
    u: np.ndarray          # [n_tau, nb, H_l] coefficients of U(., tau_b) in the x basis
    v: np.ndarray          # [nb, H_l]
    X: float
    nb: int

    def U(self, x: np.ndarray, b: int) -> np.ndarray:
        return _orthonormal_jacobi01(self.nb, np.asarray(x, float), self.X).T @ self.u[b]

    def V(self, y: np.ndarray) -> np.ndarray:
        return _orthonormal_jacobi01(self.nb, np.asarray(y, float), 1.0).T @ self.v


def modal_svd_ctf(l: int, W: float, eps: float, K: float, taus, phase: float, nb: int | None = None,
                  nq: int | None = None) -> CtfModalSVD:
    """Joint operator SVD of J_l(x y) C(K y; tau_b) over (x, tau_b) and y, by projection as in
    Remark r:svd (one x-basis block per defocus value, stacked with weight 1/sqrt(n_tau))."""
    X = 2.0 * math.pi * W
    taus = tuple(float(t) for t in taus)
    if nb is None:
        nb = int(math.ceil(X)) + 40 + int(math.ceil(2 * max(abs(t) for t in taus)))
    if nq is None:
        nq = nb + 24
    xq, wx = _gauss_jacobi01(nq, X)
    yq, wy = _gauss_jacobi01(nq, 1.0)
    Px = _orthonormal_jacobi01(nb, xq, X)
    Py = _orthonormal_jacobi01(nb, yq, 1.0)
    Jm = sps.jv(l, np.outer(xq, yq))
    blocks = [(Px * wx) @ (Jm * ctf(K * yq, K, t, phase)[None, :]) @ (Py * wy).T for t in taus]
    Cst = np.concatenate(blocks, axis=0) / math.sqrt(len(taus))     # [n_tau nb, nb]
    u, s, vt = np.linalg.svd(Cst, full_matrices=False)
    H = int(np.sum(s > eps))
    uu = (u[:, :H] * math.sqrt(len(taus))).reshape(len(taus), nb, H)
    return CtfModalSVD(l=l, sigma=s[:H].copy(), sigma_all=s, u=uu, v=vt[:H].T.copy(), X=X, nb=nb)


def build_plan_ctf(W: float, eps: float, K: float, taus, phase: float, nb: int | None = None,
                   nq: int | None = None) -> Plan:
    L_scan = int(math.ceil(2.0 * theorem1_calH(W, eps)))
    modes = {}
    for l in range(-L_scan, L_scan + 1):
        m = modal_svd_ctf(l, W, eps, K, taus, phase, nb, nq)
        if m.sigma.size > 0:
            modes[l] = m
    return Plan(W=W, eps=eps, K=K, modes=modes, taus=tuple(float(t) for t in taus), phase=float(phase))
