"""FP64 reference of the template-proposal network and its gradients
(oracle; test infrastructure only).

The network (no counterpart in the paper; it shortlists templates and a shift
window for the FTK search) maps Fourier--Bessel coefficients a(k_m; q) of one
image to template logits and a shift estimate:

  features   x0[m][q] = log(eps_f + |a(k_m; q)|), q = 0..Q-1 (rotation acts on a as a
             phase, so |a| does not depend on the in-plane rotation);
             lin = (Re a(k_m; 0), Im a(k_m; 0), Re a(k_m; 1), Im a(k_m; 1)) for all m
  conv1..4   3x3 convolutions with zero padding 1, bias, ReLU; a 2x2 average pool
             after conv1, conv2, conv3; a global average pool after conv4
  head       fc1 on [pooled conv4 features, lin] + ReLU, fc2 -> NT logits + 2 shift outputs
  loss       mean over the batch of  CE(logits, label) + lam * ||shift_out - shift_target||^2

Every operation is written out plainly with numpy; `tests/test_oracle_nn.py` pins
the backward pass with finite differences of the forward pass.
"""

from __future__ import annotations

import numpy as np


def features(a: np.ndarray, eps_f: float):
    """a: [B, M, 2Q] complex -> (x0 [B, 1, M, Q], lin [B, 4M])."""
    B, M, two_Q = a.shape
    Q = two_Q // 2
    x0 = np.log(eps_f + np.abs(a[:, :, :Q]))[:, None]
    lin = np.concatenate([a[:, :, 0].real, a[:, :, 0].imag, a[:, :, 1].real, a[:, :, 1].imag], axis=1)
    return x0.astype(np.float64), lin.astype(np.float64)


def conv3x3(x, w, b):
    """x [B, Ci, H, W], w [Co, Ci, 3, 3], b [Co] -> [B, Co, H, W] (zero padding 1)."""
    B, Ci, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((B, w.shape[0], H, W))
    for kh in range(3):
        for kw in range(3):
            y += np.einsum("bchw,oc->bohw", xp[:, :, kh:kh + H, kw:kw + W], w[:, :, kh, kw])
    return y + b[None, :, None, None]


def conv3x3_backward(x, w, dy):
    """Gradients of conv3x3 w.r.t. x, w, b."""
    B, Ci, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for kh in range(3):
        for kw in range(3):
            dw[:, :, kh, kw] = np.einsum("bohw,bchw->oc", dy, xp[:, :, kh:kh + H, kw:kw + W])
            dxp[:, :, kh:kh + H, kw:kw + W] += np.einsum("bohw,oc->bchw", dy, w[:, :, kh, kw])
    return dxp[:, :, 1:-1, 1:-1], dw, dy.sum(axis=(0, 2, 3))


def pool2(x):
    B, C, H, W = x.shape
    return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def pool2_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=2), 2, axis=3) / 4.0


def init_params(M: int, Q: int, NT: int, rng: np.random.Generator, ch=(32, 64, 64, 64), hidden=256):
    """He-normal weights, zero biases (float64)."""
    c1, c2, c3, c4 = ch
    p = {}
    for name, co, ci in [("w1", c1, 1), ("w2", c2, c1), ("w3", c3, c2), ("w4", c4, c3)]:
        p[name] = rng.normal(scale=np.sqrt(2.0 / (ci * 9)), size=(co, ci, 3, 3))
        p["b" + name[1:]] = np.zeros(co)
    fin = c4 + 4 * M
    p["f1"] = rng.normal(scale=np.sqrt(2.0 / fin), size=(hidden, fin))
    p["g1"] = np.zeros(hidden)
    p["f2"] = rng.normal(scale=np.sqrt(1.0 / hidden), size=(NT + 2, hidden))
    p["g2"] = np.zeros(NT + 2)
    return p


def forward(p, x0, lin):
    """Returns (out [B, NT + 2], cache)."""
    c = {"x0": x0, "lin": lin}
    z1 = conv3x3(x0, p["w1"], p["b1"]); a1 = np.maximum(z1, 0); h1 = pool2(a1)
    z2 = conv3x3(h1, p["w2"], p["b2"]); a2 = np.maximum(z2, 0); h2 = pool2(a2)
    z3 = conv3x3(h2, p["w3"], p["b3"]); a3 = np.maximum(z3, 0); h3 = pool2(a3)
    z4 = conv3x3(h3, p["w4"], p["b4"]); a4 = np.maximum(z4, 0)
    g = a4.mean(axis=(2, 3))
    u = np.concatenate([g, lin], axis=1)
    v = u @ p["f1"].T + p["g1"]; hv = np.maximum(v, 0)
    out = hv @ p["f2"].T + p["g2"]
    c.update(z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3, z4=z4, a4=a4, u=u, v=v, hv=hv)
    return out, c


def loss_and_grad_out(out, label, shift_target, NT: int, lam: float):
    """Mean cross-entropy over the NT logits + lam * squared error of the 2 shift outputs."""
    B = out.shape[0]
    logits = out[:, :NT]
    mx = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - mx)
    prob = e / e.sum(axis=1, keepdims=True)
    ce = -np.log(prob[np.arange(B), label])
    d = out[:, NT:NT + 2] - shift_target
    loss = float(np.mean(ce + lam * np.sum(d * d, axis=1)))
    g = np.zeros_like(out)
    g[:, :NT] = prob
    g[np.arange(B), label] -= 1.0
    g[:, NT:NT + 2] = 2.0 * lam * d
    return loss, g / B


def backward(p, c, dout):
    """Gradients of every parameter given d loss / d out."""
    gr = {}
    gr["f2"] = dout.T @ c["hv"]; gr["g2"] = dout.sum(axis=0)
    dhv = dout @ p["f2"]
    dv = dhv * (c["v"] > 0)
    gr["f1"] = dv.T @ c["u"]; gr["g1"] = dv.sum(axis=0)
    du = dv @ p["f1"]
    C4 = p["w4"].shape[0]
    dg = du[:, :C4]
    H4, W4 = c["a4"].shape[2:]
    da4 = np.repeat(np.repeat(dg[:, :, None, None], H4, axis=2), W4, axis=3) / (H4 * W4)
    dz4 = da4 * (c["z4"] > 0)
    dh3, gr["w4"], gr["b4"] = conv3x3_backward(c["h3"], p["w4"], dz4)
    dz3 = pool2_backward(dh3) * (c["z3"] > 0)
    dh2, gr["w3"], gr["b3"] = conv3x3_backward(c["h2"], p["w3"], dz3)
    dz2 = pool2_backward(dh2) * (c["z2"] > 0)
    dh1, gr["w2"], gr["b2"] = conv3x3_backward(c["h1"], p["w2"], dz2)
    dz1 = pool2_backward(dh1) * (c["z1"] > 0)
    _, gr["w1"], gr["b1"] = conv3x3_backward(c["x0"], p["w1"], dz1)
    return gr


def adam(p, g, m, v, t: int, lr: float, b1: float, b2: float, eps: float):
    """One Adam step (Kingma & Ba, Algorithm 1) on float64 copies; returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def topk(logits, k: int):
    """Per row, the k largest values' indices, descending; equal values: lower index first."""
    order = np.argsort(-np.asarray(logits, dtype=np.float64), axis=1, kind="stable")
    return order[:, :k]


def confidence(logits, idx=None):
    """Per row, the softmax mass on the indices idx[row] (a shortlist), or the largest probability."""
    x = np.asarray(logits, dtype=np.float64)
    e = np.exp(x - x.max(axis=1, keepdims=True))
    p = e / e.sum(axis=1, keepdims=True)
    if idx is None:
        return p.max(axis=1)
    return np.take_along_axis(p, np.asarray(idx), axis=1).sum(axis=1)


# ---- rotation-equivariant template head -------------------------------------------------
#
# For image i and template j, with learned filters W_j(m, q) on the rings m < Mh and the
# angular frequencies |q| <= Qh (stored at u = q + Qh):
#   X_ij(r)  = Re sum_{m, q} W_j(m, q) a_i(k_m; q) exp(-i q gamma_r),  gamma_r = 2 pi r / (2Q)
#   logit_ij = alpha * max_r X_ij(r) + beta_j       (first maximising r on ties)
# A rotation of the image multiplies a_i(k_m; q) by a phase exp(-i q gamma) (Section 3), which
# moves the maximum over r without changing its value on the rotation grid, so the logit is
# invariant to grid rotations.


def eqhead_forward(W, beta, a, alpha: float):
    """W [NT, Mh, 2Qh+1] complex, beta [NT], a [B, M, 2Q] complex -> (logits [B, NT], rstar [B, NT])."""
    NT, Mh, U = W.shape
    Qh = (U - 1) // 2
    B, M, two_Q = a.shape
    q = np.arange(-Qh, Qh + 1)
    aq = a[:, :Mh, q % two_Q]                                      # [B, Mh, U]
    gam = 2.0 * np.pi * np.arange(two_Q) / two_Q
    E = np.exp(-1j * np.outer(q, gam))                             # [U, 2Q]
    P = np.einsum("jmu,bmu->bju", W, aq)                           # [B, NT, U]
    X = (P @ E).real                                               # [B, NT, 2Q]
    rstar = X.argmax(axis=2)
    return alpha * X.max(axis=2) + beta[None, :], rstar


def eqhead_backward(a, rstar, g, alpha: float, Mh: int, Qh: int):
    """Gradients of sum_ij g_ij logit_ij: (dW as dRe + i dIm [NT, Mh, 2Qh+1], dbeta [NT])."""
    B, M, two_Q = a.shape
    q = np.arange(-Qh, Qh + 1)
    aq = a[:, :Mh, q % two_Q]                                      # [B, Mh, U]
    gam = 2.0 * np.pi * rstar / two_Q                              # [B, NT]
    ph = np.exp(-1j * q[None, None, :] * gam[:, :, None])          # [B, NT, U]
    # d X / d Re W = Re(a e^{-iq gamma}), d X / d Im W = -Im(a e^{-iq gamma})
    z = aq[:, None, :, :] * ph[:, :, None, :]                      # [B, NT, Mh, U]
    dW = alpha * np.einsum("bj,bjmu->jmu", g, np.conj(z))
    return dW, g.sum(axis=0)


def scale_filters(W0, rho):
    """Template-head filters with a spectral weight shared by all templates:
    W_j(m, u) = rho(m, u) W0_j(m, u). W0 [NT, Mh, U] complex, rho [Mh, U] real."""
    return rho[None, :, :] * W0


def scale_filters_backward(W0, dW):
    """Gradient of a loss in W = rho W0 with respect to rho, from dW = dL/dRe W + i dL/dIm W:
    dL/drho(m, u) = sum_j Re dW_j Re W0_j + Im dW_j Im W0_j (the chain rule through both parts)."""
    return np.sum(dW.real * W0.real + dW.imag * W0.imag, axis=0)
