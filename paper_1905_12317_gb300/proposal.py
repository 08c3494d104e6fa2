"""Learned template proposals for the FTK search (the paper has no counterpart).

A small network maps an image's Fourier--Bessel coefficients a(k_m; q) (Section 3)
to template logits and a shift estimate. The k templates of largest logit (and,
optionally, a window of shifts around the estimate) restrict the exact FTK
search (ftk_align_best_shortlist); an image whose shortlist holds too little of
the softmax mass falls back to the full search (ftk_align_best). Training
labels come from the full FTK search itself.

Network (include/ftk.h, "Template-proposal network"):
  * CNN branch: x0 = log(eps_f + |a(k_m; q)|) (rotation invariant), 4 conv3x3 layers
    (ReLU; 2x2 average pools after the first three, a global average after the
    fourth), then fc1 (ReLU) on [pooled features, Re/Im a(k_m; 0), Re/Im a(k_m; 1)]
    and fc2 -> NT template logits + 2 shift outputs;
  * template head (optional, head_rings > 0): for each template j a filter
    W_j(m, q) on the lowest rings and angular band, logit_j = max over the 2Q grid
    rotations of Re sum W_j a e^{-i q gamma} + beta_j; it is added to the CNN's
    template logits. W_j starts from 2 pi w_m conj b_j(k_m; q), the zero-shift
    term of the FTK inner product. head_weight="template" refines every W_j on FTK
    labels; head_weight="shared" keeps that analytic filter and learns one real
    spectral weight rho(m, q) for all templates, W_j = rho W0_j (about a thousand
    parameters trained on every image instead of NT times as many).
Every forward/backward operation and the Adam update run in the library's CUDA
kernels; this module allocates buffers and sequences the calls.
"""

from __future__ import annotations

import ctypes

import os

import numpy as np

from .binding import BF16X3, FP32, _check, _ptr, _stream_ptr, load_library

_vp = ctypes.c_void_p
_i, _f, _ll = ctypes.c_int, ctypes.c_float, ctypes.c_longlong
_SIGS = {
    "ftk_nn_features": [_vp, _i, _i, _i, _f, _vp, _vp, _vp],
    "ftk_nn_conv3x3": [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp],
    "ftk_nn_conv3x3_backward": [_vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _vp],
    "ftk_nn_relu_backward": [_vp, _vp, _ll, _vp],
    "ftk_nn_pool2": [_vp, _vp, _ll, _i, _i, _vp],
    "ftk_nn_pool2_backward": [_vp, _vp, _ll, _i, _i, _vp],
    "ftk_nn_gap": [_vp, _vp, _ll, _i, _vp],
    "ftk_nn_gap_backward": [_vp, _vp, _ll, _i, _vp],
    "ftk_nn_linear": [_vp, _vp, _i, _vp, _vp, _vp, _i, _i, _i, _i, _vp],
    "ftk_nn_linear_backward": [_vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, _i, _i, _i, _vp],
    "ftk_nn_loss": [_vp, _vp, _vp, _i, _i, _f, _vp, _vp, _vp],
    "ftk_nn_adam": [_vp, _vp, _vp, _vp, _ll, _f, _f, _f, _f, _i, _vp],
    "ftk_nn_topk": [_vp, _i, _i, _i, _i, _vp, _vp],
    "ftk_nn_confidence": [_vp, _i, _i, _i, _vp, _i, _vp, _vp],
    "ftk_gather_rows": [_vp, _ll, _vp, _ll, _i, _vp, _vp],
    "ftk_scatter_rows": [_vp, _vp, _ll, _i, _vp, _ll, _vp],
    "ftk_select_below": [_vp, _ll, _f, _vp, _vp, _vp],
    "ftk_nn_snap_to_shifts": [_vp, _i, _vp, _i, _vp, _vp],
    "ftk_nn_eqhead": [_vp, _i, _i, _i, _vp, _vp, _i, _i, _i, _f, _vp, _i, _i, _vp, _vp],
    "ftk_nn_eqhead_backward": [_vp, _i, _i, _i, _vp, _i, _vp, _i, _i, _i, _f, _vp, _vp, _vp],
    "ftk_nn_scale_filters": [_vp, _vp, _i, _i, _vp, _vp],
    "ftk_nn_scale_filters_backward": [_vp, _vp, _i, _i, _vp, _vp],
    "ftk_align_best_shortlist": [_vp, _i, _vp, _i, _vp, _i, _vp, _i, _vp, _f, _vp, _vp, _vp, _vp, _vp,
                                 ctypes.c_size_t, _vp],
    "ftk_shortlist_workspace_size": [_vp, _i, _i, _i, _i, ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t)],
}


def _lib():
    lib = load_library()
    if not getattr(lib, "_nn_sigs", False):
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = args
        lib._nn_sigs = True
    return lib


def _call(name, *args):
    _check(getattr(_lib(), name)(*args), name)


class ProposalNet:
    """The proposal network with FP32 parameters, gradients and Adam state on the device."""

    def __init__(self, M: int, Q: int, NT: int, ch=(32, 64, 64, 64), hidden: int = 256, seed: int = 0,
                 device="cuda", eps_f: float = 1e-3, lam: float = 0.25, shift_scale: float = 3.0,
                 head_rings: int = 0, head_band: int = 0, cnn: bool = True, head_weight: str = "template"):
        import torch
        if M % 8 or Q % 8:
            raise ValueError("M and Q must be multiples of 8 (three 2x2 pools)")
        if head_rings and not (1 <= head_rings <= M and 0 <= head_band and 2 * head_band + 1 <= 2 * Q):
            raise ValueError("head_rings in [1, M] and 2 head_band + 1 <= 2Q")
        if not cnn and not head_rings:
            raise ValueError("a network without the CNN branch needs the template head")
        if head_weight not in ("template", "shared"):
            raise ValueError("head_weight is 'template' or 'shared'")
        self.head_weight = head_weight
        self.cnn = bool(cnn)
        self.Mh, self.Qh = int(head_rings), int(head_band)
        self.M, self.Q, self.NT, self.ch, self.hidden = M, Q, NT, tuple(ch), hidden
        self.eps_f, self.lam, self.shift_scale = eps_f, lam, shift_scale
        self.device = torch.device(device)
        rng = np.random.default_rng(seed)
        c1, c2, c3, c4 = self.ch
        shapes = {"w1": (c1, 1, 3, 3), "b1": (c1,), "w2": (c2, c1, 3, 3), "b2": (c2,), "w3": (c3, c2, 3, 3),
                  "b3": (c3,), "w4": (c4, c3, 3, 3), "b4": (c4,), "f1": (hidden, c4 + 4 * M), "g1": (hidden,),
                  "f2": (NT + 2, hidden), "g2": (NT + 2,)} if cnn else {}
        self.p, self.g, self.m, self.v = {}, {}, {}, {}
        for k, sh in shapes.items():
            if k[0] in "bg":
                val = np.zeros(sh)
            else:
                fan_in = int(np.prod(sh[1:]))
                val = rng.normal(scale=np.sqrt((1.0 if k == "f2" else 2.0) / fan_in), size=sh)
            self.p[k] = torch.tensor(val, dtype=torch.float32, device=self.device)
            self.g[k] = torch.zeros(sh, dtype=torch.float32, device=self.device)
            self.m[k] = torch.zeros(sh, dtype=torch.float32, device=self.device)
            self.v[k] = torch.zeros(sh, dtype=torch.float32, device=self.device)
        if self.Mh:
            # template head: W [NT][Mh][2Qh+1] complex (as float pairs), beta [NT]; the CNN's
            # template logits start at zero and learn a correction to the head
            U = 2 * self.Qh + 1
            fshape = (NT, self.Mh, U, 2)
            shared = head_weight == "shared"
            for k, sh in ((("hr", (self.Mh, U)) if shared else ("hW", fshape)), ("hb", (NT,))):
                self.p[k] = (torch.ones if k == "hr" else torch.zeros)(sh, dtype=torch.float32, device=self.device)
                self.g[k] = torch.zeros(sh, dtype=torch.float32, device=self.device)
                self.m[k] = torch.zeros(sh, dtype=torch.float32, device=self.device)
                self.v[k] = torch.zeros(sh, dtype=torch.float32, device=self.device)
            if shared:  # the analytic filters W0, the effective filters rho W0 and their gradient
                self.hW0 = torch.zeros(fshape, dtype=torch.float32, device=self.device)
                self.hW = torch.zeros(fshape, dtype=torch.float32, device=self.device)
                self.dhW = torch.zeros(fshape, dtype=torch.float32, device=self.device)
            if cnn:
                self.p["f2"][:NT] = 0.0
        self.t = 0
        self._B = None

    # ---- checkpoints: parameters, Adam moments and step count, and the architecture ----
    def state(self):
        """Host copy of everything that training changes and of the architecture."""
        arch = dict(M=self.M, Q=self.Q, NT=self.NT, ch=list(self.ch), hidden=self.hidden, eps_f=self.eps_f,
                    lam=self.lam, shift_scale=self.shift_scale, head_rings=self.Mh, head_band=self.Qh, cnn=self.cnn,
                    head_weight=self.head_weight)
        tensors = {}
        if self._shared():
            tensors["buf.hW0"] = self.hW0.detach().cpu().numpy()
        for k in self.p:
            for tag, d in (("p", self.p), ("m", self.m), ("v", self.v)):
                tensors[f"{tag}.{k}"] = d[k].detach().cpu().numpy()
        return {"arch": arch, "t": self.t, "tensors": tensors}

    def save(self, path: str):
        """Writes a checkpoint (numpy .npz: arch as JSON, step count, p / m / v of every parameter)."""
        import json
        st = self.state()
        tmp = path + ".tmp.npz"
        np.savez(tmp, __arch__=np.frombuffer(json.dumps(st["arch"]).encode(), dtype=np.uint8),
                 __t__=np.array(st["t"], dtype=np.int64), **st["tensors"])
        os.replace(tmp, path)   # a checkpoint is either the old one or the complete new one

    def load_state(self, path: str):
        """Restores parameters, Adam moments and step count from a checkpoint of the same architecture."""
        import json
        import torch
        with np.load(path) as z:
            arch = json.loads(bytes(z["__arch__"]).decode())
            mine = self.state()["arch"]
            if arch != mine:
                raise ValueError(f"checkpoint architecture {arch} != {mine}")
            for k in self.p:
                for tag, d in (("p", self.p), ("m", self.m), ("v", self.v)):
                    d[k].copy_(torch.from_numpy(z[f"{tag}.{k}"]).to(d[k].device))
            if self._shared():
                self.hW0.copy_(torch.from_numpy(z["buf.hW0"]).to(self.device))
            self.t = int(z["__t__"])

    @classmethod
    def load(cls, path: str, device="cuda"):
        """A network rebuilt from a checkpoint's architecture, with its state restored."""
        import json
        with np.load(path) as z:
            a = json.loads(bytes(z["__arch__"]).decode())
        net = cls(a["M"], a["Q"], a["NT"], ch=tuple(a["ch"]), hidden=a["hidden"], device=device, eps_f=a["eps_f"],
                  lam=a["lam"], shift_scale=a["shift_scale"], head_rings=a["head_rings"], head_band=a["head_band"],
                  cnn=a["cnn"], head_weight=a.get("head_weight", "template"))
        net.load_state(path)
        return net

    def init_head(self, b_coeffs, radial_w, a_sample=None, spread: float = 3.0):
        """Head filters from the templates: W_j(m, q) = c 2 pi w_m conj b_j(k_m; q) on the band.

        With ``a_sample`` (coefficients of a few images) c is set so that the head's logits
        spread with standard deviation ``spread`` over the templates.
        """
        import torch
        two_Q = 2 * self.Q
        q = np.arange(-self.Qh, self.Qh + 1) % two_Q
        b = b_coeffs.detach().cpu().numpy().astype(np.complex128)[:, :self.Mh, q]
        Wc = np.conj(b) * (2.0 * np.pi * np.asarray(radial_w, dtype=np.float64)[None, :self.Mh, None])
        W = np.stack([Wc.real, Wc.imag], axis=-1).astype(np.float32)
        (self.hW0 if self._shared() else self.p["hW"]).copy_(torch.from_numpy(W))
        self.p["hb"].zero_()
        if self._shared():
            self.p["hr"].fill_(1.0)
        if a_sample is not None:
            B = a_sample.shape[0]
            logits = torch.zeros((B, self.NT), dtype=torch.float32, device=self.device)
            rstar = torch.empty((B, self.NT), dtype=torch.int32, device=self.device)
            _call("ftk_nn_eqhead", _ptr(a_sample), B, self.M, two_Q, _ptr(self._head_filters()), _ptr(self.p["hb"]),
                  self.NT,
                  self.Mh, self.Qh, 1.0, _ptr(logits), self.NT, 0, _ptr(rstar), _stream_ptr(None))
            sd = float(logits.std(dim=1).mean())
            if sd > 0:
                (self.hW0 if self._shared() else self.p["hW"]).mul_(spread / sd)

    def head_logits(self, coeffs, out=None, stream=None):
        """Head logits alone [B, NT] (and the maximising rotation index [B, NT])."""
        import torch
        B = coeffs.shape[0]
        if out is None:
            out = torch.empty((B, self.NT), dtype=torch.float32, device=self.device)
        rstar = torch.empty((B, self.NT), dtype=torch.int32, device=self.device)
        _call("ftk_nn_eqhead", _ptr(coeffs), B, self.M, 2 * self.Q, _ptr(self._head_filters(stream)),
              _ptr(self.p["hb"]), self.NT,
              self.Mh, self.Qh, 1.0, _ptr(out), out.shape[1], 0, _ptr(rstar), _stream_ptr(stream))
        return out, rstar

    def _shared(self):
        return bool(self.Mh) and self.head_weight == "shared"

    def _head_filters(self, stream=None):
        """The head's filters as the kernels read them: W_j, or rho W0_j formed now."""
        if not self._shared():
            return self.p["hW"]
        _call("ftk_nn_scale_filters", _ptr(self.hW0), _ptr(self.p["hr"]), self.NT, self.Mh * (2 * self.Qh + 1),
              _ptr(self.hW), _stream_ptr(stream))
        return self.hW

    # ---- buffers ----
    def _alloc(self, B):
        import torch
        if self._B == B:
            return
        M, Q = self.M, self.Q
        c1, c2, c3, c4 = self.ch
        e = lambda *s: torch.empty(s, dtype=torch.float32, device=self.device)  # noqa: E731
        if not self.cnn:
            self.buf = dict(out=torch.zeros((B, self.NT + 2), dtype=torch.float32, device=self.device),
                            dout=e(B, self.NT + 2), loss=e(B), conf=e(B),
                            rstar=torch.empty((B, self.NT), dtype=torch.int32, device=self.device))
            self._B = B
            return
        self.buf = dict(
            x0=e(B, 1, M, Q), lin=e(B, 4 * M),
            a1=e(B, c1, M, Q), h1=e(B, c1, M // 2, Q // 2),
            a2=e(B, c2, M // 2, Q // 2), h2=e(B, c2, M // 4, Q // 4),
            a3=e(B, c3, M // 4, Q // 4), h3=e(B, c3, M // 8, Q // 8),
            a4=e(B, c4, M // 8, Q // 8), gp=e(B, c4), hv=e(B, self.hidden), out=e(B, self.NT + 2),
            dout=e(B, self.NT + 2), loss=e(B), dhv=e(B, self.hidden), dgp=e(B, c4),
            da4=e(B, c4, M // 8, Q // 8), dh3=e(B, c3, M // 8, Q // 8), da3=e(B, c3, M // 4, Q // 4),
            dh2=e(B, c2, M // 4, Q // 4), da2=e(B, c2, M // 2, Q // 2), dh1=e(B, c1, M // 2, Q // 2),
            da1=e(B, c1, M, Q), conf=e(B))
        if self.Mh:
            self.buf["rstar"] = torch.empty((B, self.NT), dtype=torch.int32, device=self.device)
        self._B = B

    # ---- forward / backward ----
    def forward(self, coeffs, stream=None):
        B = coeffs.shape[0]
        self._alloc(B)
        M, Q, s = self.M, self.Q, _stream_ptr(stream)
        c1, c2, c3, c4 = self.ch
        b, p = self.buf, self.p
        self._coeffs = coeffs
        if not self.cnn:   # template head alone; the two shift outputs stay zero
            _call("ftk_nn_eqhead", _ptr(coeffs), B, M, 2 * Q, _ptr(self._head_filters(stream)), _ptr(p["hb"]),
                  self.NT, self.Mh, self.Qh, 1.0, _ptr(b["out"]), self.NT + 2, 0, _ptr(b["rstar"]), s)
            return b["out"]
        _call("ftk_nn_features", _ptr(coeffs), B, M, 2 * Q, self.eps_f, _ptr(b["x0"]), _ptr(b["lin"]), s)
        _call("ftk_nn_conv3x3", _ptr(b["x0"]), _ptr(p["w1"]), _ptr(p["b1"]), _ptr(b["a1"]), B, 1, c1, M, Q, 1, s)
        _call("ftk_nn_pool2", _ptr(b["a1"]), _ptr(b["h1"]), B * c1, M, Q, s)
        _call("ftk_nn_conv3x3", _ptr(b["h1"]), _ptr(p["w2"]), _ptr(p["b2"]), _ptr(b["a2"]), B, c1, c2, M // 2, Q // 2, 1, s)
        _call("ftk_nn_pool2", _ptr(b["a2"]), _ptr(b["h2"]), B * c2, M // 2, Q // 2, s)
        _call("ftk_nn_conv3x3", _ptr(b["h2"]), _ptr(p["w3"]), _ptr(p["b3"]), _ptr(b["a3"]), B, c2, c3, M // 4, Q // 4, 1, s)
        _call("ftk_nn_pool2", _ptr(b["a3"]), _ptr(b["h3"]), B * c3, M // 4, Q // 4, s)
        _call("ftk_nn_conv3x3", _ptr(b["h3"]), _ptr(p["w4"]), _ptr(p["b4"]), _ptr(b["a4"]), B, c3, c4, M // 8, Q // 8, 1, s)
        _call("ftk_nn_gap", _ptr(b["a4"]), _ptr(b["gp"]), B * c4, (M // 8) * (Q // 8), s)
        _call("ftk_nn_linear", _ptr(b["gp"]), _ptr(b["lin"]), c4, _ptr(p["f1"]), _ptr(p["g1"]), _ptr(b["hv"]), B,
              c4 + 4 * M, self.hidden, 1, s)
        _call("ftk_nn_linear", _ptr(b["hv"]), None, self.hidden, _ptr(p["f2"]), _ptr(p["g2"]), _ptr(b["out"]), B,
              self.hidden, self.NT + 2, 0, s)
        if self.Mh:
            _call("ftk_nn_eqhead", _ptr(coeffs), B, M, 2 * Q, _ptr(self._head_filters(stream)), _ptr(p["hb"]),
                  self.NT, self.Mh, self.Qh, 1.0, _ptr(b["out"]), self.NT + 2, 1, _ptr(b["rstar"]), s)
        return b["out"]

    def backward(self, stream=None):
        """Gradients of the loss whose d/d out is in buf['dout'] (after loss())."""
        B = self._B
        M, Q, s = self.M, self.Q, _stream_ptr(stream)
        c1, c2, c3, c4 = self.ch
        b, p, g = self.buf, self.p, self.g
        if self.Mh:
            dW = self.dhW if self._shared() else g["hW"]
            _call("ftk_nn_eqhead_backward", _ptr(self._coeffs), B, M, 2 * Q, _ptr(b["dout"]), self.NT + 2,
                  _ptr(b["rstar"]), self.NT, self.Mh, self.Qh, 1.0, _ptr(dW), _ptr(g["hb"]), s)
            if self._shared():
                _call("ftk_nn_scale_filters_backward", _ptr(self.hW0), _ptr(dW), self.NT,
                      self.Mh * (2 * self.Qh + 1), _ptr(g["hr"]), s)
        if not self.cnn:
            return g
        _call("ftk_nn_linear_backward", _ptr(b["hv"]), None, self.hidden, _ptr(p["f2"]), _ptr(b["dout"]),
              _ptr(b["dhv"]), _ptr(g["f2"]), _ptr(g["g2"]), B, self.hidden, self.NT + 2, s)
        _call("ftk_nn_relu_backward", _ptr(b["hv"]), _ptr(b["dhv"]), B * self.hidden, s)
        _call("ftk_nn_linear_backward", _ptr(b["gp"]), _ptr(b["lin"]), c4, _ptr(p["f1"]), _ptr(b["dhv"]),
              _ptr(b["dgp"]), _ptr(g["f1"]), _ptr(g["g1"]), B, c4 + 4 * M, self.hidden, s)
        _call("ftk_nn_gap_backward", _ptr(b["dgp"]), _ptr(b["da4"]), B * c4, (M // 8) * (Q // 8), s)
        _call("ftk_nn_relu_backward", _ptr(b["a4"]), _ptr(b["da4"]), b["da4"].numel(), s)
        _call("ftk_nn_conv3x3_backward", _ptr(b["h3"]), _ptr(p["w4"]), _ptr(b["da4"]), _ptr(b["dh3"]), _ptr(g["w4"]),
              _ptr(g["b4"]), B, c3, c4, M // 8, Q // 8, s)
        _call("ftk_nn_pool2_backward", _ptr(b["dh3"]), _ptr(b["da3"]), B * c3, M // 4, Q // 4, s)
        _call("ftk_nn_relu_backward", _ptr(b["a3"]), _ptr(b["da3"]), b["da3"].numel(), s)
        _call("ftk_nn_conv3x3_backward", _ptr(b["h2"]), _ptr(p["w3"]), _ptr(b["da3"]), _ptr(b["dh2"]), _ptr(g["w3"]),
              _ptr(g["b3"]), B, c2, c3, M // 4, Q // 4, s)
        _call("ftk_nn_pool2_backward", _ptr(b["dh2"]), _ptr(b["da2"]), B * c2, M // 2, Q // 2, s)
        _call("ftk_nn_relu_backward", _ptr(b["a2"]), _ptr(b["da2"]), b["da2"].numel(), s)
        _call("ftk_nn_conv3x3_backward", _ptr(b["h1"]), _ptr(p["w2"]), _ptr(b["da2"]), _ptr(b["dh1"]), _ptr(g["w2"]),
              _ptr(g["b2"]), B, c1, c2, M // 2, Q // 2, s)
        _call("ftk_nn_pool2_backward", _ptr(b["dh1"]), _ptr(b["da1"]), B * c1, M, Q, s)
        _call("ftk_nn_relu_backward", _ptr(b["a1"]), _ptr(b["da1"]), b["da1"].numel(), s)
        _call("ftk_nn_conv3x3_backward", _ptr(b["x0"]), _ptr(p["w1"]), _ptr(b["da1"]), None, _ptr(g["w1"]),
              _ptr(g["b1"]), B, 1, c1, M, Q, s)
        return g

    def loss(self, labels, targets_px, stream=None):
        """Fills buf['dout'] and buf['loss'] for int32 labels [B] and shift targets [B, 2] (pixels)."""
        import torch
        tgt = (targets_px / self.shift_scale).to(torch.float32).contiguous()
        _call("ftk_nn_loss", _ptr(self.buf["out"]), _ptr(labels), _ptr(tgt), self._B, self.NT,
              self.lam if self.cnn else 0.0,
              _ptr(self.buf["dout"]), _ptr(self.buf["loss"]), _stream_ptr(stream))
        return self.buf["loss"]

    def adam_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        self.t += 1
        for k in self.p:
            _call("ftk_nn_adam", _ptr(self.p[k]), _ptr(self.g[k]), _ptr(self.m[k]), _ptr(self.v[k]),
                  self.p[k].numel(), lr, b1, b2, eps, self.t, _stream_ptr(stream))

    def train_batch(self, coeffs, labels, targets_px, lr=1e-3):
        self.forward(coeffs)
        loss = self.loss(labels, targets_px)
        self.backward()
        self.adam_step(lr)
        return loss

    def propose(self, coeffs, k: int, stream=None):
        """Top-k templates [B, k] (int32), shift estimates [B, 2] (pixels), and the softmax mass of
        the k templates [B] (an estimate of the probability that the shortlist holds the best one)."""
        import torch
        out = self.forward(coeffs, stream)
        B = coeffs.shape[0]
        idx = torch.empty((B, k), dtype=torch.int32, device=self.device)
        _call("ftk_nn_topk", _ptr(out), B, self.NT + 2, self.NT, k, _ptr(idx), _stream_ptr(stream))
        _call("ftk_nn_confidence", _ptr(out), B, self.NT + 2, self.NT, _ptr(idx), k, _ptr(self.buf["conf"]),
              _stream_ptr(stream))
        shift = out[:, self.NT:] * self.shift_scale
        return idx, shift.contiguous(), self.buf["conf"]


def shortlist_workspace_size(plan, precision: int, NI: int, NT: int, K: int):
    mn, gd = ctypes.c_size_t(), ctypes.c_size_t()
    _call("ftk_shortlist_workspace_size", plan._h, precision, NI, NT, K, ctypes.byref(mn), ctypes.byref(gd))
    return mn.value, gd.value


def align_best_shortlist(plan, a, b, shortlist, center_px=None, window_px: float = 1.0, precision: int = FP32,
                         work=None, out=None, stream=None):
    """ftk_align_best_shortlist: the FTK search restricted per image to its shortlist (and shift window)."""
    import torch
    NI, NT, K = a.shape[0], b.shape[0], shortlist.shape[1]
    if work is None:
        work = torch.empty(shortlist_workspace_size(plan, precision, NI, NT, K)[1], dtype=torch.uint8,
                           device=a.device)
    if out is None:
        out = (torch.empty(NI, dtype=torch.int32, device=a.device), torch.empty(NI, dtype=torch.int32, device=a.device),
               torch.empty(NI, dtype=torch.int32, device=a.device), torch.empty(NI, dtype=torch.float32, device=a.device))
    tpl, rot, shift, score = out
    _call("ftk_align_best_shortlist", plan._h, precision, _ptr(a), NI, _ptr(b), NT, _ptr(shortlist), K,
          _ptr(center_px) if center_px is not None else None, float(window_px), _ptr(tpl), _ptr(rot), _ptr(shift),
          _ptr(score), _ptr(work), work.numel(), _stream_ptr(stream))
    return out


def gather_rows(src, rows, stream=None):
    """dst[r] = src[rows[r]] (device rows of float32 storage)."""
    import torch
    n = rows.shape[0]
    row_elems = src[0].numel() * (2 if src.is_complex() else 1)
    dst = torch.empty((n,) + tuple(src.shape[1:]), dtype=src.dtype, device=src.device)
    _call("ftk_gather_rows", _ptr(src), src.shape[0], _ptr(rows), n, row_elems, _ptr(dst), _stream_ptr(stream))
    return dst


def scatter_rows(src, rows, dst, stream=None):
    """dst[rows[r]] = src[r] (device rows of 4-byte elements)."""
    n = rows.shape[0]
    row_elems = src[0].numel() * (2 if src.is_complex() else 1)
    _call("ftk_scatter_rows", _ptr(src), _ptr(rows), n, row_elems, _ptr(dst), dst.shape[0], _stream_ptr(stream))
    return dst


def select_below(val, thr: float, stream=None):
    """Device indices b with val[b] < thr (any order); reads their count back to the host."""
    import torch
    rows = torch.empty(max(1, val.shape[0]), dtype=torch.int32, device=val.device)
    count = torch.empty(1, dtype=torch.int32, device=val.device)
    _call("ftk_select_below", _ptr(val), val.shape[0], float(thr), _ptr(rows), _ptr(count), _stream_ptr(stream))
    return rows[:int(count.item())]


def snap_to_shifts(center, shifts_px, stream=None):
    """Each window centre [B, 2] (device, pixels) moved to the nearest shift of shifts_px [N, 2]
    (max norm, ties: lowest index)."""
    import torch
    sh = torch.as_tensor(np.ascontiguousarray(np.asarray(shifts_px, dtype=np.float32).reshape(-1, 2)),
                         device=center.device)
    out = torch.empty_like(center)
    _call("ftk_nn_snap_to_shifts", _ptr(center), center.shape[0], _ptr(sh), sh.shape[0], _ptr(out),
          _stream_ptr(stream))
    return out


def search_with_proposals(plan, net, a, b, k: int = 32, window_px: float = 0.0, min_conf: float = 0.0,
                          precision: int = FP32, work=None):
    """Proposal path: top-k shortlist (+ shift window if window_px > 0) search; images whose
    shortlist holds less than ``min_conf`` of the softmax mass take the full search instead.

    Returns (tpl, rot, shift, score) on the device and the number of fallback images.
    """
    idx, center, conf = net.propose(a, k)
    if window_px > 0:  # the window around the shift nearest to the regressed centre is never empty
        center = snap_to_shifts(center, plan.shifts_px)
    tpl, rot, shift, score = align_best_shortlist(plan, a, b, idx, center if window_px > 0 else None, window_px,
                                                  precision, work=work)
    n_fb = 0
    if min_conf > 0:
        low = select_below(conf, min_conf)
        n_fb = int(low.shape[0])
        if n_fb:
            fb = plan.align_best(gather_rows(a, low), b, precision)
            for dst, src in zip((tpl, rot, shift, score), fb):
                scatter_rows(src, low, dst)
    return (tpl, rot, shift, score), n_fb


def fit(net, coeffs, labels, target_px, epochs: int = 10, batch: int = 256, lr: float = 1e-3, seed: int = 0,
        checkpoint: str = None, every: int = 1):
    """Minibatch Adam on (coeffs [B, M, 2Q] complex64, labels [B] int32, target_px [B, 2]).

    With ``checkpoint``, the network's state is written there every ``every`` epochs (and
    after the last), together with the epoch count; if the file exists when fit starts,
    training resumes after the epochs it records, with the same minibatch order as an
    uninterrupted run. Returns the mean loss of each epoch run by this call (host floats).
    """
    import torch
    B = coeffs.shape[0]
    gen = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    start = 0
    if checkpoint and os.path.exists(checkpoint):
        net.load_state(checkpoint)
        with np.load(checkpoint) as z:
            start = int(z["__epoch__"]) if "__epoch__" in z else 0
    for e in range(epochs):
        perm_cpu = torch.randperm(B, generator=gen)   # drawn for every epoch, so a resume sees the same order
        if e < start:
            continue
        perm = perm_cpu.to(torch.int32).to(coeffs.device)
        tot = torch.zeros((), dtype=torch.float64, device=coeffs.device)
        for s in range(0, B - batch + 1, batch):
            rows = perm[s:s + batch].contiguous()
            xb = gather_rows(coeffs, rows)
            yb = labels[rows.long()].contiguous()
            tb = target_px[rows.long()].contiguous()
            tot += net.train_batch(xb, yb, tb, lr).double().sum()
        hist.append(float(tot) / (B - B % batch))
        if checkpoint and ((e + 1) % every == 0 or e + 1 == epochs):
            _save_with_epoch(net, checkpoint, e + 1)
    return hist


def _save_with_epoch(net, path, epoch):
    import json
    st = net.state()
    tmp = path + ".tmp.npz"
    np.savez(tmp, __arch__=np.frombuffer(json.dumps(st["arch"]).encode(), dtype=np.uint8),
             __t__=np.array(st["t"], dtype=np.int64), __epoch__=np.array(epoch, dtype=np.int64), **st["tensors"])
    os.replace(tmp, path)


def calibrate_min_conf(conf, hit, target: float):
    """Smallest shortlist-mass threshold whose path recall on a calibration set reaches ``target``.

    conf: shortlist masses [B]; hit: whether each image's shortlist holds the full search's
    pose [B] (bool). Images below the threshold take the full search (always recalled).
    """
    c = np.asarray(conf, dtype=np.float64)
    h = np.asarray(hit, dtype=bool)
    order = np.argsort(c)
    # threshold just above the t-th smallest mass: the t smallest fall back
    misses_kept = np.concatenate([np.cumsum((~h[order])[::-1])[::-1], [0]])  # misses among order[t:]
    n = len(c)
    for t in range(n + 1):
        if 1.0 - misses_kept[t] / n >= target:
            return 0.0 if t == 0 else float(np.nextafter(c[order[t - 1]], np.inf))
    return float("inf")


def recall_at_k(shortlist, best_tpl):
    """Fraction of images whose full-search best template is on their shortlist."""
    return float((shortlist == best_tpl[:, None].to(shortlist.dtype)).any(dim=1).double().mean())


def train_with_ftk_labels(plan, net, b, clean, noise_sd, shifts_px, epochs: int, precision: int = BF16X3,
                          batch: int = 256, lr: float = 1e-3, seed: int = 0):
    """Train ``net`` on images labelled by the full FTK search.

    Each epoch draws fresh white noise (standard deviation ``noise_sd`` [B, 1, 1]) on the clean
    training images ``clean`` [B, n, n], transforms them, labels every image with the full
    search's best template and shift (``shifts_px`` [N, 2], device), then runs one pass of Adam.
    Returns the mean loss of each epoch.
    """
    import torch
    B = clean.shape[0]
    work = torch.empty(plan.workspace_size(precision, B, b.shape[0])[1], dtype=torch.uint8, device=clean.device)
    gen = torch.Generator(device=clean.device)
    losses = []
    for ep in range(epochs):
        gen.manual_seed(seed * 100003 + ep)
        a = plan.transform(clean + noise_sd * torch.randn(clean.shape, generator=gen, device=clean.device))
        tpl, _, sh, _ = plan.align_best(a, b, precision, work=work)
        losses += fit(net, a, tpl.contiguous(), shifts_px[sh.long()].contiguous(), epochs=1, batch=batch, lr=lr,
                      seed=seed * 100003 + ep)
    return losses


def calibrate_path(plan, net, a_cal, b, k: int, target: float, precision: int = BF16X3, work=None):
    """Shortlist-mass threshold for ``target`` path recall on calibration images ``a_cal``."""
    full = plan.align_best(a_cal, b, precision)
    idx, _, conf = net.propose(a_cal, k)
    conf = conf.clone()
    res = align_best_shortlist(plan, a_cal, b, idx, None, 0.0, precision, work=work)
    hit = ((res[0] == full[0]) & (res[1] == full[1]) & (res[2] == full[2])).cpu().numpy()
    return calibrate_min_conf(conf.cpu().numpy(), hit, target)
