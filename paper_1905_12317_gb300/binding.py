"""ctypes binding of libftk (include/ftk.h). Argument marshalling only: every
step of the computation runs in the library's CUDA kernels. PyTorch supplies
device memory and the current stream.

The shared library must have been built (``python -m paper_1905_12317_gb300.build``
or ``__graft_entry__.build()``); loading fails loudly otherwise.
"""

from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libftk.so")
HEADER = os.path.join(HERE, "..", "include", "ftk.h")

FP32, BF16X3, BF16, FP16 = 0, 1, 2, 3
PRECISIONS = {"fp32": FP32, "bf16x3": BF16X3, "bf16": BF16, "fp16": FP16}

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_size_p = ctypes.POINTER(ctypes.c_size_t)
_vp = ctypes.c_void_p

class _Group(ctypes.Structure):
    """ftk_group of include/ftk.h."""
    _fields_ = [("plan", _vp), ("d_img_coeffs", _vp), ("NI", ctypes.c_int), ("d_tpl_coeffs", _vp),
                ("NT", ctypes.c_int), ("d_tpl", _vp), ("d_rot", _vp), ("d_shift", _vp), ("d_score", _vp)]


_SIGNATURES = {
    "ftk_groups_workspace_size": (ctypes.c_int, [ctypes.POINTER(_Group), ctypes.c_int, ctypes.c_int, _c_size_p,
                                                 _c_size_p]),
    "ftk_align_best_groups": (ctypes.c_int, [ctypes.POINTER(_Group), ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t,
                                             _vp]),
    "ftk_selftest_timeout": (ctypes.c_int, [_vp, ctypes.c_uint, _vp]),
    "ftk_plan_create_ctf": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_int, _c_double_p, ctypes.c_int, _c_double_p,
                                           ctypes.c_int, ctypes.c_double, ctypes.POINTER(_vp)]),
    "ftk_plan_defocus_count": (ctypes.c_int, [_vp]),
    "ftk_plan_create_weighted": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_int, ctypes.c_int, _c_double_p, ctypes.c_int,
                                                ctypes.c_double, ctypes.POINTER(_vp)]),
    "ftk_plan_spectral_decay": (ctypes.c_double, [_vp]),
    "ftk_rank_profile_weighted": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                 _c_int_p, _c_double_p, ctypes.c_int, _c_int_p]),
    "ftk_plan_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "ftk_plan_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_vp)]),
    "ftk_plan_set_rotations": (ctypes.c_int, [_vp, ctypes.c_int]),
    "ftk_plan_rotations": (ctypes.c_int, [_vp]),
    "ftk_plan_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, _c_double_p, ctypes.c_int,
                                       ctypes.POINTER(_vp)]),
    "ftk_plan_destroy": (None, [_vp]),
    "ftk_rank_profile": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_int, _c_int_p, _c_double_p,
                                        ctypes.c_int, _c_int_p]),
    "ftk_plan_info": (ctypes.c_int, [_vp, _c_int_p, _c_int_p, _c_int_p, _c_int_p, _c_int_p, _c_int_p, _c_int_p]),
    "ftk_plan_terms": (ctypes.c_int, [_vp, _c_int_p, _c_double_p]),
    "ftk_plan_radial_rule": (ctypes.c_int, [_vp, _c_double_p, _c_double_p]),
    "ftk_transform": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    "ftk_workspace_size": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_size_p, _c_size_p]),
    "ftk_align_scores": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp,
                                        ctypes.c_size_t, _vp]),
    "ftk_align_best": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp,
                                      _vp, _vp, ctypes.c_size_t, _vp]),
    "ftk_search_workspace_size": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_size_p,
                                                 _c_size_p]),
    "ftk_search_host": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp,
                                       _vp, _vp, ctypes.c_size_t, _vp]),
    "ftk_stream_check": (ctypes.c_int, [_vp, _vp]),
    "ftk_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ftk_plan_launch_count": (ctypes.c_longlong, [_vp]),
    "ftk_plan_tune": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_int]),
    "ftk_plan_tuning": (ctypes.c_int, [_vp, _c_int_p, _c_int_p, _c_int_p]),
    "ftk_profile_begin": (ctypes.c_int, [_vp]),
    "ftk_profile_end": (ctypes.c_int, [_vp, _vp]),
    "ftk_profile_kernel": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
}
NUM_KERNELS = 15  # FTK_NUM_KERNELS of include/ftk.h

_lib = None


class FtkError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = load_library().ftk_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})")


def load_library():
    """Loads the in-tree libftk.so (no fallback: a missing library is an error)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libftk.so not built: {LIB_PATH} is missing; run "
                           "`python -m paper_1905_12317_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/ftk.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(ftk_\w+)\s*\(", text, re.M)))


def rank_profile(W: float, eps: float, max_l: int, n_sigma: int = 4, decay: float = 0.0):
    """Host-only modal ranks H_l (l = 0..max_l), leading Sigma_eta(l), and total H; with
    `decay` > 0 those of the spectrally weighted SVD (ftk_rank_profile_weighted)."""
    lib = load_library()
    H = (ctypes.c_int * (max_l + 1))()
    sig = (ctypes.c_double * ((max_l + 1) * max(n_sigma, 1)))()
    tot = ctypes.c_int()
    _check(lib.ftk_rank_profile_weighted(float(W), float(eps), float(decay), int(max_l), H, sig, int(n_sigma),
                                         ctypes.byref(tot)),
           "ftk_rank_profile_weighted")
    return np.array(H[:]), np.array(sig[:]).reshape(max_l + 1, max(n_sigma, 1))[:, :n_sigma], tot.value


def _check(status: int, what: str):
    if status != 0:
        raise FtkError(status, what)


def _stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Plan:
    """An FTK plan (ftk_plan_create): radial rule, rank-H factors, transform tables."""

    def __init__(self, n: int, W: float, eps: float, M: int, two_Q: int, shifts_px, K: float = 0.0,
                 defocus=None, phase: float = 0.0, decay: float = 0.0):
        """defocus: CTF defocus values (ftk_plan_create_ctf); the plan's rows are then
        (defocus b, shift s) at b * N_shift + s. decay > 0: the modal SVDs in the spectral
        weight exp(-decay (k/K)^2) (ftk_plan_create_weighted; not with defocus)."""
        lib = load_library()
        sh = np.ascontiguousarray(np.asarray(shifts_px, dtype=np.float64).reshape(-1, 2))
        self.shifts_px = sh.copy()
        h = _vp()
        if decay and defocus is not None:
            raise ValueError("a spectral weight is not offered with CTF defocus values")
        if decay:
            _check(lib.ftk_plan_create_weighted(int(n), float(K), float(W), float(eps), int(M), int(two_Q),
                                                sh.ctypes.data_as(_c_double_p), int(sh.shape[0]), float(decay),
                                                ctypes.byref(h)),
                   "ftk_plan_create_weighted")
        elif defocus is None:
            _check(lib.ftk_plan_create(int(n), float(K), float(W), float(eps), int(M), int(two_Q),
                                       sh.ctypes.data_as(_c_double_p), int(sh.shape[0]), ctypes.byref(h)),
                   "ftk_plan_create")
        else:
            tau = np.ascontiguousarray(np.asarray(defocus, dtype=np.float64).reshape(-1))
            _check(lib.ftk_plan_create_ctf(int(n), float(K), float(W), float(eps), int(M), int(two_Q),
                                           sh.ctypes.data_as(_c_double_p), int(sh.shape[0]),
                                           tau.ctypes.data_as(_c_double_p), int(tau.size), float(phase),
                                           ctypes.byref(h)),
                   "ftk_plan_create_ctf")
        self._adopt(lib, h, W, eps)

    def _adopt(self, lib, h, W, eps):
        self._h = h
        self._lib = lib
        vals = [ctypes.c_int() for _ in range(7)]
        _check(lib.ftk_plan_info(h, *[ctypes.byref(v) for v in vals]), "ftk_plan_info")
        self.H, self.H_half, self.L, self.M, self.two_Q, self.N, self.n = [v.value for v in vals]
        self.W, self.eps = W, eps
        self.n_defocus = int(lib.ftk_plan_defocus_count(h))
        self.N_shift = self.N // self.n_defocus
        self.decay = float(lib.ftk_plan_spectral_decay(h))

    def save(self, path: str):
        """Writes the plan's precomputation, shifts, rotation count and knobs (ftk_plan_save)."""
        _check(self._lib.ftk_plan_save(self._h, os.fsencode(path)), "ftk_plan_save")

    @classmethod
    def load(cls, path: str) -> "Plan":
        """A plan read from a file of Plan.save, with its device tables rebuilt on the
        current device (ftk_plan_load); no modal SVD is computed."""
        lib = load_library()
        h = _vp()
        _check(lib.ftk_plan_load(os.fsencode(path), ctypes.byref(h)), "ftk_plan_load")
        with open(path, "rb") as f:   # K, W, eps follow the magic and 18 int32 header words
            raw = f.read()
        hdr = np.frombuffer(raw[8:8 + 18 * 4], dtype="<i4")
        K, W, eps = np.frombuffer(raw[8 + 18 * 4:8 + 18 * 4 + 24], dtype="<f8")
        # then phase (and the spectral decay from version 2 on), the defocus values, the shifts
        off = 8 + 18 * 4 + 8 * (4 + (1 if hdr[0] >= 2 else 0)) + 8 * int(hdr[16])
        self = cls.__new__(cls)
        self._adopt(lib, h, float(W), float(eps))
        self.shifts_px = np.frombuffer(raw[off:off + 16 * int(hdr[4])], dtype="<f8").reshape(-1, 2).copy()
        return self

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ftk_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- plan contents ----
    def terms(self):
        l = (ctypes.c_int * self.H_half)()
        s = (ctypes.c_double * self.H_half)()
        _check(self._lib.ftk_plan_terms(self._h, l, s), "ftk_plan_terms")
        return np.array(l[:], dtype=np.int64), np.array(s[:])

    def radial_rule(self):
        k = (ctypes.c_double * self.M)()
        w = (ctypes.c_double * self.M)()
        _check(self._lib.ftk_plan_radial_rule(self._h, k, w), "ftk_plan_radial_rule")
        return np.array(k[:]), np.array(w[:])

    @property
    def rotations(self) -> int:
        """Rotation count R of the grid gamma_r = 2 pi r / R (2Q unless set_rotations changed it)."""
        return int(self._lib.ftk_plan_rotations(self._h))

    def set_rotations(self, n_rot: int):
        """Finer rotation grid by zero-padding Step 2 (Section 3.2); n_rot a multiple of 2Q."""
        _check(self._lib.ftk_plan_set_rotations(self._h, int(n_rot)), "ftk_plan_set_rotations")

    @property
    def launch_count(self) -> int:
        return int(self._lib.ftk_plan_launch_count(self._h))

    # ---- device calls ----
    def transform(self, images, out=None, stream=None):
        import torch
        assert images.is_cuda and images.dtype == torch.float32 and images.is_contiguous()
        B = images.shape[0]
        if out is None:
            out = torch.empty((B, self.M, self.two_Q), dtype=torch.complex64, device=images.device)
        _check(self._lib.ftk_transform(self._h, _ptr(images), B, _ptr(out), _stream_ptr(stream)), "ftk_transform")
        return out

    def workspace_size(self, precision: int, NI: int, NT: int):
        mn, gd = ctypes.c_size_t(), ctypes.c_size_t()
        _check(self._lib.ftk_workspace_size(self._h, precision, NI, NT, ctypes.byref(mn), ctypes.byref(gd)),
               "ftk_workspace_size")
        return mn.value, gd.value

    def _work(self, precision, NI, NT, work, device):
        import torch
        if work is None:
            _, gd = self.workspace_size(precision, NI, NT)
            work = torch.empty(gd, dtype=torch.uint8, device=device)
        return work

    def align_scores(self, a, b, precision: int = FP32, work=None, out=None, stream=None):
        import torch
        NI, NT = a.shape[0], b.shape[0]
        if out is None:
            out = torch.empty((NI, NT, self.N, self.rotations), dtype=torch.float32, device=a.device)
        work = self._work(precision, NI, NT, work, a.device)
        _check(self._lib.ftk_align_scores(self._h, precision, _ptr(a), NI, _ptr(b), NT, _ptr(out), _ptr(work),
                                          work.numel(), _stream_ptr(stream)), "ftk_align_scores")
        return out

    def align_best(self, a, b, precision: int = FP32, work=None, out=None, stream=None):
        import torch
        NI, NT = a.shape[0], b.shape[0]
        if out is None:
            out = (torch.empty(NI, dtype=torch.int32, device=a.device),
                   torch.empty(NI, dtype=torch.int32, device=a.device),
                   torch.empty(NI, dtype=torch.int32, device=a.device),
                   torch.empty(NI, dtype=torch.float32, device=a.device))
        work = self._work(precision, NI, NT, work, a.device)
        tpl, rot, shift, score = out
        _check(self._lib.ftk_align_best(self._h, precision, _ptr(a), NI, _ptr(b), NT, _ptr(tpl), _ptr(rot),
                                        _ptr(shift), _ptr(score), _ptr(work), work.numel(), _stream_ptr(stream)),
               "ftk_align_best")
        return out

    def search_workspace_size(self, precision: int, NI: int, NT: int):
        mn, gd = ctypes.c_size_t(), ctypes.c_size_t()
        _check(self._lib.ftk_search_workspace_size(self._h, precision, NI, NT, ctypes.byref(mn), ctypes.byref(gd)),
               "ftk_search_workspace_size")
        return mn.value, gd.value

    def search_host(self, images, templates, precision: int, work, out, stream=None):
        """images/templates: host (pinned) float32 torch tensors; out: 4 host tensors [NI]."""
        NI, NT = images.shape[0], templates.shape[0]
        tpl, rot, shift, score = out
        _check(self._lib.ftk_search_host(self._h, precision, _ptr(images), NI, _ptr(templates), NT, _ptr(tpl),
                                         _ptr(rot), _ptr(shift), _ptr(score), _ptr(work), work.numel(),
                                         _stream_ptr(stream)), "ftk_search_host")
        return out

    def selftest_timeout(self, limit_us: int = 20000, stream=None):
        """Launches a bounded wait that nothing completes (ftk_selftest_timeout)."""
        _check(self._lib.ftk_selftest_timeout(self._h, int(limit_us), _stream_ptr(stream)), "ftk_selftest_timeout")

    def stream_check(self, stream=None):
        _check(self._lib.ftk_stream_check(self._h, _stream_ptr(stream)), "ftk_stream_check")

    # ---- launch-shape knobs ----
    def tune(self, knob: str, value: int):
        _check(self._lib.ftk_plan_tune(self._h, knob.encode(), int(value)), f"ftk_plan_tune({knob})")

    def tuning(self):
        g, ng, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._lib.ftk_plan_tuning(self._h, ctypes.byref(g), ctypes.byref(ng), ctypes.byref(st)),
               "ftk_plan_tuning")
        return {"step3_group": g.value, "step3_groups": ng.value, "step3_a_stages": st.value}

    # ---- launch profiler ----
    def profile_begin(self):
        _check(self._lib.ftk_profile_begin(self._h), "ftk_profile_begin")

    def profile_end(self, stream=None):
        """Stops recording; returns {kernel name: (total ms, launches)} for launched kernels."""
        _check(self._lib.ftk_profile_end(self._h, _stream_ptr(stream)), "ftk_profile_end")
        out = {}
        for kid in range(NUM_KERNELS):
            name, ms, n = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_longlong()
            _check(self._lib.ftk_profile_kernel(self._h, kid, ctypes.byref(name), ctypes.byref(ms),
                                                ctypes.byref(n)), "ftk_profile_kernel")
            if n.value:
                out[name.value.decode()] = (ms.value, n.value)
        return out


def _group_array(groups, outs):
    arr = (_Group * len(groups))()
    for k, ((plan, a, b), out) in enumerate(zip(groups, outs)):
        tpl, rot, shift, score = out if out is not None else (None,) * 4
        arr[k] = _Group(plan._h, _ptr(a).value, int(a.shape[0]), _ptr(b).value, int(b.shape[0]),
                        _ptr(tpl).value, _ptr(rot).value, _ptr(shift).value, _ptr(score).value)
    return arr


def groups_workspace_size(groups, precision: int):
    """(min, good) workspace bytes of align_best_groups; groups: [(plan, a, b), ...]."""
    lib = load_library()
    arr = _group_array(groups, [None] * len(groups))
    mn, gd = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib.ftk_groups_workspace_size(arr, len(groups), int(precision), ctypes.byref(mn), ctypes.byref(gd)),
           "ftk_groups_workspace_size")
    return mn.value, gd.value


def align_best_groups(groups, precision: int = BF16X3, work=None, outs=None, stream=None):
    """ftk_align_best_groups: the best pose of every image of every group in one call.
    groups: [(plan, a, b), ...] with device coefficients; returns [(tpl, rot, shift, score), ...]."""
    import torch
    lib = load_library()
    dev = groups[0][1].device
    if outs is None:
        outs = [tuple(torch.empty(a.shape[0], dtype=d, device=dev)
                      for d in (torch.int32, torch.int32, torch.int32, torch.float32)) for _, a, _ in groups]
    if work is None:
        work = torch.empty(max(groups_workspace_size(groups, precision)[1], 256), dtype=torch.uint8, device=dev)
    arr = _group_array(groups, outs)
    _check(lib.ftk_align_best_groups(arr, len(groups), int(precision), _ptr(work), work.numel(), _stream_ptr(stream)),
           "ftk_align_best_groups")
    return outs
