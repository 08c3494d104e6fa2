"""C-ABI checks that need no GPU: the library loads, exports every function that
include/ftk.h declares, validates arguments before touching the device, and its
host-only FP64 planning agrees with the oracle's plan."""

import ctypes

import numpy as np
import pytest

import paper_1905_12317_gb300 as ftk
from oracle import svd_plan


@pytest.fixture(scope="module")
def lib():
    return ftk.load_library()


def test_library_exports_every_header_function(lib):
    names = ftk.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for st in range(8):
        assert lib.ftk_status_string(st)


def _create(lib, n=32, W=1.0, eps=1e-2, M=16, two_Q=96, shifts=((0.0, 0.0),)):
    sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    h = ctypes.c_void_p()
    st = lib.ftk_plan_create(n, 0.0, W, eps, M, two_Q, sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             sh.shape[0], ctypes.byref(h))
    return st, h


def test_plan_rejects_shift_outside_disk(lib):
    # Section 2: shifts are limited to |delta| <= D, i.e. |s_px| <= 2W.
    st, h = _create(lib, W=1.0, shifts=((0.0, 0.0), (1.5, 1.5)))
    assert st == 2 and not h.value


@pytest.mark.parametrize("kw", [dict(two_Q=100), dict(two_Q=7), dict(n=7), dict(M=0), dict(eps=0.0),
                                dict(eps=1.5), dict(W=-1.0), dict(shifts=np.zeros((0, 2)))])
def test_plan_rejects_bad_arguments(lib, kw):
    st, h = _create(lib, **kw)
    assert st == 1 and not h.value


def test_null_plan_is_rejected(lib):
    assert lib.ftk_transform(None, None, 1, None, None) == 1
    assert lib.ftk_align_best(None, 0, None, 1, None, 1, None, None, None, None, None, 0, None) == 1
    lib.ftk_plan_destroy(None)


@pytest.mark.parametrize("W,eps", [(1.0, 1e-2), (1.5, 1e-3), (2.0, 1e-4)])
def test_host_rank_profile_matches_oracle(W, eps):
    # Two independent discretizations of the operator SVD of J_l (Nystrom on
    # Gauss-Jacobi nodes in the library, Jacobi-polynomial projection in the
    # oracle) must agree on the retained ranks and the leading singular values.
    H_l, sig, H = ftk.rank_profile(W, eps, 30, n_sigma=3)
    plan = svd_plan.build_plan(W, eps, K=1.0)
    assert H == plan.H
    for l in range(31):
        assert H_l[l] == plan.H_l(l)
        ref = svd_plan.modal_svd(l, W, eps).sigma_all[:3]
        assert np.allclose(sig[l], ref, rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("W,eps,decay", [(1.0, 1e-2, 10.0), (1.5, 1e-3, 10.0), (1.0, 1e-3, 40.0)])
def test_host_weighted_rank_profile_matches_oracle(W, eps, decay):
    # the spectrally weighted SVD (Section 4.5, alternative weights): Nystrom with the
    # weight inside the kernel (library) vs projection of J_l sqrt(rho) (oracle)
    H_l, sig, H = ftk.rank_profile(W, eps, 30, n_sigma=3, decay=decay)
    plan = svd_plan.build_plan(W, eps, K=1.0, decay=decay)
    assert H == plan.H < svd_plan.build_plan(W, eps, K=1.0).H
    for l in range(31):
        assert H_l[l] == plan.H_l(l)
        ref = svd_plan.modal_svd(l, W, eps, decay=decay).sigma_all[:3]
        assert np.allclose(sig[l], ref, rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("decay", [-1.0, 300.0, float("nan"), float("inf")])
def test_weighted_plan_rejects_bad_decay_before_touching_the_device(lib, decay):
    sh = np.zeros((1, 2))
    h = ctypes.c_void_p(1)
    st = lib.ftk_plan_create_weighted(32, 0.0, 1.0, 1e-2, 16, 96, sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      1, decay, ctypes.byref(h))
    assert st == 1 and not h.value
    assert lib.ftk_rank_profile_weighted(1.0, 1e-2, decay, 4, None, None, 0, None) == 1
    assert lib.ftk_plan_spectral_decay(None) == -1.0


def _plan_file(path, hdr_over=None, tail=b"", drop=0, decay=0.0):
    """A plan file laid out as ftk_plan_save documents: magic, 18 int32 header words
    (version, n, M, 2Q, N_shift, n_tau, H, H_half, L, R, four Step-1/3 knobs, fft_lanes,
    transform, #defocus, step23), K, W, eps, phase (and the spectral decay from version 2
    on), then taus, shifts, k, w, l, Sigma, G, Y."""
    n, M, two_Q, N, Hh = 32, 4, 96, 2, 3
    hdr = dict(version=2, n=n, M=M, two_Q=two_Q, N=N, n_tau=1, H=5, Hh=Hh, L=1, R=two_Q, g=0, a=0, s1=0, c1=0,
               lanes=0, xf=0, ntaus=0, step23=1)
    hdr.update(hdr_over or {})
    body = b"FTKPLAN1" + np.array(list(hdr.values()), dtype="<i4").tobytes()
    body += np.array([50.0, 1.0, 1e-2, 0.0] + ([decay] if hdr["version"] == 2 else []), dtype="<f8").tobytes()
    body += np.zeros(2 * N, "<f8").tobytes() + np.linspace(1, 40, M).astype("<f8").tobytes()
    body += np.ones(M, "<f8").tobytes() + np.array([0, 1, 1], "<i4").tobytes() + np.ones(Hh, "<f8").tobytes()
    body += np.ones(Hh * M, "<f4").tobytes() + np.ones(2 * N * Hh, "<f4").tobytes()
    with open(path, "wb") as f:
        f.write(body[:len(body) - drop] + tail)
    return str(path).encode()


@pytest.mark.parametrize("case", ["missing", "magic", "version", "two_Q", "L", "knob", "step23", "truncated",
                                  "decay_nan", "decay_range", "v1_with_decay",
                                  "extra"])
def test_plan_load_rejects_bad_files_before_touching_the_device(lib, tmp_path, case):
    p = tmp_path / "plan.bin"
    if case == "missing":
        path = str(tmp_path / "none.bin").encode()
    elif case == "magic":
        path = _plan_file(p)
        data = bytearray(open(p, "rb").read())
        data[7] = ord("2")
        open(p, "wb").write(bytes(data))
    else:
        over = dict(version=dict(version=3), two_Q=dict(two_Q=100, R=100), L=dict(L=96), knob=dict(lanes=12),
                    step23=dict(step23=2), v1_with_decay=dict(version=1))
        decay = dict(decay_nan=float("nan"), decay_range=300.0).get(case, 0.0)
        # a version-1 file is one double shorter: the trailing bytes of a version-2 body are left over
        tail = b"\0" if case == "extra" else (b"\0" * 8 if case == "v1_with_decay" else b"")
        path = _plan_file(p, over.get(case), tail=tail, drop=4 if case == "truncated" else 0, decay=decay)
    h = ctypes.c_void_p(1)
    assert lib.ftk_plan_load(path, ctypes.byref(h)) == 1
    assert not h.value
    assert lib.ftk_plan_save(None, path) == 1


def test_grouped_call_rejects_bad_arguments_before_touching_the_device(lib):
    assert lib.ftk_align_best_groups(None, 1, 1, None, 0, None) == 1
    assert lib.ftk_groups_workspace_size(None, 1, 1, None, None) == 1
    arr = (ftk.binding._Group * 2)()          # NULL plans
    assert lib.ftk_groups_workspace_size(arr, 2, 1, None, None) == 1
    assert lib.ftk_align_best_groups(arr, 0, 1, None, 0, None) == 1
    big = (ftk.binding._Group * 65)()
    assert lib.ftk_align_best_groups(big, 65, 1, None, 0, None) == 1   # more than FTK_MAX_GROUPS


def test_binding_rejects_weight_with_ctf_before_the_library():
    with pytest.raises(ValueError):
        ftk.Plan(32, 1.0, 1e-2, 16, 96, np.zeros((1, 2)), defocus=[0.5], decay=10.0)
