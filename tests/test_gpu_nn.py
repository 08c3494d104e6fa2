"""GPU parity of the template-proposal network and the shortlist search.

Every CUDA operation of the network (features, conv3x3, pools, linear, loss,
their backward passes, Adam, top-k, confidence, row gather) is compared with
the FP64 oracle in oracle/nn.py on the same FP32-representable inputs.
Tolerance: FP32 accumulation over at most ~1e5 terms, 2e-4 relative to the
largest magnitude of the compared tensor. Index outputs are compared exactly.

The shortlist search (ftk_align_best_shortlist) is compared with the oracle's
Steps 1-3 restricted to the same templates and shift window.
"""

import numpy as np
import pytest

import torch

pytestmark = pytest.mark.gpu

import paper_1905_12317_gb300 as ftk
from paper_1905_12317_gb300 import proposal as pr
from oracle import nn as onn, brute, ftk_steps, quadrature as quad, svd_plan, transform as tr
from oracle.best import best_pose
from workloads import make_workload

TOL = 2e-4


def _rel(x, ref):
    x, ref = np.asarray(x), np.asarray(ref)
    dt = np.complex128 if (np.iscomplexobj(x) or np.iscomplexobj(ref)) else np.float64
    x, ref = x.astype(dt), ref.astype(dt)
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-30))


def _net_case(B, M, Q, NT, ch, hidden, seed):
    rng = np.random.default_rng(seed)
    a = (rng.normal(size=(B, M, 2 * Q)) + 1j * rng.normal(size=(B, M, 2 * Q))).astype(np.complex64)
    net = pr.ProposalNet(M, Q, NT, ch=ch, hidden=hidden, seed=seed, lam=0.3, shift_scale=1.0)
    p = onn.init_params(M, Q, NT, rng, ch=ch, hidden=hidden)
    for k in p:
        if k.startswith(("b", "g")):
            p[k] = rng.normal(scale=0.1, size=p[k].shape)
        p[k] = p[k].astype(np.float32).astype(np.float64)
        net.p[k].copy_(torch.from_numpy(p[k].astype(np.float32)))
    label = rng.integers(0, NT, B)
    target = rng.normal(size=(B, 2)).astype(np.float32)
    return a, net, p, label, target


@pytest.mark.parametrize("B,M,Q,NT,ch,hidden", [
    (3, 16, 16, 20, (4, 8, 8, 8), 16),      # several tiles of every kernel
    (1, 8, 8, 3, (2, 3, 3, 2), 5),          # smallest: the last conv runs on 1 x 1
    (37, 16, 24, 50, (8, 8, 16, 8), 33),    # ragged batch and widths
])
def test_network_forward_backward_match_oracle(B, M, Q, NT, ch, hidden):
    a, net, p, label, target = _net_case(B, M, Q, NT, ch, hidden, seed=B)
    x0, lin = onn.features(a.astype(np.complex128), net.eps_f)
    ref_out, cache = onn.forward(p, x0, lin)
    loss_ref, dout_ref = onn.loss_and_grad_out(ref_out, label, target.astype(np.float64), NT, 0.3)
    gr = onn.backward(p, cache, dout_ref)

    ad = torch.from_numpy(a).cuda()
    out = net.forward(ad).cpu().numpy()
    assert _rel(net.buf["x0"].cpu().numpy(), x0) < 1e-6
    assert _rel(net.buf["lin"].cpu().numpy(), lin) < 1e-7
    for k, r in [("a1", cache["z1"]), ("h2", cache["h2"]), ("a4", cache["a4"])]:
        assert _rel(net.buf[k].cpu().numpy(), np.maximum(r, 0)) < TOL, k
    assert _rel(out, ref_out) < TOL
    loss = net.loss(torch.from_numpy(label.astype(np.int32)).cuda(), torch.from_numpy(target).cuda())
    assert abs(float(loss.double().mean()) - loss_ref) < TOL * max(1.0, abs(loss_ref))
    assert _rel(net.buf["dout"].cpu().numpy(), dout_ref) < TOL
    g = net.backward()
    torch.cuda.synchronize()
    for k in gr:
        assert _rel(g[k].cpu().numpy(), gr[k]) < TOL, k


def test_adam_matches_oracle():
    rng = np.random.default_rng(11)
    n = 1000
    p0 = rng.normal(size=n).astype(np.float32)
    net_p = torch.from_numpy(p0.copy()).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    pr_, mr, vr = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        g = rng.normal(size=n).astype(np.float32)
        gd = torch.from_numpy(g).cuda()
        pr._call("ftk_nn_adam", pr._ptr(net_p), pr._ptr(gd), pr._ptr(m), pr._ptr(v), n, 1e-2, 0.9, 0.999, 1e-8, t,
                 pr._stream_ptr())
        pr_, mr, vr = onn.adam(pr_, g.astype(np.float64), mr, vr, t, 1e-2, 0.9, 0.999, 1e-8)
    assert np.abs(net_p.cpu().numpy() - pr_).max() < 1e-6


def test_topk_confidence_gather_exact():
    rng = np.random.default_rng(12)
    B, NT, k = 9, 700, 32
    logits = rng.integers(-20, 20, size=(B, NT + 2)).astype(np.float32)   # many ties
    logits[3] = 1.5                                                      # all equal
    d = torch.from_numpy(logits).cuda()
    idx = torch.empty((B, k), dtype=torch.int32, device="cuda")
    pr._call("ftk_nn_topk", pr._ptr(d), B, NT + 2, NT, k, pr._ptr(idx), pr._stream_ptr())
    assert np.array_equal(idx.cpu().numpy(), onn.topk(logits[:, :NT], k))
    conf = torch.empty(B, device="cuda")
    pr._call("ftk_nn_confidence", pr._ptr(d), B, NT + 2, NT, None, 0, pr._ptr(conf), pr._stream_ptr())
    assert _rel(conf.cpu().numpy(), onn.confidence(logits[:, :NT])) < 1e-6
    pr._call("ftk_nn_confidence", pr._ptr(d), B, NT + 2, NT, pr._ptr(idx), k, pr._ptr(conf), pr._stream_ptr())
    assert _rel(conf.cpu().numpy(), onn.confidence(logits[:, :NT], idx.cpu().numpy())) < 1e-5
    src = torch.from_numpy(rng.normal(size=(50, 7, 3)).astype(np.float32)).cuda()
    rows = torch.tensor([49, 0, 7, 7, 13], dtype=torch.int32, device="cuda")
    assert torch.equal(pr.gather_rows(src, rows), src[rows.long()])


def test_nn_rejects_bad_sizes():
    x = torch.zeros(64, device="cuda")
    with pytest.raises(ftk.FtkError):
        pr._call("ftk_nn_pool2", pr._ptr(x), pr._ptr(x), 1, 3, 4, pr._stream_ptr())   # odd H
    idx = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(ftk.FtkError):
        pr._call("ftk_nn_topk", pr._ptr(x), 1, 64, 64, 65, pr._ptr(idx), pr._stream_ptr())   # k > NT


class _Tiny:
    def __init__(self):
        self.wl = wl = make_workload("n32_tiny", n_images=6, n_templates=16)
        K = quad.nyquist_K(wl.n)
        self.k, self.w = quad.radial_rule(wl.M, K)
        self.delta = brute.shift_vectors(wl.shifts_px, wl.n)
        self.a = tr.ring_coefficients(tr.polar_fourier(wl.images, self.k, wl.two_Q))
        self.b = tr.ring_coefficients(tr.polar_fourier(wl.templates, self.k, wl.two_Q))
        self.plan_o = svd_plan.build_plan(wl.W, wl.eps, K)
        self.plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
        self.ad = torch.from_numpy(self.a.astype(np.complex64)).cuda()
        self.bd = torch.from_numpy(self.b.astype(np.complex64)).cuda()


@pytest.fixture(scope="module")
def tiny():
    return _Tiny()


@pytest.mark.parametrize("precision", [ftk.FP32, ftk.BF16X3])
def test_shortlist_of_all_templates_equals_full_search(tiny, precision):
    # per pair the arithmetic is that of the full search, so results are identical
    NI, NT = tiny.a.shape[0], tiny.b.shape[0]
    rng = np.random.default_rng(3)
    sl = np.stack([rng.permutation(NT) for _ in range(NI)]).astype(np.int32)
    got = pr.align_best_shortlist(tiny.plan, tiny.ad, tiny.bd, torch.from_numpy(sl).cuda(), precision=precision)
    ref = tiny.plan.align_best(tiny.ad, tiny.bd, precision)
    for g, r in zip(got, ref):
        assert torch.equal(g, r)


def test_tensor_core_shortlist_over_several_tiles_and_chunks():
    # n = 64 grid, 300 templates: a 300-long list spans three 128-row template tiles, a
    # 40-long list one tile with padding rows; the smallest workspace runs one image per launch
    wl = make_workload("n64_1k", n_images=6, n_templates=300)
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
    a = plan.transform(torch.from_numpy(wl.images).cuda())
    b = plan.transform(torch.from_numpy(wl.templates).cuda())
    ref = plan.align_best(a, b, ftk.BF16X3)
    rng = np.random.default_rng(5)
    sl = torch.from_numpy(np.stack([rng.permutation(300) for _ in range(6)]).astype(np.int32)).cuda()
    mn, gd = pr.shortlist_workspace_size(plan, ftk.BF16X3, 6, 300, 300)
    for work_bytes in (mn, gd):
        work = torch.empty(work_bytes, dtype=torch.uint8, device="cuda")
        got = pr.align_best_shortlist(plan, a, b, sl, precision=ftk.BF16X3, work=work)
        for g, r in zip(got, ref):
            assert torch.equal(g, r)
    # a 40-long list: the best over those 40 templates, bit for bit that of the written
    # scores when both run the separate Step-2 and Step-3 kernels
    X = plan.align_scores(a, b, ftk.BF16X3)
    sub = sl[:, :40].contiguous()
    plan.tune("step23", 0)
    try:
        tpl, rot, shift, score = pr.align_best_shortlist(plan, a, b, sub, precision=ftk.BF16X3)
    finally:
        plan.tune("step23", 1)
    for i in range(6):
        Xi = X[i, sub[i].long()]
        assert float(score[i]) == float(Xi.max())
        assert float(X[i, tpl[i], shift[i], rot[i]]) == float(score[i])
    # the fused Steps 2-3 (default): the same maximum up to the rounding of Z before its split
    tpl, rot, shift, score = pr.align_best_shortlist(plan, a, b, sub, precision=ftk.BF16X3)
    for i in range(6):
        Xi = X[i, sub[i].long()]
        assert abs(float(score[i]) - float(Xi.max())) <= 5e-5 * float(Xi.abs().max())
        assert int(tpl[i]) in sub[i].tolist()


@pytest.mark.parametrize("precision,tol", [(ftk.FP32, 2e-5), (ftk.BF16X3, 2e-4)])
@pytest.mark.parametrize("window", [0.8, None])
def test_shortlist_matches_oracle(tiny, precision, tol, window):
    NI, NT, K = tiny.a.shape[0], tiny.b.shape[0], 5
    rng = np.random.default_rng(4)
    sl = np.stack([rng.choice(NT, K, replace=False) for _ in range(NI)]).astype(np.int32)
    centre = rng.uniform(-1.0, 1.0, size=(NI, 2)).astype(np.float32)
    cd = torch.from_numpy(centre).cuda() if window is not None else None
    tpl, rot, shift, score = [t.cpu().numpy() for t in pr.align_best_shortlist(
        tiny.plan, tiny.ad, tiny.bd, torch.from_numpy(sl).cuda(), cd, window or 0.0, precision)]
    sh = tiny.wl.shifts_px
    for i in range(NI):
        X = ftk_steps.ftk_scores(tiny.a[i], tiny.b[sl[i]], tiny.k, tiny.w, tiny.plan_o, tiny.delta)
        inside = (np.max(np.abs(sh - centre[i].astype(np.float64)), axis=1) <= window if window is not None
                  else np.ones(len(sh), dtype=bool))
        assert inside.any()
        Xw = np.where(inside[None, :, None], X, -np.inf)
        t, r, s, v = best_pose(Xw)
        scale = np.abs(X).max()
        assert abs(score[i] - v) < tol * scale
        assert inside[shift[i]] and tpl[i] in sl[i]
        j = int(np.nonzero(sl[i] == tpl[i])[0][0])
        assert abs(X[j, shift[i], rot[i]] - v) < 2 * tol * scale


def test_out_of_range_indices_are_contained(tiny):
    # a bad shortlist entry is replaced and latched (FTK_ERR_ARG at the next check);
    # a bad gather row yields NaN; neither touches memory outside the buffers
    NI, NT = tiny.a.shape[0], tiny.b.shape[0]
    sl = np.tile(np.arange(4, dtype=np.int32), (NI, 1))
    sl[2, 1] = NT + 5
    sl[4, 3] = -1
    for precision in (ftk.FP32, ftk.BF16X3):
        pr.align_best_shortlist(tiny.plan, tiny.ad, tiny.bd, torch.from_numpy(sl).cuda(), precision=precision)
        with pytest.raises(ftk.FtkError) as e:
            tiny.plan.stream_check()
        assert e.value.status == 1   # FTK_ERR_ARG
        tiny.plan.stream_check()     # latch cleared
    src = torch.arange(12, dtype=torch.float32, device="cuda").reshape(4, 3)
    got = pr.gather_rows(src, torch.tensor([3, 4, -1, 0], dtype=torch.int32, device="cuda")).cpu().numpy()
    assert np.array_equal(got[0], [9, 10, 11]) and np.array_equal(got[3], [0, 1, 2])
    assert np.isnan(got[1]).all() and np.isnan(got[2]).all()


@pytest.mark.parametrize("B,M,two_Q,NT,Mh,Qh", [
    (5, 6, 48, 19, 4, 7),      # direct-sum kernel (2Q not a multiple of 32)
    (1, 3, 12, 1, 3, 5),       # smallest
    (33, 8, 96, 40, 8, 47),    # FFT kernel, full band, ragged image and template blocks
    (9, 16, 192, 13, 12, 48),  # FFT kernel at the proposal workload's grid
])
def test_eqhead_matches_oracle(B, M, two_Q, NT, Mh, Qh):
    rng = np.random.default_rng(B + NT)
    U = 2 * Qh + 1
    a = (rng.normal(size=(B, M, two_Q)) + 1j * rng.normal(size=(B, M, two_Q))).astype(np.complex64)
    W = (rng.normal(size=(NT, Mh, U)) + 1j * rng.normal(size=(NT, Mh, U))).astype(np.complex64)
    beta = rng.normal(size=NT).astype(np.float32)
    alpha, stride = 0.8, NT + 3
    base = rng.normal(size=(B, stride)).astype(np.float32)
    ad, Wd, bd = (torch.from_numpy(x).cuda() for x in (a, W, beta))
    out = torch.from_numpy(base.copy()).cuda()
    rstar = torch.empty((B, NT), dtype=torch.int32, device="cuda")
    pr._call("ftk_nn_eqhead", pr._ptr(ad), B, M, two_Q, pr._ptr(Wd), pr._ptr(bd), NT, Mh, Qh, alpha, pr._ptr(out),
             stride, 1, pr._ptr(rstar), pr._stream_ptr())
    ref, rref = onn.eqhead_forward(W.astype(np.complex128), beta.astype(np.float64), a.astype(np.complex128), alpha)
    got = out.cpu().numpy()
    assert _rel(got[:, :NT] - base[:, :NT], ref) < 1e-5
    assert np.array_equal(got[:, NT:], base[:, NT:])                 # untouched padding columns
    # the maximising rotation: exact where the oracle's top two rotations are apart
    q = np.arange(-Qh, Qh + 1)
    E = np.exp(-1j * np.outer(q, 2 * np.pi * np.arange(two_Q) / two_Q))
    X = (np.einsum("jmu,bmu->bju", W.astype(np.complex128), a.astype(np.complex128)[:, :Mh, q % two_Q]) @ E).real
    rs = rstar.cpu().numpy()
    Xs = np.sort(X, axis=2)
    clear = (Xs[:, :, -1] - Xs[:, :, -2]) > 1e-4 * np.abs(X).max()
    assert np.array_equal(rs[clear], rref[clear])
    assert np.all(np.take_along_axis(X, rs[:, :, None], 2)[:, :, 0] >= Xs[:, :, -1] - 1e-4 * np.abs(X).max())
    # backward at the GPU's maximising rotations
    g = rng.normal(size=(B, stride)).astype(np.float32)
    gd = torch.from_numpy(g).cuda()
    dW = torch.empty_like(Wd)
    db = torch.empty_like(bd)
    pr._call("ftk_nn_eqhead_backward", pr._ptr(ad), B, M, two_Q, pr._ptr(gd), stride, pr._ptr(rstar), NT, Mh, Qh,
             alpha, pr._ptr(dW), pr._ptr(db), pr._stream_ptr())
    dW_ref, db_ref = onn.eqhead_backward(a.astype(np.complex128), rs, g[:, :NT].astype(np.float64), alpha, Mh, Qh)
    assert _rel(dW.cpu().numpy(), dW_ref) < 1e-5
    assert _rel(db.cpu().numpy(), db_ref) < 1e-5


@pytest.mark.parametrize("NT,S", [(1, 1), (7, 97), (300, 1164)])
def test_shared_spectral_weight_matches_oracle(NT, S):
    # W = rho W0 (one real weight per ring and angular frequency for all templates) and the
    # gradient of rho from dW, against oracle/nn.py
    rng = np.random.default_rng(NT + S)
    W0 = (rng.normal(size=(NT, S)) + 1j * rng.normal(size=(NT, S))).astype(np.complex64)
    rho = rng.uniform(0.2, 2.0, size=S).astype(np.float32)
    dW = (rng.normal(size=(NT, S)) + 1j * rng.normal(size=(NT, S))).astype(np.complex64)
    W0d, rhod, dWd = (torch.from_numpy(x).cuda() for x in (W0, rho, dW))
    W = torch.empty_like(W0d)
    pr._call("ftk_nn_scale_filters", pr._ptr(W0d), pr._ptr(rhod), NT, S, pr._ptr(W), pr._stream_ptr())
    ref = onn.scale_filters(W0.astype(np.complex128)[:, None, :], rho.astype(np.float64)[None, :])[:, 0, :]
    assert _rel(W.cpu().numpy(), ref) < 1e-6
    drho = torch.empty_like(rhod)
    pr._call("ftk_nn_scale_filters_backward", pr._ptr(W0d), pr._ptr(dWd), NT, S, pr._ptr(drho), pr._stream_ptr())
    dref = onn.scale_filters_backward(W0.astype(np.complex128)[:, None, :], dW.astype(np.complex128)[:, None, :])[0]
    assert _rel(drho.cpu().numpy(), dref) < 2e-5


@pytest.mark.parametrize("two_Q", [64, 192])
def test_eqhead_is_invariant_to_grid_rotations(two_Q):
    rng = np.random.default_rng(21)
    B, M, NT, Mh, Qh = 2, 4, 6, 4, 20
    a = rng.normal(size=(B, M, two_Q)) + 1j * rng.normal(size=(B, M, two_Q))
    q = np.arange(two_Q)
    q = np.where(q >= two_Q // 2, q - two_Q, q)
    a_rot = a * np.exp(-1j * q * (2 * np.pi * 11 / two_Q))[None, None, :]
    W = rng.normal(size=(NT, Mh, 2 * Qh + 1)) + 1j * rng.normal(size=(NT, Mh, 2 * Qh + 1))
    res = []
    for x in (a, a_rot):
        xd = torch.from_numpy(x.astype(np.complex64)).cuda()
        Wd = torch.from_numpy(W.astype(np.complex64)).cuda()
        bd = torch.zeros(NT, device="cuda")
        out = torch.empty((B, NT), device="cuda")
        rstar = torch.empty((B, NT), dtype=torch.int32, device="cuda")
        pr._call("ftk_nn_eqhead", pr._ptr(xd), B, M, two_Q, pr._ptr(Wd), pr._ptr(bd), NT, Mh, Qh, 1.0, pr._ptr(out),
                 NT, 0, pr._ptr(rstar), pr._stream_ptr())
        res.append((out.cpu().numpy(), rstar.cpu().numpy()))
    assert _rel(res[1][0], res[0][0]) < 1e-5
    assert np.array_equal((res[0][1] - res[1][1]) % two_Q, np.full((B, NT), 11))


@pytest.mark.parametrize("head_weight", ["template", "shared"])
def test_network_checkpoint_round_trip_and_resume(tmp_path, head_weight):
    # A checkpoint restores parameters, Adam moments and step count exactly; fit with a
    # checkpoint resumes after the recorded epochs with the minibatch order of an
    # uninterrupted run, so 1 + 1 epochs equal 2 epochs (up to FP32 summation order).
    rng = np.random.default_rng(11)
    B, M, Q, NT = 64, 16, 16, 20
    coeffs = torch.from_numpy((rng.normal(size=(B, M, 2 * Q)) + 1j * rng.normal(size=(B, M, 2 * Q)))
                              .astype(np.complex64)).cuda()
    labels = torch.from_numpy(rng.integers(0, NT, B).astype(np.int32)).cuda()
    target = torch.from_numpy(rng.normal(size=(B, 2)).astype(np.float32)).cuda()
    kw = dict(ch=(4, 8, 8, 8), hidden=16, head_rings=4, head_band=3)
    if head_weight == "shared":   # head alone: fixed filters W0 (a buffer the checkpoint keeps), learned rho
        kw = dict(head_rings=4, head_band=3, cnn=False, head_weight="shared")
    W0 = torch.from_numpy(rng.normal(size=(NT, 4, 7, 2)).astype(np.float32)).cuda()

    def make():
        net = pr.ProposalNet(M, Q, NT, seed=3, **kw)
        if head_weight == "shared":
            net.hW0.copy_(W0)
        return net

    ref = make()
    pr.fit(ref, coeffs, labels, target, epochs=2, batch=16, seed=5)

    ck = str(tmp_path / "net.npz")
    a = make()
    pr.fit(a, coeffs, labels, target, epochs=1, batch=16, seed=5, checkpoint=ck)
    b = pr.ProposalNet.load(ck)                       # architecture from the file, state restored
    for k in a.p:
        for d1, d2 in ((a.p, b.p), (a.m, b.m), (a.v, b.v)):
            assert torch.equal(d1[k], d2[k]), k
    if head_weight == "shared":
        assert torch.equal(b.hW0, W0) and "hr" in b.p and "hW" not in b.p
    assert b.t == a.t > 0
    pr.fit(b, coeffs, labels, target, epochs=2, batch=16, seed=5, checkpoint=ck)   # resumes at epoch 1
    assert b.t == ref.t
    for k in ref.p:
        assert _rel(b.p[k].cpu().numpy(), ref.p[k].cpu().numpy()) < 1e-5, k
    if head_weight == "shared":
        assert not torch.equal(b.p["hr"], torch.ones_like(b.p["hr"]))   # the shared weight was trained
    other = pr.ProposalNet(M, Q, NT + 1, seed=3, **kw)
    with pytest.raises(ValueError):
        other.load_state(ck)
