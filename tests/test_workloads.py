"""The seeded synthetic inputs (stand-ins for Section 6's projections): unit-L2
templates, exact rotated and shifted images, the stated noise level, the shift sets
and their sizes, and seeding (no GPU)."""

import math

import numpy as np
import pytest

from workloads import BATCH_GROUPS, CONFIGS, make_workload, render_blobs, shift_lattice


@pytest.mark.parametrize("name,N", [("n32_tiny", 49), ("n64_1k", 441), ("n128_8k", 797), ("b64_2k", 197),
                                    ("b192_256", 1793)])
def test_shift_sets_have_the_stated_sizes(name, N):
    cfg = CONFIGS[name]
    s = shift_lattice(cfg["shift_h"], cfg["shift_r"])
    assert s.shape == (N, 2)
    assert np.all(np.hypot(s[:, 0], s[:, 1]) <= cfg["shift_r"] + 1e-9)
    # every lattice point of the disk, each once
    k = np.rint(s / cfg["shift_h"]).astype(int)
    assert np.allclose(k * cfg["shift_h"], s) and len({tuple(v) for v in k}) == N
    # |s| <= 2W with W = radius / 2 (Section 2)
    assert np.max(np.hypot(s[:, 0], s[:, 1])) <= 2 * (cfg["shift_r"] / 2.0) + 1e-12


def test_templates_have_unit_norm_and_images_their_noise():
    wl = make_workload("n64_1k", n_images=6, n_templates=4)
    dx = 2.0 / wl.n
    for t in wl.templates.astype(np.float64):
        assert abs(dx * dx * np.sum(t * t) - 1.0) < 1e-5      # unit L2 on [-1, 1]^2 (float32 storage)
    clean = make_workload("n64_1k", n_images=6, n_templates=4, noise=False)
    assert np.array_equal(clean.templates, wl.templates)
    noise = wl.images.astype(np.float64) - clean.images.astype(np.float64)
    snr = CONFIGS["n64_1k"]["snr"]
    for i in range(6):
        want = np.mean(clean.images[i].astype(np.float64) ** 2) / snr
        assert abs(np.var(noise[i]) / want - 1.0) < 0.1      # variance mean(I^2) / SNR, 4096 samples


def test_noise_free_image_is_the_exactly_rotated_and_shifted_template():
    wl = make_workload("n32_tiny", n_images=3, n_templates=3, noise=False)
    for i in range(3):
        c, s, a = wl.template_blobs[wl.true_template[i]]
        th, sh = wl.true_theta[i], wl.true_shift_px[i]
        rot = np.stack([math.cos(th) * c[:, 0] - math.sin(th) * c[:, 1],
                        math.sin(th) * c[:, 0] + math.cos(th) * c[:, 1]], axis=1)
        ref = render_blobs(wl.n, rot + sh * (2.0 / wl.n), s, a)
        assert np.allclose(wl.images[i], ref, rtol=1e-6, atol=1e-6)
        assert np.hypot(*sh) <= CONFIGS["n32_tiny"]["image_shift_r"] + 1e-12


def test_seeding_is_deterministic_and_streams_are_separate():
    a = make_workload("n32_tiny", n_images=2, n_templates=2)
    b = make_workload("n32_tiny", n_images=2, n_templates=2)
    assert np.array_equal(a.images, b.images) and np.array_equal(a.templates, b.templates)
    c = make_workload("n32_tiny", n_images=2, n_templates=2, image_seed=5)
    assert np.array_equal(c.templates, a.templates) and not np.array_equal(c.images, a.images)
    d = make_workload("n32_tiny", n_images=2, n_templates=2, seed=7)
    assert not np.array_equal(d.templates, a.templates)


def test_centred_templates_have_their_intensity_centroid_at_the_origin():
    wl = make_workload("n64_prop", n_images=1, n_templates=3)
    for c, s, a in wl.template_blobs:
        mass = a * s * s
        assert np.allclose((mass[:, None] * c).sum(axis=0), 0.0, atol=1e-12)


def test_uneven_groups_follow_n_over_32_shift_radius():
    for g in BATCH_GROUPS:
        cfg = CONFIGS[g]
        assert cfg["shift_r"] == cfg["n"] / 32 and cfg["M"] == cfg["n"] // 2 and cfg["two_Q"] == 3 * cfg["n"]
