"""Seeded synthetic template-matching workloads.

The paper's experiment (Section 6) aligns noisy images against templates that
are unit-L2 projections of a 3D density, with images made by rotating the
templates by random real angles and shifting them by random sub-pixel shifts.
That density is not available here, so templates are sums of isotropic 2D
Gaussians evaluated analytically at the pixel centres x_ij = (i dx - 1, j dx - 1),
i, j = 0..n-1, dx = 2/n (Section 2.1; first array index = x). Rotation and shift
are applied to the Gaussian centres, so they are exact, not resampled.

An image made from template B with rotation theta and shift s (pixels) has
centres c -> R_theta c + s * dx. With the inner product X(delta, gamma) of
eq. (Xdg) (translate the image by delta, then rotate by gamma), its best match is
template B at delta = -s * dx and gamma = -theta (mod 2 pi).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

# Workload table. Each entry: image size n, radial nodes M, angular nodes 2Q,
# precision target eps, counts, blob recipe, SNR, shift-lattice spacing/radius
# (pixels). W = radius / 2 (the maximum shift is 2W pixels, Section 2).
CONFIGS = {
    "n32_tiny": dict(n=32, M=16, two_Q=96, eps=1e-2, n_templates=16, n_images=16,
                     blobs=8, sigma_px=(1.0, 4.0), snr=1.0, shift_h=0.5, shift_r=2.0,
                     image_shift_r=2.0, image_template="cyclic", projected=False),
    "n64_1k": dict(n=64, M=32, two_Q=192, eps=1e-3, n_templates=1024, n_images=1024,
                   blobs=16, sigma_px=(1.0, 6.0), snr=0.1, shift_h=0.25, shift_r=3.0,
                   image_shift_r=3.0, image_template="cyclic", projected=False),
    # the n = 64 recipe with 256 x 256 pairs: a small case for profiling captures
    "n64_256": dict(n=64, M=32, two_Q=192, eps=1e-3, n_templates=256, n_images=256,
                    blobs=16, sigma_px=(1.0, 6.0), snr=0.1, shift_h=0.25, shift_r=3.0,
                    image_shift_r=3.0, image_template="cyclic", projected=False),
    # the n = 64 recipe with 64 x 256 pairs (one 16384-pair chunk, ~2.5 GB on the device):
    # the case for full ncu captures of single kernels
    "n64_64x256": dict(n=64, M=32, two_Q=192, eps=1e-3, n_templates=256, n_images=64,
                       blobs=16, sigma_px=(1.0, 6.0), snr=0.1, shift_h=0.25, shift_r=3.0,
                       image_shift_r=3.0, image_template="cyclic", projected=False),
    # template-proposal workload: the n = 64 grid, templates centred on their
    # intensity centroid (as projections of a centred density are), so that an
    # image's best shift is set by the image alone
    "n64_prop": dict(n=64, M=32, two_Q=192, eps=1e-3, n_templates=512, n_images=2048,
                     blobs=16, sigma_px=(1.0, 6.0), snr=0.1, shift_h=0.25, shift_r=3.0,
                     image_shift_r=3.0, image_template="random", projected=False, centered=True),
    "n128_8k": dict(n=128, M=64, two_Q=384, eps=1e-3, n_templates=4096, n_images=8192,
                    blobs=32, sigma_px=(1.0, 6.0), snr=0.05, shift_h=0.25, shift_r=4.0,
                    image_shift_r=4.0, image_template="random", projected=True),
    # the n = 128 recipe with 64 x 256 pairs (one 16384-pair chunk, about 8 GB on the device): the
    # case for full ncu captures of single kernels on the benchmark's grid
    "n128_64x256": dict(n=128, M=64, two_Q=384, eps=1e-3, n_templates=256, n_images=64,
                        blobs=32, sigma_px=(1.0, 6.0), snr=0.05, shift_h=0.25, shift_r=4.0,
                        image_shift_r=4.0, image_template="random", projected=True),
    # uneven groups of image sizes searched together (one group per size, each against its
    # own 1024 templates); shift radius n / 32 px at 0.25 px spacing, W = radius / 2
    "b64_2k": dict(n=64, M=32, two_Q=192, eps=1e-3, n_templates=1024, n_images=2048,
                   blobs=32, sigma_px=(1.0, 6.0), snr=0.1, shift_h=0.25, shift_r=2.0,
                   image_shift_r=2.0, image_template="random", projected=True),
    "b96_1k": dict(n=96, M=48, two_Q=288, eps=1e-3, n_templates=1024, n_images=1024,
                   blobs=32, sigma_px=(1.0, 6.0), snr=0.1, shift_h=0.25, shift_r=3.0,
                   image_shift_r=3.0, image_template="random", projected=True),
    "b128_512": dict(n=128, M=64, two_Q=384, eps=1e-3, n_templates=1024, n_images=512,
                     blobs=32, sigma_px=(1.0, 6.0), snr=0.1, shift_h=0.25, shift_r=4.0,
                     image_shift_r=4.0, image_template="random", projected=True),
    "b192_256": dict(n=192, M=96, two_Q=576, eps=1e-3, n_templates=1024, n_images=256,
                     blobs=32, sigma_px=(1.0, 6.0), snr=0.1, shift_h=0.25, shift_r=6.0,
                     image_shift_r=6.0, image_template="random", projected=True),
    # the proposal workload on the precision grid: n = 128, 2048 centred projected templates
    "n128_prop": dict(n=128, M=64, two_Q=384, eps=1e-3, n_templates=2048, n_images=8192,
                      blobs=32, sigma_px=(1.0, 6.0), snr=0.05, shift_h=0.25, shift_r=4.0,
                      image_shift_r=4.0, image_template="random", projected=True, centered=True),
    # the learned-proposal configuration at its stated size: n = 128, 16384 centred projected
    # templates, 65536 images at SNR 0.05; shift set and eps as the precision workload (the
    # configuration states neither); NT * 2Q * N = 5.0e9 pose indices per image
    "n128_16k": dict(n=128, M=64, two_Q=384, eps=1e-3, n_templates=16384, n_images=65536,
                     blobs=32, sigma_px=(1.0, 6.0), snr=0.05, shift_h=0.25, shift_r=4.0,
                     image_shift_r=4.0, image_template="random", projected=True, centered=True),
}

# the uneven-groups workload: its four member workloads
BATCH_GROUPS = ("b64_2k", "b96_1k", "b128_512", "b192_256")


def shift_lattice(h: float, r: float) -> np.ndarray:
    """All lattice shifts (a h, b h), a, b integers, with norm <= r (pixels).

    Returned as float64 [N, 2] in row-major lattice order (a outer, b inner).
    """
    m = int(math.floor(r / h + 1e-9))
    out = []
    for a in range(-m, m + 1):
        for b in range(-m, m + 1):
            if (a * h) ** 2 + (b * h) ** 2 <= r * r + 1e-9:
                out.append((a * h, b * h))
    return np.asarray(out, dtype=np.float64)


def blob_params(rng: np.random.Generator, n: int, count: int, sigma_px, projected: bool):
    """Random Gaussian blobs: centres (in [-1,1]^2 units), widths, amplitudes.

    Centres are uniform in the disk of radius 0.5. With ``projected`` the blobs
    are 3D isotropic Gaussians projected along a random direction, which is again
    a set of 2D isotropic Gaussians at the projected centres.
    """
    dx = 2.0 / n
    if projected:
        # uniform in the 3D ball of radius 0.5, projected along a random axis
        v = rng.normal(size=(count, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        rad = 0.5 * rng.uniform(0.0, 1.0, count) ** (1.0 / 3.0)
        p3 = v * rad[:, None]
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        e1 = np.cross(axis, [1.0, 0.0, 0.0] if abs(axis[0]) < 0.9 else [0.0, 1.0, 0.0])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(axis, e1)
        centres = np.stack([p3 @ e1, p3 @ e2], axis=1)
    else:
        rad = 0.5 * np.sqrt(rng.uniform(0.0, 1.0, count))
        th = rng.uniform(0.0, 2.0 * math.pi, count)
        centres = np.stack([rad * np.cos(th), rad * np.sin(th)], axis=1)
    sigma = rng.uniform(sigma_px[0], sigma_px[1], count) * dx
    amp = rng.uniform(0.5, 1.0, count)
    return centres, sigma, amp


def render_blobs(n: int, centres: np.ndarray, sigma: np.ndarray, amp: np.ndarray) -> np.ndarray:
    """Evaluate sum_g amp_g exp(-|x - c_g|^2 / (2 sigma_g^2)) at the pixel centres."""
    dx = 2.0 / n
    xs = np.arange(n) * dx - 1.0
    gx = np.exp(-((xs[None, :] - centres[:, 0:1]) ** 2) / (2.0 * sigma[:, None] ** 2))  # [G, n]
    gy = np.exp(-((xs[None, :] - centres[:, 1:2]) ** 2) / (2.0 * sigma[:, None] ** 2))
    return np.einsum("g,gi,gj->ij", amp, gx, gy)


@dataclasses.dataclass
class Workload:
    name: str
    n: int
    M: int
    two_Q: int
    eps: float
    W: float
    shifts_px: np.ndarray          # [N, 2] float64, pixels
    templates: np.ndarray          # [NT, n, n] float32
    images: np.ndarray             # [NI, n, n] float32
    true_template: np.ndarray      # [NI] int
    true_theta: np.ndarray         # [NI] float64 (radians)
    true_shift_px: np.ndarray      # [NI, 2] float64
    template_blobs: list           # per template (centres, sigma, amp)


def make_workload(name: str, seed: int | None = None, n_images: int | None = None,
                  n_templates: int | None = None, noise: bool = True,
                  dtype=np.float32, image_seed: int | None = None) -> Workload:
    """Build the named workload deterministically.

    ``n_images`` / ``n_templates`` override the counts (a prefix of the same
    seeded streams is not guaranteed; overrides draw their own sets).
    ``image_seed`` draws the images from their own stream while keeping the
    templates of ``seed`` (fresh images of the same template set).
    """
    cfg = CONFIGS[name]
    n = cfg["n"]
    dx = 2.0 / n
    base = 1905 + list(CONFIGS).index(name) if seed is None else seed
    ss = np.random.SeedSequence(base)
    s_tpl, s_img = ss.spawn(2)
    if image_seed is not None:
        s_img = np.random.SeedSequence([base, 77, image_seed])
    rng_t = np.random.Generator(np.random.PCG64(s_tpl))
    rng_i = np.random.Generator(np.random.PCG64(s_img))
    NT = cfg["n_templates"] if n_templates is None else n_templates
    NI = cfg["n_images"] if n_images is None else n_images

    templates = np.empty((NT, n, n), dtype=np.float64)
    blobs = []
    for t in range(NT):
        c, s, a = blob_params(rng_t, n, cfg["blobs"], cfg["sigma_px"], cfg["projected"])
        if cfg.get("centered"):
            mass = a * s * s          # integral of each blob is 2 pi amp sigma^2
            c = c - (mass[:, None] * c).sum(axis=0) / mass.sum()
        img = render_blobs(n, c, s, a)
        norm = math.sqrt(dx * dx * float(np.sum(img * img)))  # unit L2 norm on [-1,1]^2
        a = a / norm
        templates[t] = img / norm
        blobs.append((c, s, a))

    images = np.empty((NI, n, n), dtype=np.float64)
    true_t = np.empty(NI, dtype=np.int64)
    theta = rng_i.uniform(0.0, 2.0 * math.pi, NI)
    rad = cfg["image_shift_r"] * np.sqrt(rng_i.uniform(0.0, 1.0, NI))
    phi = rng_i.uniform(0.0, 2.0 * math.pi, NI)
    shift = np.stack([rad * np.cos(phi), rad * np.sin(phi)], axis=1)
    for i in range(NI):
        t = i % NT if cfg["image_template"] == "cyclic" else int(rng_i.integers(NT))
        true_t[i] = t
        c, s, a = blobs[t]
        ct, st = math.cos(theta[i]), math.sin(theta[i])
        rot = np.stack([ct * c[:, 0] - st * c[:, 1], st * c[:, 0] + ct * c[:, 1]], axis=1)
        img = render_blobs(n, rot + shift[i] * dx, s, a)
        if noise:
            var = float(np.mean(img * img)) / cfg["snr"]
            img = img + rng_i.normal(scale=math.sqrt(var), size=img.shape)
        images[i] = img

    return Workload(name=name, n=n, M=cfg["M"], two_Q=cfg["two_Q"], eps=cfg["eps"],
                    W=cfg["shift_r"] / 2.0,
                    shifts_px=shift_lattice(cfg["shift_h"], cfg["shift_r"]),
                    templates=templates.astype(dtype), images=images.astype(dtype),
                    true_template=true_t, true_theta=theta, true_shift_px=shift,
                    template_blobs=blobs)
