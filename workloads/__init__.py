"""Seeded synthetic workloads for rigid image alignment (template matching).

This package only draws random inputs: Gaussian-blob templates, rotated and
shifted noisy images made from them, and shift sets. It holds none of the
alignment method's arithmetic, so both the CPU oracle and the GPU library may
use it.
"""

from .synthetic import (  # noqa: F401
    BATCH_GROUPS,
    CONFIGS,
    Workload,
    make_workload,
    shift_lattice,
    blob_params,
    render_blobs,
)
