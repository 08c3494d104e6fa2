"""Best pose per image (oracle; test infrastructure only).

Section 6: after all inner products are computed, each image's maximum over
(template, rotation, shift) is its estimated pose. Ties are broken by the
lowest (template, rotation, shift) index, in that order of significance.
"""

from __future__ import annotations

import numpy as np


def best_pose(X: np.ndarray):
    """X: [NT, N, 2Q] scores of one image. Returns (template, rot, shift, score)."""
    NT, N, two_Q = X.shape
    # order (template, r, s) lexicographically; argmax returns the first maximum
    Xt = np.transpose(X, (0, 2, 1)).reshape(-1)
    idx = int(np.argmax(Xt))
    t, rem = divmod(idx, two_Q * N)
    r, s = divmod(rem, N)
    return t, r, s, float(Xt[idx])

