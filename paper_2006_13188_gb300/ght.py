"""Pattern detection with the generalised Hough transform of Sec. 5.

Orchestration only: the gradient signal and field, the voted consensus
filter, its angular decomposition and the extended convolution all run in
the library's kernels; this module sequences the calls.
"""
from __future__ import annotations

import numpy as np

from . import _binding as b


def consensus_filter(plan, P, centre, eps, K, dr=0.25, n_theta=128):
    """The consensus filter of pattern P (float64 array) about `centre` =
    (cy, cx) with support radius eps, as a SAMPLED FilterSO2 band-limited to
    |k| <= K, and the raw voted grid (float64, (2R+1)^2)."""
    P = np.ascontiguousarray(np.asarray(P, np.float64))
    R = b.ext_consensus_radius(eps)
    F = np.zeros((2 * R + 1, 2 * R + 1), np.float64)
    b.ext_consensus_filter(plan, P, P.shape[0], P.shape[1], centre[0], centre[1], eps, F)
    return b.FilterSO2.sampled(F, K, dr, n_theta), F


def detect(plan, I, h, w, filt, out, stream=None):
    """Detection response {|grad I|, theta_grad I} * F (Eq. Def-EConv) of image
    I into `out` (h x w float32, host or device)."""
    b.ext_ght_detect(plan, I, h, w, filt, out, stream)
    return out
