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


def detect(plan, I, h, w, filt, out, H=None, theta=None, stream=None):
    """Detection response {|grad I|, theta_grad I} * F (Eq. Def-EConv) of image
    I into `out` (h x w float32); H and theta (h x w float32 scratch, device
    when I is) receive the signal and the field."""
    import torch
    dev = I.device if hasattr(I, "device") else None
    if H is None:
        H = torch.empty((h, w), dtype=torch.float32, device=dev) if dev is not None else np.empty((h, w), np.float32)
    if theta is None:
        theta = torch.empty((h, w), dtype=torch.float32, device=dev) if dev is not None else np.empty((h, w), np.float32)
    b.ext_gradient_field(plan, I, h, w, H, theta, stream)
    b.ext_conv_so2(plan, H, h, w, filt, theta, out, stream)
    return out
