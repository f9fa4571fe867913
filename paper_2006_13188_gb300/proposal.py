"""Training of the learned SO(3) proposal from planted volumes.

Orchestration only: every step (component correlations, the grid sweep
that labels the samples, their refinement, the gathering of channel rows,
augmentation, the network's forward/backward passes and Adam) runs in the
library's kernels; this module picks sample voxels and sequences the calls.
Random draws (minibatch rows, augmentation rotations) are inputs.
"""
from __future__ import annotations

import numpy as np

from . import _binding as b


def neighbourhood_voxels(centres, shape, reach=2):
    """Flat indices of the (2 reach + 1)^3 voxels around each centre (periodic)."""
    nz, ny, nx = shape
    d = np.arange(-reach, reach + 1)
    out = []
    for c in centres:
        zz, yy, xx = np.meshgrid((c[0] + d) % nz, (c[1] + d) % ny, (c[2] + d) % nx, indexing="ij")
        out.append(((zz * ny + yy) * nx + xx).ravel())
    return np.concatenate(out).astype(np.int32)


def training_rows(plan, V, shape, tables, dr, radius, grid, vox, precision=b.EXT_PREC_BF16X3):
    """Channel rows at voxels `vox` of volume V (device tensor) and their
    labels: the grid argmax refined by gradient ascent.  Returns (X [n][C],
    q [n][4], grid max at vox) as device tensors."""
    import torch
    nz, ny, nx = shape
    P = nz * ny * nx
    L = len(tables) - 1
    C = b.ext_so3_channels(L)
    dev = V.device
    G = torch.empty((C, P), dtype=torch.float32, device=dev)
    b.ext_corr_so3_components(plan, V, nz, ny, nx, tables, dr, radius, G)
    mx = torch.empty(P, dtype=torch.float32, device=dev)
    am = torch.empty(P, dtype=torch.int32, device=dev)
    b.ext_sweep_so3(plan, G, P, L, grid, mx, am, precision)
    vt = torch.from_numpy(np.ascontiguousarray(vox)).to(dev)
    n = len(vox)
    X = torch.empty((n, C), dtype=torch.float32, device=dev)
    b.ext_so3_gather(plan, G, P, L, vt, n, X)
    gq = torch.from_numpy(np.ascontiguousarray(np.asarray(grid, np.float32))).to(dev)
    q0 = gq[am[vt.long()].long()].contiguous()
    q = torch.empty((n, 4), dtype=torch.float32, device=dev)
    s = torch.empty(n, dtype=torch.float32, device=dev)
    b.ext_so3_refine(plan, X, n, L, q0, q, s)
    plan.sync()
    return X, q, mx[vt.long()].clone()


def training_set(plan, problems, grid, reach=2, precision=b.EXT_PREC_BF16X3):
    """Rows, labels and the grid maxima at the planted centres from planted
    volumes (dicts with V, centres, tables, dr, radius, e.g. from
    synth.so3_training_volumes): every planted centre and its (2 reach + 1)^3
    neighbourhood.  Returns (X, q) as device tensors and the centre maxima."""
    import torch
    rows, labels, peaks = [], [], []
    mid = ((2 * reach + 1) ** 3) // 2
    for prob in problems:
        shape = prob["V"].shape
        vox = neighbourhood_voxels(prob["centres"], shape, reach)
        V = torch.from_numpy(np.ascontiguousarray(prob["V"])).cuda()
        X, q, mx = training_rows(plan, V, shape, prob["tables"], prob["dr"], prob["radius"], grid, vox, precision)
        rows.append(X)
        labels.append(q)
        peaks.extend(mx.cpu().numpy()[mid::(2 * reach + 1) ** 3].tolist())
    return torch.cat(rows), torch.cat(labels), np.asarray(peaks)


def train(net, X, q, L, rows, Q, steps, batch, lrs=(1e-3, 2.5e-4)):
    """Adam on (X, q) with rotation augmentation, the steps split evenly over
    the learning rates `lrs`; rows (int32 [steps*batch]) and Q (float32
    [steps*batch][4]) are the random draws.  Returns the per-step losses."""
    losses = np.zeros(steps, np.float32)
    n = X.shape[0]
    bounds = np.linspace(0, steps, len(lrs) + 1).astype(int)
    for lr, s0, s1 in zip(lrs, bounds[:-1], bounds[1:]):
        if s1 <= s0:
            continue
        part = np.zeros(s1 - s0, np.float32)
        b.ext_mlp_train(net, X, q, n, L, rows[s0 * batch:s1 * batch], Q[s0 * batch:s1 * batch], s1 - s0, batch,
                        lr, part)
        losses[s0:s1] = part
    return losses
