"""FP64 oracle for fixed-budget component selection (Sec. 5 "Band-Limiting
Revisited": with a budget of standard convolutions, the best choice in the
least-squares sense, averaged over all rotations, is the components with the
largest coefficients), test infrastructure only.

* Energy of component k on the lattice box B = [-R, R]^2:
      E_k = sum_{d in B} |F_k(d)|^2,  F_k(d) = f_k(|d|) e^{ik theta(d)}
  (F_k(0) = 0 for k != 0).  For every lattice point, orthogonality of
  e^{-ik alpha} over the rotation angle alpha gives
      (1/2pi) int |T_alpha F(d) - T_alpha F_S(d)|^2 d alpha = sum_{k not in S} |F_k(d)|^2,
  so the rotation-averaged squared error of steering with the subset S is
  the dropped energy, and keeping the largest E_k minimises it.
* Reading: a real filter's components come in pairs +-k of equal energy
  (a pair costs one complex correlation); G_0 (one real correlation, the
  angle-independent mean) is always kept, and the remaining budget - 1
  components are the k >= 1 of largest E_k (ties to the smaller k).
* Subset sweep: S(p, j) = G_0(p) + 2 sum_{k in S, k >= 1} Re(e^{ik alpha_j} G_k(p)).
* The alternative the paper compares against (Fig. f:frequency): with a
  budget of B standard correlations, correlate the image with B rotated
  copies of the pattern itself (no band limit), alpha_j = 2 pi j / B, and
  keep per pixel the largest response.  The copies are the sampled pattern
  rotated by cubic-spline interpolation (a library step), the correlations
  FFTs (a library step).
"""
from __future__ import annotations

import numpy as np

from .so2 import box_offsets, sweep_from_components


def component_energy(filt, K: int, radius: int):
    """E_k, k = 0..K, of a filter object with ``radial(k, r)`` on the box."""
    dx, dy = box_offsets(radius)
    r = np.hypot(dx, dy).astype(np.float64)
    E = np.zeros(K + 1)
    for k in range(K + 1):
        f = filt.radial(k, r)
        if k != 0:
            f = np.where(r == 0, 0.0, f)
        E[k] = float(np.sum(np.abs(f) ** 2))
    return E


def select_components(E, budget: int):
    """Component list [0, k_1 < k_2 < ...] of length min(budget, K + 1): G_0 plus
    the budget - 1 components k >= 1 of largest energy."""
    E = np.asarray(E, np.float64)
    K = len(E) - 1
    order = sorted(range(1, K + 1), key=lambda k: (-E[k], k))
    return [0] + sorted(order[:max(budget, 1) - 1])


def steered_error_sq(filt, K: int, radius: int, ks, n_alpha: int):
    """Rotation-averaged squared error sum_d mean_alpha |T_alpha F(d) - T_alpha F_S(d)|^2
    by direct evaluation on n_alpha equispaced angles (exact for n_alpha > 2K)."""
    dx, dy = box_offsets(radius)
    r = np.hypot(dx, dy).astype(np.float64)
    th = np.arctan2(dy, dx).astype(np.float64)
    keep = set(ks)
    total = 0.0
    for j in range(n_alpha):
        a = 2 * np.pi * j / n_alpha
        full = np.zeros(r.shape, np.complex128)
        part = np.zeros(r.shape, np.complex128)
        for k in range(-K, K + 1):
            f = filt.radial(k, r)
            if k != 0:
                f = np.where(r == 0, 0.0, f)
            term = f * np.exp(1j * k * (th - a))
            full += term
            if abs(k) in keep:
                part += term
        total += float(np.sum(np.abs(full - part) ** 2))
    return total / n_alpha


def sweep_subset_from_components(G, ks, J: int):
    """Subset sweep from the full component list G = [G_0, ..., G_K]: the
    components outside ``ks`` contribute nothing.  Returns (J, ...), real."""
    K = len(G) - 1
    keep = set(ks)
    Gs = [G[k] if k in keep else np.zeros_like(G[k]) for k in range(K + 1)]
    return sweep_from_components(Gs, K, J).real


def rotate_pattern(img, alpha):
    """The sampled pattern rotated by alpha, (T_alpha P)(d) = P(R(-alpha) d) on
    the same (2R+1)^2 box (d = (column, row) offset from the centre), by cubic
    spline interpolation (scipy.ndimage.map_coordinates; zero outside)."""
    from scipy import ndimage
    img = np.asarray(img, np.float64)
    n = img.shape[0]
    R = (n - 1) // 2
    dy, dx = np.mgrid[-R:R + 1, -R:R + 1].astype(np.float64)
    c, s = np.cos(alpha), np.sin(alpha)
    x = c * dx + s * dy                     # R(-alpha) d
    y = -s * dx + c * dy
    return ndimage.map_coordinates(img, [y + R, x + R], order=3, mode="constant", cval=0.0)


def rotated_copies_sweep(H, pattern, B: int, workers: int = -1):
    """Max over B rotated copies of the pattern of the plain correlation
    sum_d H(p + d) (T_{alpha_j} P)(d), alpha_j = 2 pi j / B; returns (max,
    first argmax j).  Periodic, the box wrapped as in the other operators."""
    import scipy.fft as sfft
    H = np.asarray(H, np.float64)
    h, w = H.shape
    n = np.shape(pattern)[0]
    R = (n - 1) // 2
    dy, dx = np.mgrid[-R:R + 1, -R:R + 1]
    Hf = sfft.rfft2(H, workers=workers)
    best = np.full((h, w), -np.inf)
    arg = np.zeros((h, w), np.int64)
    for j in range(B):
        f = rotate_pattern(pattern, 2 * np.pi * j / B)
        grid = np.zeros((h, w))
        np.add.at(grid, (dy.ravel() % h, dx.ravel() % w), f.ravel())
        s = sfft.irfft2(Hf * np.conj(sfft.rfft2(grid, workers=workers)), s=(h, w), workers=workers)
        upd = s > best
        arg = np.where(upd, j, arg)
        best = np.where(upd, s, best)
    return best, arg
