"""FP64 oracle for SO(3) extended correlation (Sec. 9; test infrastructure only).

Spherical harmonics are the orthonormal complex Y_l^m with the Condon-Shortley
phase (the associated Legendre functions come from scipy.special.lpmv, a
library step); theta is the polar angle from +z, phi = atan2(y, x); voxel
offsets d = (dx, dy, dz) with x = column, y = row, z = slice.

Filter (Sec. 9 "Filter Decomposition"):
    F(x) = sum_{l <= L} sum_{|a| <= l} f_l^a(|x|) Y_l^a(x^),
f_l^a given as radial tables with the cubic Hermite interpolant of
oracle.filters_so2.RadialTable; at x = 0 only l = 0 contributes.

Rotations act by (T_R F)(x) = F(R^-1 x).  The matrix C^l(R) is defined by
    T_R Y_l^a = sum_b C^l_ab(R) Y_l^b
and computed here straight from that definition, by projecting Y_l^a(R^-1 x)
onto Y_l^b with a quadrature that is exact for band-limited products.
(Sec. 9 calls these the Wigner-D functions; its index roles are fixed by this
definition.)

Extended correlation (Eq. Def-ECorr) with a rotation R at every voxel, or
swept over a list of rotations:
    S(p, R) = sum_{d in B} V(p + d) conj(F(R^-1 d)),   B = [-Rb, Rb]^3,
periodic mod the volume shape.  The component form of Sec. 9,
    S(p, R) = sum_{l,a,b} conj(C^l_ab(R)) G_l^{ab}(p),
    G_l^{ab} = V (*) (f_l^a Y_l^b),
is provided separately (component_correlation, sweep_from_components) and is
pinned against the brute force.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import lpmv, roots_legendre

from .filters_so2 import hermite_eval


def sph_harm(l: int, m: int, theta, phi):
    """Orthonormal Y_l^m(theta, phi) with the Condon-Shortley phase."""
    theta = np.asarray(theta, np.float64)
    phi = np.asarray(phi, np.float64)
    am = abs(m)
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    y = norm * lpmv(am, l, np.cos(theta)) * np.exp(1j * am * phi)
    if m < 0:
        y = ((-1) ** am) * np.conj(y)
    return y


def to_spherical(x, y, z):
    r = np.sqrt(x * x + y * y + z * z)
    theta = np.arccos(np.clip(np.where(r > 0, z / np.where(r > 0, r, 1.0), 1.0), -1.0, 1.0))
    phi = np.arctan2(y, x)
    return r, theta, phi


class SHFilter:
    """F(x) = sum_{l,a} f_l^a(|x|) Y_l^a(x^); tables[l] has shape (2l+1, n_r),
    row a + l holding f_l^a(i dr).  The radial profiles of degree l have
    parity (-1)^l (f_l^a ~ r^l near the origin for a smooth F)."""

    def __init__(self, tables, dr: float):
        self.tables = [np.asarray(t, np.complex128) for t in tables]
        self.L = len(self.tables) - 1
        self.dr = float(dr)

    def radial(self, l, a, r):
        return hermite_eval(self.tables[l][a + l], self.dr, l, r)


def filter_eval(F: SHFilter, x, y, z):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    z = np.asarray(z, np.float64)
    r, th, ph = to_spherical(x, y, z)
    out = np.zeros(np.broadcast(x, y, z).shape, np.complex128)
    at0 = r == 0
    for l in range(F.L + 1):
        for a in range(-l, l + 1):
            term = F.radial(l, a, r) * sph_harm(l, a, th, ph)
            if l > 0:
                term = np.where(at0, 0.0, term)
            out += term
    return out


def rotated_filter_eval(F: SHFilter, Rm, dx, dy, dz):
    """(T_R F)(d) = F(R^-1 d) with the rotated coordinate formed explicitly."""
    Ri = np.asarray(Rm, np.float64).T
    x = Ri[0, 0] * dx + Ri[0, 1] * dy + Ri[0, 2] * dz
    y = Ri[1, 0] * dx + Ri[1, 1] * dy + Ri[1, 2] * dz
    z = Ri[2, 0] * dx + Ri[2, 1] * dy + Ri[2, 2] * dz
    return filter_eval(F, x, y, z)


# ------------------------------------------------------------- rotations ---

def quat_to_matrix(q):
    """Unit quaternion (w, x, y, z) -> rotation matrix."""
    w, x, y, z = (float(v) for v in q)
    n = math.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / n, x / n, y / n, z / n
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _sphere_quadrature(L):
    n_t = L + 2
    n_p = 2 * L + 3
    xs, ws = roots_legendre(n_t)
    th = np.arccos(xs)
    ph = 2 * math.pi * np.arange(n_p) / n_p
    T, Pp = np.meshgrid(th, ph, indexing="ij")
    W = np.repeat(ws[:, None], n_p, axis=1) * (2 * math.pi / n_p)
    return T.ravel(), Pp.ravel(), W.ravel()


def wigner_by_projection(l: int, Rm):
    """C^l(R) from its definition: C_ab = < Y_l^a(R^-1 x), Y_l^b(x) > on S^2,
    by a Gauss-Legendre x uniform quadrature exact for degree <= 2l."""
    th, ph, wq = _sphere_quadrature(2 * l + 1)
    x, y, z = np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)
    Ri = np.asarray(Rm, np.float64).T
    xr = Ri[0, 0] * x + Ri[0, 1] * y + Ri[0, 2] * z
    yr = Ri[1, 0] * x + Ri[1, 1] * y + Ri[1, 2] * z
    zr = Ri[2, 0] * x + Ri[2, 1] * y + Ri[2, 2] * z
    _, thr, phr = to_spherical(xr, yr, zr)
    C = np.zeros((2 * l + 1, 2 * l + 1), np.complex128)
    Yb = np.stack([sph_harm(l, b, th, ph) for b in range(-l, l + 1)])        # (2l+1, nq)
    for a in range(-l, l + 1):
        Ya_rot = sph_harm(l, a, thr, phr)
        C[a + l] = (Ya_rot[None, :] * np.conj(Yb) * wq[None, :]).sum(axis=1)
    return C


# ------------------------------------------------------------- operators ---

def box_offsets3(radius: int):
    dz, dy, dx = np.mgrid[-radius:radius + 1, -radius:radius + 1, -radius:radius + 1]
    return dx.ravel(), dy.ravel(), dz.ravel()


def corr_so3_at(V, F: SHFilter, radius: int, rotations, voxels):
    """S(p, R) for every p in `voxels` (rows (z, y, x)) and every rotation
    matrix in `rotations`; returns (n_vox, n_rot) complex."""
    V = np.asarray(V, np.float64)
    nz, ny, nx = V.shape
    dx, dy, dz = box_offsets3(radius)
    vox = np.asarray(voxels, np.int64).reshape(-1, 3)
    patches = V[(vox[:, 0:1] + dz[None]) % nz, (vox[:, 1:2] + dy[None]) % ny, (vox[:, 2:3] + dx[None]) % nx]
    bank = np.stack([rotated_filter_eval(F, Rm, dx.astype(np.float64), dy.astype(np.float64),
                                         dz.astype(np.float64)) for Rm in rotations])
    return patches @ np.conj(bank).T


def component_correlation(V, F: SHFilter, l: int, a: int, b: int, radius: int):
    """G_l^{ab}(p) = sum_d V(p + d) conj(f_l^a(|d|) Y_l^b(d^)) over the box."""
    V = np.asarray(V, np.float64)
    dx, dy, dz = box_offsets3(radius)
    r, th, ph = to_spherical(dx.astype(np.float64), dy.astype(np.float64), dz.astype(np.float64))
    phi_c = F.radial(l, a, r) * sph_harm(l, b, th, ph)
    if l > 0:
        phi_c = np.where(r == 0, 0.0, phi_c)
    out = np.zeros(V.shape, np.complex128)
    for n in range(dx.size):
        if phi_c[n] != 0:
            out += np.roll(V, (-dz[n], -dy[n], -dx[n]), axis=(0, 1, 2)) * np.conj(phi_c[n])
    return out


def sweep_from_components(G, Cs):
    """S = sum_{l,a,b} conj(C^l_ab) G_l^{ab}; G[l] has shape (2l+1, 2l+1, ...),
    Cs[l] the (2l+1, 2l+1) matrix of one rotation."""
    S = 0
    for l in range(len(G)):
        S = S + np.tensordot(np.conj(Cs[l]), G[l], axes=([0, 1], [0, 1]))
    return S


def component_correlation_at(V, F: SHFilter, l: int, a: int, b: int, radius: int, voxels):
    """G_l^{ab} at the given voxels (rows (z, y, x)), summed directly."""
    V = np.asarray(V, np.float64)
    nz, ny, nx = V.shape
    dx, dy, dz = box_offsets3(radius)
    r, th, ph = to_spherical(dx.astype(np.float64), dy.astype(np.float64), dz.astype(np.float64))
    phi_c = F.radial(l, a, r) * sph_harm(l, b, th, ph)
    if l > 0:
        phi_c = np.where(r == 0, 0.0, phi_c)
    vox = np.asarray(voxels, np.int64).reshape(-1, 3)
    patches = V[(vox[:, 0:1] + dz[None]) % nz, (vox[:, 1:2] + dy[None]) % ny, (vox[:, 2:3] + dx[None]) % nx]
    return patches @ np.conj(phi_c)


def channel_layout(L: int):
    """Unique (l, a, b) up to the pairing (a, b) <-> (-a, -b): per l the self
    pair (0, 0), then (0, b > 0), then (a > 0, b = -l..l); with their first
    real channel (self: 1 channel, others: Re and Im)."""
    out, ch = [], 0
    for l in range(L + 1):
        out.append((l, 0, 0, ch))
        ch += 1
        for a in range(0, l + 1):
            for b in range(-l, l + 1):
                if a == 0 and b <= 0:
                    continue
                out.append((l, a, b, ch))
                ch += 2
    return out, ch


# ------------------------------------------------------- proposal support ---

def full_components(chan, L: int):
    """Per-l (2l+1, 2l+1) complex G_l^{ab} at one voxel from its real channels."""
    lay, _ = channel_layout(L)
    G = [np.zeros((2 * l + 1, 2 * l + 1), np.complex128) for l in range(L + 1)]
    for (l, a, b, ch) in lay:
        if a == 0 and b == 0:
            G[l][l, l] = chan[ch]
        else:
            g = chan[ch] + 1j * chan[ch + 1]
            G[l][a + l, b + l] = g
            G[l][-a + l, -b + l] = (-1) ** (a + b) * np.conj(g)
    return G


def score_from_channels(chan, L: int, Rm):
    """S(p, R) = sum_{l,a,b} conj(C^l_ab(R)) G_l^{ab}(p) (real for a real filter)."""
    G = full_components(np.asarray(chan, np.float64), L)
    return float(sum(np.sum(np.conj(wigner_by_projection(l, Rm)) * G[l]) for l in range(L + 1)).real)


def upper_bound(chan, L: int):
    """sum_l sqrt(2l+1) |G_l|_F >= |S(p, R)| for every R (Cauchy-Schwarz with
    the unitary C^l, |C^l|_F = sqrt(2l+1))."""
    G = full_components(np.asarray(chan, np.float64), L)
    return float(sum(np.sqrt(2 * l + 1) * np.linalg.norm(G[l]) for l in range(L + 1)))


def nuclear_bound(chan, L: int):
    """sum_l |G_l|_* (nuclear norm, by numpy's SVD) >= |S(p, R)| for every R:
    Re tr(U^H G) <= |G|_* for every unitary U, C^l(R) among them.  Never
    above upper_bound (|G|_* <= sqrt(rank) |G|_F)."""
    G = full_components(np.asarray(chan, np.float64), L)
    return float(sum(np.linalg.svd(G[l], compute_uv=False).sum() for l in range(L + 1)))


def quat_mul(p, q):
    w1, x1, y1, z1 = p
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def quat_exp(v):
    """Unit quaternion of the rotation vector v (angle |v| about v/|v|)."""
    v = np.asarray(v, np.float64)
    t = np.linalg.norm(v)
    if t == 0:
        return np.array([1.0, 0.0, 0.0, 0.0])
    return np.concatenate([[np.cos(t / 2)], np.sin(t / 2) * v / t])


def rotation_generators(l: int):
    """A_i = d/dt C^l(exp(t e_i)) at t = 0 for i = x, y, z.  With
    (T_R F)(x) = F(R^-1 x), d/dt Y(exp(-t e_i) x) = -(e_i x x).grad Y = -i L_i Y
    (L = -i x x grad), so (A_i)_ab = -i <Y_l^b, L_i Y_l^a>, from the textbook
    relations L_z Y_l^m = m Y_l^m, L_+- Y_l^m = sqrt(l(l+1) - m(m+-1)) Y_l^{m+-1},
    L_x = (L_+ + L_-)/2, L_y = (L_+ - L_-)/(2i)."""
    d = 2 * l + 1
    Lp = np.zeros((d, d), np.complex128)       # <Y^b, L_+ Y^a> at [b, a]
    for a in range(-l, l):
        Lp[a + 1 + l, a + l] = math.sqrt(l * (l + 1) - a * (a + 1))
    Lm = Lp.conj().T
    Lz = np.diag(np.arange(-l, l + 1)).astype(np.complex128)
    Lx, Ly = (Lp + Lm) / 2, (Lp - Lm) / 2j
    return [(-1j * Li).T for Li in (Lx, Ly, Lz)]   # [a, b] = -i <Y^b, L_i Y^a>


def score_gradient(chan, L: int, Rm):
    """Body-frame gradient of the score: d/dxi_i S(R exp(xi e_i)) at 0 =
    Re sum_l tr((A_i C^l(R))^H G_l), since C(R exp(xi)) = C(exp(xi)) C(R)."""
    G = full_components(np.asarray(chan, np.float64), L)
    g = np.zeros(3)
    for l in range(L + 1):
        C = wigner_by_projection(l, Rm)
        for i, A in enumerate(rotation_generators(l)):
            g[i] += float(np.sum(np.conj(A @ C) * G[l]).real)
    return g


def refine(chan, L: int, q0, steps: int = 5, theta0: float = 0.25, tries: int = 6):
    """Gradient ascent on the exact score over SO(3), in the body frame: the
    gradient g from the rotation generators (score_gradient); each step moves
    q -> q exp(t g/|g|), t halved until the score increases (at most `tries`
    times, stopping if none does); an accepted step keeps t for the next one.
    Returns (quaternion, score)."""
    q = np.asarray(q0, np.float64) / np.linalg.norm(q0)
    s = score_from_channels(chan, L, quat_to_matrix(q))
    theta = theta0
    for _ in range(steps):
        g = score_gradient(chan, L, quat_to_matrix(q))
        gn = np.linalg.norm(g)
        if gn == 0:
            break
        u = g / gn
        moved = False
        t = theta
        for _ in range(tries):
            qn = quat_mul(q, quat_exp(t * u))
            sn = score_from_channels(chan, L, quat_to_matrix(qn))
            if sn > s:
                q, s, theta, moved = qn / np.linalg.norm(qn), sn, t, True
                break
            t *= 0.5
        if not moved:
            break
    return q, s


# ------------------------------------------- extended convolution (scatter) ---
# Eq. Def-EConv with a rotation at every INPUT voxel (Sec. 2.2; Sec. 9 for the
# SO(3) component form):
#     O(p) = sum_q V(q) (T_{R(q)} F)(p - q) = sum_{d in B} V(p - d) F(R(p - d)^-1 d),
# periodic mod the volume shape.  Expanding T_R F = sum_{l,a,b} f_l^a C^l_ab(R) Y_l^b
# gives the component form
#     O = sum_{l,a,b} (V C^l_ab(R(.))) (*) (f_l^a Y_l^b)      (standard convolution),
# i.e. the signal is modulated by each matrix entry of its own voxel's rotation
# and convolved with one fixed function per (l, a, b) (the SO(3) analogue of
# pre-multiplying H by e^{-ik Theta} in Sec. 4.1).

def quat_field_matrices(Q):
    """Rotation matrices (..., 3, 3) of a field of quaternions (..., 4) = (w, x, y, z)."""
    Q = np.asarray(Q, np.float64)
    n = np.linalg.norm(Q, axis=-1, keepdims=True)
    w, x, y, z = np.moveaxis(Q / n, -1, 0)
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def conv_so3_at(V, F: SHFilter, radius: int, Q, voxels):
    """O(p) at the given output voxels (rows (z, y, x)) by the brute-force sum
    over the box, each input voxel's filter rotated by its own rotation and
    evaluated at R^-1 d straight from the closed form.  Q: (nz, ny, nx, 4)."""
    V = np.asarray(V, np.float64)
    nz, ny, nx = V.shape
    dx, dy, dz = box_offsets3(radius)
    fx, fy, fz = dx.astype(np.float64), dy.astype(np.float64), dz.astype(np.float64)
    out = np.zeros(len(voxels), np.complex128)
    for i, (pz, py, px) in enumerate(np.asarray(voxels, np.int64).reshape(-1, 3)):
        qz, qy, qx = (pz - dz) % nz, (py - dy) % ny, (px - dx) % nx
        Rm = quat_field_matrices(np.asarray(Q)[qz, qy, qx])          # (n_d, 3, 3)
        # R^-1 d = R^T d
        x = Rm[:, 0, 0] * fx + Rm[:, 1, 0] * fy + Rm[:, 2, 0] * fz
        y = Rm[:, 0, 1] * fx + Rm[:, 1, 1] * fy + Rm[:, 2, 1] * fz
        z = Rm[:, 0, 2] * fx + Rm[:, 1, 2] * fy + Rm[:, 2, 2] * fz
        out[i] = np.sum(V[qz, qy, qx] * filter_eval(F, x, y, z))
    return out


def conv_so3(V, F: SHFilter, radius: int, Q):
    """O at every voxel by the brute force (small volumes only)."""
    nz, ny, nx = np.asarray(V).shape
    vox = np.stack(np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij"), -1).reshape(-1, 3)
    return conv_so3_at(V, F, radius, Q, vox).reshape(nz, ny, nx)


def conv_so3_from_components(V, F: SHFilter, radius: int, Q):
    """O by the component form: every voxel's C^l(R(q)) from its definition
    (wigner_by_projection), the modulated signals V C^l_ab, and a direct
    periodic convolution of each with f_l^a Y_l^b over the box."""
    V = np.asarray(V, np.float64)
    shape = V.shape
    Rms = quat_field_matrices(np.asarray(Q).reshape(-1, 4))
    dx, dy, dz = box_offsets3(radius)
    r, th, ph = to_spherical(dx.astype(np.float64), dy.astype(np.float64), dz.astype(np.float64))
    out = np.zeros(shape, np.complex128)
    for l in range(F.L + 1):
        Cs = np.stack([wigner_by_projection(l, Rm) for Rm in Rms])   # (P, 2l+1, 2l+1)
        for a in range(-l, l + 1):
            for b in range(-l, l + 1):
                g = F.radial(l, a, r) * sph_harm(l, b, th, ph)
                if l > 0:
                    g = np.where(r == 0, 0.0, g)
                U = V * Cs[:, a + l, b + l].reshape(shape)
                for n in range(dx.size):
                    if g[n] != 0:
                        out += np.roll(U, (dz[n], dy[n], dx[n]), axis=(0, 1, 2)) * g[n]
    return out
