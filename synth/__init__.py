"""Seeded synthetic inputs for the extended convolution/correlation workloads.

This module only draws data: images, transformation fields, filter
coefficients, template images and planted positions/angles.  It holds none of
the method's arithmetic (no filter decomposition, no steering, no transform of
a filter by a group element); both the CUDA path and the CPU oracle consume
what it returns, and each computes everything else on its own.

Seeds follow ``13188 * 10 + workload`` so that every workload is reproducible
from its number alone.  Workload numbering:

1. SO(2) extended convolution, 256 x 256, analytic filter with |k| <= 4.
2. SO(2) rotation-independent pattern matching, 2048 x 2048, 20 planted
   65 x 65 templates, |k| <= 16, 64 sweep angles.
3. Scale-adaptive smoothing, Voronoi image with block noise, scale field in
   [1, 8] px (see :func:`scale_smoothing_problem`).
4. Batched uneven SO(2) correlation (see :func:`batched_descriptors`).
5. SO(3) matching, 128^3 volume, 16 planted templates, L = 6.
6. Pattern detection (gradient signal and field, consensus filter).
7. Normalised orientation-adaptive smoothing (line integral convolution).
8. Depth-defocus blur with a Mellin disk filter.
9. SO(3) orientation-adaptive filtering, 128^3 volume, L = 6, smooth
   rotation field (see :func:`so3_conv_problem`).
10. Smoothing under joint rotation and scale fields, 2048^2 x 3 (see
    :func:`similarity_problem`).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import ndimage

SEED_BASE = 13188 * 10


def seed_for(workload: int) -> int:
    return SEED_BASE + int(workload)


# ---------------------------------------------------------------- helpers ---

def periodic_gaussian_blur(img: np.ndarray, sigma: float) -> np.ndarray:
    """Gaussian blur with wrap-around boundaries (input preparation only)."""
    return ndimage.gaussian_filter(np.asarray(img, np.float64), sigma, mode="wrap")


def smooth_random_template(rng: np.random.Generator, radius: int, blur: float,
                           taper: float = 4.0) -> np.ndarray:
    """(2R+1)^2 random smooth template: N(0,1) on a canvas padded by 4*blur,
    Gaussian blur, centre crop, then a raised-cosine taper to zero on
    r in [R - taper, R] (zero for r >= R)."""
    side = 2 * radius + 1
    pad = int(math.ceil(4 * blur))
    canvas = rng.standard_normal((side + 2 * pad, side + 2 * pad))
    canvas = ndimage.gaussian_filter(canvas, blur, mode="reflect")
    t = canvas[pad:pad + side, pad:pad + side].copy()
    yy, xx = np.mgrid[-radius:radius + 1, -radius:radius + 1]
    r = np.hypot(xx, yy)
    w = np.where(r <= radius - taper, 1.0,
                 np.where(r >= radius, 0.0,
                          0.5 * (1 + np.cos(np.pi * (r - (radius - taper)) / taper))))
    return t * w


def _place_centres(rng, h, w, n, min_sep, margin=0):
    """Seeded rejection sampling of n integer centres whose torus distance is
    at least ``min_sep``."""
    centres = []
    tries = 0
    while len(centres) < n:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place centres")
        cy = int(rng.integers(margin, h - margin)) if h > 2 * margin else int(rng.integers(0, h))
        cx = int(rng.integers(margin, w - margin)) if w > 2 * margin else int(rng.integers(0, w))
        ok = True
        for (py, px) in centres:
            dy = min(abs(cy - py), h - abs(cy - py))
            dx = min(abs(cx - px), w - abs(cx - px))
            if math.hypot(dx, dy) < min_sep:
                ok = False
                break
        if ok:
            centres.append((cy, cx))
    return np.array(centres, dtype=np.int64).reshape(-1, 2)


def plant_rotated(img: np.ndarray, template: np.ndarray, centre, beta: float) -> None:
    """Add a copy of ``template`` rotated by ``beta`` (radians, counter-clockwise
    in (x = column, y = row) coordinates) centred on ``centre`` = (row, col),
    wrapping periodically.  The copy at offset d is the template sampled at
    R(-beta) d with scipy's cubic spline; this is data generation, unrelated
    to the filter model either side builds from the template."""
    radius = template.shape[0] // 2
    h, w = img.shape
    dy, dx = np.mgrid[-radius:radius + 1, -radius:radius + 1].astype(np.float64)
    c, s = math.cos(beta), math.sin(beta)
    sx = c * dx + s * dy
    sy = -s * dx + c * dy
    vals = ndimage.map_coordinates(template, [sy + radius, sx + radius], order=3,
                                   mode="constant", cval=0.0)
    rows = (centre[0] + dy.astype(np.int64)) % h
    cols = (centre[1] + dx.astype(np.int64)) % w
    np.add.at(img, (rows, cols), vals)


# ------------------------------------------------------------- workload 1 ---

def so2_conv_problem(seed: int | None = None, size: int = 256, K: int = 4,
                     sigma: float = 6.0, radius: int = 15):
    """SO(2) extended convolution input.

    * H: size^2 uniform[0,1] noise, periodic Gaussian blur sigma = 2 px, float32.
    * a_k (k = -K..K, stored at index k+K): a_0 ~ N(0,1) real,
      a_k = (N + iN)/sqrt(2) for k >= 1, a_{-k} = conj(a_k) (real filter).
    * alpha: sum of 4 sinusoids sum_i A_i sin(2 pi (u_i x + v_i y)/size + phi_i),
      integer (u_i, v_i) in [-3,3]^2 minus the origin, A_i ~ U[0, pi],
      phi_i ~ U[0, 2 pi), reduced mod 2 pi, float32.
    """
    rng = np.random.default_rng(seed_for(1) if seed is None else seed)
    H = periodic_gaussian_blur(rng.uniform(0.0, 1.0, (size, size)), 2.0).astype(np.float32)
    a = np.zeros(2 * K + 1, np.complex128)
    a[K] = rng.standard_normal()
    for k in range(1, K + 1):
        a[K + k] = (rng.standard_normal() + 1j * rng.standard_normal()) / math.sqrt(2)
        a[K - k] = np.conj(a[K + k])
    alpha = _angle_field(rng, size, size)
    return dict(H=H, alpha=alpha, a=a, sigma=sigma, radius=radius, K=K)


def _angle_field(rng, h, w, n_terms=4):
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    field = np.zeros((h, w))
    for _ in range(n_terms):
        while True:
            u, v = rng.integers(-3, 4, size=2)
            if u != 0 or v != 0:
                break
        A = rng.uniform(0, math.pi)
        phi = rng.uniform(0, 2 * math.pi)
        field += A * np.sin(2 * math.pi * (u * xx / w + v * yy / h) + phi)
    return np.mod(field, 2 * math.pi).astype(np.float32)


def random_angle_field(seed: int, h: int, w: int) -> np.ndarray:
    """Low-frequency angle field in [0, 2 pi), float32 (same recipe as workload 1)."""
    return _angle_field(np.random.default_rng(seed), h, w)


def random_gauss_pow_coeffs(seed: int, K: int) -> np.ndarray:
    """Hermitian-symmetric a_k, k = -K..K at index k+K (real filter)."""
    rng = np.random.default_rng(seed)
    a = np.zeros(2 * K + 1, np.complex128)
    a[K] = rng.standard_normal()
    for k in range(1, K + 1):
        a[K + k] = (rng.standard_normal() + 1j * rng.standard_normal()) / math.sqrt(2)
        a[K - k] = np.conj(a[K + k])
    return a


# ------------------------------------------------------------- workload 2 ---

def so2_match_problem(seed: int | None = None, size: int | tuple = 2048, n_plant: int = 20,
                      radius: int = 32, K: int = 16, J: int = 64,
                      noise_sigma: float = 0.1, blur: float = 3.0):
    """Rotation-independent pattern matching input.

    * template: (2R+1)^2 smooth random template (N(0,1), blur sigma = 3 px,
      taper to zero on r in [R-4, R]), float64.
    * H: Gaussian noise sigma = 0.1 plus ``n_plant`` copies of the template
      rotated by beta ~ U[0, 2 pi) at centres at least 2R+1 apart, float32.
    * The filter is the template's angular band-limit |k| <= K, polar-sampled
      at dr = 0.25 px with 128 angles; J sweep angles alpha_j = 2 pi j / J.
    """
    rng = np.random.default_rng(seed_for(2) if seed is None else seed)
    h, w = (size, size) if np.isscalar(size) else size
    template = smooth_random_template(rng, radius, blur)
    H = rng.normal(0.0, noise_sigma, (h, w))
    centres = _place_centres(rng, h, w, n_plant, 2 * radius + 1)
    betas = rng.uniform(0.0, 2 * math.pi, n_plant)
    for c, b in zip(centres, betas):
        plant_rotated(H, template, c, b)
    return dict(H=H.astype(np.float32), template=template, centres=centres, betas=betas,
                radius=radius, K=K, J=J, dr=0.25, n_theta=128)


# ------------------------------------------------- pattern detection (GHT) ---

def ght_problem(seed: int | None = None, size: int | tuple = 2048, n_plant: int = 12, radius: int = 24,
                noise_sigma: float = 0.05, blur: float = 3.0):
    """Pattern-detection input for the generalised Hough transform of Sec. 5:
    a smooth random pattern ((2R+1)^2, as smooth_random_template, scaled to
    peak |value| 1) and an image of Gaussian noise (sigma 0.05, periodic blur
    sigma 1) plus ``n_plant`` copies of the pattern rotated by
    beta ~ U[0, 2 pi) at centres at least 2R+1 apart, float32."""
    rng = np.random.default_rng(seed_for(6) if seed is None else seed)
    h, w = (size, size) if np.isscalar(size) else size
    pattern = smooth_random_template(rng, radius, blur)
    pattern /= np.abs(pattern).max()
    I = periodic_gaussian_blur(rng.normal(0.0, noise_sigma, (h, w)), 1.0)
    centres = _place_centres(rng, h, w, n_plant, 2 * radius + 1)
    betas = rng.uniform(0.0, 2 * math.pi, n_plant)
    for c, b in zip(centres, betas):
        plant_rotated(I, pattern, c, b)
    return dict(I=I.astype(np.float32), pattern=pattern, centres=centres, betas=betas, radius=radius)


# ------------------------------------------------------------- workload 4 ---

def batched_descriptors(seed: int | None = None, n_images: int = 512,
                        sides=tuple(range(128, 1025, 64)),
                        template_sizes=tuple(range(33, 98, 2)),
                        Ks=(4, 8, 16), Js=tuple(range(32, 129, 4))):
    """Per-image (h, w, template side, K, J, image seed) for the batched
    uneven workload; images are drawn lazily with :func:`batched_image`."""
    rng = np.random.default_rng(seed_for(4) if seed is None else seed)
    out = []
    for i in range(n_images):
        h = int(rng.choice(sides))
        w = int(rng.choice(sides))
        ts = int(rng.choice(template_sizes))
        K = int(rng.choice(Ks))
        J = int(rng.choice(Js))
        out.append(dict(h=h, w=w, side=ts, radius=(ts - 1) // 2, K=K, J=J,
                        seed=int(rng.integers(0, 2**31 - 1))))
    return out


def batched_image(desc: dict, noise_sigma: float = 0.1, blur: float = 3.0):
    """One image of the batched workload: noise + one planted template."""
    rng = np.random.default_rng(desc["seed"])
    R = desc["radius"]
    template = smooth_random_template(rng, R, blur)
    H = rng.normal(0.0, noise_sigma, (desc["h"], desc["w"]))
    centre = (int(rng.integers(0, desc["h"])), int(rng.integers(0, desc["w"])))
    beta = float(rng.uniform(0, 2 * math.pi))
    plant_rotated(H, template, centre, beta)
    return dict(H=H.astype(np.float32), template=template, centres=np.array([centre]),
                betas=np.array([beta]), radius=R, K=desc["K"], J=desc["J"], dr=0.25,
                n_theta=128)


# ------------------------------------------------------------- workload 3 ---

def _mellin_fit(target, n_h, log_period, u_lo, u_hi, ridge, n_fit):
    """Least-squares coefficients c_k, k = 0..n_h-1 (c_{-k} = conj(c_k)), of
    P(u) = sum_k c_k exp(i w_k u), w_k = 2 pi k / log_period, fitted (ridge
    ``ridge``) to target(u) on u in [u_lo, u_hi].  Returns complex128 (n_h,)."""
    u = np.linspace(u_lo, u_hi, n_fit)
    w = 2 * math.pi * np.arange(n_h) / log_period
    cols = [np.ones_like(u)]
    for k in range(1, n_h):
        cols += [np.cos(w[k] * u), np.sin(w[k] * u)]
    A = np.stack(cols, axis=1)
    coef = np.linalg.solve(A.T @ A + ridge * np.eye(A.shape[1]), A.T @ target(u))
    c = np.zeros(n_h, np.complex128)
    c[0] = coef[0]
    for k in range(1, n_h):
        # 2 Re(c_k e^{iwu}) = 2 Re(c_k) cos - 2 Im(c_k) sin
        c[k] = 0.5 * (coef[2 * k - 1] - 1j * coef[2 * k])
    return c


def mellin_gaussian_coeffs(n_h: int = 24, log_period: float = 8.0,
                           u_lo: float = -math.log(8.0), u_hi: float = math.log(64.0),
                           ridge: float = 1e-10, n_fit: int = 4001):
    """Filter design for scale-adaptive smoothing: coefficients c_k,
    k = 0..n_h-1 (c_{-k} = conj(c_k)), of P(u) = sum_k c_k exp(i w_k u),
    w_k = 2 pi k / log_period, least-squares fitted (ridge ``ridge``) to the
    unit Gaussian profile exp(-e^{2u}/2) on u in [u_lo, u_hi].  With
    u = ln r - ln s this gives exp(-r^2 / (2 s^2)).  Returns complex128 (n_h,)."""
    return _mellin_fit(lambda u: np.exp(-np.exp(2 * u) / 2), n_h, log_period, u_lo, u_hi, ridge, n_fit)


def mellin_disk_coeffs(n_h: int = 64, log_period: float = 8.0, tau: float = 0.1,
                       u_lo: float = -math.log(8.0), u_hi: float = math.log(64.0),
                       ridge: float = 1e-10, n_fit: int = 4001):
    """The depth-defocus filter of Sec. 8: the indicator of the disk of radius
    s, smoothed along the radial direction, as P(u) = 1 / (1 + e^{u / tau})
    (u = ln r - ln s, so P ~ 1 inside the disk, 0 outside, a logistic edge
    of width tau in log-radius), fitted with n_h = 64 Mellin frequencies."""
    return _mellin_fit(lambda u: 1.0 / (1.0 + np.exp(u / tau)), n_h, log_period, u_lo, u_hi, ridge, n_fit)


def voronoi_image(rng, h, w, n_cells=500, block=8, noise=0.05):
    """Piecewise-constant colour image (3, h, w): torus Voronoi cells with
    U[0,1]^3 colours plus a per-block, per-channel offset U[-noise, noise]."""
    from scipy.spatial import cKDTree
    seeds = rng.uniform(0, 1, (n_cells, 2)) * np.array([h, w])
    colours = rng.uniform(0, 1, (n_cells, 3))
    tree = cKDTree(seeds, boxsize=[h, w])
    img = np.empty((3, h, w), np.float32)
    rows_per = max(1, (1 << 22) // w)
    xs = np.arange(w) + 0.5
    for y0 in range(0, h, rows_per):
        y1 = min(h, y0 + rows_per)
        yy, xx = np.meshgrid(np.arange(y0, y1) + 0.5, xs, indexing="ij")
        _, lab = tree.query(np.stack([yy.ravel(), xx.ravel()], 1), k=1)
        img[:, y0:y1, :] = colours[lab].T.reshape(3, y1 - y0, w)
    bh, bw = -(-h // block), -(-w // block)
    offs = rng.uniform(-noise, noise, (3, bh, bw))
    img += np.repeat(np.repeat(offs, block, axis=1), block, axis=2)[:, :h, :w]
    return img


def scale_field_from_image(img, s_min=1.0, s_max=8.0, blur=4.0):
    """s = s_max - (s_max - s_min) * clip(m / p99(m), 0, 1), m = Gaussian
    blur (sigma 4, wrap) of the central-difference gradient magnitude of the
    channel mean.  Small scale at strong edges, large in flat regions."""
    g = np.asarray(img, np.float64).mean(axis=0)
    gx = 0.5 * (np.roll(g, -1, 1) - np.roll(g, 1, 1))
    gy = 0.5 * (np.roll(g, -1, 0) - np.roll(g, 1, 0))
    m = ndimage.gaussian_filter(np.hypot(gx, gy), blur, mode="wrap")
    p99 = np.percentile(m, 99)
    t = np.clip(m / p99, 0, 1) if p99 > 0 else np.zeros_like(m)
    return (s_max - (s_max - s_min) * t).astype(np.float32)


def scale_smoothing_problem(seed: int | None = None, size: int | tuple = 4096,
                            n_cells: int = 500, n_h: int = 24, log_period: float = 8.0,
                            r_min: float = 1.0, r_max: float = 64.0, centre_tap: float = 1.0):
    """Scale-adaptive smoothing input: image (3, h, w) float32, scale field
    s (h, w) float32 in [1, 8], Mellin coefficients of the Gaussian family."""
    rng = np.random.default_rng(seed_for(3) if seed is None else seed)
    h, w = (size, size) if np.isscalar(size) else size
    img = voronoi_image(rng, h, w, n_cells)
    s = scale_field_from_image(img)
    c = mellin_gaussian_coeffs(n_h, log_period)
    return dict(img=img, s=s, c=c, log_period=log_period, r_min=r_min, r_max=r_max,
                centre_tap=centre_tap)


# ------------------------------------------------------------ workload 10 ---

def similarity_brush_coeffs(K: int = 4, n_h: int = 8, kappa: float = 1.5, sigma: float = 2.0,
                            log_period: float = 6.0, u_lo: float = -math.log(3.0), u_hi: float = math.log(16.0),
                            ridge: float = 1e-10, n_fit: int = 4001):
    """Filter design for smoothing under rotation and scale fields: an oriented
    brush F(r, phi) = A(phi) B(ln r), separable in log-polar coordinates, with
    A(phi) = exp(kappa (cos phi - 1)) (a comet-shaped stroke pointing along
    phi = 0) band-limited to |k| <= K by its Fourier coefficients a_k (from
    512 equispaced samples), and B(u) = exp(-e^{2u} / (2 sigma^2)) (a Gaussian
    in r) fitted with n_h Mellin harmonics on [u_lo, u_hi].  Returns
    c[k, j + n_h - 1] = a_k b_j, k = 0..K, |j| < n_h (complex128)."""
    phi = 2 * math.pi * np.arange(512) / 512
    a = np.fft.fft(np.exp(kappa * (np.cos(phi) - 1.0))) / 512
    b = _mellin_fit(lambda u: np.exp(-np.exp(2 * u) / (2 * sigma * sigma)), n_h, log_period, u_lo, u_hi,
                    ridge, n_fit)
    bj = np.concatenate([np.conj(b[:0:-1]), b])        # j = -(n_h-1) .. n_h-1
    return np.outer(a[:K + 1], bj)


def similarity_problem(seed: int | None = None, size: int | tuple = 2048, K: int = 4, n_h: int = 8,
                       s_min: float = 1.0, s_max: float = 3.0, log_period: float = 6.0, r_min: float = 1.0,
                       r_max: float = 16.0, centre_tap: float = 1.0):
    """Smoothing under joint rotation and scale fields: a 3-channel torus
    Voronoi image (300 cells, as workload 3), the low-frequency angle field of
    workload 1, a smooth scale field (periodic blur sigma 48 of N(0,1) noise,
    rescaled to [s_min, s_max]) and the brush of similarity_brush_coeffs."""
    rng = np.random.default_rng(seed_for(10) if seed is None else seed)
    h, w = (size, size) if np.isscalar(size) else size
    img = voronoi_image(rng, h, w, 300)
    alpha = random_angle_field(int(rng.integers(0, 2**31 - 1)), h, w).astype(np.float32)
    z = periodic_gaussian_blur(rng.standard_normal((h, w)), 48.0)
    z = (z - z.min()) / max(z.max() - z.min(), 1e-12)
    s = (s_min + (s_max - s_min) * z).astype(np.float32)
    c = similarity_brush_coeffs(K, n_h, log_period=log_period)
    return dict(img=img, alpha=alpha, s=s, c=c, log_period=log_period, r_min=r_min, r_max=r_max,
                centre_tap=centre_tap)


# ------------------------------------------------------------- workload 8 ---

def depth_defocus_problem(seed: int | None = None, size: int | tuple = 2048, n_lines: int = 600,
                          s_min: float = 1.0, s_max: float = 8.0):
    """Depth-defocus input (Sec. 8, the wire-frame example): a 3-channel image
    of one-pixel-wide random line segments (random colours) on a dark
    background, a smooth depth field Z in [0, 1] (periodic blur sigma 64 of
    Gaussian noise, rescaled) and the scale field
    s = s_min + (s_max - s_min) |Z - Z(p0)| / max |Z - Z(p0)|, p0 the image
    centre (the focal point).  float32 arrays (3, h, w) and (h, w)."""
    rng = np.random.default_rng(seed_for(8) if seed is None else seed)
    h, w = (size, size) if np.isscalar(size) else size
    img = np.full((3, h, w), 0.05)
    for _ in range(n_lines):
        y0, x0 = rng.uniform(0, h), rng.uniform(0, w)
        ang, length = rng.uniform(0, math.pi), rng.uniform(20, 200)
        col = rng.uniform(0.3, 1.0, 3)
        t = np.linspace(0.0, length, int(4 * length) + 1)
        ys = np.round(y0 + t * math.sin(ang)).astype(np.int64) % h
        xs = np.round(x0 + t * math.cos(ang)).astype(np.int64) % w
        for c in range(3):
            img[c, ys, xs] = col[c]
    Z = periodic_gaussian_blur(rng.standard_normal((h, w)), 64.0)
    Z = (Z - Z.min()) / (Z.max() - Z.min())
    dz = np.abs(Z - Z[h // 2, w // 2])
    s = s_min + (s_max - s_min) * dz / dz.max()
    return dict(img=img.astype(np.float32), s=s.astype(np.float32), Z=Z)


def so3_filter_tables(seed: int, L: int = 6, r_max: float = 8.0, dr: float = 0.125):
    """Random smooth radial profiles f_l^a(r), l <= L, |a| <= l, sampled at
    i*dr <= r_max: three Gaussian bumps (centres U[1.5, 6], width 0.8) with
    complex N(0,1) weights, times r^l exp(-r^2/32) near the origin and a
    raised-cosine taper to zero on [r_max - 1.5, r_max].  Real-function
    symmetry f_l^{-a} = (-1)^a conj(f_l^a).  Returns a list over l of
    (2l+1, n_r) complex arrays."""
    rng = np.random.default_rng(seed)
    n_r = int(round(r_max / dr)) + 1
    r = np.arange(n_r) * dr
    taper = np.where(r <= r_max - 1.5, 1.0,
                     0.5 * (1 + np.cos(np.pi * np.clip(r - (r_max - 1.5), 0, 1.5) / 1.5)))
    taper[r >= r_max] = 0.0
    tables = []
    for l in range(L + 1):
        t = np.zeros((2 * l + 1, n_r), np.complex128)
        g = (r ** l) * np.exp(-r * r / 32.0) * taper
        g /= max(np.max(np.abs(g)), 1e-12)
        for a in range(0, l + 1):
            prof = np.zeros(n_r, np.complex128)
            for _ in range(3):
                mu = rng.uniform(1.5, 6.0)
                wgt = rng.standard_normal() + 1j * rng.standard_normal()
                prof += wgt * np.exp(-(r - mu) ** 2 / (2 * 0.8 ** 2))
            prof *= g
            if a == 0:
                prof = prof.real.astype(np.complex128)
            t[a + l] = prof
            t[-a + l] = ((-1) ** a) * np.conj(prof)
        tables.append(t)
    return tables


def haar_quaternion(rng):
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


def _quat_matrix(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _quat_from_zyz(alpha, beta, gamma):
    # q = q_z(alpha) q_y(beta) q_z(gamma)
    def qz(t):
        return np.array([math.cos(t / 2), 0.0, 0.0, math.sin(t / 2)])

    def qy(t):
        return np.array([math.cos(t / 2), 0.0, math.sin(t / 2), 0.0])

    def mul(p, q):
        w1, x1, y1, z1 = p
        w2, x2, y2, z2 = q
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    return mul(mul(qz(alpha), qy(beta)), qz(gamma))


def so3_rotation_grid(n_dirs: int = 192, n_psi: int = 24):
    """n_dirs * n_psi rotations R = R_z(phi) R_y(theta) R_z(psi): (theta, phi)
    on a Fibonacci sphere of n_dirs near-uniform directions (the base of a
    Hopf-fibration grid), psi = 2 pi j / n_psi.  Quaternions (w, x, y, z),
    shape (n_dirs * n_psi, 4)."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for i in range(n_dirs):
        zc = 1.0 - (2.0 * i + 1.0) / n_dirs
        theta = math.acos(zc)
        phi = (golden * i) % (2 * math.pi)
        for j in range(n_psi):
            out.append(_quat_from_zyz(phi, theta, 2 * math.pi * j / n_psi))
    return np.array(out)


def so3_rotation_grid_factors(n_dirs: int = 192, n_psi: int = 24):
    """The factors of so3_rotation_grid: the n_dirs direction rotations
    R_z(phi) R_y(theta) as quaternions [n_dirs][4] and n_psi, so that rotation
    d * n_psi + j of the grid is R_dir(d) R_z(2 pi j / n_psi)."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for i in range(n_dirs):
        zc = 1.0 - (2.0 * i + 1.0) / n_dirs
        out.append(_quat_from_zyz((golden * i) % (2 * math.pi), math.acos(zc), 0.0))
    return np.array(out), n_psi


def _sample_template(tables, dr, radius, Rm=None):
    """Samples sum_{l,a} f_l^a(|x|) Y_l^a(x^) at x = R^-1 d on the (2R+1)^3 box
    (data generation for planting; linear interpolation of the radial
    profiles, scipy's associated Legendre functions)."""
    from scipy.special import lpmv
    dz, dy, dx = np.mgrid[-radius:radius + 1, -radius:radius + 1, -radius:radius + 1].astype(np.float64)
    pts = np.stack([dx.ravel(), dy.ravel(), dz.ravel()])
    if Rm is not None:
        pts = Rm.T @ pts
    x, y, z = pts
    r = np.sqrt(x * x + y * y + z * z)
    ct = np.where(r > 0, z / np.where(r > 0, r, 1), 1.0)
    ph = np.arctan2(y, x)
    n_r = tables[0].shape[1]
    rr = np.arange(n_r) * dr
    out = np.zeros(r.shape, np.complex128)
    for l, t in enumerate(tables):
        for a in range(-l, l + 1):
            am = abs(a)
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            yv = norm * lpmv(am, l, np.clip(ct, -1, 1)) * np.exp(1j * am * ph)
            if a < 0:
                yv = ((-1) ** am) * np.conj(yv)
            prof = np.interp(r, rr, t[a + l].real, right=0.0) + 1j * np.interp(r, rr, t[a + l].imag, right=0.0)
            out += prof * yv
    return out.real.reshape(2 * radius + 1, 2 * radius + 1, 2 * radius + 1)


def so3_match_problem(seed: int | None = None, size: int = 128, n_plant: int = 16, L: int = 6,
                      radius: int = 8, dr: float = 0.125, noise_sigma: float = 0.1, tables=None):
    """3D matching input: Gaussian noise sigma 0.1 plus n_plant copies of the
    band-limited template (profiles from so3_filter_tables, or the given
    `tables`) rotated by Haar-random rotations at centres >= 2R+1 apart
    (torus distance).  Volume float32 (z, y, x)."""
    rng = np.random.default_rng(seed_for(5) if seed is None else seed)
    filter_seed = int(rng.integers(0, 2**31 - 1))
    if tables is None:
        tables = so3_filter_tables(filter_seed, L, float(radius), dr)
    V = rng.normal(0.0, noise_sigma, (size, size, size))
    centres = []
    while len(centres) < n_plant:
        c = rng.integers(0, size, 3)
        if all(np.linalg.norm(np.minimum(np.abs(c - p), size - np.abs(c - p))) >= 2 * radius + 1 for p in centres):
            centres.append(c)
    quats = np.array([haar_quaternion(rng) for _ in range(n_plant)])
    d = np.arange(-radius, radius + 1)
    for c, q in zip(centres, quats):
        block = _sample_template(tables, dr, radius, _quat_matrix(q))
        zi = (c[0] + d) % size
        yi = (c[1] + d) % size
        xi = (c[2] + d) % size
        V[np.ix_(zi, yi, xi)] += block
    return dict(V=V.astype(np.float32), tables=tables, dr=dr, radius=radius, L=L,
                centres=np.array(centres), quats=quats)


def so3_training_volumes(seed: int, tables, n_volumes: int = 64, size: int = 64, n_plant: int = 6):
    """The proposal network's training data source: n_volumes planted volumes
    (so3_match_problem with seeds seed, seed + 1, ...) sharing one filter,
    generated one at a time."""
    for i in range(n_volumes):
        yield so3_match_problem(seed=seed + i, size=size, n_plant=n_plant, L=len(tables) - 1, tables=tables)


def aniso_gauss_template(sigma_u: float, sigma_v: float, radius: int):
    """The anisotropic Gaussian exp(-x^2 / 2 sigma_u^2 - y^2 / 2 sigma_v^2)
    sampled on the (2R+1)^2 box (x = column offset, y = row offset): the
    oriented brush of line integral convolution, as a template image."""
    d = np.arange(-radius, radius + 1, dtype=np.float64)
    y, x = np.meshgrid(d, d, indexing="ij")
    return np.exp(-x * x / (2 * sigma_u ** 2) - y * y / (2 * sigma_v ** 2))


def so3_rotation_field(seed: int, shape, sigma: float = 4.0):
    """Smooth field of unit quaternions (w, x, y, z), float32 (*shape, 4): four
    i.i.d. N(0,1) volumes, each Gaussian-blurred (sigma voxels, periodic) and
    rescaled to unit variance, then normalised per voxel."""
    rng = np.random.default_rng(seed)
    comps = []
    for _ in range(4):
        c = ndimage.gaussian_filter(rng.standard_normal(shape), sigma, mode="wrap")
        comps.append(c / c.std())
    q = np.stack(comps, axis=-1)
    q /= np.linalg.norm(q, axis=-1, keepdims=True)
    return q.astype(np.float32)


def so3_conv_problem(seed: int | None = None, shape=(128, 128, 128), L: int = 6, radius: int = 8,
                     dr: float = 0.125, field_sigma: float = 4.0):
    """Orientation-adaptive 3D filtering input: a volume of Gaussian-blurred
    (sigma 1.5, periodic) N(0,1) noise, the band-limited random filter of
    so3_filter_tables (degree L, support radius `radius`) and a smooth rotation
    field (so3_rotation_field).  Volume float32 (z, y, x)."""
    rng = np.random.default_rng(seed_for(9) if seed is None else seed)
    tables = so3_filter_tables(int(rng.integers(0, 2**31 - 1)), L, float(radius), dr)
    V = ndimage.gaussian_filter(rng.standard_normal(shape), 1.5, mode="wrap")
    V = (V / V.std()).astype(np.float32)
    Q = so3_rotation_field(int(rng.integers(0, 2**31 - 1)), shape, field_sigma)
    return dict(V=V, Q=Q, tables=tables, dr=dr, radius=radius, L=L)


def mlp_init(seed: int, n_in: int, hidden: int = 256):
    """Initial weights of the proposal network (He-normal, zero biases; the
    output layer scaled by 0.5), FP32, shapes W1 [hidden][n_in], b1 [hidden],
    W2 [hidden][hidden], b2 [hidden], W3 [4][hidden], b3 [4]."""
    rng = np.random.default_rng(seed)

    def he(o, i):
        return (rng.standard_normal((o, i)) * np.sqrt(2.0 / i)).astype(np.float32)
    return dict(W1=he(hidden, n_in), b1=np.zeros(hidden, np.float32), W2=he(hidden, hidden),
                b2=np.zeros(hidden, np.float32), W3=(he(4, hidden) * 0.5).astype(np.float32),
                b3=np.zeros(4, np.float32))


def training_draws(seed: int, n_train: int, steps: int, batch: int):
    """Minibatch row indices (int32 [steps*batch]) and Haar-random
    augmentation rotations (float32 [steps*batch][4]) for training the
    proposal network."""
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, n_train, steps * batch).astype(np.int32)
    q = rng.standard_normal((steps * batch, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return rows, q.astype(np.float32)
