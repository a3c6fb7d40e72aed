"""Seeded synthetic images and initial label images for the segmentation workloads.

This module holds input generation only: no part of the segmentation method's
arithmetic lives here, so both the CUDA path and the CPU oracle can be fed from it.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the i-th
draw of a stream is the SplitMix64 output function applied to base + i * golden.
Gaussians use the Box-Muller transform; Poisson variates use CDF inversion for
small means and Hoermann's PTRS transformed-rejection method ("The transformed
rejection method for generating Poisson random variables", 1993) for means >= 10.

Workloads (the paper's own images are not available, so these stand in for them):

* ``disks``      - 2D float32 piecewise-constant scene: background 0, disks of
                   intensity 1, additive Gaussian noise (sigma 0.3); initial label is
                   one centred square.  ``disks(128, 128, seed=0)`` is the 128x128
                   two-disk case (radii 20 and 30, centres (40,40) and (84,84)).
* ``ellipses``   - 2D float32 piecewise-smooth scene: random ellipses (semi-axes
                   10-60 px) with amplitude U[0.5,1.5] times a linear bias field
                   0.5 + x/(W-1), Poisson noise at 20 photons per unit; initial labels
                   are 32x32 squares on a 64 px pitch.
* ``deconv_scene`` - 2D float32 scene for the deconvolving model (Eq. 8): four objects
                   over a faint background, blurred by a Gaussian PSF (sigma 15 px, as in
                   Figure 3), Poisson noise; the PSF profile travels with the workload.
* ``ellipsoids`` - 3D uint16 scene: random ellipsoids (semi-axes 4-20 vox) at 300
                   over background 100, Gaussian blur sigma 1.5 (radius 6, clamped
                   edges), Poisson noise; initial labels are 16^3 cubes on a 32 pitch.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """A counter-based SplitMix64 stream identified by (seed, stream id)."""

    def __init__(self, seed: int, stream: int = 0):
        s = np.array([(seed * 0x100000001B3 + stream * 0xC2B2AE3D27D4EB4F) & (2**64 - 1)],
                     dtype=np.uint64)
        self.base = splitmix64_mix(s)[0]
        self.ctr = 0

    def u64(self, n: int) -> np.ndarray:
        i = np.arange(self.ctr + 1, self.ctr + 1 + n, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return splitmix64_mix(self.base + i * _GOLDEN)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform_range(self, lo: float, hi: float, n: int) -> np.ndarray:
        return lo + (hi - lo) * self.uniform(n)

    def integers(self, lo: int, hi_incl: int, n: int) -> np.ndarray:
        span = hi_incl - lo + 1
        return lo + np.minimum((self.uniform(n) * span).astype(np.int64), span - 1)

    def normal(self, n: int) -> np.ndarray:
        """Box-Muller: one normal per pair of uniforms (cosine branch)."""
        u1 = 1.0 - self.uniform(n)          # (0, 1]
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)

    def poisson(self, mean: np.ndarray) -> np.ndarray:
        mean = np.asarray(mean, dtype=np.float64)
        out = np.zeros(mean.shape, dtype=np.int64)
        flat_m = mean.reshape(-1)
        flat_o = out.reshape(-1)
        small = np.nonzero((flat_m > 0) & (flat_m < 10.0))[0]
        large = np.nonzero(flat_m >= 10.0)[0]
        if small.size:
            flat_o[small] = self._poisson_inversion(flat_m[small])
        if large.size:
            flat_o[large] = self._poisson_ptrs(flat_m[large])
        return out

    def _poisson_inversion(self, lam: np.ndarray) -> np.ndarray:
        u = self.uniform(lam.size)
        k = np.zeros(lam.size, dtype=np.int64)
        p = np.exp(-lam)
        cdf = p.copy()
        active = u > cdf
        kk = 0
        while active.any() and kk < 1000:
            kk += 1
            idx = np.nonzero(active)[0]
            p[idx] *= lam[idx] / kk
            cdf[idx] += p[idx]
            k[idx] = kk
            active[idx] = u[idx] > cdf[idx]
        return k

    def _poisson_ptrs(self, lam: np.ndarray) -> np.ndarray:
        from scipy.special import gammaln
        slam = np.sqrt(lam)
        loglam = np.log(lam)
        b = 0.931 + 2.53 * slam
        a = -0.059 + 0.02483 * b
        inv_alpha = 1.1239 + 1.1328 / (b - 3.4)
        v_r = 0.9277 - 3.6224 / (b - 2.0)
        out = np.zeros(lam.size, dtype=np.int64)
        todo = np.arange(lam.size)
        rounds = 0
        while todo.size and rounds < 200:
            rounds += 1
            uu = self.uniform(todo.size) - 0.5
            vv = self.uniform(todo.size)
            us = 0.5 - np.abs(uu)
            aa, bb, lm = a[todo], b[todo], lam[todo]
            k = np.floor((2.0 * aa / us + bb) * uu + lm + 0.43)
            quick = (us >= 0.07) & (vv <= v_r[todo])
            bad = (k < 0) | ((us < 0.013) & (vv > us))
            with np.errstate(divide="ignore", invalid="ignore"):
                lhs = np.log(vv) + np.log(inv_alpha[todo]) - np.log(aa / (us * us) + bb)
                rhs = -lm + k * loglam[todo] - gammaln(k + 1.0)
            ok = quick | (~bad & (lhs <= rhs))
            out[todo[ok]] = k[ok].astype(np.int64)
            todo = todo[~ok]
        return out


@dataclass
class Workload:
    """One segmentation job: image, initial labels and the method's parameters."""
    name: str
    image: np.ndarray            # float32 (2D) or uint16 (3D); shape (H, W) or (D, H, W)
    labels0: np.ndarray          # int32, same shape; 0 = background
    model: str                   # "pc" | "ps" | "psp" | "pcd"
    connectivity: int            # 4 (2D) | 6 (3D)
    lam: float                   # length weight lambda (Eq. 10)
    cutoff: float                # interaction cutoff E/2 in pixels
    ps_radius: float = 0.0       # local-mean radius (piecewise-smooth model)
    iterations: int = 50
    extra: dict = field(default_factory=dict)
    psf: np.ndarray | None = None  # deconvolving model: 1D PSF profile, 2r+1 taps (float64)

    @property
    def ndim(self) -> int:
        return self.image.ndim


def centred_square_labels(H: int, W: int, side_h: int, side_w: int, label: int = 1) -> np.ndarray:
    L = np.zeros((H, W), dtype=np.int32)
    y0 = (H - side_h) // 2
    x0 = (W - side_w) // 2
    L[y0:y0 + side_h, x0:x0 + side_w] = label
    return L


def square_grid_labels(H: int, W: int, pitch: int = 64, side: int = 32) -> np.ndarray:
    L = np.zeros((H, W), dtype=np.int32)
    lab = 1
    off = (pitch - side) // 2
    for ty in range(H // pitch):
        for tx in range(W // pitch):
            L[ty * pitch + off: ty * pitch + off + side, tx * pitch + off: tx * pitch + off + side] = lab
            lab += 1
    if lab == 1:   # image smaller than one pitch: one centred square of half the side
        L = centred_square_labels(H, W, max(1, H // 2), max(1, W // 2))
    return L


def cube_grid_labels(D: int, H: int, W: int, pitch: int = 32, side: int = 16) -> np.ndarray:
    L = np.zeros((D, H, W), dtype=np.int32)
    lab = 1
    off = (pitch - side) // 2
    for tz in range(D // pitch):
        for ty in range(H // pitch):
            for tx in range(W // pitch):
                L[tz * pitch + off: tz * pitch + off + side,
                  ty * pitch + off: ty * pitch + off + side,
                  tx * pitch + off: tx * pitch + off + side] = lab
                lab += 1
    if lab == 1:
        s = max(1, min(D, H, W) // 2)
        L[(D - s) // 2:(D - s) // 2 + s, (H - s) // 2:(H - s) // 2 + s, (W - s) // 2:(W - s) // 2 + s] = 1
    return L


def disks(H: int = 128, W: int = 128, seed: int = 0, n_disks: int | None = None,
          sigma: float = 0.3, lam: float = 0.04, cutoff: float = 3.0, iterations: int = 50) -> Workload:
    """Piecewise-constant 2D disk scene with Gaussian noise and a centred-square start.

    With the defaults (128x128, seed 0) the scene is the fixed two-disk layout.  Other
    sizes draw ``n_disks`` (default U{1..8}) disks of radius U[0.08, 0.25] * min(H, W).
    """
    rs = Stream(seed, 1)
    yy, xx = np.mgrid[0:H, 0:W]
    clean = np.zeros((H, W), dtype=np.float64)
    if (H, W) == (128, 128) and n_disks is None:
        circles = [(40.0, 40.0, 20.0), (84.0, 84.0, 30.0)]
    else:
        k = int(rs.integers(1, 8, 1)[0]) if n_disks is None else n_disks
        r = rs.uniform_range(0.08, 0.25, k) * min(H, W)
        cy = rs.uniform_range(0, H, k)
        cx = rs.uniform_range(0, W, k)
        circles = list(zip(cy, cx, r))
    for cy, cx, r in circles:
        clean[(yy - cy) ** 2 + (xx - cx) ** 2 <= r * r] = 1.0
    noise = rs.normal(H * W).reshape(H, W) * sigma
    image = (clean + noise).astype(np.float32)
    labels0 = centred_square_labels(H, W, H // 2, W // 2)
    return Workload("disks", image, labels0, "pc", 4, lam, cutoff, 0.0, iterations,
                    {"seed": seed, "sigma": sigma})


def ellipses(H: int = 1024, W: int = 1024, seed: int = 1, n_ellipses: int | None = None,
             photons: float = 20.0, lam: float = 0.04, cutoff: float = 5.0, ps_radius: float = 8.0,
             iterations: int = 200, axis_lo: float = 10.0, axis_hi: float = 60.0) -> Workload:
    """Piecewise-smooth 2D scene: biased ellipses with Poisson noise, square-grid start."""
    rs = Stream(seed, 2)
    if n_ellipses is None:
        n_ellipses = max(1, int(round(40 * H * W / (1024 * 1024))))
    clean = np.zeros((H, W), dtype=np.float64)
    a = rs.uniform_range(axis_lo, axis_hi, n_ellipses)
    b = rs.uniform_range(axis_lo, axis_hi, n_ellipses)
    th = rs.uniform_range(0.0, math.pi, n_ellipses)
    cy = rs.uniform_range(0, H, n_ellipses)
    cx = rs.uniform_range(0, W, n_ellipses)
    amp = rs.uniform_range(0.5, 1.5, n_ellipses)
    for i in range(n_ellipses):
        r = math.ceil(max(a[i], b[i]))
        y0, y1 = max(0, int(cy[i]) - r - 1), min(H, int(cy[i]) + r + 2)
        x0, x1 = max(0, int(cx[i]) - r - 1), min(W, int(cx[i]) + r + 2)
        if y0 >= y1 or x0 >= x1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1]
        dy, dx = yy - cy[i], xx - cx[i]
        c, s = math.cos(th[i]), math.sin(th[i])
        u = (dx * c + dy * s) / a[i]
        v = (-dx * s + dy * c) / b[i]
        m = u * u + v * v <= 1.0
        clean[y0:y1, x0:x1][m] = amp[i]
    bias = 0.5 + np.arange(W, dtype=np.float64) / max(1, W - 1)
    clean *= bias[None, :]
    counts = rs.poisson(photons * clean)
    image = (counts.astype(np.float64) / photons).astype(np.float32)
    labels0 = square_grid_labels(H, W, 64, 32)
    return Workload("ellipses", image, labels0, "ps", 4, lam, cutoff, ps_radius, iterations,
                    {"seed": seed, "photons": photons})


def _gauss_blur_axis(x: np.ndarray, axis: int, sigma: float, radius: int) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-0.5 * (t / sigma) ** 2)
    w /= w.sum()
    n = x.shape[axis]
    out = np.zeros_like(x)
    for k, wk in zip(range(-radius, radius + 1), w):
        src = np.clip(np.arange(n) + k, 0, n - 1)
        out += wk * np.take(x, src, axis=axis)
    return out


def gaussian_psf(sigma: float, radius: int | None = None) -> np.ndarray:
    """Sampled Gaussian profile exp(-u^2 / (2 sigma^2)), u = -r..r (r = ceil(3 sigma) by
    default), normalised to unit sum; exactly symmetric."""
    r = int(math.ceil(3.0 * sigma)) if radius is None else int(radius)
    u = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-(u * u) / (2.0 * sigma * sigma))
    return w / w.sum()


def _blur_zero(x: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Separable blur with profile k on every axis, zero outside the array."""
    r = (k.size - 1) // 2
    out = x.astype(np.float64)
    for axis in range(x.ndim):
        n = out.shape[axis]
        pad = [(0, 0)] * x.ndim
        pad[axis] = (r, r)
        xp = np.pad(out, pad)
        acc = np.zeros_like(out)
        for j, wk in enumerate(k):
            acc += wk * np.take(xp, np.arange(j, j + n), axis=axis)
        out = acc
    return out


def deconv_scene(H: int = 512, W: int = 512, seed: int = 11, sigma: float = 15.0, photons: float = 10.0,
                 lam: float = 0.04, cutoff: float = 5.0, iterations: int = 200) -> Workload:
    """Deconvolution scene: four objects (two disks, a square, an ellipse) at intensities
    2-4 over background 0.25, blurred by a Gaussian PSF of width sigma (zero outside the
    image), Poisson noise at `photons` per unit; initial labels are squares on a grid."""
    rs = Stream(seed, 4)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    clean = np.full((H, W), 0.25)
    amp = rs.uniform_range(2.0, 4.0, 4)
    jit = rs.uniform_range(-0.05, 0.05, 8).reshape(4, 2)
    s = min(H, W)
    cy = np.array([0.28, 0.30, 0.72, 0.70]) * H + jit[:, 0] * s
    cx = np.array([0.28, 0.72, 0.30, 0.70]) * W + jit[:, 1] * s
    clean[(yy - cy[0]) ** 2 + (xx - cx[0]) ** 2 <= (0.12 * s) ** 2] = amp[0]
    clean[(yy - cy[1]) ** 2 + (xx - cx[1]) ** 2 <= (0.08 * s) ** 2] = amp[1]
    clean[(np.abs(yy - cy[2]) <= 0.10 * s) & (np.abs(xx - cx[2]) <= 0.10 * s)] = amp[2]
    clean[((yy - cy[3]) / (0.06 * s)) ** 2 + ((xx - cx[3]) / (0.14 * s)) ** 2 <= 1.0] = amp[3]
    psf = gaussian_psf(sigma)
    blurred = _blur_zero(clean, psf)
    counts = rs.poisson(photons * blurred)
    image = (counts.astype(np.float64) / photons).astype(np.float32)
    pitch = max(8, s // 4)
    labels0 = square_grid_labels(H, W, pitch, pitch // 2)
    return Workload("deconv", image, labels0, "pcd", 4, lam, cutoff, 0.0, iterations,
                    {"seed": seed, "sigma": sigma, "photons": photons}, psf)


def ellipsoids(D: int = 256, H: int = 256, W: int = 256, seed: int = 2, n_ellipsoids: int | None = None,
               lam: float = 1600.0, cutoff: float = 4.0, iterations: int = 100,
               axis_lo: float = 4.0, axis_hi: float = 20.0) -> Workload:
    """3D uint16 scene: ellipsoids at 300 over 100, blurred, Poisson noise, cube-grid start."""
    rs = Stream(seed, 3)
    if n_ellipsoids is None:
        n_ellipsoids = max(1, int(round(200 * D * H * W / 256 ** 3)))
    clean = np.full((D, H, W), 100.0, dtype=np.float64)
    ax = rs.uniform_range(axis_lo, axis_hi, 3 * n_ellipsoids).reshape(n_ellipsoids, 3)
    q = rs.uniform(3 * n_ellipsoids).reshape(n_ellipsoids, 3)
    cz = rs.uniform_range(0, D, n_ellipsoids)
    cy = rs.uniform_range(0, H, n_ellipsoids)
    cx = rs.uniform_range(0, W, n_ellipsoids)
    for i in range(n_ellipsoids):
        # uniform random rotation from a uniform unit quaternion (Shoemake 1992)
        u1, u2, u3 = q[i]
        qa = math.sqrt(1 - u1) * math.sin(2 * math.pi * u2)
        qb = math.sqrt(1 - u1) * math.cos(2 * math.pi * u2)
        qc = math.sqrt(u1) * math.sin(2 * math.pi * u3)
        qd = math.sqrt(u1) * math.cos(2 * math.pi * u3)
        R = np.array([
            [1 - 2 * (qc * qc + qd * qd), 2 * (qb * qc - qa * qd), 2 * (qb * qd + qa * qc)],
            [2 * (qb * qc + qa * qd), 1 - 2 * (qb * qb + qd * qd), 2 * (qc * qd - qa * qb)],
            [2 * (qb * qd - qa * qc), 2 * (qc * qd + qa * qb), 1 - 2 * (qb * qb + qc * qc)]])
        r = math.ceil(ax[i].max())
        z0, z1 = max(0, int(cz[i]) - r - 1), min(D, int(cz[i]) + r + 2)
        y0, y1 = max(0, int(cy[i]) - r - 1), min(H, int(cy[i]) + r + 2)
        x0, x1 = max(0, int(cx[i]) - r - 1), min(W, int(cx[i]) + r + 2)
        if z0 >= z1 or y0 >= y1 or x0 >= x1:
            continue
        zz, yy, xx = np.mgrid[z0:z1, y0:y1, x0:x1]
        p = np.stack([xx - cx[i], yy - cy[i], zz - cz[i]], axis=-1) @ R
        m = ((p / ax[i]) ** 2).sum(axis=-1) <= 1.0
        clean[z0:z1, y0:y1, x0:x1][m] = 300.0
    for axis in range(3):
        clean = _gauss_blur_axis(clean, axis, 1.5, 6)
    counts = np.clip(rs.poisson(clean), 0, 65535).astype(np.uint16)
    labels0 = cube_grid_labels(D, H, W, 32, 16)
    return Workload("ellipsoids", counts, labels0, "pc", 6, lam, cutoff, 0.0, iterations, {"seed": seed})


def batch_disk(i: int, seed0: int = 1000, lo: int = 64, hi: int = 512, iterations: int = 50) -> Workload:
    """Image i of the uneven batch: a disk scene with seed seed0 + i, sides U{lo..hi}."""
    rs = Stream(seed0 + i, 7)
    H, W = (int(v) for v in rs.integers(lo, hi, 2))
    w = disks(H, W, seed=seed0 + i, iterations=iterations)
    w.name = f"batch{i}"
    return w


def batch_disks(n_images: int = 512, seed0: int = 1000, lo: int = 64, hi: int = 512,
                iterations: int = 50) -> list[Workload]:
    """Many uneven 2D disk scenes (seeds seed0 + i), sides U{lo..hi} drawn independently."""
    return [batch_disk(i, seed0, lo, hi, iterations) for i in range(n_images)]


@dataclass
class Arrival:
    t: float                 # arrival time in seconds
    kind: str                # "pc2d" | "ps2d" | "pc3d"
    side: int
    seed: int


def arrival_stream(n_jobs: int = 2000, rate: float = 200.0, seed: int = 42) -> list[Arrival]:
    """Poisson-process job arrivals: 80% 2D (half pc, half ps), 20% 3D."""
    rs = Stream(seed, 11)
    gaps = -np.log(1.0 - rs.uniform(n_jobs)) / rate
    times = np.cumsum(gaps)
    kind_u = rs.uniform(n_jobs)
    half_u = rs.uniform(n_jobs)
    side2 = rs.integers(128, 1024, n_jobs)
    side3 = rs.integers(64, 256, n_jobs)
    out = []
    for i in range(n_jobs):
        if kind_u[i] < 0.8:
            kind = "pc2d" if half_u[i] < 0.5 else "ps2d"
            side = int(side2[i])
        else:
            kind, side = "pc3d", int(side3[i])
        out.append(Arrival(float(times[i]), kind, side, seed * 100000 + i))
    return out


def make_job(a: Arrival, iterations: int = 100) -> Workload:
    if a.kind == "pc2d":
        return disks(a.side, a.side, seed=a.seed, iterations=iterations)
    if a.kind == "ps2d":
        return ellipses(a.side, a.side, seed=a.seed, iterations=iterations)
    return ellipsoids(a.side, a.side, a.side, seed=a.seed, iterations=iterations)


def served_job_key(a: Arrival) -> tuple:
    """The pooled job an arrival of the served stream runs: its kind, its side rounded to a
    bucket (32 voxels in 3D within 64..256, 64 pixels in 2D within 128..1024) and one seed per
    bucket. Arrivals of one bucket run the same image, so that the stream needs only a few
    dozen distinct images (a 256^3 volume takes seconds to generate)."""
    if a.kind == "pc3d":
        side = max(64, min(256, int(round(a.side / 32.0)) * 32))
    else:
        side = max(128, min(1024, int(round(a.side / 64.0)) * 64))
    return (a.kind, side, 7 * side + len(a.kind))


def served_job(key: tuple, iterations: int = 100) -> Workload:
    kind, side, seed = key
    return make_job(Arrival(0.0, kind, side, seed), iterations=iterations)


def config(index: int) -> Workload | list:
    """The five standard workloads by index (0: 128^2 disks, 1: 1024^2 ellipses,
    2: 256^3 ellipsoids, 3: 512 uneven disk images, 4: served arrival stream)."""
    if index == 0:
        return disks()
    if index == 1:
        return ellipses()
    if index == 2:
        return ellipsoids()
    if index == 3:
        return batch_disks()
    if index == 4:
        return arrival_stream()
    raise ValueError(f"no workload {index}")
