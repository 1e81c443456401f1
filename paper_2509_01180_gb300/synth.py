"""Seeded synthetic workloads: blob phantoms, rotations, noise, missing wedge, random starts.

This module is the one piece of input preparation that the CUDA path and the
FP64 oracle both use.  It contains none of the alignment method's arithmetic
(no basis, no expansion, no Wigner matrices, no score): it only draws random
numbers and renders test volumes.

Synthetic data stand in for the SHREC 2020 simulated tomograms the paper
evaluates on (Sec. III); no SHREC item is reproduced.  Recipe:
  * template: ``n_blobs`` isotropic Gaussians exp(-|p - c|^2 / (2 sigma^2)) in
    voxel units, centres uniform in volume inside radius 0.75 * N/2 around the
    box centre N/2, amplitudes U[0.5, 1];
  * subtomogram p: the template rotated by a uniform random rotation R_p
    (rendered analytically at R_p c, no interpolation), so f_p = R_p t with
    (R t)(x) = t(R^{-1} x);
  * optional white Gaussian noise with SNR = var(signal in the ball) / sigma_n^2,
    added before the wedge mask;
  * optional missing wedge about the y axis (beam along z): Fourier components
    with |k_z| > tan(theta_max) |k_x| are zeroed, the k_x = k_z = 0 line kept;
  * starts: uniform random rotations (Shoemake's method), per particle.
Seeds: master seed 2509; the generator of particle i is seeded with
splitmix64(master + i).  Volumes are float32 in [z][y][x] order; quaternions
(w, x, y, z) are float32, and the FP64 oracle reads the same float32 values.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 2509
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One output of the SplitMix64 generator (Steele, Lea, Flood 2014) for state x."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def rng_for(stream: int, index: int, master: int = MASTER_SEED) -> np.random.Generator:
    """Independent generator for (stream, index); streams separate templates, particles and starts."""
    return np.random.default_rng(splitmix64((master * 1000003 + stream * 7919 + index) & _M64))


def uniform_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """n uniform random unit quaternions (w, x, y, z), Shoemake's subgroup algorithm; w >= 0."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3)], axis=1)
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    return q


def _rotation_matrix(q) -> np.ndarray:
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


@dataclass
class BlobTemplate:
    centres: np.ndarray  # (n, 3) voxel units relative to the box centre, (x, y, z)
    amps: np.ndarray  # (n,)
    sigma: float


def blob_template(rng: np.random.Generator, n_blobs: int, sigma: float, r_max: float) -> BlobTemplate:
    """Blob centres uniform in volume in the ball of radius r_max (voxels), amplitudes U[0.5, 1]."""
    d = rng.normal(size=(n_blobs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = r_max * rng.random(n_blobs) ** (1.0 / 3.0)
    return BlobTemplate(d * r[:, None], 0.5 + 0.5 * rng.random(n_blobs), float(sigma))


def render(N: int, tpl: BlobTemplate, q=None, offset=None) -> np.ndarray:
    """Volume vol[z, y, x] of the blobs (rotated by q, then displaced by `offset` voxels (x, y, z), when
    given), centre at voxel N/2 along each axis."""
    c = tpl.centres if q is None else tpl.centres @ _rotation_matrix(q).T
    if offset is not None:
        c = c + np.asarray(offset, dtype=np.float64)[None, :]
    p = np.arange(N, dtype=np.float64) - N / 2
    s2 = 2.0 * tpl.sigma ** 2
    ex = np.exp(-(p[None, :] - c[:, 0:1]) ** 2 / s2) * tpl.amps[:, None]
    ey = np.exp(-(p[None, :] - c[:, 1:2]) ** 2 / s2)
    ez = np.exp(-(p[None, :] - c[:, 2:3]) ** 2 / s2)
    zy = (ez[:, :, None] * ey[:, None, :]).reshape(len(c), N * N)
    return (zy.T @ ex).reshape(N, N, N)


def ball_mask(N: int) -> np.ndarray:
    h = N // 2
    i = np.arange(N) - h
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    return (x * x + y * y + z * z) < h * h


def wedge_mask(N: int, half_angle_deg: float) -> np.ndarray:
    """Fourier mask keeping |k_z| <= tan(theta) |k_x| (tilt axis y, beam z) plus the k_x = k_z = 0 line."""
    k = np.fft.fftfreq(N)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    keep = np.abs(kz) <= math.tan(math.radians(half_angle_deg)) * np.abs(kx) + 1e-12
    keep |= (kx == 0) & (kz == 0)
    return keep


def degrade(vol: np.ndarray, rng: np.random.Generator, snr: float | None, wedge_deg: float | None) -> np.ndarray:
    """Add white noise at the given SNR (signal variance inside the ball) and apply the missing wedge."""
    out = vol
    if snr is not None:
        var = float(np.var(vol[ball_mask(vol.shape[0])]))
        out = out + rng.normal(scale=math.sqrt(var / snr), size=vol.shape)
    if wedge_deg is not None:
        out = np.fft.ifftn(np.fft.fftn(out) * wedge_mask(vol.shape[0], wedge_deg)).real
    return out


@dataclass
class Workload:
    """One alignment workload: a template, B subtomograms and S starts per subtomogram."""

    name: str
    N: int
    Lmax: int
    lam_max: float
    stages: list
    steps: int
    S: int
    template: np.ndarray  # (N, N, N) float32
    vols: np.ndarray  # (B, N, N, N) float32
    q_true: np.ndarray  # (B, 4) float64: f_p = R(q_true[p]) t
    starts: np.ndarray  # (B, S, 4) float32
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return self.vols.shape[0]


# name: (N, Lmax, blobs, sigma, snr, wedge, stages, steps, starts, count)
CONFIGS = {
    # FP64 plain method, one noiseless pair (16^3, l <= 8, marching 2-4-8, 8 starts, 50 steps)
    "pair16": (16, 8, 20, 1.2, None, None, [2, 4, 8], 50, 8, 1),
    # FP32 plain method on the GPU: 1024 x 32^3, SNR 0.1, +-60 deg wedge, l <= 16, 4-8-16, 16 starts, 30 steps
    "batch32": (32, 16, 60, 1.5, 0.1, 60.0, [4, 8, 16], 30, 16, 1024),
    # precision form: 4096 x 64^3, SNR 0.05, +-60 deg, l <= 32, 4-8-16-32, 32 starts, 30 steps
    "precision64": (64, 32, 200, 2.0, 0.05, 60.0, [4, 8, 16, 32], 30, 32, 4096),
}


def _workload_particle(tpl: BlobTemplate, N: int, p: int, master: int, snr, wedge):
    """Ground-truth rotation and degraded volume of particle p (its own seeded generator)."""
    rng = rng_for(2, p, master)
    q = uniform_quaternions(rng, 1)[0]
    return q, degrade(render(N, tpl, q), rng, snr, wedge)


def _workload_chunk(job):
    """Worker (spawned process): rotations and volumes of particles lo..hi-1 of a workload."""
    count, name, first, lo, hi, master, snr, wedge, dtype = job
    N, _, nb, sigma = CONFIGS[name][:4]
    tpl = blob_template(rng_for(1, 0, master), nb, sigma, 0.75 * N / 2)
    qs = np.empty((hi - lo, 4))
    vols = np.empty((hi - lo, N, N, N), dtype=dtype)
    for j in range(lo, hi):
        qs[j - lo], v = _workload_particle(tpl, N, first + j, master, snr, wedge)
        vols[j - lo] = v.astype(dtype)
    return lo, qs, vols


def _parallel_chunks(fn, jobs, workers: int):
    """fn over jobs in a pool of `workers` spawned processes (results in job order)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(fn, jobs, chunksize=1)


def _chunks(count: int, workers: int):
    step = max(1, -(-count // (4 * workers)))
    return [(lo, min(count, lo + step)) for lo in range(0, count, step)]


def make_workload(name: str, count: int | None = None, first: int = 0, master: int = MASTER_SEED,
                  snr=..., wedge=..., dtype=np.float32, workers: int = 1) -> Workload:
    """Build particles first .. first+count-1 of a named workload (all deterministic in the seeds; the same
    arrays whatever `workers`, the number of spawned processes that render the volumes)."""
    N, Lmax, nb, sigma, snr0, wedge0, stages, steps, S, B = CONFIGS[name]
    snr = snr0 if snr is ... else snr
    wedge = wedge0 if wedge is ... else wedge
    count = B if count is None else count
    tpl = blob_template(rng_for(1, 0, master), nb, sigma, 0.75 * N / 2)
    template = render(N, tpl).astype(dtype)
    q_true = np.empty((count, 4))
    starts = np.empty((count, S, 4), dtype=np.float32)
    vols = np.empty((count, N, N, N), dtype=dtype)
    if workers > 1 and count > 1:
        jobs = [(count, name, first, lo, hi, master, snr, wedge, np.dtype(dtype)) for lo, hi in _chunks(count, workers)]
        for lo, qs, vs in _parallel_chunks(_workload_chunk, jobs, workers):
            q_true[lo:lo + len(qs)] = qs
            vols[lo:lo + len(qs)] = vs
    else:
        for j in range(count):
            q_true[j], v = _workload_particle(tpl, N, first + j, master, snr, wedge)
            vols[j] = v.astype(dtype)
    for j in range(count):
        starts[j] = uniform_quaternions(rng_for(3, first + j, master), S).astype(np.float32)
    return Workload(name, N, Lmax, math.pi * N / 2, list(stages), steps, S, template, vols, q_true, starts,
                    {"blobs": nb, "sigma": sigma, "snr": snr, "wedge_deg": wedge, "first": first})


# ---------------------------------------------------------------------------------- mixed batch
@dataclass
class ClassWorkload:
    """One box class of a mixed batch: its templates and particles (sorted by start count)."""

    N: int
    Lmax: int
    lam_max: float
    stages: list
    steps: int
    templates: np.ndarray  # (n_templates, N, N, N) float32
    vols: np.ndarray  # (B, N, N, N) float32
    tmpl_index: np.ndarray  # (B,) int32
    q_true: np.ndarray  # (B, 4)
    S: np.ndarray  # (B,) starts per particle, ascending
    starts: np.ndarray  # (B, max S, 4) float32 (rows beyond S[b] unused)

    @property
    def B(self) -> int:
        return self.vols.shape[0]

    def groups(self):
        """Contiguous (first, count, S) runs of equal start count."""
        out, b = [], 0
        while b < self.B:
            e = b
            while e < self.B and self.S[e] == self.S[b]:
                e += 1
            out.append((b, e - b, int(self.S[b])))
            b = e
        return out


# mixed batch: (box edge, count) per class; bands Lmax/4 -> Lmax/2 -> Lmax with Lmax = N/2
MIXED_CLASSES = [(24, 3000), (40, 2000), (64, 1000)]
MIXED_BLOBS = [40, 93, 146, 200]


def _mixed_class_templates(ci: int, N: int, master: int):
    sigma = 1.2 + 0.8 * (N - 16) / 48
    return [blob_template(rng_for(10 + ci, t, master), nb, sigma, 0.75 * N / 2) for t, nb in enumerate(MIXED_BLOBS)]


def _mixed_particle(tpls, ci: int, N: int, j: int, master: int):
    """Template index, rotation, start count and degraded volume of particle j of class ci."""
    rng = rng_for(20 + ci, j, master)
    t = int(rng.integers(0, len(tpls)))
    q = uniform_quaternions(rng, 1)[0]
    snr = rng.uniform(0.03, 0.2)
    wedge = rng.uniform(50.0, 70.0)
    vol = degrade(render(N, tpls[t], q), rng, snr, wedge)
    S = (8, 16, 32)[rng.integers(0, 3)]
    return t, q, S, vol


def _mixed_chunk(job):
    """Worker (spawned process): particles lo..hi-1 of one mixed class."""
    ci, N, lo, hi, master = job
    tpls = _mixed_class_templates(ci, N, master)
    vols = np.empty((hi - lo, N, N, N), dtype=np.float32)
    meta = []
    for j in range(lo, hi):
        t, q, S, v = _mixed_particle(tpls, ci, N, j, master)
        vols[j - lo] = v.astype(np.float32)
        meta.append((t, q, S))
    return lo, meta, vols


def make_mixed(scale: float = 1.0, distinct: int | None = None, master: int = MASTER_SEED, workers: int = 1) -> list:
    """Batched uneven workload: classes of 24^3 (l <= 12), 40^3 (l <= 20) and 64^3 (l <= 32) subtomograms,
    4 blob templates per class (40-200 blobs), SNR ~ U[0.03, 0.2], wedge half-angle ~ U[50, 70] deg,
    starts per particle ~ uniform on {8, 16, 32}, 30 steps per band.  `scale` multiplies the class
    counts; with `distinct`, only that many particles per class are generated and the rest repeat them.
    `workers` > 1 renders the volumes in that many spawned processes (same arrays)."""
    out = []
    for ci, (N, count) in enumerate(MIXED_CLASSES):
        count = max(1, int(round(count * scale)))
        L = N // 2
        tpls = _mixed_class_templates(ci, N, master)
        templates = np.stack([render(N, t) for t in tpls]).astype(np.float32)
        n_gen = count if distinct is None else min(count, distinct)
        tidx = np.empty(n_gen, dtype=np.int32)
        q_true = np.empty((n_gen, 4))
        S = np.empty(n_gen, dtype=np.int32)
        starts = np.zeros((n_gen, 32, 4), dtype=np.float32)
        vols = np.empty((n_gen, N, N, N), dtype=np.float32)
        if workers > 1 and n_gen > 1:
            jobs = [(ci, N, lo, hi, master) for lo, hi in _chunks(n_gen, workers)]
            for lo, meta, vs in _parallel_chunks(_mixed_chunk, jobs, workers):
                vols[lo:lo + len(meta)] = vs
                for i, (t, q, s_) in enumerate(meta):
                    tidx[lo + i], q_true[lo + i], S[lo + i] = t, q, s_
        else:
            for j in range(n_gen):
                tidx[j], q_true[j], S[j], v = _mixed_particle(tpls, ci, N, j, master)
                vols[j] = v.astype(np.float32)
        for j in range(n_gen):
            starts[j, :S[j]] = uniform_quaternions(rng_for(30 + ci, j, master), S[j]).astype(np.float32)
        if n_gen < count:
            rep = np.arange(count) % n_gen
            vols, tidx, q_true, S, starts = vols[rep], tidx[rep], q_true[rep], S[rep], starts[rep]
        order = np.argsort(S, kind="stable")
        stages = [s for s in (L // 4, L // 2, L) if s >= 1]
        out.append(ClassWorkload(N, L, math.pi * N / 2, stages, 30, templates, vols[order], tidx[order],
                                 q_true[order], S[order], starts[order]))
    return out


# ---------------------------------------------------------------------------------- rotation grids
def super_fibonacci(n: int) -> np.ndarray:
    """n quasi-uniform rotations (w, x, y, z) from super-Fibonacci spirals (M. Alexa, "Super-Fibonacci
    Spirals: Fast, Low-Discrepancy Sampling of SO(3)", CVPR 2022): s_i = i + 1/2, r = sqrt(s/n),
    R = sqrt(1 - s/n), alpha = 2 pi s / phi, beta = 2 pi s / psi with phi = sqrt(2) and psi the real root
    of psi^4 = psi + 4; q_i = (r sin alpha, r cos alpha, R sin beta, R cos beta).  Returned as float32 with
    w >= 0 (q and -q are the same rotation)."""
    phi = math.sqrt(2.0)
    psi = 1.533751168755204288118041
    s = np.arange(n, dtype=np.float64) + 0.5
    r, R = np.sqrt(s / n), np.sqrt(1.0 - s / n)
    a, b = 2 * math.pi * s / phi, 2 * math.pi * s / psi
    q = np.stack([r * np.sin(a), r * np.cos(a), R * np.sin(b), R * np.cos(b)], axis=1)
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    return q.astype(np.float32)
