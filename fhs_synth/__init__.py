"""Seeded synthetic inputs shaped like the workloads of Faceted HyperSARA
(Thouvenin et al., arXiv 2003.07358, Section 4.1).

This module is shared by the FP64 oracle (test infrastructure) and by the GPU
library's tests and benchmark.  It holds no arithmetic of the reconstruction
method itself: it draws skies, uv points, block partitions and unit-variance
noise, nothing more.  Noise scaling (iSNR -> sigma), l2-ball radii, operator
norms and regularisation parameters belong to the method and are computed by
whoever consumes these inputs.

Every draw comes from ``numpy.random.default_rng(seed)`` (PCG64) in the order
documented on each function, so equal seeds give bit-identical inputs.

Stand-ins (the paper's data is not available): the Cyg A map becomes a sum of
Gaussian blobs and point sources with power-law spectra (the spectral model of
Section 4.1, with optional curvature); the VLA coverage becomes isotropic
Gaussian uv points scaled with frequency (uv coverage of channel l is the
reference coverage dilated by nu_l / nu_1, Section 4.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

__all__ = [
    "CubeSpec", "WORKLOADS", "workload", "frequencies", "subcube_channels",
    "sky_sources", "render_channel", "sky_cube", "base_uv", "channel_uv", "radial_blocks", "unit_noise",
    "ProblemInputs", "make_inputs", "DdeInputs", "dde_inputs", "BATCH_SIDES", "batch_specs",
]


@dataclass(frozen=True)
class CubeSpec:
    """Shape of one synthetic wide-band problem.

    n      : image side (the image is n x n)
    L      : total channels; C interleaved spectral sub-cubes of L/C channels
    Q      : spatial facets per dimension (Q x Q facets)
    overlap: nuclear-norm facet overlap, fraction of the tile side
    window : "triangular" or "sine" apodisation
    m_ratio: visibilities per channel = round(m_ratio * n * n) (or m_abs)
    B      : data blocks per channel (uv-radial)
    """
    name: str
    n: int
    L: int
    C: int = 1
    Q: int = 1
    overlap: float = 0.1
    window: str = "triangular"
    m_ratio: float = 0.5
    m_abs: int | None = None
    B: int = 1
    isnr_db: float = 40.0
    n_blobs: int = 20
    n_points: int = 0
    curvature: float = 0.0
    nu_min: float = 1.0
    nu_max: float = 2.0
    sigma_uv: float = math.pi / 4
    seed: int = 0

    @property
    def M(self) -> int:
        return int(self.m_abs) if self.m_abs is not None else int(round(self.m_ratio * self.n * self.n))

    @property
    def Lc(self) -> int:
        return self.L // self.C


# Workloads with the shapes of the paper-derived configurations.
WORKLOADS = {
    "tiny": CubeSpec("tiny: 64x64, L=4, Q=1, M=2000, B=1", n=64, L=4, C=1, Q=1,
                     m_abs=2000, B=1, isnr_db=40.0, n_blobs=20, seed=0),
    "faceted": CubeSpec("faceted: 256x256, L=20, 4x4 facets, 10% sine overlap, M=0.5N, B=2",
                        n=256, L=20, C=1, Q=4, overlap=0.1, window="sine",
                        m_ratio=0.5, B=2, isnr_db=40.0, n_blobs=20, seed=1000),
    "precision": CubeSpec("precision: 1024x1024, L=32, 8x8 facets, M=N, B=4",
                          n=1024, L=32, C=1, Q=8, overlap=0.1, m_ratio=1.0, B=4,
                          isnr_db=30.0, n_blobs=250, n_points=250, curvature=0.01,
                          seed=2000),
    "large": CubeSpec("large: 4096x4096, L=64 (4 interleaved sub-cubes of 16), 16x16 facets, M=0.5N, B=8",
                      n=4096, L=64, C=4, Q=16, overlap=0.1, m_ratio=0.5, B=8,
                      isnr_db=30.0, n_blobs=250, n_points=250, curvature=0.01,
                      seed=4000),
    # the large workload's geometry (image, grid, facets, visibility density) on two
    # channels of one sub-cube: a few GB on the device, for profiler captures
    "large_slice": CubeSpec("large_slice: 4096x4096, L=2 (1 sub-cube), 16x16 facets, M=0.5N, B=8",
                            n=4096, L=2, C=1, Q=16, overlap=0.1, m_ratio=0.5, B=8,
                            isnr_db=30.0, n_blobs=250, n_points=250, curvature=0.01,
                            seed=4000),
    # the large workload's nuclear facets (256 + 25 pixels a side) and sub-cube channel
    # count (16) on a 1024 x 1024 image: about 2 GB on the device, for profiler captures
    # of the facet kernels
    "facet_slice": CubeSpec("facet_slice: 1024x1024, L=16 (1 sub-cube), 4x4 facets of 281^2, M=0.5N, B=8",
                            n=1024, L=16, C=1, Q=4, overlap=0.1, m_ratio=0.5, B=8,
                            isnr_db=30.0, n_blobs=60, n_points=60, curvature=0.01,
                            seed=4100),
}


def workload(name: str, **over) -> CubeSpec:
    return replace(WORKLOADS[name], **over)


# The mixed-size batch: 16 independent cubes of uneven shapes (Section 2.4.1: sub-cubes
# are separate problems), image sides 128..768 (including 3 * 2^m sides), 8..48
# channels, 1..6 facets a side, 0.3..2 visibilities per pixel.
BATCH_SIDES = (128, 192, 256, 384, 512, 768)


def batch_specs(n_cubes: int = 16, seed: int = 3000) -> list[CubeSpec]:
    """Seeded shapes of the mixed-size batch (draw order: side, channels, facets,
    visibility ratio, blocks, per cube); cube k has seed `seed + k`.  The largest side
    appears at least once."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_cubes):
        n = int(BATCH_SIDES[rng.integers(len(BATCH_SIDES))]) if k else BATCH_SIDES[-1]
        L = int(rng.integers(8, 49))
        Q = int(rng.integers(1, 7))
        mr = float(rng.uniform(0.3, 2.0))
        B = int(rng.integers(1, 5))
        out.append(CubeSpec(f"batch cube {k}: {n}x{n}, L={L}, {Q}x{Q} facets, M={mr:.2f}N, B={B}", n=n, L=L, C=1,
                            Q=Q, overlap=0.1, m_ratio=mr, B=B, isnr_db=40.0, n_blobs=20, seed=seed + k))
    return out


def frequencies(spec: CubeSpec) -> np.ndarray:
    """Channel frequencies in GHz, uniform on [nu_min, nu_max]."""
    if spec.L == 1:
        return np.array([spec.nu_min])
    return np.linspace(spec.nu_min, spec.nu_max, spec.L)


def subcube_channels(spec: CubeSpec, c: int) -> np.ndarray:
    """Channels of interleaved sub-cube c: l = c, c + C, c + 2C, ... (Section 3 spectral faceting)."""
    return np.arange(c, spec.L, spec.C)


def sky_sources(spec: CubeSpec, rng: np.random.Generator) -> dict:
    """Source parameters of the synthetic sky.

    Draw order: for each blob (n_blobs): row, col ~ U[lo, hi), sigma ~ U[1,4],
    amplitude ~ U[0.1, 1], spectral index ~ U[-1, 1], curvature sign (U[0,1] < 0.5
    gives +1); then for each point source (n_points): row, col (integers in
    [lo, hi)), amplitude, index, curvature sign.  lo = min(8, n/4), hi = n - lo.
    """
    n = spec.n
    lo, hi = min(8, n // 4), max(n - 8, 3 * n // 4)
    blobs = []
    for _ in range(spec.n_blobs):
        r0 = rng.uniform(lo, hi)
        c0 = rng.uniform(lo, hi)
        sig = rng.uniform(1.0, 4.0)
        amp = rng.uniform(0.1, 1.0)
        a = rng.uniform(-1.0, 1.0)
        b = spec.curvature * (1.0 if rng.uniform() < 0.5 else -1.0)
        blobs.append((r0, c0, sig, amp, a, b))
    points = []
    for _ in range(spec.n_points):
        r0 = int(rng.integers(lo, hi))
        c0 = int(rng.integers(lo, hi))
        amp = rng.uniform(0.1, 1.0)
        a = rng.uniform(-1.0, 1.0)
        b = spec.curvature * (1.0 if rng.uniform() < 0.5 else -1.0)
        points.append((r0, c0, amp, a, b))
    return {"blobs": blobs, "points": points}


def render_channel(spec: CubeSpec, sources: dict, l: int) -> np.ndarray:
    """Channel l of the sky [n][n] float64:
    x_l = x_1 (nu_l/nu_1)^(a + b log(nu_l/nu_1)) per source (Section 4.1 spectral model)."""
    n = spec.n
    nu = frequencies(spec)
    lr = math.log(nu[l] / nu[0])
    x = np.zeros((n, n))
    for (r0, c0, sig, amp, a, b) in sources["blobs"]:
        rad = int(math.ceil(4 * sig))
        r_lo, r_hi = max(0, int(r0) - rad), min(n, int(r0) + rad + 2)
        c_lo, c_hi = max(0, int(c0) - rad), min(n, int(c0) + rad + 2)
        rr = np.arange(r_lo, r_hi)[:, None]
        cc = np.arange(c_lo, c_hi)[None, :]
        g = amp * np.exp(-((rr - r0) ** 2 + (cc - c0) ** 2) / (2 * sig * sig))
        x[r_lo:r_hi, c_lo:c_hi] += math.exp((a + b * lr) * lr) * g
    for (r0, c0, amp, a, b) in sources["points"]:
        x[r0, c0] += amp * math.exp((a + b * lr) * lr)
    return x


def sky_cube(spec: CubeSpec, rng: np.random.Generator, chans=None) -> np.ndarray:
    """Ground-truth cube [len(chans)][n][n] float64 (all channels by default), non-negative."""
    src = sky_sources(spec, rng)
    chans = range(spec.L) if chans is None else chans
    return np.stack([render_channel(spec, src, l) for l in chans])


def base_uv(spec: CubeSpec, rng: np.random.Generator) -> np.ndarray:
    """Reference-frequency uv points [M][2] (u, v) in rad/pixel, float64.

    Isotropic Gaussian N(0, sigma_uv^2 I), rejection-clipped so that the
    highest channel's dilated point still lies in [-pi, pi)^2.
    Draws: batches of standard normals of shape (2*M, 2) until M accepted.
    """
    M = spec.M
    smax = spec.nu_max / spec.nu_min
    out = np.empty((0, 2))
    while out.shape[0] < M:
        d = rng.standard_normal((2 * M, 2)) * spec.sigma_uv
        keep = np.max(np.abs(d), axis=1) * smax < math.pi * (1 - 1e-6)
        out = np.concatenate([out, d[keep]])
    return out[:M]


def channel_uv(base: np.ndarray, spec: CubeSpec, l: int) -> np.ndarray:
    """uv points of channel l: reference points dilated by nu_l / nu_1, float32."""
    nu = frequencies(spec)
    return (base * (nu[l] / nu[0])).astype(np.float32)


def radial_blocks(base: np.ndarray, B: int) -> list[np.ndarray]:
    """Partition of visibility indices into B uv-radial blocks of (nearly) equal
    count, by quantiles of |omega| of the reference points (Fig. 1 blocking).
    Returns B index arrays, each sorted ascending; ties broken by index."""
    r = np.hypot(base[:, 0], base[:, 1])
    order = np.lexsort((np.arange(r.size), r))
    bounds = [int(round(b * r.size / B)) for b in range(B + 1)]
    return [np.sort(order[bounds[b]:bounds[b + 1]]) for b in range(B)]


def unit_noise(M: int, rng: np.random.Generator) -> np.ndarray:
    """Complex white Gaussian noise CN(0, 1): E|n|^2 = 1 (real, imag each N(0, 1/2)).
    Draws: standard normals of shape (M, 2)."""
    d = rng.standard_normal((M, 2))
    return (d[:, 0] + 1j * d[:, 1]) / math.sqrt(2.0)


@dataclass
class ProblemInputs:
    """Inputs of one sub-cube, channel-major, visibilities block-contiguous per channel.

    x_true : [Lc][n][n] float64 ground truth
    uv     : [Lc*M][2] float32 (u, v) rad/pixel, channel-major, block-contiguous
    M_lb   : [Lc][B] visibilities per (channel, block)
    noise  : [Lc*M] complex128 unit-variance noise, same order as uv
    chans  : global channel indices of this sub-cube
    """
    spec: CubeSpec
    cube: int
    x_true: np.ndarray
    uv: np.ndarray
    M_lb: np.ndarray
    noise: np.ndarray
    chans: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=int))
    perm: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int64))   # block order of the reference points


def make_inputs(spec: CubeSpec, cube: int = 0, with_noise: bool = True) -> ProblemInputs:
    """All inputs of sub-cube `cube` of `spec`.

    Draw order with rng = default_rng(spec.seed): sky cube (all L channels),
    reference uv points, then (if with_noise) unit noise for every channel of
    every sub-cube in global channel order, so that each sub-cube sees the
    same draws whichever sub-cube is generated.
    """
    rng = np.random.default_rng(spec.seed)
    chans = subcube_channels(spec, cube)
    x = sky_cube(spec, rng, chans)
    base = base_uv(spec, rng)
    blocks = radial_blocks(base, spec.B)
    Lc = chans.size
    perm = np.concatenate(blocks)
    uv = np.concatenate([channel_uv(base, spec, l)[perm] for l in chans])
    M_lb = np.array([[b.size for b in blocks] for _ in chans], dtype=np.int64)
    if with_noise:
        noise_all = [unit_noise(spec.M, rng) for _ in range(spec.L)]
        noise = np.concatenate([noise_all[l][perm] for l in chans])
    else:
        noise = np.zeros(Lc * spec.M, dtype=np.complex128)
    return ProblemInputs(spec=spec, cube=cube, x_true=x, uv=uv, M_lb=M_lb,
                         noise=noise, chans=chans, perm=perm)


@dataclass
class DdeInputs:
    """Synthetic direction-dependent effects of one sub-cube (Section 2.1, after Eq. 1).

    Each antenna a and channel l has a pattern D_{a,l}(p) with an S_a x S_a Fourier-domain
    representation d_{a,l} on the lattice of the 2x oversampled grid (centre coefficient 1,
    the other coefficients small, decaying away from the centre).  Visibility m of
    baseline (a, b) sees the sky multiplied by D_a conj(D_b), whose representation is the
    S_d x S_d = (2 S_a - 1)^2 convolution of d_a with d~_b[j] = conj(d_b[-j]).

    kern : [Lc * n_bl][S_d][S_d] complex128, kernel of (channel i of the sub-cube,
           baseline k) at index i * n_bl + k; first index along grid rows (v)
    kidx : [Lc * M] int32, kernel of each visibility, in the order of ProblemInputs.uv
    """
    kern: np.ndarray
    kidx: np.ndarray
    n_ant: int
    S_a: int


def dde_inputs(inp: ProblemInputs, n_ant: int = 8, S_a: int = 5, amp: float = 0.05) -> DdeInputs:
    """DDE kernels and per-visibility kernel indices for `inp`.

    Draw order with rng = default_rng(spec.seed + 7919): the baseline of every reference
    visibility (integers in [0, n_bl)), then for every channel of the cube in global
    order and every antenna, S_a x S_a x 2 standard normals (real, imaginary parts),
    scaled by amp * exp(-|j|^2 / 2); the centre coefficient is then set to 1.
    """
    spec = inp.spec
    rng = np.random.default_rng(spec.seed + 7919)
    pairs = [(a, b) for a in range(n_ant) for b in range(a + 1, n_ant)]
    n_bl = len(pairs)
    bl = rng.integers(0, n_bl, size=spec.M)
    R = S_a // 2
    j = np.arange(-R, R + 1)
    taper = amp * np.exp(-(j[:, None] ** 2 + j[None, :] ** 2) / 2.0)
    d_all = {}
    for l in range(spec.L):
        d = rng.standard_normal((n_ant, S_a, S_a, 2))
        d = (d[..., 0] + 1j * d[..., 1]) * taper
        d[:, R, R] = 1.0
        d_all[l] = d
    S_d = 2 * S_a - 1
    kern = np.zeros((inp.chans.size * n_bl, S_d, S_d), dtype=np.complex128)
    for i, l in enumerate(inp.chans):
        d = d_all[int(l)]
        for k, (a, b) in enumerate(pairs):
            db = np.conj(d[b][::-1, ::-1])                          # d~_b[j] = conj(d_b[-j])
            out = kern[i * n_bl + k]
            for r in range(S_a):
                for c in range(S_a):
                    out[r:r + S_a, c:c + S_a] += d[a][r, c] * db
    # visibilities are block-ordered in ProblemInputs (inp.perm)
    perm = inp.perm
    kidx = np.concatenate([i * n_bl + bl[perm] for i in range(inp.chans.size)]).astype(np.int32)
    return DdeInputs(kern=kern, kidx=kidx, n_ant=n_ant, S_a=S_a)
