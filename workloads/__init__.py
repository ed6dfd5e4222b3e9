"""Seeded synthetic inputs for the compressed control-step GEMV.

This module holds NO arithmetic of the method: it only builds the matrices and
vectors that both the CUDA path and the CPU oracle consume.  The paper's own
matrices (the deformation matrices C_d of Sec. 2.1, from a 150x200 mesh) are
proprietary, so smooth-kernel matrices on a regular grid stand in for them:

    A_ij = exp(-|p_i - p_j|^2 / l^2) + 1e-3 * n_ij,   n_ij ~ N(0, 1)

with p on a g x g uniform grid over the square inscribed in the unit disk,
[-1/sqrt(2), 1/sqrt(2)]^2, taken row-major.  Indices beyond the n valid grid
points (when the matrix order is padded up, e.g. 181^2 = 32761 -> 32768) are
all-zero rows and columns.  The noise of row i is drawn from its own Philox
stream, Generator(Philox(key=seed, counter=[0, i, 0, 0])).standard_normal(n),
so any band of rows can be built independently and in parallel.

The per-step heat load of the control loop (Sec. 2.1: the scanner moves field
by field, slit by slit) is a Gaussian spot, sigma = 2 grid cells, whose centre
moves along a serpentine path: 100 exposure fields on a 10 x 10 lattice over
the grid, visited boustrophedon (left to right on even lattice rows, right to
left on odd ones), 20 steps per field; within a field the centre moves
linearly along y from one edge to the other, alternating direction from one
field to the next.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20190208
HALF = 1.0 / math.sqrt(2.0)


def grid_points(g: int, n: int) -> np.ndarray:
    """(n, 2) array: the first n points, row-major, of a g x g grid over [-HALF, HALF]^2."""
    if n > g * g:
        raise ValueError("n exceeds the grid size")
    ax = np.linspace(-HALF, HALF, g)
    k = np.arange(n)
    return np.stack([ax[k % g], ax[k // g]], axis=1)


def _row_noise(seed: int, i: int, n: int) -> np.ndarray:
    gen = np.random.Generator(np.random.Philox(key=seed, counter=[0, i, 0, 0]))
    return gen.standard_normal(n)


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


@dataclass(frozen=True)
class KernelMatrix:
    """Lazily-built smooth-kernel matrix of order `order` over `n_valid` grid points."""

    order: int
    g: int
    n_valid: int
    length: float
    seed: int
    noise: float = 1e-3

    @property
    def shape(self):
        return (self.order, self.order)

    def rows(self, r0: int, r1: int, out: np.ndarray | None = None) -> np.ndarray:
        """FP64 rows [r0, r1) as a (r1 - r0, order) C-contiguous array."""
        n = self.n_valid
        if out is None:
            out = np.empty((r1 - r0, self.order), dtype=np.float64)
        pts = grid_points(self.g, n)
        inv_l2 = 1.0 / (self.length * self.length)

        def one(i):
            row = out[i - r0]
            if i >= n:
                row[:] = 0.0
                return
            d2 = (pts[:, 0] - pts[i, 0]) ** 2 + (pts[:, 1] - pts[i, 1]) ** 2
            row[:n] = np.exp(-d2 * inv_l2) + self.noise * _row_noise(self.seed, i, n)
            row[n:] = 0.0

        nrows = r1 - r0
        if nrows <= 8:
            for i in range(r0, r1):
                one(i)
        else:
            with ThreadPoolExecutor(_threads()) as ex:
                list(ex.map(one, range(r0, r1)))
        return out

    def dense(self) -> np.ndarray:
        return self.rows(0, self.order)

    def bands(self, band_rows: int):
        """Yield (r0, rows) bands of `band_rows` rows covering the matrix."""
        for r0 in range(0, self.order, band_rows):
            r1 = min(self.order, r0 + band_rows)
            yield r0, self.rows(r0, r1)


@dataclass(frozen=True)
class RectKernelMatrix:
    """M x N smooth-kernel matrix between two point sets over the same square:
    the first M points of a ceil(sqrt(M))-grid (outputs) and the first N points
    of a ceil(sqrt(N))-grid (inputs), A_ij = exp(-|p_i - q_j|^2 / l^2) plus
    1e-3 N(0,1) noise; the noise of rows 64k..64k+63 is one (64, N) draw from
    Philox keyed by seed at counter (0, k, 1, 0).  The shape of the paper's
    slit models (Sec. 4.4, Sec. 5.1): wide 378 x 256000 maps heat loads to the slit,
    tall 256000 x 378 the reverse."""

    M: int
    N: int
    length: float
    seed: int
    noise: float = 1e-3

    @property
    def shape(self):
        return (self.M, self.N)

    def rows(self, r0: int, r1: int) -> np.ndarray:
        out = np.empty((r1 - r0, self.N), dtype=np.float64)
        p = grid_points(int(np.ceil(np.sqrt(self.M))), self.M)
        q = grid_points(int(np.ceil(np.sqrt(self.N))), self.N)
        inv_l2 = 1.0 / (self.length * self.length)

        def group(k):
            g0, g1 = 64 * k, min(self.M, 64 * k + 64)
            gen = np.random.Generator(np.random.Philox(key=self.seed, counter=[0, k, 1, 0]))
            nz = gen.standard_normal((64, self.N))
            a, b = max(g0, r0), min(g1, r1)
            for i in range(a, b):
                d2 = (q[:, 0] - p[i, 0]) ** 2 + (q[:, 1] - p[i, 1]) ** 2
                out[i - r0] = np.exp(-d2 * inv_l2) + self.noise * nz[i - g0]

        groups = range(r0 // 64, (r1 + 63) // 64)
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(group, groups))
        return out

    def dense(self) -> np.ndarray:
        return self.rows(0, self.M)


# The paper's GEMV shapes (Sec. 5.1, Fig. results_throughput): (name, M, N)
PAPER_SHAPES = (("wide", 378, 256000), ("tall", 256000, 378), ("square", 10000, 10000))


def gaussian_x(n_valid: int, order: int, seed: int, R: int = 1) -> np.ndarray:
    """FP64 x ~ N(0,1), shape (order, R), zero beyond n_valid; column r from Philox key seed+r."""
    X = np.zeros((order, R), dtype=np.float64)
    for r in range(R):
        gen = np.random.Generator(np.random.Philox(key=seed + r))
        X[:n_valid, r] = gen.standard_normal(n_valid)
    return X


def serpentine_centres(steps: int, fields_per_side: int = 10, steps_per_field: int = 20) -> np.ndarray:
    """(steps, 2) spot centres in grid coordinates [-HALF, HALF]^2; the path repeats after one wafer."""
    side = 2 * HALF / fields_per_side
    out = np.empty((steps, 2))
    per_wafer = fields_per_side * fields_per_side * steps_per_field
    for k in range(steps):
        kk = k % per_wafer
        f, s = divmod(kk, steps_per_field)
        fr, fc = divmod(f, fields_per_side)
        if fr % 2 == 1:
            fc = fields_per_side - 1 - fc
        cx = -HALF + (fc + 0.5) * side
        cy0 = -HALF + fr * side
        t = (s + 0.5) / steps_per_field
        if f % 2 == 1:
            t = 1.0 - t
        out[k] = (cx, cy0 + t * side)
    return out


def heat_load(g: int, n_valid: int, order: int, centre, sigma_cells: float = 2.0) -> np.ndarray:
    """FP64 x[i] = exp(-|p_i - c|^2 / (2 sigma^2)), sigma in grid cells; zero beyond n_valid."""
    h = 2 * HALF / (g - 1)
    sigma = sigma_cells * h
    pts = grid_points(g, n_valid)
    x = np.zeros(order, dtype=np.float64)
    d2 = (pts[:, 0] - centre[0]) ** 2 + (pts[:, 1] - centre[1]) ** 2
    x[:n_valid] = np.exp(-d2 / (2 * sigma * sigma))
    return x


def heat_loads(g: int, n_valid: int, order: int, steps: int, sigma_cells: float = 2.0) -> np.ndarray:
    """(order, steps) FP64, column k = the heat load of control step k."""
    C = serpentine_centres(steps)
    X = np.empty((order, steps), dtype=np.float64)
    for k in range(steps):
        X[:, k] = heat_load(g, n_valid, order, C[k], sigma_cells)
    return X


# ------------------------------------------------------------------ configs
@dataclass(frozen=True)
class Config:
    name: str
    matrix: KernelMatrix
    rate: int
    steps: int = 1
    R: int = 1
    notes: str = ""
    extra: dict = field(default_factory=dict)


def config(idx: int) -> Config:
    """The five measurement workloads (1: small plain GEMV, 2: control loop, 3: precision
    sweep, 4: batched uneven instances, 5: serving)."""
    seed = SEED_BASE + idx
    if idx == 1:
        return Config("plain-4096-rate16", KernelMatrix(4096, 64, 4096, 0.1, seed), rate=16)
    if idx == 2:
        return Config("control-loop-32768-rate16", KernelMatrix(32768, 181, 181 * 181, 0.05, seed), rate=16,
                      steps=2000, notes="s_{k+1} = 0.99 s_k + A x_k, serpentine heat load")
    if idx == 3:
        return Config("precision-sweep-32768", KernelMatrix(32768, 181, 181 * 181, 0.05, SEED_BASE + 2), rate=16,
                      extra={"formats": ["zfp8", "zfp12", "zfp16", "bf16", "fp16", "fp8e4m3"], "R": [1, 32]})
    if idx == 4:
        return Config("batched-64-uneven-rate12", KernelMatrix(0, 0, 0, 0.05, seed), rate=12,
                      extra={"instances": batched_instances()})
    if idx == 5:
        return Config("serving-8-models-rate8", KernelMatrix(0, 0, 0, 0.05, seed), rate=8,
                      extra={"orders": [8192, 16384, 32768, 49152, 65536, 65536, 32768, 16384],
                             "arrival_hz": 2000.0, "deadline_us": 500.0})
    raise ValueError(idx)


def batched_instances(count: int = 64, seed: int = 4, lo: int = 2048, hi: int = 16384):
    """[(N_m, R_m)]: N_m = round(exp(U[ln lo, ln hi])), R_m uniform over {1, 4, 8, 32}."""
    gen = np.random.Generator(np.random.Philox(key=seed))
    ns = np.rint(np.exp(gen.uniform(math.log(lo), math.log(hi), size=count))).astype(int)
    rs = gen.choice(np.array([1, 4, 8, 32]), size=count)
    return [(int(n), int(r)) for n, r in zip(ns, rs)]


def instance_matrix(N: int, length: float = 0.05, seed: int = SEED_BASE + 4) -> KernelMatrix:
    g = int(math.ceil(math.sqrt(N)))
    return KernelMatrix(N, g, N, length, seed + N)


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream: seeded exponential inter-arrival gaps."""
    gen = np.random.Generator(np.random.Philox(key=seed))
    n = int(rate_hz * duration_s * 1.5) + 16
    t = np.cumsum(gen.exponential(1.0 / rate_hz, size=n))
    return t[t < duration_s]
