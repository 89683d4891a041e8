"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *generates* discrete SDF samples (p_i, s_i) and query points.
It contains none of the consistent-interpolation arithmetic: both the FP64
oracle and the CUDA library consume its arrays, and neither is imported here.

The paper evaluates on meshes (TetWild shapes, artist assets) that are not
available; analytic shapes sampled on node-aligned grids over [-1, 1]^3 stand
in for them (grid sizes 16^3 .. 128^3 match the paper's 12^3 .. 50^3 scale and
above).  Every generator is deterministic in its seed
(``numpy.random.default_rng(seed)``, seed = workload index * 1000 + shape).

Index order of a grid is x-major: sample (ix, iy, iz) has linear index
``(ix * N + iy) * N + iz`` and position ``(g[ix], g[iy], g[iz])`` with
``g = numpy.linspace(-1, 1, N)``.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# --------------------------------------------------------------------------
# analytic signed distance functions (FP64, numpy)
# --------------------------------------------------------------------------


def sdf_sphere(p: np.ndarray, c, r: float) -> np.ndarray:
    d = p - np.asarray(c, dtype=np.float64)
    return np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]) - r


def sdf_box(p: np.ndarray, c, half) -> np.ndarray:
    """Exact distance to an axis-aligned box (negative inside)."""
    q = np.abs(p - np.asarray(c, dtype=np.float64)) - np.asarray(half, dtype=np.float64)
    qp = np.maximum(q, 0.0)
    outside = np.sqrt(qp[:, 0] ** 2 + qp[:, 1] ** 2 + qp[:, 2] ** 2)
    inside = np.minimum(np.max(q, axis=1), 0.0)
    return outside + inside


def sdf_torus(p: np.ndarray, c, R: float, r: float, axis: int = 2) -> np.ndarray:
    """Exact distance to a torus with major radius R, minor radius r."""
    d = p - np.asarray(c, dtype=np.float64)
    a = [0, 1, 2]
    a.remove(axis)
    ring = np.sqrt(d[:, a[0]] ** 2 + d[:, a[1]] ** 2) - R
    return np.sqrt(ring * ring + d[:, axis] ** 2) - r


# --------------------------------------------------------------------------
# grids and workload containers
# --------------------------------------------------------------------------


def grid_points(N: int) -> np.ndarray:
    """Node-aligned N^3 grid on [-1,1]^3, x-major, shape (N^3, 3) FP64."""
    g = np.linspace(-1.0, 1.0, N)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def grid_spacing(N: int) -> float:
    return 2.0 / (N - 1)


@dataclasses.dataclass
class Workload:
    name: str
    p: np.ndarray          # (n, 3) float64 sample positions
    s: np.ndarray          # (n,) float64 signed distance samples
    tau: int               # icosphere subdivision depth
    h: float               # sample spacing (grid) or 2 / n^(1/3) (scattered)
    queries: object        # callable () -> (m, 3) array, or None
    m: int                 # number of query points
    query_dtype: str       # "f64" or "f32"

    @property
    def n(self) -> int:
        return int(self.s.shape[0])

    def make_queries(self) -> np.ndarray:
        return self.queries()


# --------------------------------------------------------------------------
# the five workload families
# --------------------------------------------------------------------------


def sphere_grid(N: int = 16, up: int = 2, tau: int = 2) -> Workload:
    """16^3 grid of the exact SDF of a sphere r=0.6 at (0.05,-0.03,0.02);
    queries on the 2x upsampled node grid (31^3)."""
    p = grid_points(N)
    s = sdf_sphere(p, (0.05, -0.03, 0.02), 0.6)
    Nq = up * (N - 1) + 1
    return Workload(f"sphere_grid{N}", p, s, tau, grid_spacing(N),
                    lambda: grid_points(Nq), Nq ** 3, "f64")


def union_field(seed: int = 2000):
    """The field of union_grid: pointwise min of 6 spheres (r ~ U[0.15,0.4])
    and 4 axis-aligned boxes (half-extents ~ U[0.1,0.3]^3), centres
    ~ U[-0.6,0.6]^3, as a function of (m, 3) points.

    The min of exact primitive SDFs is exact outside the union and a lower
    bound of the distance inside overlaps of primitives."""
    rng = np.random.default_rng(seed)
    sph = [(rng.uniform(-0.6, 0.6, 3), rng.uniform(0.15, 0.4)) for _ in range(6)]
    box = [(rng.uniform(-0.6, 0.6, 3), rng.uniform(0.1, 0.3, 3)) for _ in range(4)]

    def field(p: np.ndarray) -> np.ndarray:
        s = np.full(p.shape[0], np.inf)
        for c, r in sph:
            s = np.minimum(s, sdf_sphere(p, c, r))
        for c, b in box:
            s = np.minimum(s, sdf_box(p, c, b))
        return s
    return field


def union_grid(N: int = 64, up: int = 4, tau: int = 3, seed: int = 2000) -> Workload:
    """N^3 grid samples of union_field(seed); queries on the up-times
    upsampled node grid."""
    p = grid_points(N)
    s = union_field(seed)(p)
    Nq = up * (N - 1) + 1
    return Workload(f"union_grid{N}", p, s, tau, grid_spacing(N),
                    lambda: grid_points(Nq), Nq ** 3, "f64")


def _random_primitive(rng, kinds=("sphere", "box", "torus")):
    kind = kinds[int(rng.integers(len(kinds)))]
    c = rng.uniform(-0.55, 0.55, 3)
    if kind == "sphere":
        r = rng.uniform(0.12, 0.35)
        return lambda P, c=c, r=r: sdf_sphere(P, c, r)
    if kind == "box":
        b = rng.uniform(0.08, 0.28, 3)
        return lambda P, c=c, b=b: sdf_box(P, c, b)
    R = rng.uniform(0.15, 0.35)
    r = rng.uniform(0.04, 0.1)
    ax = int(rng.integers(3))
    return lambda P, c=c, R=R, r=r, ax=ax: sdf_torus(P, c, R, r, ax)


def csg_pseudo_grid(N: int = 128, tau: int = 3, seed: int = 3000,
                    n_prims: int = 12, noise_frac: float = 0.05) -> Workload:
    """Pseudo-SDF: a CSG tree over seeded spheres/boxes/tori -- pairs of
    primitives combined by union (min), difference (max(a, -b)) or
    intersection with a dilated partner (max(a, b - 0.15)), and the pairs
    joined by union -- plus N(0, 0.1 h) noise on a seeded 5% of the samples.
    max/min combinations are not Euclidean distances, hence "pseudo"."""
    rng = np.random.default_rng(seed)
    prims = [_random_primitive(rng) for _ in range(n_prims)]
    p = grid_points(N)
    vals = [f(p) for f in prims]
    acc = None
    for j in range(0, n_prims - 1, 2):
        a, b = vals[j], vals[j + 1]
        op = rng.choice(["union", "diff", "inter"])
        if op == "union":
            blob = np.minimum(a, b)
        elif op == "diff":
            blob = np.maximum(a, -b)
        else:
            blob = np.maximum(a, b - 0.15)
        if not np.any(blob < 0):            # an empty pair falls back to its union
            blob = np.minimum(a, b)
        acc = blob if acc is None else np.minimum(acc, blob)
    h = grid_spacing(N)
    s = acc.copy()
    idx = rng.choice(s.shape[0], size=int(noise_frac * s.shape[0]), replace=False)
    s[idx] += rng.normal(0.0, 0.1 * h, size=idx.shape[0])
    return Workload(f"csg_pseudo_grid{N}", p, s, tau, h, None, 0, "f64")


def torus_grid(N: int = 128, m: int = 1 << 22, tau: int = 3, seed: int = 4000) -> Workload:
    """Grid samples of a seeded torus (R=0.5, r=0.2); m uniform FP32 queries."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-0.05, 0.05, 3)
    p = grid_points(N)
    s = sdf_torus(p, c, 0.5, 0.2, 2)

    def q():
        r2 = np.random.default_rng(seed + 1)
        return r2.uniform(-1.0, 1.0, size=(m, 3)).astype(np.float32)

    return Workload(f"torus_grid{N}", p, s, tau, grid_spacing(N), q, m, "f32")


def union_of_primitives(rng, k: int):
    prims = [_random_primitive(rng) for _ in range(k)]

    def f(P):
        out = prims[0](P)
        for g in prims[1:]:
            out = np.minimum(out, g(P))
        return out
    return f


def batch_shape(index: int, tau: int = 3, base_seed: int = 5000,
                scale: float = 1.0) -> Workload:
    """Shape ``index`` of the 256-shape batch: even indices are grids of side
    U{16..96} (2x upsampled queries), odd indices are scattered samples
    (U[10k,200k] uniform points with exact values, 8 n uniform queries).
    ``scale`` < 1 shrinks sizes for small test runs."""
    rng = np.random.default_rng(base_seed + index)
    f = union_of_primitives(rng, int(rng.integers(1, 9)))
    if index % 2 == 0:
        N = int(rng.integers(16, 97))
        N = max(4, int(round(N * scale)))
        p = grid_points(N)
        s = f(p)
        Nq = 2 * (N - 1) + 1
        return Workload(f"batch{index}_grid{N}", p, s, tau, grid_spacing(N),
                        lambda: grid_points(Nq), Nq ** 3, "f64")
    n = int(rng.integers(10_000, 200_001))
    n = max(64, int(round(n * scale)))
    p = rng.uniform(-1.0, 1.0, size=(n, 3))
    s = f(p)
    mq = 8 * n
    qseed = base_seed + 100_000 + index

    def q():
        return np.random.default_rng(qseed).uniform(-1.0, 1.0, size=(mq, 3))
    return Workload(f"batch{index}_scatter{n}", p, s, tau, 2.0 / n ** (1 / 3), q, mq, "f64")


def tiny_random(n: int, seed: int, valid: bool = True, spread: float = 0.5):
    """Tiny random discrete SDF for brute-force pins: samples of the exact
    SDF of one or two random spheres at random points (so the input is valid
    by construction when ``valid``), else random values."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(-spread, spread, size=(n, 3))
    if valid:
        c1 = rng.uniform(-0.2, 0.2, 3)
        r1 = rng.uniform(0.15, 0.35)
        c2 = rng.uniform(-0.2, 0.2, 3)
        r2 = rng.uniform(0.1, 0.3)
        s = np.minimum(sdf_sphere(p, c1, r1), sdf_sphere(p, c2, r2))
        # union of two spheres: exact outside; inside use the (valid,
        # conservative) min so that no sphere penetrates the surface.
    else:
        s = rng.uniform(-0.3, 0.3, size=n)
    return p, s


WORKLOADS = {
    "sphere16": sphere_grid,
    "union64": union_grid,
    "csg128": csg_pseudo_grid,
    "torus128": torus_grid,
}
