"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the stencil method itself: it only draws random
fields, samples manufactured right-hand sides and lays out patch lattices and request
streams.  Both the CPU oracle and the GPU library receive exactly the arrays made here.

Random numbers come from numpy's Philox bit generator keyed by the seed, whose stream
is fixed across platforms, so the x86 and Arm hosts produce identical bits.
Arrays are float64, C-contiguous, x fastest: (nz+1, ny+1, nx+1) in 3D, (ny+1, nx+1) in 2D.
"""
import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def grid_shape(dim: int, n) -> tuple:
    """Vertex-array shape for cells n (int or per-axis tuple x, y[, z])."""
    if isinstance(n, (int, np.integer)):
        n = (int(n),) * dim
    if dim == 3:
        return (n[2] + 1, n[1] + 1, n[0] + 1)
    return (n[1] + 1, n[0] + 1)


def zero_boundary(a: np.ndarray) -> np.ndarray:
    """Sets every boundary vertex (first/last index on any axis) to 0, in place."""
    for ax in range(a.ndim):
        idx = [slice(None)] * a.ndim
        idx[ax] = 0
        a[tuple(idx)] = 0.0
        idx[ax] = -1
        a[tuple(idx)] = 0.0
    return a


def uniform_field(shape, seed: int, zero_bc: bool = True, gen=None) -> np.ndarray:
    """u ~ U[-1, 1) per vertex (53-bit doubles), boundary zeroed unless zero_bc=False."""
    g = gen if gen is not None else rng(seed)
    a = g.random(size=int(np.prod(shape))).reshape(shape) * 2.0 - 1.0
    a = np.ascontiguousarray(a)
    if zero_bc:
        zero_boundary(a)
    return a


def coords(dim: int, n: int):
    """Vertex coordinates x_i = i/n on the unit square/cube, broadcastable (z, y, x)."""
    x = np.arange(n + 1, dtype=np.float64) / n
    if dim == 3:
        return x[None, None, :], x[None, :, None], x[:, None, None]
    return x[None, :], x[:, None]


def sin_rhs(dim: int, n: int, modes=(1, 1, 1)) -> np.ndarray:
    """Manufactured right-hand side f = -Laplace(u*) for u* = prod_a sin(m_a pi x_a):
    f = pi^2 (sum m_a^2) u*, sampled at the vertices (zero on the boundary)."""
    cs = coords(dim, n)
    m = list(modes)[:dim]
    ustar = np.ones(grid_shape(dim, n))
    for c, ma in zip(cs, m):
        ustar = ustar * np.sin(ma * math.pi * c)
    f = math.pi ** 2 * sum(ma * ma for ma in m) * ustar
    f = np.ascontiguousarray(f)
    zero_boundary(f)
    return f


def sin_solution(dim: int, n: int, modes=(1, 1, 1)) -> np.ndarray:
    """u* = prod_a sin(m_a pi x_a) at the vertices (the continuous solution)."""
    cs = coords(dim, n)
    u = np.ones(grid_shape(dim, n))
    for c, ma in zip(cs, list(modes)[:dim]):
        u = u * np.sin(ma * math.pi * c)
    u = np.ascontiguousarray(u)
    zero_boundary(u)
    return u


# ------------------------------------------------------------------ patch lattice

PATCH_EDGES = (8, 12, 16, 24, 32)


class PatchLattice:
    """A lat[0] x lat[1] x lat[2] lattice of cubic patches, patch p = Px + lat0*(Py +
    lat1*Pz), edge n_p drawn uniformly from PATCH_EDGES, packed one after another,
    each a dense (n_p+1)^3 array (h = 1/n_p).  u starts at 0, f ~ U[-1,1) per patch
    (boundary shell zero), drawn from the same seeded stream after the edges."""

    def __init__(self, lat=(16, 16, 16), seed: int = 2, edges=PATCH_EDGES, u_random=False):
        self.lat = np.array(lat, dtype=np.int32)
        npatch = int(np.prod(self.lat))
        g = rng(seed)
        self.np_sizes = np.asarray(g.choice(np.array(edges), size=npatch), dtype=np.int32)
        sizes = (self.np_sizes.astype(np.int64) + 1) ** 3
        self.offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        self.total = int(sizes.sum())
        self.f = np.empty(self.total)
        self.u = np.zeros(self.total)
        for p in range(npatch):
            n = int(self.np_sizes[p])
            sl = slice(int(self.offsets[p]), int(self.offsets[p]) + (n + 1) ** 3)
            self.f[sl] = uniform_field((n + 1,) * 3, 0, gen=g).ravel()
            if u_random:
                self.u[sl] = uniform_field((n + 1,) * 3, 0, gen=g).ravel()

    def view(self, a: np.ndarray, p: int) -> np.ndarray:
        n = int(self.np_sizes[p])
        o = int(self.offsets[p])
        return a[o:o + (n + 1) ** 3].reshape((n + 1,) * 3)

    def neighbours27(self) -> np.ndarray:
        """(npatch, 27) int32 table: entry (dx+1) + 3(dy+1) + 9(dz+1) is the patch at
        lattice offset (dx, dy, dz), -1 outside the lattice (the centre entry is p)."""
        lx, ly, lz = (int(v) for v in self.lat)
        npatch = lx * ly * lz
        nb = np.full((npatch, 27), -1, dtype=np.int32)
        for p in range(npatch):
            px, py, pz = p % lx, (p // lx) % ly, p // (lx * ly)
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        qx, qy, qz = px + dx, py + dy, pz + dz
                        if 0 <= qx < lx and 0 <= qy < ly and 0 <= qz < lz:
                            nb[p, (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] = qx + lx * (qy + ly * qz)
        return nb

    @property
    def interior_updates_per_sweep(self) -> int:
        return int(((self.np_sizes.astype(np.int64) - 1) ** 3).sum())


# ------------------------------------------------------------------ SplitMix64 fields

_GOLDEN = 0x9E3779B97F4A7C15


def splitmix_field(n: int, seed: int) -> np.ndarray:
    """(n+1)^3 field whose interior value at flat index i (x fastest) is the top 53
    bits of SplitMix64 (Steele, Lea & Flood, 2014) evaluated at counter
    seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64), mapped to U[-1, 1); boundary 0.
    The request server draws the same numbers on the device for seeded requests."""
    W = n + 1
    with np.errstate(over="ignore"):
        i = np.arange(W ** 3, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (i + np.uint64(1)) * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    v = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0
    v = np.ascontiguousarray(v.reshape(W, W, W))
    zero_boundary(v)
    return v


# ------------------------------------------------------------------ request stream

def request_stream(count: int, rate_per_s: float, seed: int = 3, edge_lo: int = 16,
                   edge_hi: int = 256, p_solve: float = 0.5):
    """A seeded stream of smoothing / solve requests: Poisson arrivals at rate_per_s,
    cubic edge log-uniform in [edge_lo, edge_hi] rounded to the nearest integer,
    kind SOLVE with probability p_solve (Bernoulli), else SMOOTH.
    Returns a list of dicts with arrival time (s), edge, kind, and a per-request seed
    for its right-hand side."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    edges = np.rint(np.exp(g.uniform(math.log(edge_lo), math.log(edge_hi), size=count)))
    kinds = g.random(size=count) < p_solve
    seeds = g.integers(0, 2 ** 31 - 1, size=count)
    return [dict(t=float(t[i]), edge=int(edges[i]), kind="solve" if kinds[i] else "smooth",
                 seed=int(seeds[i])) for i in range(count)]
