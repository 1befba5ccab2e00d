"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the smoother: only a counter-based random
stream (splitmix64, Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) and the recipes that turn it into macro-tetrahedra,
right-hand sides, macro-meshes and request arrival times.  Every workload in
this repository is drawn from here so that the oracle and the CUDA path see
identical inputs.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first n outputs of splitmix64 started from `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniform in [lo, hi): the top 53 bits of each splitmix64 output."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


REFERENCE_TET = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def macro_tet(seed: int, amp: float = 0.1) -> np.ndarray:
    """Reference tetrahedron with each of its 12 coordinates moved by U(-amp, amp)."""
    return REFERENCE_TET + uniform(seed, 12, -amp, amp).reshape(4, 3)


def num_nodes(level: int) -> int:
    """Points of the logical grid of a macro-tetrahedron at this level: C(N+3, 3)."""
    n = 2 ** level
    return (n + 1) * (n + 2) * (n + 3) // 6


def rhs(level: int, seed: int) -> np.ndarray:
    """Right-hand side over the full logical grid, every entry U(-1, 1)
    (the smoother reads only the interior entries)."""
    return uniform(seed, num_nodes(level), -1.0, 1.0)


def boundary_data(level: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """A full-grid vector U(-scale, scale), used as Dirichlet data / start vector."""
    return uniform(seed, num_nodes(level), -scale, scale)


def interior_error(level: int, seed: int) -> np.ndarray:
    """A full-grid start error: U(-1, 1) on the interior points, 0 on the
    boundary (lexicographic order, z slowest, then y, then x)."""
    n = 2 ** level
    v = uniform(seed, num_nodes(level), -1.0, 1.0)
    k = 0
    for z in range(n + 1):
        for y in range(n + 1 - z):
            m = n + 1 - z - y  # points of the row, x = 0 .. n - z - y
            row = v[k:k + m]
            row[0] = 0.0
            row[m - 1] = 0.0
            if y == 0 or z == 0:
                row[:] = 0.0
            k += m
    return v


def _aspect(P: np.ndarray) -> float:
    """Circumradius / (3 * inradius); 1 for a regular tetrahedron."""
    a, b, c, d = P
    M = np.array([b - a, c - a, d - a])
    vol = abs(np.linalg.det(M)) / 6.0
    faces = [(a, b, c), (a, b, d), (a, c, d), (b, c, d)]
    area = sum(0.5 * np.linalg.norm(np.cross(q - p, r - p)) for p, q, r in faces)
    inr = 3.0 * vol / area
    rhs_ = 0.5 * np.array([b @ b - a @ a, c @ c - a @ a, d @ d - a @ a])
    cc = np.linalg.solve(M, rhs_)
    R = np.linalg.norm(cc - a)
    return R / (3.0 * inr)


def macro_mesh(seed: int, n_tets: int = 256, cubes=(4, 4, 3), jitter: float = 0.15,
               max_aspect: float = 3.0) -> list:
    """Macro-tetrahedra of a jittered structured mesh: a grid of unit cubes, six
    Kuhn tetrahedra per cube, interior vertices moved by U(-jitter, jitter);
    tetrahedra with aspect ratio above max_aspect are dropped; the first
    n_tets are returned as (4,3) arrays."""
    nx, ny, nz = cubes
    verts = np.array([[i, j, k] for k in range(nz + 1) for j in range(ny + 1) for i in range(nx + 1)], float)
    interior = np.all((verts > 0) & (verts < np.array([nx, ny, nz])), axis=1)
    u = uniform(seed, verts.size, -jitter, jitter).reshape(-1, 3)
    verts = verts + u * interior[:, None]

    def vid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i

    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    unit = np.eye(3, dtype=int)
    out = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for p in perms:
                    q = np.array([i, j, k])
                    path = [q, q + unit[p[0]], q + unit[p[0]] + unit[p[1]], q + 1]
                    P = np.array([verts[vid(*v)] for v in path])
                    if _aspect(P) <= max_aspect:
                        out.append(P)
    return out[:n_tets]


def batch_levels(seed: int, n: int, lo: int = 5, hi: int = 8) -> np.ndarray:
    """Levels drawn uniformly from lo..hi."""
    return lo + np.minimum((uniform(seed, n) * (hi - lo + 1)).astype(int), hi - lo)


def poisson_arrivals(seed: int, n: int, mean_gap_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    gaps = -np.log1p(-uniform(seed, n)) * mean_gap_s
    return np.cumsum(gaps)
