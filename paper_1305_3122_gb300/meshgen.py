"""Seeded synthetic inputs: jittered, node-permuted triangulations of the unit square (and
tetrahedralisations of the unit cube).

This module generates *inputs only* (vertex coordinates, connectivity, vertex weights,
upstream gradients, sample indices). It holds none of the assembly arithmetic, so it can
feed both the CUDA path and the CPU oracle with identical arrays.

Layout follows the mesh description of Section 2 of the paper (the table of ``q``, ``me``):
``q`` is ``[2, nq]`` float64 (row 0 = x, row 1 = y) and ``me`` is ``[3, nme]`` int32 with
0-based vertex ids (the paper is 1-based), every triangle counter-clockwise.

Random numbers come from one counter-based generator: the output sequence of splitmix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
started at a key derived from ``(seed, stream)``. Value ``i`` of a stream is
``mix(key + (i + 1) * 0x9E3779B97F4A7C15)`` with the splitmix64 finaliser ``mix``; a uniform
double in [0, 1) is the top 53 bits times 2**-53. Because every value depends only on its
counter, the arrays are identical on every machine and independent of numpy's own RNGs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids (one per purpose, so that changing one draw never shifts another)
S_JITTER_X, S_JITTER_Y, S_PERM, S_WNOISE, S_SIZES, S_GRAD_S, S_GRAD_M, S_SAMPLE, S_JITTER_Z, S_DIAG = range(1, 11)
S_DISK_A, S_DISK_B = range(11, 13)

# seeds of the standard workloads: SEED_BASE + 1 mass on 64 x 64 cells, + 2 stiffness and weighted
# mass on 2048 x 2048, + 3 elasticity on 1024 x 1024, + 4 the batch of 256 meshes, + 5 the
# differentiated assembly on 1024 x 1024
SEED_BASE = 13053122


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Values ``offset .. offset+n-1`` of the splitmix64 sequence of ``(seed, stream)``."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([(seed * 0x100000001B3 + stream * 0x632BE59BD9B4E019) & (2**64 - 1)],
                            dtype=np.uint64))[0]
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(key + ctr * _GAMMA)


def stream_uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform float64 in [0, 1) with 53 random bits."""
    return (stream_u64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def stream_normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normal float64 by the Box-Muller transform on pairs of uniforms."""
    m = (n + 1) // 2
    u = stream_uniform(seed, stream, 2 * m)
    u1 = 1.0 - u[0::2]                      # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n]


def random_permutation(seed: int, stream: int, n: int) -> np.ndarray:
    """A uniformly random permutation of ``0..n-1`` (ranks of 64-bit random keys, ties by index)."""
    keys = stream_u64(seed, stream, n)
    order = np.argsort(keys, kind="stable")
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n, dtype=np.int64)
    return rank


@dataclass
class Mesh:
    q: np.ndarray      # [2, nq] float64
    me: np.ndarray     # [3, nme] int32, 0-based, counter-clockwise
    N: int             # cells per side

    @property
    def nq(self) -> int:
        return self.q.shape[1]

    @property
    def nme(self) -> int:
        return self.me.shape[1]


def square_mesh(N: int, seed: int, jitter: float = 0.2, permute: bool = True, random_diagonals: bool = False,
                hole: bool = False, stretch: float = 1.0) -> Mesh:
    """Unit square cut into N x N cells, each cell split into two triangles.

    Node (i, j) has id ``j*(N+1)+i`` at ``(i/N, j/N)`` before the permutation. Cell (i, j) with
    corners a=(i,j), b=(i+1,j), c=(i+1,j+1), d=(i,j+1) gives triangles (a,b,c) and (a,c,d), both
    counter-clockwise, numbered ``2*(j*N+i)`` and ``2*(j*N+i)+1`` (cell-major element order).
    Interior nodes move by independent offsets drawn uniformly from [-jitter*h, jitter*h) in x
    and in y (h = 1/N); boundary nodes stay put, so the domain stays the unit square. With
    jitter <= 0.2 no triangle can invert. Then the node ids are randomly permuted (element order
    and the local vertex order of each triangle are kept).

    Unstructured variants (the method applies to any triangulation):

    - ``random_diagonals``: each cell takes the diagonal a-c (as above) or b-d, with probability
      1/2 each from the stream ``S_DIAG``; the b-d split gives (a,b,d) and (b,c,d), also
      counter-clockwise. An interior vertex then lies in 4 to 8 triangles (4 plus the number of
      its four cells whose diagonal ends at it), so closed fans of every size 4..8 occur, and
      boundary vertices have open fans of 1 to 4 triangles. Every triangle is still a right
      isosceles triangle of legs h before the jitter, so none can invert for jitter <= 0.2.
    - ``hole`` (needs N >= 8): the cells with N/4 <= i, j < N/2 are removed (a square hole; the
      nodes strictly inside it belong to no triangle and keep their ids, giving empty rows), and
      so are the cells (p+1, p) and (p, p+1) with p = (3N)//4, so that node (p+1, p+1) belongs
      only to the cells (p, p) and (p+1, p+1): two fans that touch at one vertex.
    - ``stretch``: x is multiplied by this factor after the jitter (the domain becomes
      [0, stretch] x [0, 1]); triangles keep their orientation but get angles far from 45/90
      degrees (about 8 to 165 degrees for stretch 7).
    """
    if N < 1:
        raise ValueError("N must be >= 1")
    if hole and N < 8:
        raise ValueError("hole needs N >= 8")
    n1 = N + 1
    h = 1.0 / N
    nq = n1 * n1
    ii = np.tile(np.arange(n1), n1)
    jj = np.repeat(np.arange(n1), n1)
    x = ii * h
    y = jj * h
    interior = (ii > 0) & (ii < N) & (jj > 0) & (jj < N)
    if jitter != 0.0:
        jx = (2.0 * stream_uniform(seed, S_JITTER_X, nq) - 1.0) * (jitter * h)
        jy = (2.0 * stream_uniform(seed, S_JITTER_Y, nq) - 1.0) * (jitter * h)
        x = np.where(interior, x + jx, x)
        y = np.where(interior, y + jy, y)
    ci = np.tile(np.arange(N), N)
    cj = np.repeat(np.arange(N), N)
    a = cj * n1 + ci
    b = a + 1
    c = a + n1 + 1
    d = a + n1
    me = np.empty((3, 2 * N * N), dtype=np.int64)
    me[0, 0::2], me[1, 0::2], me[2, 0::2] = a, b, c
    me[0, 1::2], me[1, 1::2], me[2, 1::2] = a, c, d
    if random_diagonals:
        flip = stream_uniform(seed, S_DIAG, N * N) >= 0.5
        me[0, 0::2] = np.where(flip, a, me[0, 0::2])
        me[1, 0::2] = np.where(flip, b, me[1, 0::2])
        me[2, 0::2] = np.where(flip, d, me[2, 0::2])
        me[0, 1::2] = np.where(flip, b, me[0, 1::2])
        me[1, 1::2] = np.where(flip, c, me[1, 1::2])
        me[2, 1::2] = np.where(flip, d, me[2, 1::2])
    if hole:
        lo, hi, p = N // 4, N // 2, (3 * N) // 4
        gone = (ci >= lo) & (ci < hi) & (cj >= lo) & (cj < hi)
        gone |= ((ci == p + 1) & (cj == p)) | ((ci == p) & (cj == p + 1))
        me = me[:, np.repeat(~gone, 2)]
    x = x * stretch
    q = np.stack([x, y]).astype(np.float64)
    if permute:
        newid = random_permutation(seed, S_PERM, nq)
        qp = np.empty_like(q)
        qp[:, newid] = q
        q = qp
        me = newid[me]
    return Mesh(q=np.ascontiguousarray(q), me=np.ascontiguousarray(me.astype(np.int32)), N=N)


def cube_mesh(N: int, seed: int, jitter: float = 0.05, permute: bool = True) -> Mesh:
    """Unit cube cut into N^3 cells, each cell split into six tetrahedra around its main diagonal.

    Node (i, j, k) has id ``(k*(N+1)+j)*(N+1)+i`` at ``(i/N, j/N, k/N)`` before the permutation.
    Cell (i, j, k) with corner v0 = (i, j, k) gives, for each order (d1, d2, d3) of the three
    axes, the tetrahedron (v0, v0+e_d1, v0+e_d1+e_d2, v0+e_d1+e_d2+e_d3), its last two vertices
    exchanged when the order is odd so that every one has positive signed volume
    det[p1-p0 | p2-p0 | p3-p0]; elements are cell-major, six per cell. Interior nodes move by
    independent offsets drawn uniformly from [-jitter*h, jitter*h) per coordinate; boundary nodes
    stay put. Then the node ids are randomly permuted, as for ``square_mesh``. ``q`` is [3, nq]
    float64 and ``me`` [4, nme] int32."""
    if N < 1:
        raise ValueError("N must be >= 1")
    n1 = N + 1
    h = 1.0 / N
    nq = n1 ** 3
    ii = np.tile(np.arange(n1), n1 * n1)
    jj = np.tile(np.repeat(np.arange(n1), n1), n1)
    kk = np.repeat(np.arange(n1), n1 * n1)
    x, y, z = ii * h, jj * h, kk * h
    interior = (ii > 0) & (ii < N) & (jj > 0) & (jj < N) & (kk > 0) & (kk < N)
    if jitter != 0.0:
        x = np.where(interior, x + (2.0 * stream_uniform(seed, S_JITTER_X, nq) - 1.0) * (jitter * h), x)
        y = np.where(interior, y + (2.0 * stream_uniform(seed, S_JITTER_Y, nq) - 1.0) * (jitter * h), y)
        z = np.where(interior, z + (2.0 * stream_uniform(seed, S_JITTER_Z, nq) - 1.0) * (jitter * h), z)
    ci = np.tile(np.arange(N), N * N)
    cj = np.tile(np.repeat(np.arange(N), N), N)
    ck = np.repeat(np.arange(N), N * N)
    v0 = (ck * n1 + cj) * n1 + ci
    step = (1, n1, n1 * n1)                      # id offset of a unit move along x, y, z
    orders = ((0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1), (2, 1, 0), (1, 0, 2))   # three even, three odd
    me = np.empty((4, 6 * N ** 3), dtype=np.int64)
    for t, (d1, d2, d3) in enumerate(orders):
        p1 = v0 + step[d1]
        p2 = p1 + step[d2]
        p3 = p2 + step[d3]
        if t >= 3:
            p2, p3 = p3, p2
        me[0, t::6], me[1, t::6], me[2, t::6], me[3, t::6] = v0, p1, p2, p3
    q = np.stack([x, y, z]).astype(np.float64)
    if permute:
        newid = random_permutation(seed, S_PERM, nq)
        qp = np.empty_like(q)
        qp[:, newid] = q
        q = qp
        me = newid[me]
    return Mesh(q=np.ascontiguousarray(q), me=np.ascontiguousarray(me.astype(np.int32)), N=N)


def disk_mesh(n: int, seed: int, points: str = "poisson", permute: bool = True) -> Mesh:
    """The unit disk, the paper's test domain (its meshes come from FreeFEM++'s Delaunay mesher),
    triangulated by Delaunay with about ``n`` vertices.

    Points: ``nb = round(2 pi / h)`` on the unit circle at equal angles, where
    ``h = sqrt(2 pi / (sqrt(3) n))`` is the spacing of a hexagonal lattice of ``n`` points in the
    disk, and interior points:
      - ``points="poisson"``: ``n - nb`` points uniform in the disk of radius ``1 - h/2``
        (valences 3 to about 20, about 4% of the vertices in more than 8 triangles);
      - ``points="lattice"``: the hexagonal lattice of spacing ``h`` inside radius ``1 - h/2``,
        each point moved by up to ``0.15 h`` per coordinate (valence 6 almost everywhere, like a
        quality mesher's output).
    Triangulation by ``scipy.spatial.Delaunay`` (Qhull), every triangle made counter-clockwise.
    Triangles are put in scanline order of their centroids (rows of height h, then x), since a
    mesher's output has that kind of locality, and the node ids are randomly permuted unless
    ``permute=False``. ``N`` of the result is 0 (no cell grid)."""
    from scipy.spatial import Delaunay

    if n < 8:
        raise ValueError("n must be >= 8")
    h = math.sqrt(2.0 * math.pi / (math.sqrt(3.0) * n))
    nb = max(8, int(round(2.0 * math.pi / h)))
    t = 2.0 * math.pi * np.arange(nb) / nb
    bnd = np.stack([np.cos(t), np.sin(t)], axis=1)
    rmax = 1.0 - 0.5 * h
    if points == "poisson":
        k = max(n - nb, 1)
        r = rmax * np.sqrt(stream_uniform(seed, S_DISK_A, k))
        a = 2.0 * math.pi * stream_uniform(seed, S_DISK_B, k)
        inner = np.stack([r * np.cos(a), r * np.sin(a)], axis=1)
    elif points == "lattice":
        dy = h * math.sqrt(3.0) / 2.0
        rows = []
        for j in range(-int(1.0 / dy) - 1, int(1.0 / dy) + 2):
            xs = np.arange(-int(1.0 / h) - 1, int(1.0 / h) + 2) * h + (0.5 * h if j % 2 else 0.0)
            rows.append(np.stack([xs, np.full_like(xs, j * dy)], axis=1))
        inner = np.concatenate(rows)
        inner = inner[(inner ** 2).sum(axis=1) < rmax * rmax]
        k = inner.shape[0]
        inner = inner + (2.0 * np.stack([stream_uniform(seed, S_DISK_A, k), stream_uniform(seed, S_DISK_B, k)], axis=1)
                         - 1.0) * (0.15 * h)
    else:
        raise ValueError("points must be 'poisson' or 'lattice'")
    P = np.concatenate([bnd, inner])
    tri = np.asarray(Delaunay(P).simplices, dtype=np.int64)
    a, b, c = P[tri[:, 0]], P[tri[:, 1]], P[tri[:, 2]]
    d = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1])
    if not (np.abs(d) > 1e-12 * h * h).all():
        raise RuntimeError("degenerate triangle in the Delaunay triangulation")
    flip = d < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    cen = (a + b + c) / 3.0
    order = np.lexsort((cen[:, 0], np.floor((cen[:, 1] + 1.0) / h)))
    tri = tri[order]
    nq = P.shape[0]
    if permute:
        perm = random_permutation(seed, S_PERM, nq)
        q = np.empty((2, nq))
        q[:, perm] = P.T
        me = perm[tri.T]
    else:
        q = P.T.copy()
        me = tri.T
    return Mesh(q=np.ascontiguousarray(q), me=np.ascontiguousarray(me.astype(np.int32)), N=0)


def vertex_weights3(mesh: Mesh, seed: int) -> np.ndarray:
    """w_i = 1 + 0.5*sin(2*pi*x_i)*cos(2*pi*y_i)*cos(2*pi*z_i) + U(0, 0.1) at the vertices of a
    tetrahedral mesh."""
    x, y, z = mesh.q
    noise = 0.1 * stream_uniform(seed, S_WNOISE, mesh.nq)
    return 1.0 + 0.5 * np.sin(2.0 * math.pi * x) * np.cos(2.0 * math.pi * y) * np.cos(2.0 * math.pi * z) + noise


def vertex_weights(mesh: Mesh, seed: int) -> np.ndarray:
    """w_i = 1 + 0.5*sin(2*pi*x_i)*cos(2*pi*y_i) + U(0, 0.1), sampled at the (jittered) vertices."""
    x, y = mesh.q
    noise = 0.1 * stream_uniform(seed, S_WNOISE, mesh.nq)
    return 1.0 + 0.5 * np.sin(2.0 * math.pi * x) * np.cos(2.0 * math.pi * y) + noise


def batch_sizes(seed: int, count: int = 256, lo: int = 16, hi: int = 512) -> np.ndarray:
    """Cells per side of each mesh of a batch: round(exp(U(ln lo, ln hi)))."""
    u = stream_uniform(seed, S_SIZES, count)
    n = np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return np.clip(n, lo, hi)


def batch_meshes(seed: int, count: int = 256, lo: int = 16, hi: int = 512) -> list[Mesh]:
    """``count`` independent jittered, permuted meshes; mesh m uses seed*1000003 + m."""
    return [square_mesh(int(n), seed * 1000003 + m) for m, n in enumerate(batch_sizes(seed, count, lo, hi))]


def upstream_gradients(seed: int, nnz: int) -> tuple[np.ndarray, np.ndarray]:
    """G_S, G_M ~ N(0, 1), one value per stored non-zero of S and of M^[w]."""
    return stream_normal(seed, S_GRAD_S, nnz), stream_normal(seed, S_GRAD_M, nnz)


def sample_indices(seed: int, count: int, upper: int) -> np.ndarray:
    """``count`` indices drawn uniformly from [0, upper) (with replacement)."""
    u = stream_u64(seed, S_SAMPLE, count)
    return (u % np.uint64(upper)).astype(np.int64)
