"""Seeded synthetic triangle meshes shaped like the paper's workloads.

The paper (Sec. 5) measures on scanned models (bunny, armadillo, dragon, ...)
and on a regular grid of 1,002,001 vertices (Sec. 5.2.2).  Those models are
not available here, so these generators stand in for them: flat jittered
grids (exact answer = Euclidean distance), subdivided spheres (exact answer =
great-circle distance), noisy tori, bumpy spheres and fractal heightfields.
Valence is 6 almost everywhere, as in the paper's degree histogram (App. B).

This module holds no part of the distance method itself: it only produces
vertex positions, faces and source indices, and it is shared by the CUDA
path's tests, the oracle's tests and the benchmark.

Every generator returns ``(V, F)`` with ``V`` a float64 array ``[n, 3]`` and
``F`` an int32 array ``[nf, 3]`` of 0-based vertex indices.
"""
from __future__ import annotations

import math

import numpy as np


def _grid_faces(nx: int, ny: int, wrap_x: bool = False, wrap_y: bool = False) -> np.ndarray:
    """Faces of an nx-by-ny vertex lattice, index = j*nx + i.

    Every quad (i,j),(i+1,j),(i+1,j+1),(i,j+1) is split along the same
    diagonal (i,j)-(i+1,j+1), so every interior vertex has valence 6.
    With wrap_x / wrap_y the lattice closes on itself (torus)."""
    qx = nx if wrap_x else nx - 1
    qy = ny if wrap_y else ny - 1
    i = np.arange(qx, dtype=np.int64)
    j = np.arange(qy, dtype=np.int64)
    I, J = np.meshgrid(i, j, indexing="xy")
    I = I.ravel()
    J = J.ravel()
    I1 = (I + 1) % nx
    J1 = (J + 1) % ny
    v00 = J * nx + I
    v10 = J * nx + I1
    v11 = J1 * nx + I1
    v01 = J1 * nx + I
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    F = np.empty((2 * t1.shape[0], 3), dtype=np.int64)
    F[0::2] = t1
    F[1::2] = t2
    return F.astype(np.int32)


def grid(nx: int, ny: int, jitter: float = 0.0, seed: int = 0,
         size: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Flat grid over [0,size]^2 at z=0; interior vertices are jittered
    uniformly by +-jitter grid spacings in x and y (boundary vertices stay
    on the boundary so the domain stays a square)."""
    hx = size / (nx - 1)
    hy = size / (ny - 1)
    xs = np.arange(nx) * hx
    ys = np.arange(ny) * hy
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    V = np.zeros((nx * ny, 3), dtype=np.float64)
    V[:, 0] = X.ravel()
    V[:, 1] = Y.ravel()
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        jx = rng.uniform(-jitter, jitter, size=(ny, nx)) * hx
        jy = rng.uniform(-jitter, jitter, size=(ny, nx)) * hy
        interior = np.zeros((ny, nx), dtype=bool)
        interior[1:-1, 1:-1] = True
        V[:, 0] += np.where(interior, jx, 0.0).ravel()
        V[:, 1] += np.where(interior, jy, 0.0).ravel()
    return V, _grid_faces(nx, ny)


def tri_lattice(nx: int, ny: int, h: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Equilateral triangle lattice (every triangle has side h)."""
    V = np.zeros((nx * ny, 3), dtype=np.float64)
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    V[:, 0] = (i + 0.5 * j).ravel() * h
    V[:, 1] = (j * math.sqrt(3.0) / 2.0).ravel() * h
    # with x = i + j/2 the short diagonal of each rhombus joins (i+1,j)-(i,j+1)
    qi, qj = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="xy")
    qi = qi.ravel().astype(np.int64)
    qj = qj.ravel().astype(np.int64)
    v00 = qj * nx + qi
    v10 = qj * nx + qi + 1
    v01 = (qj + 1) * nx + qi
    v11 = (qj + 1) * nx + qi + 1
    t1 = np.stack([v00, v10, v01], axis=1)
    t2 = np.stack([v10, v11, v01], axis=1)
    F = np.concatenate([t1, t2], axis=0).astype(np.int32)
    return V, F


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere: icosahedron, `level` times split every triangle into
    four at the edge midpoints and push the new vertices onto the sphere.
    Vertex count 10*4**level + 2."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    for _ in range(level):
        nv = V.shape[0]
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
        lo = np.minimum(e[:, 0], e[:, 1])
        hi = np.maximum(e[:, 0], e[:, 1])
        key = lo * nv + hi
        uk, inv = np.unique(key, return_inverse=True)
        ulo = uk // nv
        uhi = uk % nv
        mid = V[ulo] + V[uhi]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        V = np.concatenate([V, mid], axis=0)
        nf = F.shape[0]
        m01 = nv + inv[0:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:3 * nf]
        a, b, c = F[:, 0], F[:, 1], F[:, 2]
        F = np.concatenate([
            np.stack([a, m01, m20], 1), np.stack([b, m12, m01], 1),
            np.stack([c, m20, m12], 1), np.stack([m01, m12, m20], 1)], axis=0)
    return V, F.astype(np.int32)


def bumpy_icosphere(level: int, n_bumps: int = 64, amplitude: float = 0.05,
                    width: float = 0.1, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Icosphere with Gaussian radial bumps:
    radius(p) = 1 + amplitude * sum_i exp(-|p - c_i|^2 / (2 width^2)),
    c_i uniform on the unit sphere, |.| the chord distance."""
    V, F = icosphere(level)
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(n_bumps, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    rad = np.ones(V.shape[0])
    for ci in c:
        d2 = np.sum((V - ci) ** 2, axis=1)
        rad += amplitude * np.exp(-d2 / (2.0 * width * width))
    return V * rad[:, None], F


def torus(nu: int, nv: int, R: float = 1.0, r: float = 0.4, noise: float = 0.0,
          seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Closed torus from an nu-by-nv parametric lattice.  Each vertex is
    moved along the tube normal by a uniform amount in [-noise*r, +noise*r]."""
    u = 2.0 * math.pi * np.arange(nu) / nu
    v = 2.0 * math.pi * np.arange(nv) / nv
    Vv, Uu = np.meshgrid(v, u, indexing="ij")   # row j = v index, column i = u index
    Uu = Uu.ravel()
    Vv = Vv.ravel()
    nrm = np.stack([np.cos(Uu) * np.cos(Vv), np.sin(Uu) * np.cos(Vv), np.sin(Vv)], axis=1)
    ctr = np.stack([R * np.cos(Uu), R * np.sin(Uu), np.zeros_like(Uu)], axis=1)
    rr = np.full(Uu.shape, r)
    if noise > 0.0:
        rng = np.random.default_rng(seed)
        rr = rr + rng.uniform(-noise * r, noise * r, size=Uu.shape)
    V = ctr + rr[:, None] * nrm
    return V, _grid_faces(nu, nv, wrap_x=True, wrap_y=True)


def _value_noise(nx: int, ny: int, freq: int, rng: np.random.Generator) -> np.ndarray:
    """Smoothstep-interpolated lattice value noise on an (freq+1)^2 lattice,
    sampled on an ny-by-nx grid over the unit square, values in [-1, 1]."""
    lat = rng.uniform(-1.0, 1.0, size=(freq + 1, freq + 1))
    x = np.linspace(0.0, freq, nx, endpoint=True)
    y = np.linspace(0.0, freq, ny, endpoint=True)
    ix = np.minimum(np.floor(x).astype(np.int64), freq - 1)
    iy = np.minimum(np.floor(y).astype(np.int64), freq - 1)
    fx = x - ix
    fy = y - iy
    sx = fx * fx * (3.0 - 2.0 * fx)
    sy = fy * fy * (3.0 - 2.0 * fy)
    out = np.empty((ny, nx))
    for row in range(ny):
        a = lat[iy[row], ix] * (1 - sx) + lat[iy[row], ix + 1] * sx
        b = lat[iy[row] + 1, ix] * (1 - sx) + lat[iy[row] + 1, ix + 1] * sx
        out[row] = a * (1 - sy[row]) + b * sy[row]
    return out


def terrain(nx: int, ny: int, octaves: int = 8, amplitude: float = 0.1,
            seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Heightfield over [0,1]^2: fractal value noise with `octaves` octaves
    (lacunarity 2, gain 0.5, base frequency 2), scaled so max |z| = amplitude."""
    rng = np.random.default_rng(seed)
    z = np.zeros((ny, nx))
    gain = 1.0
    freq = 2
    for _ in range(octaves):
        z += gain * _value_noise(nx, ny, freq, rng)
        gain *= 0.5
        freq *= 2
    z *= amplitude / max(np.max(np.abs(z)), 1e-30)
    V, F = grid(nx, ny)
    V[:, 2] = z.ravel()
    return V, F


def random_planar(n: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Delaunay triangulation of n seeded random points in the unit square
    (an irregular mesh with mixed valences and obtuse triangles)."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    P = rng.uniform(0.0, 1.0, size=(n, 2))
    tri = Delaunay(P)
    V = np.zeros((n, 3))
    V[:, :2] = P
    return V, tri.simplices.astype(np.int32)


def _zip_rows(rows: list[tuple[np.ndarray, np.ndarray]]) -> np.ndarray:
    """Faces stitching consecutive rows of vertices whose x increases along
    each row: a monotone merge (zipper) walks both rows and always advances
    the one whose next vertex lies further left, so every strip between two
    rows is triangulated without overlap, whatever the rows' densities and
    offsets.  `rows[r]` is (vertex indices, x positions)."""
    F = []
    for (li, lx), (hi_, hx) in zip(rows[:-1], rows[1:]):
        a, b = 0, 0
        while a < len(li) - 1 or b < len(hi_) - 1:
            if b == len(hi_) - 1 or (a < len(li) - 1 and lx[a + 1] <= hx[b + 1]):
                F.append((li[a], li[a + 1], hi_[b]))
                a += 1
            else:
                F.append((li[a], hi_[b + 1], hi_[b]))
                b += 1
    return np.asarray(F, dtype=np.int32)


def sliver_plane(nx: int = 48, bands: int = 6, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """A flat mesh full of near-degenerate triangles, built row by row over
    [0,1] x [0,~1] and stitched by `_zip_rows`.  Between regular rows
    (spacing h = 1/(nx-1), interior x jittered by +-0.2 h) every band adds:

    * a needle row: the previous row's x positions lifted by g*h, so the
      triangles between them have one angle of about g radians;
    * a cap row at a gap g*h whose interior points sit at the midpoints of
      the row below, so its triangles have one angle of about pi - 4 g;
    * a dense row (spacing h/4) at a gap g*h above a regular row and below
      another: the regular row's vertices then have about a dozen
      neighbours (more than a one-ring slot holds) and needle triangles;

    with g cycling through 1e-3, 1e-4, 1e-5 and 3e-6, i.e. squared sines of
    the small angle from about 1e-6 down to 1e-11 (the smallest gaps are a
    few float32 ulps, so the float32 positions define the slivers).  All
    coordinates are exactly representable in float32, and consecutive rows
    differ in float32 y."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (nx - 1)
    gaps = [1e-3, 1e-4, 1e-5, 3e-6]
    base = np.linspace(0.0, 1.0, nx)

    def regular():
        x = base.copy()
        x[1:-1] += rng.uniform(-0.2, 0.2, nx - 2) * h
        return x

    row_x: list[np.ndarray] = []
    row_y: list[float] = []

    def push(x, dy):
        y = np.float32(0.0) if not row_y else np.float32(row_y[-1] + dy)
        if row_y and not y > np.float32(row_y[-1]):
            y = np.nextafter(np.float32(row_y[-1]), np.float32(np.inf))
        row_x.append(np.asarray(x, dtype=np.float32).astype(np.float64))
        row_y.append(float(y))

    push(regular(), 0.0)
    for b in range(bands):
        g = gaps[b % len(gaps)]
        push(regular(), h)
        push(row_x[-1], g * h)                       # needles
        push(regular(), h)
        mid = 0.5 * (row_x[-1][:-1] + row_x[-1][1:])
        push(np.concatenate([[0.0], mid, [1.0]]), g * h)  # caps
        push(regular(), h)
        push(np.linspace(0.0, 1.0, 4 * (nx - 1) + 1), g * h)  # dense, just above a regular row
        push(regular(), h)
        push(np.linspace(0.0, 1.0, 4 * (nx - 1) + 1), h)
    push(regular(), h)
    V, rows, k = [], [], 0
    for x, y in zip(row_x, row_y):
        rows.append((np.arange(k, k + len(x)), x))
        V.append(np.stack([x, np.full(len(x), y), np.zeros(len(x))], axis=1))
        k += len(x)
    return np.concatenate(V), _zip_rows(rows)


def random_source(n: int, seed: int) -> int:
    """A seeded uniformly random vertex index."""
    return int(np.random.default_rng(seed).integers(0, n))


def bbox_diagonal(V: np.ndarray) -> float:
    """Length of the bounding-box diagonal, used as the mesh diameter."""
    return float(np.linalg.norm(V.max(axis=0) - V.min(axis=0)))


# --------------------------------------------------------------------------
# The named workloads.  Sizes, distributions and seeds are fixed here so the
# tests, the oracle timings and the benchmark all see the same inputs.
# --------------------------------------------------------------------------

def flat65(seed: int = 0):
    """65x65 jittered unit-square grid, 4,225 vertices, 8,192 triangles,
    interior jitter +-0.2 spacing, one source at the centre vertex."""
    V, F = grid(65, 65, jitter=0.2, seed=seed)
    return V, F, np.array([32 * 65 + 32], dtype=np.int32)


def sphere_l7(seed: int = 0):
    """Level-7 unit icosphere, 163,842 vertices, 327,680 triangles,
    one seeded random source."""
    V, F = icosphere(7)
    return V, F, np.array([random_source(V.shape[0], seed)], dtype=np.int32)


def torus_1m(seed: int = 0):
    """Noisy torus R=1, r=0.4 on a 1024x1024 lattice (1,048,576 vertices,
    2,097,152 triangles), radial noise +-0.01*r, one seeded random source."""
    V, F = torus(1024, 1024, 1.0, 0.4, noise=0.01, seed=seed)
    return V, F, np.array([random_source(V.shape[0], seed + 1)], dtype=np.int32)


def bumpy_l8(seed: int = 0):
    """Level-8 icosphere (655,362 vertices) with 64 Gaussian bumps of
    amplitude 0.05 and width 0.1; one seeded random first sample."""
    V, F = bumpy_icosphere(8, 64, 0.05, 0.1, seed=seed)
    return V, F, np.array([random_source(V.shape[0], seed + 1)], dtype=np.int32)


def terrain_4096(seed: int = 0):
    """4096x4096 heightfield, 16,777,216 vertices, 33,538,050 triangles
    (an open 4096^2 lattice has 2*4095^2 triangles), 8-octave value noise of
    amplitude 0.1, one seeded random source."""
    V, F = terrain(4096, 4096, octaves=8, amplitude=0.1, seed=seed)
    return V, F, np.array([random_source(V.shape[0], seed + 1)], dtype=np.int32)


def uneven_batch(count: int = 32, n_min: int = 10_000, n_max: int = 2_000_000, seed: int = 0):
    """A batch of independent single-source problems of uneven size: vertex
    counts log-uniform in [n_min, n_max], even entries jittered unit-square
    grids (jitter +-0.2 spacing, aspect ratio in [1, 2]), odd entries noisy
    tori (R=1, r=0.4, radial noise +-0.01 r), each with one seeded random
    source.  Returns a list of ``(V, F, S)``."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = float(np.exp(rng.uniform(math.log(n_min), math.log(n_max))))
        s = int(rng.integers(0, 2**31 - 1))
        if b % 2 == 0:
            aspect = float(rng.uniform(1.0, 2.0))
            ny = max(3, int(round(math.sqrt(n / aspect))))
            nx = max(3, int(round(n / ny)))
            V, F = grid(nx, ny, jitter=0.2, seed=s)
        else:
            side = max(4, int(round(math.sqrt(n))))
            V, F = torus(side, side, 1.0, 0.4, noise=0.01, seed=s)
        out.append((V, F, np.array([random_source(V.shape[0], s + 1)], dtype=np.int32)))
    return out
