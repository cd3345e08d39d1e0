"""Seeded synthetic meshes and initial states for the finite-volume Euler step.

This module only makes inputs: node coordinates, triangles, boundary tags and
initial conserved states.  It holds none of the scheme's arithmetic (no flux,
residual, update, time step or totals) and is the one module that both the
CUDA library's tests and the FP64 oracle's tests draw inputs from.

The paper's own meshes (Gmsh, forward-facing step, Sec. 7.1) are not
available; these generators stand in for them with the structure the paper
describes: a cell-centred triangle mesh where every triangle has three
neighbours or a ghost cell at the boundary (Sec. 7).

Boundary tags in ``bnd`` triples (node a, node b, tag): 1 slip wall,
2 far field (free-stream ghost), 3 extrapolation.  ``canon`` maps every node
to the node it is identified with on a periodic domain.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4  # ratio of specific heats (Sec. 6.1)

TAG_WALL, TAG_FARFIELD, TAG_EXTRAP = 1, 2, 3


@dataclass
class MeshInput:
    xy: np.ndarray                 # (n_nodes, 2) float64
    tri: np.ndarray                # (n_tri, 3) int32
    canon: np.ndarray | None = None  # (n_nodes,) int32 periodic identification
    bnd: np.ndarray | None = None    # (n_bnd, 3) int32 (a, b, tag)
    default_bc: int = 0
    info: dict = field(default_factory=dict)

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])

    def centroids(self) -> np.ndarray:
        return self.xy[self.tri].mean(axis=1)


def _quad_split(nx, ny, node_id, coin):
    """Two triangles per lattice quad, counter-clockwise, split along a
    diagonal picked per quad by ``coin`` (0: a-c, 1: b-d)."""
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    a = node_id(i, j)
    b = node_id(i + 1, j)
    c = node_id(i + 1, j + 1)
    d = node_id(i, j + 1)
    coin = coin.reshape(ny, nx).astype(bool)
    t1 = np.where(coin[..., None], np.stack([a, b, d], -1), np.stack([a, b, c], -1))
    t2 = np.where(coin[..., None], np.stack([b, c, d], -1), np.stack([a, c, d], -1))
    tri = np.stack([t1, t2], axis=2).reshape(-1, 3)
    return tri.astype(np.int32)


def _signed_areas(xy, tri):
    p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    return 0.5 * ((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1])
                  - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1]))


def periodic_square(nx: int, ny: int, seed: int, jitter: float = 0.2,
                    lx: float = 1.0, ly: float = 1.0) -> MeshInput:
    """Periodic [0,lx]x[0,ly] lattice of nx*ny quads (2*nx*ny triangles).

    Every node is moved by U(-jitter, jitter) times the lattice spacing in each
    axis; identified copies on opposite sides move together (the offset is
    drawn per canonical node).  Diagonals are chosen by a seeded coin.  With
    jitter <= 0.2 no triangle falls below 1/5 of its lattice area.
    """
    if nx < 2 or ny < 2:
        raise ValueError("periodic lattice needs nx, ny >= 2")
    rng = np.random.default_rng(seed)
    hx, hy = lx / nx, ly / ny
    off = rng.uniform(-jitter, jitter, size=(ny, nx, 2)) * np.array([hx, hy])
    coin = rng.integers(0, 2, size=nx * ny)
    jj, ii = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    canon_ij = (jj % ny) * nx + (ii % nx)
    xy = np.stack([ii * hx, jj * hy], -1).astype(np.float64)
    xy += off.reshape(-1, 2)[canon_ij]
    node_id = lambda i, j: j * (nx + 1) + i  # noqa: E731
    tri = _quad_split(nx, ny, node_id, coin)
    # canonical id expressed as a node index of the (nx+1)*(ny+1) lattice
    cj, ci = canon_ij // nx, canon_ij % nx
    canon = (cj * (nx + 1) + ci).reshape(-1).astype(np.int32)
    xy = xy.reshape(-1, 2)
    assert _signed_areas(xy, tri).min() > 0.0
    return MeshInput(xy, tri, canon=canon, bnd=None, default_bc=0,
                     info=dict(kind="periodic_square", nx=nx, ny=ny, seed=seed, jitter=jitter))


def _graded(n: int, density, lo: float, hi: float) -> np.ndarray:
    """n+1 points on [lo, hi] whose spacing is inversely proportional to the
    given density function (equidistribution)."""
    s = np.linspace(lo, hi, 20001)
    w = density(s)
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (w[1:] + w[:-1]) * np.diff(s))])
    cum /= cum[-1]
    pts = np.interp(np.linspace(0.0, 1.0, n + 1), cum, s)
    pts[0], pts[-1] = lo, hi
    return pts


def bump_height(x: np.ndarray, x0: float = 1.0, x1: float = 2.0, h: float = 0.1) -> np.ndarray:
    """Lower wall of the channel: a circular arc of height h over [x0, x1]."""
    half = 0.5 * (x1 - x0)
    radius = (half * half + h * h) / (2.0 * h)
    xc, yc = 0.5 * (x0 + x1), h - radius
    y = yc + np.sqrt(np.maximum(radius * radius - (x - xc) ** 2, 0.0))
    return np.where((x > x0) & (x < x1), np.maximum(y, 0.0), 0.0)


def channel_bump(nx: int, ny: int, seed: int, jitter: float = 0.2, h: float = 0.1,
                 refine: float = 4.0) -> MeshInput:
    """Channel [0,3]x[0,1] with a circular-arc bump of thickness h on the lower
    wall over x in [1,2]; nx*ny quads (2*nx*ny triangles).

    The x-spacing is ``refine`` times denser over the bump and the y-spacing
    ``refine`` times denser at the lower wall (smooth tanh blends).  Interior
    nodes are jittered by U(-jitter, jitter) of the local spacing.  Left and
    right ends are far field (tag 2), lower and upper walls slip walls (tag 1).
    """
    rng = np.random.default_rng(seed)
    delta = 0.08
    dens_x = lambda x: 1.0 + (refine - 1.0) * 0.5 * (np.tanh((x - 1.0) / delta)  # noqa: E731
                                                      - np.tanh((x - 2.0) / delta))
    dens_y = lambda e: 1.0 + (refine - 1.0) * (1.0 - np.tanh(e / 0.12))  # noqa: E731
    xs = _graded(nx, dens_x, 0.0, 3.0)
    es = _graded(ny, dens_y, 0.0, 1.0)
    # local spacings (the smaller neighbouring interval) for the jitter
    dx = np.diff(xs)
    hx = np.minimum(np.concatenate([[dx[0]], dx]), np.concatenate([dx, [dx[-1]]]))
    de = np.diff(es)
    he = np.minimum(np.concatenate([[de[0]], de]), np.concatenate([de, [de[-1]]]))
    X, E = np.meshgrid(xs, es, indexing="xy")  # (ny+1, nx+1)
    jx = rng.uniform(-jitter, jitter, size=X.shape) * hx[None, :]
    je = rng.uniform(-jitter, jitter, size=X.shape) * he[:, None]
    interior = np.zeros(X.shape, bool)
    interior[1:-1, 1:-1] = True
    X = np.where(interior, X + jx, X)
    E = np.where(interior, E + je, E)
    yb = bump_height(X, h=h)
    Y = yb + E * (1.0 - yb)
    xy = np.stack([X, Y], -1).reshape(-1, 2).astype(np.float64)
    coin = rng.integers(0, 2, size=nx * ny)
    node_id = lambda i, j: j * (nx + 1) + i  # noqa: E731
    tri = _quad_split(nx, ny, node_id, coin)
    i = np.arange(nx)
    j = np.arange(ny)
    bnd = np.concatenate([
        np.stack([node_id(i, 0), node_id(i + 1, 0), np.full(nx, TAG_WALL)], -1),
        np.stack([node_id(i, ny), node_id(i + 1, ny), np.full(nx, TAG_WALL)], -1),
        np.stack([node_id(0, j), node_id(0, j + 1), np.full(ny, TAG_FARFIELD)], -1),
        np.stack([node_id(nx, j), node_id(nx, j + 1), np.full(ny, TAG_FARFIELD)], -1),
    ]).astype(np.int32)
    assert _signed_areas(xy, tri).min() > 0.0
    return MeshInput(xy, tri, canon=None, bnd=bnd, default_bc=0,
                     info=dict(kind="channel_bump", nx=nx, ny=ny, seed=seed, jitter=jitter,
                               h=h, refine=refine))


def shock_tube_strip(nx: int, ny: int, seed: int, jitter: float = 0.2,
                     lx: float = 1.0, ly: float = 0.05) -> MeshInput:
    """Strip [0,lx]x[0,ly] of nx*ny jittered quads: slip walls at top and
    bottom (tag 1), extrapolation at both ends (tag 3)."""
    rng = np.random.default_rng(seed)
    hx, hy = lx / nx, ly / ny
    X, Y = np.meshgrid(np.arange(nx + 1) * hx, np.arange(ny + 1) * hy, indexing="xy")
    interior = np.zeros(X.shape, bool)
    interior[1:-1, 1:-1] = True
    X = np.where(interior, X + rng.uniform(-jitter, jitter, X.shape) * hx, X)
    Y = np.where(interior, Y + rng.uniform(-jitter, jitter, Y.shape) * hy, Y)
    xy = np.stack([X, Y], -1).reshape(-1, 2).astype(np.float64)
    coin = rng.integers(0, 2, size=nx * ny)
    node_id = lambda i, j: j * (nx + 1) + i  # noqa: E731
    tri = _quad_split(nx, ny, node_id, coin)
    i = np.arange(nx)
    j = np.arange(ny)
    bnd = np.concatenate([
        np.stack([node_id(i, 0), node_id(i + 1, 0), np.full(nx, TAG_WALL)], -1),
        np.stack([node_id(i, ny), node_id(i + 1, ny), np.full(nx, TAG_WALL)], -1),
        np.stack([node_id(0, j), node_id(0, j + 1), np.full(ny, TAG_EXTRAP)], -1),
        np.stack([node_id(nx, j), node_id(nx, j + 1), np.full(ny, TAG_EXTRAP)], -1),
    ]).astype(np.int32)
    assert _signed_areas(xy, tri).min() > 0.0
    return MeshInput(xy, tri, canon=None, bnd=bnd, default_bc=0,
                     info=dict(kind="shock_tube_strip", nx=nx, ny=ny, seed=seed))


def two_cells(default_bc: int = TAG_WALL) -> MeshInput:
    """Unit square split on its (0,0)-(1,1) diagonal: L = (0,0),(1,0),(1,1)
    and R = (0,0),(1,1),(0,1), both counter-clockwise."""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return MeshInput(xy, tri, default_bc=default_bc, info=dict(kind="two_cells"))


# --------------------------------------------------------------------------
# initial states (point values at the cell centroids)
# --------------------------------------------------------------------------
def conserved(rho, u, v, p) -> np.ndarray:
    """(rho, rho u, rho v, E) with E = p/(gamma-1) + rho |v|^2 / 2 (Eq. 2)."""
    rho, u, v, p = np.broadcast_arrays(*(np.asarray(a, np.float64) for a in (rho, u, v, p)))
    return np.stack([rho, rho * u, rho * v, p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v)], -1)


def freestream(mach: float, angle: float = 0.0, rho: float = 1.0, p: float = 1.0) -> tuple:
    """Primitive free stream (rho, u, v, p) of Mach number ``mach``."""
    c = math.sqrt(GAMMA * p / rho)
    return (rho, mach * c * math.cos(angle), mach * c * math.sin(angle), p)


def isentropic_vortex(xy_c: np.ndarray, mach: float = 0.5, beta: float = 5.0,
                      radius: float = 0.1, center=(0.5, 0.5)) -> np.ndarray:
    """Isentropic vortex of strength beta and core radius ``radius`` advected
    by a free stream of Mach ``mach`` along +x (rho_inf = p_inf = 1)."""
    x0, y0 = center
    dx = (xy_c[:, 0] - x0) / radius
    dy = (xy_c[:, 1] - y0) / radius
    r2 = dx * dx + dy * dy
    amp = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    u_inf = mach * math.sqrt(GAMMA)
    u = u_inf - amp * dy
    v = amp * dx
    T = 1.0 - (GAMMA - 1.0) * beta * beta / (8.0 * GAMMA * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (GAMMA - 1.0))
    return conserved(rho, u, v, rho * T)


def uniform_state(n: int, prim) -> np.ndarray:
    rho, u, v, p = prim
    return np.repeat(conserved(rho, u, v, p)[None, :], n, axis=0)


def sod_state(xy_c: np.ndarray, x0: float = 0.5) -> np.ndarray:
    """Sod's shock tube: (1, 0, 1) left of x0, (0.125, 0, 0.1) right."""
    left = xy_c[:, 0] < x0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    return conserved(rho, 0.0 * rho, 0.0 * rho, p)


def random_smooth_state(xy_c: np.ndarray, seed: int, amp: float = 0.2) -> np.ndarray:
    """A smooth random positive state (a few Fourier modes per field)."""
    rng = np.random.default_rng(seed)
    fields = []
    for base in (1.0, 0.3, -0.2, 1.0):
        k = rng.integers(1, 4, size=(3, 2))
        ph = rng.uniform(0, 2 * math.pi, size=3)
        a = rng.uniform(-amp, amp, size=3)
        f = base + sum(a[m] * np.sin(2 * math.pi * (k[m, 0] * xy_c[:, 0] + k[m, 1] * xy_c[:, 1])
                                     + ph[m]) for m in range(3))
        fields.append(f)
    rho, u, v, p = fields
    return conserved(np.abs(rho) + 0.2, u, v, np.abs(p) + 0.2)


# --------------------------------------------------------------------------
# the benchmark workloads
# --------------------------------------------------------------------------
def vortex_square_small(seed: int = 1) -> MeshInput:
    """Periodic unit square, 64x32 lattice, 4,096 triangles."""
    return periodic_square(64, 32, seed)


def channel_bump_1m(seed: int = 2) -> MeshInput:
    """Channel with bump, 1250x400 quads: 1,000,000 triangles."""
    return channel_bump(1250, 400, seed)


def vortex_square_16m(seed: int = 4) -> MeshInput:
    """Periodic unit square, 4096x2048 lattice: 16,777,216 triangles."""
    return periodic_square(4096, 2048, seed)


def batch_lattices(n_meshes: int = 256, lo: int = 5000, hi: int = 200000, seed: int = 3):
    """Lattice sizes (nx, ny) for a batch of periodic squares whose triangle
    counts are log-uniform in [lo, hi]: ny = round(sqrt(N/4)), nx = 2 ny."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_meshes))
    ny = np.maximum(np.rint(np.sqrt(n / 4.0)).astype(int), 2)
    return [(2 * int(a), int(a)) for a in ny]


def vortex_batch(n_meshes: int = 256, lo: int = 5000, hi: int = 200000, seed: int = 3):
    """A batch of periodic jittered squares with triangle counts log-uniform in
    [lo, hi]; each mesh gets a free-stream Mach number U(0.3, 0.8) and, by a
    seeded coin, a vortex or a uniform initial state.  Returns a list of
    (MeshInput, primitive free stream, initial state)."""
    rng = np.random.default_rng(seed + 7919)
    out = []
    for k, (nx, ny) in enumerate(batch_lattices(n_meshes, lo, hi, seed)):
        mi = periodic_square(nx, ny, seed=1000 * seed + k)
        mach = float(rng.uniform(0.3, 0.8))
        prim = freestream(mach)
        if rng.integers(0, 2):
            U0 = isentropic_vortex(mi.centroids(), mach=mach)
        else:
            U0 = uniform_state(mi.n_tri, prim)
        out.append((mi, prim, U0))
    return out


def refine_midpoint(mi: MeshInput, levels: int = 2):
    """Splits every triangle into four through its edge midpoints, ``levels``
    times (16 children per triangle for two levels).  New nodes on boundary
    edges stay on the straight edge, so the children tile their parent
    exactly.  Returns (fine MeshInput, parent) where parent[f] is the coarse
    triangle of fine triangle f; the children of coarse triangle c are the
    consecutive fine triangles 4**levels * c ... 4**levels * (c + 1) - 1.
    Periodic meshes are not supported."""
    if mi.canon is not None:
        raise ValueError("refinement of periodic meshes is not supported")
    xy, tri = mi.xy, mi.tri.astype(np.int64)
    bnd = None if mi.bnd is None else mi.bnd.astype(np.int64)
    parent = np.arange(tri.shape[0], dtype=np.int64)
    for _ in range(levels):
        nn = xy.shape[0]
        e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
        key = np.sort(e, axis=1)
        uniq, inv = np.unique(key[:, 0] * nn + key[:, 1], return_inverse=True)
        a, b = uniq // nn, uniq % nn
        mid_xy = 0.5 * (xy[a] + xy[b])
        mid = nn + inv.reshape(3, -1)  # midpoint node of edges 01, 12, 20 per triangle
        m01, m12, m20 = mid[0], mid[1], mid[2]
        v0, v1, v2 = tri[:, 0], tri[:, 1], tri[:, 2]
        kids = np.stack([np.stack([v0, m01, m20], -1), np.stack([m01, v1, m12], -1),
                         np.stack([m20, m12, v2], -1), np.stack([m01, m12, m20], -1)], axis=1)
        tri = kids.reshape(-1, 3)
        parent = np.repeat(parent, 4)
        if bnd is not None:
            bk = np.sort(bnd[:, :2], axis=1)
            pos = np.searchsorted(uniq, bk[:, 0] * nn + bk[:, 1])
            m = nn + pos
            bnd = np.concatenate([np.stack([bnd[:, 0], m, bnd[:, 2]], -1),
                                  np.stack([m, bnd[:, 1], bnd[:, 2]], -1)])
        xy = np.concatenate([xy, mid_xy])
    fine = MeshInput(xy, tri.astype(np.int32), None,
                     None if bnd is None else bnd.astype(np.int32), mi.default_bc,
                     dict(mi.info, refined=levels))
    return fine, parent


def _graded_toward(n: int, lo: float, hi: float, at_hi: bool, ratio: float) -> np.ndarray:
    """n+1 points on [lo, hi] whose spacing shrinks geometrically by `ratio`
    toward one end (the hi end if at_hi)."""
    if n < 1:
        raise ValueError("need at least one interval")
    q = ratio ** (1.0 / max(n - 1, 1))  # growth factor between neighbouring intervals
    w = q ** np.arange(n)
    w = w[::-1] if at_hi else w  # large intervals away from the refined end
    x = lo + (hi - lo) * np.concatenate([[0.0], np.cumsum(w)]) / w.sum()
    x[0], x[-1] = lo, hi
    return x


def forward_step(nx1: int, nx2: int, ny1: int, ny2: int, seed: int, jitter: float = 0.2,
                 length: float = 3.0, height: float = 1.0, step_x: float = 0.6,
                 step_h: float = 0.2, corner_refine: float = 12.5) -> MeshInput:
    """Channel [0, length] x [0, height] with a forward-facing step occupying
    x > step_x, y < step_h (these dimensions are this generator's choice).
    Grid lines run through the step corner; the spacing shrinks toward the
    corner by `corner_refine` (Sec. 7.1 refines the characteristic length
    near the corner by 12.5).  Interior nodes are jittered.  Tags: inflow at
    x = 0 far field (2), outflow at x = length extrapolation (3), all walls
    slip (1)."""
    rng = np.random.default_rng(seed)
    xs = np.concatenate([_graded_toward(nx1, 0.0, step_x, True, corner_refine),
                         _graded_toward(nx2, step_x, length, False, corner_refine)[1:]])
    ys = np.concatenate([_graded_toward(ny1, 0.0, step_h, True, corner_refine),
                         _graded_toward(ny2, step_h, height, False, corner_refine)[1:]])
    nx, ny = nx1 + nx2, ny1 + ny2
    dx = np.diff(xs)
    hx = np.minimum(np.concatenate([[dx[0]], dx]), np.concatenate([dx, [dx[-1]]]))
    dy = np.diff(ys)
    hy = np.minimum(np.concatenate([[dy[0]], dy]), np.concatenate([dy, [dy[-1]]]))
    X, Y = np.meshgrid(xs, ys, indexing="xy")  # (ny+1, nx+1)
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    # nodes on a boundary (outer walls, inflow, outflow, step faces) stay put
    on_bnd = (ii == 0) | (ii == nx) | (jj == 0) | (jj == ny) | \
             ((ii == nx1) & (jj <= ny1)) | ((jj == ny1) & (ii >= nx1))
    inside_step = (ii > nx1) & (jj < ny1)
    move = ~on_bnd & ~inside_step
    X = np.where(move, X + rng.uniform(-jitter, jitter, X.shape) * hx[None, :], X)
    Y = np.where(move, Y + rng.uniform(-jitter, jitter, Y.shape) * hy[:, None], Y)
    node_id = lambda i, j: j * (nx + 1) + i  # noqa: E731
    coin = rng.integers(0, 2, size=nx * ny)
    tri = _quad_split(nx, ny, node_id, coin).reshape(ny, nx, 2, 3)
    qi, qj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    keep = ~((qi >= nx1) & (qj < ny1))  # quads inside the step are removed
    tri = tri[keep].reshape(-1, 3)
    xy = np.stack([X, Y], -1).reshape(-1, 2).astype(np.float64)
    segs = []

    def add(i0, j0, i1, j1, tag):
        if i0 == i1:
            j = np.arange(min(j0, j1), max(j0, j1))
            segs.append(np.stack([node_id(i0, j), node_id(i0, j + 1), np.full(j.size, tag)], -1))
        else:
            i = np.arange(min(i0, i1), max(i0, i1))
            segs.append(np.stack([node_id(i, j0), node_id(i + 1, j0), np.full(i.size, tag)], -1))

    add(0, 0, 0, ny, TAG_FARFIELD)          # inflow
    add(nx, ny1, nx, ny, TAG_EXTRAP)        # outflow
    add(0, 0, nx1, 0, TAG_WALL)             # floor before the step
    add(nx1, 0, nx1, ny1, TAG_WALL)         # step face
    add(nx1, ny1, nx, ny1, TAG_WALL)        # step top
    add(0, ny, nx, ny, TAG_WALL)            # ceiling
    bnd = np.concatenate(segs).astype(np.int32)
    # drop nodes no triangle uses (the inside of the step)
    used = np.unique(tri)
    remap = -np.ones(xy.shape[0], np.int64)
    remap[used] = np.arange(used.size)
    tri = remap[tri].astype(np.int32)
    bnd[:, :2] = remap[bnd[:, :2]]
    xy = xy[used]
    assert _signed_areas(xy, tri).min() > 0.0
    return MeshInput(xy, tri, canon=None, bnd=bnd, default_bc=0,
                     info=dict(kind="forward_step", nx1=nx1, nx2=nx2, ny1=ny1, ny2=ny2, seed=seed,
                               step_x=step_x, step_h=step_h, corner_refine=corner_refine))


def forward_step_394k(seed: int = 7) -> MeshInput:
    """About 394,000 triangles (410,400), the size of the paper's largest step mesh."""
    return forward_step(120, 420, 90, 360, seed)


def forward_step_65k(seed: int = 7) -> MeshInput:
    """65,664 triangles: the finest mesh of this family on which the scheme
    (averaged interface wave speed) keeps a positive pressure at the step
    corner up to t = 4."""
    return forward_step(48, 168, 36, 144, seed)


def mach3_inflow() -> tuple:
    """Primitive inflow state of the forward-facing step: Mach 3 with c = 1."""
    return freestream(3.0, rho=GAMMA, p=1.0)
