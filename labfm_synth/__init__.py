"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of the LABFM method itself.  It generates
node sets (perturbed Cartesian lattices, Sec. 4.1 of King, Lind & Nasar,
"High order difference schemes using the Local Anisotropic Basis Function
Method"), test fields with their exact derivatives, and nothing else.  Both
the oracle tests and the GPU tests draw from here so that the two sides see
identical inputs; neither side's numerics live here.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: draw ``k``
of stream ``seed`` is ``mix(seed * G + (k + 1) * G)`` with ``G`` the 64-bit
golden-ratio increment, mapped to a double in [0, 1) from its top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "splitmix64_u64",
    "uniform01",
    "normal01",
    "NodeSet",
    "jittered_lattice",
    "variable_wall_nodes",
    "dirichlet_square",
    "NeumannSet",
    "neumann_square",
    "annulus_nodes",
    "annulus_solution",
    "annulus_source",
    "HeatSteadyField",
    "ColeBurgersSolution",
    "ColeHopf2DSolution",
    "FourierField",
    "fourier_field",
    "sincos_field",
    "p6_field",
    "op_c_vector",
    "element_index",
    "p_of_k",
]

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_u64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of SplitMix64 stream ``seed`` as uint64."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) * _G + k * _G
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) built from the top 53 bits of each draw."""
    z = splitmix64_u64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normal deviates by the Box-Muller transform of two uniform streams."""
    u1 = uniform01(seed, n, offset)
    u2 = uniform01(seed ^ 0x5DEECE66D, n, offset)
    u1 = 1.0 - u1  # (0, 1]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class NodeSet:
    """A 2D node distribution.

    ``xy`` is float64 ``[n, 2]`` (row i = (x_i, y_i)), ``h`` float64 ``[n]`` the
    per-node stencil scale (stencil radius is 2h), ``s`` float64 ``[n]`` the local
    unperturbed spacing, ``order`` int8 ``[n]`` the per-node reconstruction
    order k (all equal for uniform sets), ``periodic`` whether the box
    ``[lo, hi)^2`` wraps.
    """

    xy: np.ndarray
    h: np.ndarray
    s: np.ndarray
    order: np.ndarray
    periodic: bool
    lo: tuple
    hi: tuple
    wall: np.ndarray | None = None  # bool [n]: node lies on a wall

    @property
    def n(self) -> int:
        return int(self.xy.shape[0])


def jittered_lattice(n_side: int, h_over_s: float, k: int, jitter: float = 0.3,
                     seed: int = 1, periodic: bool = True) -> NodeSet:
    """Cartesian lattice on the unit square, spacing s = 1/n_side, each node at
    ((i+1/2)s, (j+1/2)s) moved by independent U(-jitter*s, +jitter*s) offsets in x
    and y (the "noisy Cartesian" distribution of Sec. 4.1, maximum perturbation
    eps = jitter*s per coordinate).  Node index = j*n_side + i (row-major in y).
    Periodic sets are wrapped back into [0, 1).
    """
    s = 1.0 / n_side
    n = n_side * n_side
    ii, jj = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="xy")
    x = (ii.ravel() + 0.5) * s
    y = (jj.ravel() + 0.5) * s
    u = uniform01(seed, 2 * n)
    x = x + (2.0 * u[0::2] - 1.0) * jitter * s
    y = y + (2.0 * u[1::2] - 1.0) * jitter * s
    if periodic:
        x = np.where(x < 0.0, x + 1.0, x)
        x = np.where(x >= 1.0, x - 1.0, x)
        y = np.where(y < 0.0, y + 1.0, y)
        y = np.where(y >= 1.0, y - 1.0, y)
    xy = np.ascontiguousarray(np.stack([x, y], axis=1))
    return NodeSet(xy=xy, h=np.full(n, h_over_s * s), s=np.full(n, s),
                   order=np.full(n, k, dtype=np.int8), periodic=periodic,
                   lo=(0.0, 0.0), hi=(1.0, 1.0))


def lattice_clusters(n_side: int, h_over_s: float, corners, extent: float, jitter: float = 0.3,
                     seed: int = 1) -> NodeSet:
    """Dense jittered-lattice blocks in an otherwise empty, non-periodic unit box: one
    n_side x n_side block (spacing extent / n_side, h = h_over_s x spacing) with its lower-left
    corner at each point of `corners`.  The stencil radius is then tiny against the box, so a
    cell grid of side 2h would hold many more cells than nodes; a search that caps its cell
    count ends up with coarse cells holding hundreds of nodes each."""
    blocks = []
    for c, (cx, cy) in enumerate(corners):
        b = jittered_lattice(n_side, h_over_s, 4, jitter=jitter, seed=seed + c, periodic=False)
        blocks.append(np.stack([cx + b.xy[:, 0] * extent, cy + b.xy[:, 1] * extent], axis=1))
    xy = np.ascontiguousarray(np.concatenate(blocks))
    n = xy.shape[0]
    s = extent / n_side
    return NodeSet(xy=xy, h=np.full(n, h_over_s * s), s=np.full(n, s), order=np.full(n, 4, dtype=np.int8),
                   periodic=False, lo=(0.0, 0.0), hi=(1.0, 1.0))


def three_ring_stencil(delta: float, h: float = 0.05, seed: int = 7) -> NodeSet:
    """A node at (0.5, 0.5) whose 66 neighbours lie on three circles about it (radii 0.55 h,
    1.1 h and 1.6 h; 14, 22 and 30 nodes at jittered angles), each radius scaled by
    1 + delta U(-1, 1) per node; non-periodic unit box, uniform h.  On the exact circles
    x (r^2 - a^2)(r^2 - b^2)(r^2 - c^2) vanishes at every neighbour, a polynomial of degree 7
    without constant term, so the moment matrix of order k >= 7 is singular; the radial
    noise delta makes it merely ill conditioned, with a condition number growing as delta^-2."""
    u = uniform01(seed, 200)
    pts = [(0.5, 0.5)]
    t = 0
    for rad, cnt in zip((0.55 * h, 1.1 * h, 1.6 * h), (14, 22, 30)):
        for a in range(cnt):
            th = 2.0 * np.pi * (a + 0.5 * u[t]) / cnt
            rr = rad * (1.0 + delta * (2.0 * u[t + 100] - 1.0))
            t += 1
            pts.append((0.5 + rr * np.cos(th), 0.5 + rr * np.sin(th)))
    xy = np.ascontiguousarray(np.array(pts))
    n = xy.shape[0]
    return NodeSet(xy=xy, h=np.full(n, h), s=np.full(n, h / 2.2), order=np.full(n, 8, dtype=np.int8),
                   periodic=False, lo=(0.0, 0.0), hi=(1.0, 1.0))


# h/s per order for the variable-resolution set (each above the critical h/dr of Sec. 3.2).
H_OVER_S_BY_ORDER = {2: 1.0, 3: 1.1, 4: 1.4, 5: 1.6, 6: 1.8, 7: 2.0, 8: 2.2}


def variable_wall_nodes(n_side: int, seed: int = 4, jitter: float = 0.3,
                        stretch: float = 0.6, wall_order_cap: int = 4,
                        wall_h_boost: float = 1.3) -> NodeSet:
    """Non-periodic unit square with walls and a smoothly varying spacing.

    Computational coordinates xi, eta take n_side equispaced values on [0, 1];
    x = xi - stretch*sin(2 pi xi)/(2 pi) (same for y), so the local spacing
    s = (1 - stretch*cos(2 pi xi)) / (n_side - 1) varies by (1+stretch)/(1-stretch)
    (4x at stretch 0.6): fine at the walls, coarse in the middle.  Interior nodes
    are jittered by +-jitter*s per coordinate, wall nodes only along their wall,
    corners are fixed.  Order k_i = min(8, 2 + floor(7 x_i)) rises left to right,
    capped at ``wall_order_cap`` within 2h of a wall (one-sided stencils keep
    order up to 4 there, Sec. 4.1); h_i = (h/s)(k_i) * s_i, times
    ``wall_h_boost`` in that band (larger stencils at incomplete support).
    """
    m = n_side
    xi = np.linspace(0.0, 1.0, m)
    ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    xi_n = xi[ii.ravel()]
    eta_n = xi[jj.ravel()]
    tw = 2.0 * np.pi
    x = xi_n - stretch * np.sin(tw * xi_n) / tw
    y = eta_n - stretch * np.sin(tw * eta_n) / tw
    sx = (1.0 - stretch * np.cos(tw * xi_n)) / (m - 1)
    sy = (1.0 - stretch * np.cos(tw * eta_n)) / (m - 1)
    s = np.sqrt(sx * sy)  # area-equivalent spacing: pi (2h)^2 / (sx sy) neighbours = 4 pi (h/s)^2
    n = m * m
    u = uniform01(seed, 2 * n)
    on_x_wall = (ii.ravel() == 0) | (ii.ravel() == m - 1)
    on_y_wall = (jj.ravel() == 0) | (jj.ravel() == m - 1)
    jx = (2.0 * u[0::2] - 1.0) * jitter * sx
    jy = (2.0 * u[1::2] - 1.0) * jitter * sy
    x = x + np.where(on_x_wall, 0.0, jx)
    y = y + np.where(on_y_wall, 0.0, jy)
    x = np.clip(x, 0.0, 1.0)
    y = np.clip(y, 0.0, 1.0)
    k = np.minimum(8, 2 + np.floor(7.0 * x).astype(np.int64))
    hs = np.array([H_OVER_S_BY_ORDER[int(v)] for v in range(9) if v >= 2])
    h = hs[k - 2] * s
    dwall = np.minimum.reduce([x, 1.0 - x, y, 1.0 - y])
    band = dwall < 2.0 * h * wall_h_boost
    k = np.where(band, np.minimum(k, wall_order_cap), k)
    h = np.where(band, hs[k - 2] * s * wall_h_boost, hs[k - 2] * s)
    xy = np.ascontiguousarray(np.stack([x, y], axis=1))
    return NodeSet(xy=xy, h=h.astype(np.float64), s=s, order=k.astype(np.int8),
                   periodic=False, lo=(0.0, 0.0), hi=(1.0, 1.0),
                   wall=(on_x_wall | on_y_wall))


def dirichlet_square(n_side: int, h_over_s: float = 2.0, k: int = 4, eps: float = 0.5,
                     seed: int = 1, wall_band: int = 2) -> NodeSet:
    """Non-periodic unit square for the heat equation with Dirichlet walls (Sec. 5.1).

    Lattice spacing s = 1/(n_side - 1) with nodes on the walls, (i s, j s) for i, j = 0 ..
    n_side - 1.  Nodes on a wall (``wall`` mask: their values are prescribed) and the nodes
    within ``wall_band`` lattice rows of a wall stay on the lattice; every other node is
    displaced by independent U(-eps s/sqrt(2), +eps s/sqrt(2)) offsets in x and y, so that
    no node moves further than eps s (eps is the maximum perturbation distance of Sec. 4.1
    over the node spacing).  h = h_over_s * s everywhere.
    """
    m = n_side
    s = 1.0 / (m - 1)
    ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    i, j = ii.ravel(), jj.ravel()
    n = m * m
    d = np.minimum.reduce([i, m - 1 - i, j, m - 1 - j])  # lattice rows to the nearest wall
    u = uniform01(seed, 2 * n)
    a = np.where(d > wall_band, eps * s / math.sqrt(2.0), 0.0)
    x = i * s + (2.0 * u[0::2] - 1.0) * a
    y = j * s + (2.0 * u[1::2] - 1.0) * a
    xy = np.ascontiguousarray(np.stack([x, y], axis=1))
    return NodeSet(xy=xy, h=np.full(n, h_over_s * s), s=np.full(n, s),
                   order=np.full(n, k, dtype=np.int8), periodic=False,
                   lo=(0.0, 0.0), hi=(1.0, 1.0), wall=(d == 0))


@dataclass
class NeumannSet:
    """A node set with Dirichlet and Neumann boundaries (Sec. 5.2): ``ns`` holds the nodes of the
    domain followed by one ghost node per Neumann boundary node.  ``dirichlet`` (bool [n]) marks
    the Dirichlet boundary nodes; ``ghost`` / ``parent`` (int64 [n_ghost]) pair each ghost node
    with its boundary node b; ``normal`` (float64 [n_ghost, 2]) is the unit normal at b pointing
    into the domain, so that the ghost sits at r_b - n_b s, s = ``spacing``."""

    ns: NodeSet
    dirichlet: np.ndarray
    ghost: np.ndarray
    parent: np.ndarray
    normal: np.ndarray
    spacing: float


def neumann_square(n_side: int, h_over_s: float = 2.0, k: int = 4, eps: float = 0.5,
                   seed: int = 1, wall_band: int = 2) -> NeumannSet:
    """Node set for Poisson's equation with Dirichlet walls at x = 0, 1 and Neumann walls at
    y = 0, 1 (Sec. 5.2): the lattice of ``dirichlet_square`` (spacing s = 1/(n_side - 1),
    jitter beyond ``wall_band`` rows of a wall), and for every node b of the bottom and top
    walls other than the corners a ghost node at r_b - n_b s, n_b = (0, 1) at the bottom and
    (0, -1) at the top.  Ghosts share h = h_over_s s and order k; the (non-periodic) box is
    [0, 1] x [-s, 1 + s], so that it holds the ghosts."""
    base = dirichlet_square(n_side, h_over_s, k, eps, seed, wall_band)
    m = n_side
    s = 1.0 / (m - 1)
    idx = np.arange(m * m)
    i, j = idx % m, idx // m
    inner = (i > 0) & (i < m - 1)
    bottom = np.nonzero(inner & (j == 0))[0]
    top = np.nonzero(inner & (j == m - 1))[0]
    parent = np.concatenate([bottom, top]).astype(np.int64)
    normal = np.concatenate([np.tile([0.0, 1.0], (len(bottom), 1)), np.tile([0.0, -1.0], (len(top), 1))])
    gxy = base.xy[parent] - normal * s
    n0 = base.n
    ghost = np.arange(n0, n0 + len(parent), dtype=np.int64)
    xy = np.ascontiguousarray(np.concatenate([base.xy, gxy]))
    ng = len(parent)
    ns = NodeSet(xy=xy, h=np.concatenate([base.h, np.full(ng, h_over_s * s)]),
                 s=np.concatenate([base.s, np.full(ng, s)]),
                 order=np.full(n0 + ng, k, dtype=np.int8), periodic=False,
                 lo=(0.0, -s), hi=(1.0, 1.0 + s),
                 wall=np.concatenate([base.wall, np.zeros(ng, dtype=bool)]))
    dirichlet = np.zeros(n0 + ng, dtype=bool)
    dirichlet[:n0] = (i == 0) | (i == m - 1)
    return NeumannSet(ns=ns, dirichlet=dirichlet, ghost=ghost, parent=parent,
                         normal=np.ascontiguousarray(normal), spacing=s)


def annulus_nodes(m: int, k: int = 4, eps: float = 0.5, seed: int = 1, shift_iters: int = 10) -> NeumannSet:
    """Node set of the annular Poisson problem of Sec. 5.2: the annulus 1/8 < r < 1/2 about the
    origin (inner diameter H/4, outer diameter H, H = 1), spacing dr = 1/m (h/H = 2/m at
    h = 2 dr), Dirichlet on the outer circle and Neumann on the inner one.  Following the paper's
    construction: nodes at intervals of about dr along both circles; a noisy Cartesian fill of
    spacing dr (each coordinate moved by U(-eps dr/sqrt(2), +eps dr/sqrt(2)), eps the maximum
    displacement over dr) kept where dr/2 inside the domain; temporary ghosts, the same noisy
    lattice in strips of width 2h outside both circles; ``shift_iters`` passes of the shifting
    rule of Sec. 5.2 applied to the fill nodes,
        r_i <- r_i + (dr^2 / h) sum_{j: |r_ji| < h} (|r_ji| / h - 1) r_ji / |r_ji|,  r_ji = r_j - r_i,
    (all passes from the same positions of the previous pass, neighbours among every node); the
    temporary ghosts are then dropped and one ghost per inner-circle node b is added at
    r_b - n_b dr, n_b = r_b / |r_b| (into the domain).  h = 2 dr and order k at every node; the
    box for the stencil search is [-1/2 - 2h, 1/2 + 2h]^2 (non-periodic)."""
    from scipy.spatial import cKDTree

    dr = 1.0 / m
    h = 2.0 * dr
    r_in, r_out = 0.125, 0.5
    rings = []
    for rad in (r_out, r_in):
        cnt = max(3, int(round(2.0 * math.pi * rad / dr)))
        th = 2.0 * math.pi * np.arange(cnt) / cnt
        rings.append(np.stack([rad * np.cos(th), rad * np.sin(th)], axis=1))
    outer, inner = rings
    lim = r_out + 2.0 * h + dr
    g = np.arange(-int(math.ceil(lim / dr)), int(math.ceil(lim / dr)) + 1) * dr
    gx, gy = np.meshgrid(g, g, indexing="xy")
    pts = np.stack([gx.ravel(), gy.ravel()], axis=1)
    u = uniform01(seed, 2 * len(pts))
    a = eps * dr / math.sqrt(2.0)
    pts = pts + np.stack([(2.0 * u[0::2] - 1.0) * a, (2.0 * u[1::2] - 1.0) * a], axis=1)
    rr = np.hypot(pts[:, 0], pts[:, 1])
    fill = pts[(rr > r_in + 0.5 * dr) & (rr < r_out - 0.5 * dr)]
    temp = pts[((rr > r_out + 0.5 * dr) & (rr < r_out + 2.0 * h)) | ((rr < r_in - 0.5 * dr) & (rr > r_in - 2.0 * h))]
    fixed = np.concatenate([outer, inner, temp])
    for _ in range(shift_iters):
        allp = np.concatenate([fill, fixed])
        tree = cKDTree(allp)
        pairs = tree.query_pairs(h, output_type="ndarray")
        pairs = pairs[pairs[:, 0] < len(fill)]  # i a fill node (the fill comes first)
        i, j = pairs[:, 0], pairs[:, 1]
        rji = allp[j] - allp[i]
        d = np.hypot(rji[:, 0], rji[:, 1])
        keep = (d < h) & (d > 0.0)
        i, j, rji, d = i[keep], j[keep], rji[keep], d[keep]
        f = ((d / h - 1.0) / d)[:, None] * rji
        move = np.zeros_like(fill)
        np.add.at(move, i, f)
        jf = j < len(fill)  # the pair seen from the fill node j: r_ij = -r_ji
        np.add.at(move, j[jf], -f[jf])
        fill = fill + (dr * dr / h) * move
    nodes = np.concatenate([outer, inner, fill])
    n_out, n_in = len(outer), len(inner)
    parent = np.arange(n_out, n_out + n_in, dtype=np.int64)
    normal = inner / np.hypot(inner[:, 0], inner[:, 1])[:, None]
    gxy = inner - normal * dr
    n0 = len(nodes)
    xy = np.ascontiguousarray(np.concatenate([nodes, gxy]))
    n = len(xy)
    ghost = np.arange(n0, n, dtype=np.int64)
    dirichlet = np.zeros(n, dtype=bool)
    dirichlet[:n_out] = True
    wall = np.zeros(n, dtype=bool)
    wall[:n_out + n_in] = True
    box = r_out + 2.0 * h
    ns = NodeSet(xy=xy, h=np.full(n, h), s=np.full(n, dr), order=np.full(n, k, dtype=np.int8), periodic=False,
                 lo=(-box, -box), hi=(box, box), wall=wall)
    return NeumannSet(ns=ns, dirichlet=dirichlet, ghost=ghost, parent=parent, normal=np.ascontiguousarray(normal),
                      spacing=dr)


def annulus_solution(x, y):
    """Exact solution of the annular Poisson problem of Sec. 5.2: r sin(4 pi r) cos(3 theta)."""
    r, th = np.hypot(x, y), np.arctan2(y, x)
    return r * np.sin(4 * np.pi * r) * np.cos(3 * th)


def annulus_source(x, y):
    """Its source term as printed in Sec. 5.2 (the Laplacian of ``annulus_solution``):
    [12 pi cos 4 pi r - (16 pi^2 r - 1/r) sin 4 pi r] cos 3 theta - (9/r) cos 3 theta sin 4 pi r."""
    r, th = np.hypot(x, y), np.arctan2(y, x)
    return ((12 * np.pi * np.cos(4 * np.pi * r) - (16 * np.pi ** 2 * r - 1 / r) * np.sin(4 * np.pi * r)) * np.cos(3 * th)
            - 9 / r * np.cos(3 * th) * np.sin(4 * np.pi * r))


# ----------------------------------------------------------------------------------
# Index conventions of the monomial vector X and derivative vector D (Sec. 2):
# total degree n = 1, 2, ...; within a degree the power of x runs from n down to 0.
# ----------------------------------------------------------------------------------

def p_of_k(k: int) -> int:
    """Number of elements of X up to total degree k in 2D: p = (k^2 + 3k)/2 (Sec. 3.1)."""
    return (k * k + 3 * k) // 2


def element_index(a: int, b: int) -> int:
    """0-based position of x^a y^b (derivative d^(a+b)/dx^a dy^b) in X and D."""
    n = a + b
    return p_of_k(n - 1) + (n - a)


def op_c_vector(name: str, k: int) -> np.ndarray:
    """Target vector C^d (length p(k)) for the named operator.

    ``dx``, ``dy``: first derivatives; ``lap``: Laplacian (elements 3 and 5,
    Sec. 2); ``lap2``: biharmonic, ``lap3``: triharmonic, ``lap4``: nabla^8,
    each the multinomial expansion of (d_xx + d_yy)^m (Sec. 4.2 gives the
    element positions for m = 2 and m = 3; m = 4 follows the same rule).  The
    hyperviscosity coefficient and its sign are left to the caller.
    """
    p = p_of_k(k)
    c = np.zeros(p)
    if name == "dx":
        c[element_index(1, 0)] = 1.0
    elif name == "dy":
        c[element_index(0, 1)] = 1.0
    elif name.startswith("lap"):
        m = 1 if name == "lap" else int(name[3:])
        if 2 * m > k:
            raise ValueError(f"nabla^{2*m} needs order >= {2*m}, got {k}")
        for t in range(m + 1):
            c[element_index(2 * (m - t), 2 * t)] = math.comb(m, t)
    else:
        raise ValueError(name)
    return c


# ----------------------------------------------------------------------------------
# Test fields with exact derivatives.
# ----------------------------------------------------------------------------------

class _Field:
    def value(self, xy):  # pragma: no cover - interface
        raise NotImplementedError

    def deriv(self, name, xy):  # pragma: no cover - interface
        raise NotImplementedError


class SinCosField(_Field):
    """f = sin(2 pi x + ax) cos(2 pi y + ay) (period 1 in x and y; ax = ay = 0 by default)."""

    def __init__(self, ax: float = 0.0, ay: float = 0.0):
        self.ax, self.ay = ax, ay

    def value(self, xy):
        return np.sin(2 * np.pi * xy[:, 0] + self.ax) * np.cos(2 * np.pi * xy[:, 1] + self.ay)

    def deriv(self, name, xy):
        tp = 2 * np.pi
        tx, ty = tp * xy[:, 0] + self.ax, tp * xy[:, 1] + self.ay
        sx, cx = np.sin(tx), np.cos(tx)
        sy, cy = np.sin(ty), np.cos(ty)
        if name == "dx":
            return tp * cx * cy
        if name == "dy":
            return -tp * sx * sy
        if name.startswith("lap"):
            m = 1 if name == "lap" else int(name[3:])
            return (-2 * tp * tp) ** m * sx * cy
        raise ValueError(name)


def sincos_field(ax: float = 0.0, ay: float = 0.0) -> SinCosField:
    return SinCosField(ax, ay)


@dataclass
class FourierField(_Field):
    """f = sum_m a_m cos(2 pi (kx_m x + ky_m y) + phi_m): periodic on the unit square."""

    kx: np.ndarray
    ky: np.ndarray
    amp: np.ndarray
    phase: np.ndarray

    def _theta(self, xy):
        return 2 * np.pi * (np.outer(xy[:, 0], self.kx) + np.outer(xy[:, 1], self.ky)) + self.phase

    def value(self, xy):
        return np.cos(self._theta(xy)) @ self.amp

    def deriv(self, name, xy):
        th = self._theta(xy)
        tp = 2 * np.pi
        if name == "dx":
            return -np.sin(th) @ (self.amp * tp * self.kx)
        if name == "dy":
            return -np.sin(th) @ (self.amp * tp * self.ky)
        if name.startswith("lap"):
            m = 1 if name == "lap" else int(name[3:])
            k2 = (tp * tp) * (self.kx.astype(np.float64) ** 2 + self.ky.astype(np.float64) ** 2)
            return np.cos(th) @ (self.amp * (-k2) ** m)
        raise ValueError(name)


def fourier_field(n_modes: int = 16, kmax: int = 32, seed: int = 3) -> FourierField:
    """Sum of ``n_modes`` Fourier modes with integer wavenumbers uniform in
    [-kmax, kmax]^2 minus the origin, N(0,1) amplitudes and U[0, 2pi) phases."""
    kx = np.zeros(n_modes, dtype=np.int64)
    ky = np.zeros(n_modes, dtype=np.int64)
    got, off = 0, 0
    span = 2 * kmax + 1
    while got < n_modes:
        u = uniform01(seed, 2, off)
        off += 2
        a = int(u[0] * span) - kmax
        b = int(u[1] * span) - kmax
        if a == 0 and b == 0:
            continue
        kx[got], ky[got] = a, b
        got += 1
    amp = normal01(seed + 1, n_modes)
    phase = 2 * np.pi * uniform01(seed + 2, n_modes)
    return FourierField(kx=kx, ky=ky, amp=amp, phase=phase)


class HeatSteadyField(_Field):
    """Steady state of the heat equation on the unit square with u(x, 0) = sin(pi x) and
    u = 0 on the other walls (Sec. 5.1): u = sinh(pi (1 - y)) sin(pi x) / sinh(pi), a
    harmonic function (its Laplacian vanishes)."""

    def value(self, xy):
        return np.sinh(np.pi * (1.0 - xy[:, 1])) * np.sin(np.pi * xy[:, 0]) / np.sinh(np.pi)

    def boundary(self, xy, wall):
        """The prescribed wall values: sin(pi x) on y = 0, zero elsewhere (and off the walls)."""
        return np.where(wall & (xy[:, 1] == 0.0), np.sin(np.pi * xy[:, 0]), 0.0)

    def deriv(self, name, xy):
        pi = np.pi
        x, y = xy[:, 0], xy[:, 1]
        if name == "dx":
            return pi * np.sinh(pi * (1.0 - y)) * np.cos(pi * x) / np.sinh(pi)
        if name == "dy":
            return -pi * np.cosh(pi * (1.0 - y)) * np.sin(pi * x) / np.sinh(pi)
        if name.startswith("lap"):
            return np.zeros(xy.shape[0])
        raise ValueError(name)


class ColeBurgersSolution:
    """Exact solution of the periodic Burgers' problem of Sec. 5.3 (Cole 1951): on [0, 1)^2 with
    u(x, y, 0) = sin(2 pi x), v = 0, the velocity stays v = 0 and

        u(x, t) = (4 pi / Re) sum_n n A_n sin(2 n pi x) E_n / (A_0 + sum_n A_n cos(2 n pi x) E_n),
        A_0 = e^-z I_0(z),  A_n = 2 e^-z I_n(z),  z = Re / (4 pi),  E_n = exp(-4 n^2 pi^2 t / Re),

    I_n the modified Bessel functions of the first kind.  This is the Cole-Hopf transform
    u = -(2/Re) phi_x / phi of the heat-equation solution phi with phi(x, 0) = exp(Re cos(2 pi x)
    / (4 pi)) = I_0(z) + 2 sum_n I_n(z) cos(2 n pi x).  (The paper prints the decay factor as
    exp(-n^2 pi^2 t / (H^2 Re)); the factor 4 follows from phi_t = phi_xx / Re with wavenumber
    2 n pi.)  ``nterms`` terms: A_n < 1e-16 for n >= 30 at Re = 100."""

    def __init__(self, Re: float = 100.0, nterms: int = 40):
        from scipy.special import ive  # exponentially scaled I_n: e^-z I_n(z)

        self.Re = float(Re)
        z = self.Re / (4.0 * math.pi)
        self.n = np.arange(1, nterms + 1, dtype=np.float64)
        self.A0 = float(ive(0, z))
        self.An = 2.0 * ive(self.n, z)

    def u(self, x, t):
        x = np.asarray(x, dtype=np.float64)
        E = np.exp(-4.0 * self.n ** 2 * math.pi ** 2 * t / self.Re)
        th = 2.0 * math.pi * np.outer(x, self.n)
        num = (4.0 * math.pi / self.Re) * (np.sin(th) @ (self.n * self.An * E))
        den = self.A0 + np.cos(th) @ (self.An * E)
        return num / den


class ColeHopf2DSolution:
    """A two-dimensional exact solution of Burgers' equation u_t + (u . grad) u = nabla^2 u / Re
    on the periodic unit square, by the Cole-Hopf transform u = -(2/Re) grad ln(phi) of a heat-
    equation solution phi_t = nabla^2 phi / Re: phi = 1 + a sin(2 pi x) sin(2 pi y) E,
    E = exp(-8 pi^2 t / Re), 0 < a < 1 (so phi > 0).  Both components and all advection terms are
    non-zero, unlike the one-dimensional problem of Sec. 5.3."""

    def __init__(self, Re: float = 10.0, a: float = 0.5):
        self.Re, self.a = float(Re), float(a)

    def uv(self, xy, t):
        tp = 2.0 * math.pi
        x, y = xy[:, 0], xy[:, 1]
        E = self.a * math.exp(-2.0 * tp * tp * t / self.Re)
        phi = 1.0 + E * np.sin(tp * x) * np.sin(tp * y)
        c = -2.0 / self.Re * tp * E / phi
        return c * np.cos(tp * x) * np.sin(tp * y), c * np.sin(tp * x) * np.cos(tp * y)


class P6Field(_Field):
    """The polynomial test function of Eq. (p6): 1 + (xh yh)^4 + sum_{n=1..6} (xh^n + yh^n),
    xh = x - 0.1453, yh = y - 0.16401 (H = 1).  Its derivatives of order > 8 vanish."""

    X0 = 0.1453
    Y0 = 0.16401

    @staticmethod
    def _poly_terms():
        # list of (coef, a, b) with value coef * xh^a * yh^b
        t = [(1.0, 0, 0), (1.0, 4, 4)]
        for n in range(1, 7):
            t.append((1.0, n, 0))
            t.append((1.0, 0, n))
        return t

    def _d(self, xy, dx_order, dy_order):
        xh = xy[:, 0] - self.X0
        yh = xy[:, 1] - self.Y0
        out = np.zeros(xy.shape[0])
        for c, a, b in self._poly_terms():
            if dx_order > a or dy_order > b:
                continue
            ca = math.perm(a, dx_order)
            cb = math.perm(b, dy_order)
            out += c * ca * cb * xh ** (a - dx_order) * yh ** (b - dy_order)
        return out

    def value(self, xy):
        return self._d(xy, 0, 0)

    def deriv(self, name, xy):
        if name == "dx":
            return self._d(xy, 1, 0)
        if name == "dy":
            return self._d(xy, 0, 1)
        if name.startswith("lap"):
            m = 1 if name == "lap" else int(name[3:])
            return sum(math.comb(m, t) * self._d(xy, 2 * (m - t), 2 * t) for t in range(m + 1))
        raise ValueError(name)


def p6_field() -> P6Field:
    return P6Field()
