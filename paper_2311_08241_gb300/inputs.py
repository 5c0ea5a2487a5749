"""Seeded synthetic inputs for the barotropic subcycle: meshes, depths, Coriolis,
frozen forcing and initial states.

This module is shared by the CUDA path, the FP64 oracle and the benchmark. It holds
no arithmetic of the method itself (no gradient, divergence, area weighting,
time stepping or averaging): it only places points, connects them into triangles,
expresses each triangle's corners in the triangle's own planar frame and samples
the prescribed fields. Everything the method derives from a mesh (P1 gradients,
element and median-dual areas, edge lists, fluxes) is computed independently on
each side.

Workload shapes follow the idealised channel (Sect. 4.1) and the global ocean case
(Sect. 4.2) of the paper, scaled to the sizes the benchmark uses:

* ``basin_case``     closed 1000x500 km basin, regular right triangles, Gaussian bump.
* ``channel_case``   zonally periodic 4000x2000 km channel, jittered Delaunay lattice,
                     beta plane, Gaussian ridge, sinusoidal wind forcing.
* ``sphere_case``    icosahedral sphere, fractal bathymetry with land masked out.
* ``ensemble_cases`` many closed basins of uneven size.
* ``periodic_wave_case`` etc.: small doubly periodic meshes used by the closed-form pins.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

G_DEFAULT = 9.81
THETA_DEFAULT = 0.14          # Sect. 2.2, after Eq. (4.10): value recommended for the SE scheme
RHO0 = 1025.0
OMEGA = 7.292e-5
R_EARTH = 6.371e6


@dataclasses.dataclass
class Mesh:
    """Unstructured triangular mesh in the form the library and the oracle take.

    tri       (E,3) int32   vertex indices, counter-clockwise in the element frame
    xy        (E,3,2) f64   corner coordinates in the element's own planar frame (m);
                            periodic meshes are unwrapped per element, spherical meshes
                            are projected onto the plane of the flat triangle
    pos       (V,3) f64     vertex positions used only to order the mesh along a
                            space-filling curve (z = 0 for planar meshes)
    depth     (V,) f64      rest depth H0 at vertices (m)
    coriolis  (E,) f64      Coriolis parameter at the element centroid (1/s)
    """
    name: str
    tri: np.ndarray
    xy: np.ndarray
    pos: np.ndarray
    depth: np.ndarray
    coriolis: np.ndarray

    @property
    def nv(self) -> int:
        return int(self.pos.shape[0])

    @property
    def ne(self) -> int:
        return int(self.tri.shape[0])


@dataclasses.dataclass
class Params:
    g: float = G_DEFAULT
    theta: float = THETA_DEFAULT
    tau: float = 600.0
    M: int = 30
    nonlinear_h: int = 1
    scheme: int = 0            # 0: dissipative forward-backward (Eq. 4.10); 1: AB3-AM4 (Eqs. 4.7-4.8)
    sesm: tuple = None         # (beta, delta, gamma, zeta) for scheme 1; None: the library's default
    visc: tuple = None         # (A_bg m^2/s, C_v) of the barotropic viscosity, Eq. (viscosity_BT); None: off


@dataclasses.dataclass
class Case:
    """A mesh plus everything one run needs."""
    name: str
    mesh: Mesh
    params: Params
    R: np.ndarray              # (E,2) frozen forcing, m^2/s^2, element frame
    eta0: np.ndarray           # (V,) initial elevation (m)
    U0: np.ndarray             # (E,2) initial transport (m^2/s), element frame
    nsteps: int


def _contig(m: Mesh) -> Mesh:
    return Mesh(m.name,
                np.ascontiguousarray(m.tri, dtype=np.int32),
                np.ascontiguousarray(m.xy, dtype=np.float64),
                np.ascontiguousarray(m.pos, dtype=np.float64),
                np.ascontiguousarray(m.depth, dtype=np.float64),
                np.ascontiguousarray(m.coriolis, dtype=np.float64))


# ----------------------------------------------------------------------------------
# planar helpers (pure placement; no discrete operators)
# ----------------------------------------------------------------------------------

def _wrap(d, period):
    if period is None:
        return d
    return d - period * np.round(d / period)


def _unwrapped_corners(P, tri, period_x=None, period_y=None):
    """Corner coordinates of each triangle, unwrapped around corner 0."""
    c = P[tri]                                  # (E,3,2)
    out = c.copy()
    for k in (1, 2):
        out[:, k, 0] = c[:, 0, 0] + _wrap(c[:, k, 0] - c[:, 0, 0], period_x)
        out[:, k, 1] = c[:, 0, 1] + _wrap(c[:, k, 1] - c[:, 0, 1], period_y)
    return out


def _orient(xy):
    """Signed doubled area of each corner triple (orientation test only)."""
    return ((xy[:, 1, 0] - xy[:, 0, 0]) * (xy[:, 2, 1] - xy[:, 0, 1])
            - (xy[:, 2, 0] - xy[:, 0, 0]) * (xy[:, 1, 1] - xy[:, 0, 1]))


def _make_ccw(tri, xy):
    neg = _orient(xy) < 0
    tri = tri.copy()
    xy = xy.copy()
    tri[neg, 1], tri[neg, 2] = tri[neg, 2].copy(), tri[neg, 1].copy()
    xy[neg, 1], xy[neg, 2] = xy[neg, 2].copy(), xy[neg, 1].copy()
    return tri, xy


def rect_right_mesh(nx, ny, dx, periodic_x=False, periodic_y=False):
    """Regular right-triangle mesh with all diagonals in the same direction.

    Vertex (i, j) sits at (i*dx, j*dx); each cell is cut by the diagonal from its
    lower-left to its upper-right corner. Returns (P (V,2), tri (E,3), xy (E,3,2)).
    """
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    P = np.stack([ii.ravel() * dx, jj.ravel() * dx], axis=1).astype(np.float64)
    cx = nx if periodic_x else nx - 1
    cy = ny if periodic_y else ny - 1
    ci, cj = np.meshgrid(np.arange(cx), np.arange(cy), indexing="xy")
    ci = ci.ravel()
    cj = cj.ravel()
    ip = (ci + 1) % nx
    jp = (cj + 1) % ny
    v00 = cj * nx + ci
    v10 = cj * nx + ip
    v11 = jp * nx + ip
    v01 = jp * nx + ci
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tri = np.empty((2 * len(ci), 3), dtype=np.int64)
    tri[0::2] = t1
    tri[1::2] = t2
    # unwrapped corner coordinates from the cell indices (never from wrapped positions)
    x0 = ci * dx
    y0 = cj * dx
    c1 = np.stack([[x0, y0], [x0 + dx, y0], [x0 + dx, y0 + dx]], axis=0).transpose(2, 0, 1)
    c2 = np.stack([[x0, y0], [x0 + dx, y0 + dx], [x0, y0 + dx]], axis=0).transpose(2, 0, 1)
    xy = np.empty((2 * len(ci), 3, 2))
    xy[0::2] = c1
    xy[1::2] = c2
    return P, tri.astype(np.int32), xy


def _incircle(a, b, c, d):
    """>0 when d lies strictly inside the circumcircle of the CCW triangle abc."""
    ax, ay = a[:, 0] - d[:, 0], a[:, 1] - d[:, 1]
    bx, by = b[:, 0] - d[:, 0], b[:, 1] - d[:, 1]
    cx, cy = c[:, 0] - d[:, 0], c[:, 1] - d[:, 1]
    return ((ax * ax + ay * ay) * (bx * cy - cx * by)
            - (bx * bx + by * by) * (ax * cy - cx * ay)
            + (cx * cx + cy * cy) * (ax * by - bx * ay))


def lawson_flip(P, tri, period_x=None, max_rounds=200):
    """Flip interior edges until every one satisfies the empty-circumcircle test."""
    tri = tri.copy()
    for _ in range(max_rounds):
        E = tri.shape[0]
        a = tri.ravel()
        b = np.roll(tri, -1, axis=1).ravel()
        c = np.roll(tri, -2, axis=1).ravel()
        t = np.repeat(np.arange(E), 3)
        lo = np.minimum(a, b).astype(np.int64)
        hi = np.maximum(a, b).astype(np.int64)
        key = lo * (P.shape[0] + 1) + hi
        order = np.argsort(key, kind="stable")
        ks = key[order]
        same = np.nonzero(ks[1:] == ks[:-1])[0]
        h1 = order[same]
        h2 = order[same + 1]
        # quad: triangle t1 = (a, b, c), its twin has the opposite vertex d
        A = P[a[h1]]
        B = P[b[h1]]
        C = P[c[h1]]
        D = P[c[h2]]
        if period_x is not None:
            for X in (B, C, D):
                X[:, 0] = A[:, 0] + _wrap(X[:, 0] - A[:, 0], period_x)
        bad = _incircle(A, B, C, D) > 1e-9 * np.abs(
            (B[:, 0] - A[:, 0]) ** 2 + (B[:, 1] - A[:, 1]) ** 2) ** 2
        idx = np.nonzero(bad)[0]
        if len(idx) == 0:
            return tri
        used = np.zeros(E, dtype=bool)
        n_flip = 0
        for k in idx:
            t1, t2 = t[h1[k]], t[h2[k]]
            if used[t1] or used[t2]:
                continue
            va, vb, vc, vd = a[h1[k]], b[h1[k]], c[h1[k]], c[h2[k]]
            tri[t1] = (va, vd, vc)
            tri[t2] = (vd, vb, vc)
            used[t1] = used[t2] = True
            n_flip += 1
        if n_flip == 0:
            return tri
    raise RuntimeError("Lawson flipping did not converge")


def staggered_lattice(nx, ny, h, periodic_x):
    """Equilateral lattice: rows of nx points, odd rows shifted by h/2, rows h*sqrt(3)/2 apart.

    Returns (P (V,2), tri (E,3)) with counter-clockwise triangles in unwrapped space.
    """
    dy = h * math.sqrt(3.0) / 2.0
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = (i + 0.5 * (j % 2)) * h
    y = j * dy
    P = np.stack([x.ravel(), y.ravel()], axis=1).astype(np.float64)
    tris = []
    ncol = nx if periodic_x else nx - 1
    for r in range(ny - 1):
        ia = np.arange(ncol)
        ib = (ia + 1) % nx
        lo = r * nx
        up = (r + 1) * nx
        if r % 2 == 0:     # lower row unshifted, upper row shifted right by h/2
            tris.append(np.stack([lo + ia, lo + ib, up + ia], axis=1))
            tris.append(np.stack([lo + ib, up + ib, up + ia], axis=1))
        else:              # lower row shifted, upper row unshifted
            tris.append(np.stack([lo + ia, up + ib, up + ia], axis=1))
            tris.append(np.stack([lo + ia, lo + ib, up + ib], axis=1))
    tri = np.concatenate(tris, axis=0).astype(np.int32)
    return P, tri


# ----------------------------------------------------------------------------------
# value noise (seeded, smooth), used for bathymetry and forcing patterns
# ----------------------------------------------------------------------------------

class ValueNoise3:
    """Smooth seeded 3-D value noise on the integer lattice (hashed corner values)."""

    def __init__(self, seed):
        rng = np.random.default_rng(seed)
        self.perm = np.concatenate([rng.permutation(256)] * 2).astype(np.int64)
        self.vals = rng.random(256)

    def _hash(self, ix, iy, iz):
        p = self.perm
        return self.vals[p[p[p[ix & 255] + (iy & 255)] + (iz & 255)]]

    def __call__(self, X):
        f = np.floor(X)
        i = f.astype(np.int64)
        t = X - f
        s = t * t * (3.0 - 2.0 * t)
        out = np.zeros(X.shape[0])
        for dx in (0, 1):
            wx = s[:, 0] if dx else 1.0 - s[:, 0]
            for dy in (0, 1):
                wy = s[:, 1] if dy else 1.0 - s[:, 1]
                for dz in (0, 1):
                    wz = s[:, 2] if dz else 1.0 - s[:, 2]
                    out += wx * wy * wz * self._hash(i[:, 0] + dx, i[:, 1] + dy, i[:, 2] + dz)
        return out

    def fractal(self, X, octaves, base_freq=2.0, persistence=0.5, first_octave=0):
        out = np.zeros(X.shape[0])
        amp = 1.0
        norm = 0.0
        for o in range(first_octave, first_octave + octaves):
            freq = base_freq * (2.0 ** o)
            out += amp * self(X * freq + 17.0 * o)
            norm += amp
            amp *= persistence
        return out / norm


# ----------------------------------------------------------------------------------
# sphere
# ----------------------------------------------------------------------------------

def icosphere(level):
    """Vertices on the unit sphere and CCW (seen from outside) faces of a subdivided icosahedron."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    V = np.array([[-1, phi, 0], [1, phi, 0], [-1, -phi, 0], [1, -phi, 0],
                  [0, -1, phi], [0, 1, phi], [0, -1, -phi], [0, 1, -phi],
                  [phi, 0, -1], [phi, 0, 1], [-phi, 0, -1], [-phi, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
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
        mids = V[uk // nv] + V[uk % nv]
        mids /= np.linalg.norm(mids, axis=1, keepdims=True)
        nf = F.shape[0]
        m01 = nv + inv[:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:]
        F = np.concatenate([
            np.stack([F[:, 0], m01, m20], axis=1),
            np.stack([F[:, 1], m12, m01], axis=1),
            np.stack([F[:, 2], m20, m12], axis=1),
            np.stack([m01, m12, m20], axis=1)], axis=0)
        V = np.concatenate([V, mids], axis=0)
    c = V[F].mean(axis=1)
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = (n * c).sum(axis=1) < 0
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return V, F.astype(np.int32)


def sphere_element_frames(X, tri):
    """Project each flat 3-D triangle onto its own plane.

    The frame's first axis is local east (z x centroid) projected onto the triangle's
    plane, the second completes a right-handed pair with the outward normal, so
    counter-clockwise seen from outside stays counter-clockwise in the frame.
    Returns (xy (E,3,2), latitude of the centroid (E,)).
    """
    P = X[tri]
    c = P.mean(axis=1)
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    chat = c / np.linalg.norm(c, axis=1, keepdims=True)
    east = np.cross(np.array([0.0, 0.0, 1.0])[None, :], chat)
    small = np.linalg.norm(east, axis=1) < 1e-12
    east[small] = np.array([1.0, 0.0, 0.0])
    east -= (east * n).sum(axis=1, keepdims=True) * n
    east /= np.linalg.norm(east, axis=1, keepdims=True)
    north = np.cross(n, east)
    d = P - c[:, None, :]
    xy = np.stack([(d * east[:, None, :]).sum(axis=2), (d * north[:, None, :]).sum(axis=2)], axis=2)
    lat = np.arcsin(np.clip(chat[:, 2], -1.0, 1.0))
    return xy, lat


def _drop_unused(tri, nv):
    used = np.zeros(nv, dtype=bool)
    used[tri.ravel()] = True
    newid = -np.ones(nv, dtype=np.int64)
    newid[used] = np.arange(int(used.sum()))
    return newid[tri].astype(np.int32), used


# ----------------------------------------------------------------------------------
# cases
# ----------------------------------------------------------------------------------

def basin_case(nx=101, ny=51, dx=10e3, H=4000.0, f=1e-4, amp=1.0, sigma=50e3,
               M=30, tau=600.0, nsteps=20, nonlinear_h=1):
    """Closed rectangular basin (1000x500 km at the defaults), Gaussian bump, U = 0, no forcing."""
    P, tri, xy = rect_right_mesh(nx, ny, dx)
    V, E = P.shape[0], tri.shape[0]
    pos = np.concatenate([P, np.zeros((V, 1))], axis=1)
    mesh = _contig(Mesh("basin", tri, xy, pos, np.full(V, H), np.full(E, f)))
    cx, cy = 0.5 * (nx - 1) * dx, 0.5 * (ny - 1) * dx
    r2 = (P[:, 0] - cx) ** 2 + (P[:, 1] - cy) ** 2
    eta0 = amp * np.exp(-r2 / (2.0 * sigma ** 2))
    return Case("basin", mesh, Params(tau=tau, M=M, nonlinear_h=nonlinear_h),
                np.zeros((E, 2)), eta0, np.zeros((E, 2)), nsteps)


def channel_mesh(nx=588, ny=340, Lx=4000e3, Ly=2000e3, jitter=0.2, seed=20231116):
    """Zonally periodic channel: jittered equilateral lattice made Delaunay by edge flips."""
    h = Lx / nx
    P, tri = staggered_lattice(nx, ny, h, periodic_x=True)
    # stretch rows so the walls sit exactly at y = 0 and y = Ly
    P[:, 1] *= Ly / P[:, 1].max()
    rng = np.random.default_rng(seed)
    jx = rng.uniform(-jitter * h, jitter * h, P.shape[0])
    jy = rng.uniform(-jitter * h, jitter * h, P.shape[0])
    wall = (P[:, 1] <= 0.0) | (P[:, 1] >= Ly)
    jy[wall] = 0.0
    P[:, 0] = np.mod(P[:, 0] + jx, Lx)
    P[:, 1] = P[:, 1] + jy
    tri = lawson_flip(P, tri, period_x=Lx)
    xy = _unwrapped_corners(P, tri, period_x=Lx)
    tri, xy = _make_ccw(tri, xy)
    return P, tri, xy, h


def channel_case(nx=588, ny=340, Lx=4000e3, Ly=2000e3, M=40, tau=480.0, nsteps=200, seed=20231116,
                 nonlinear_h=1):
    """Wind-driven zonal channel on a beta plane with a Gaussian ridge (depth 4000 m, ridge top 1500 m)."""
    P, tri, xy, h = channel_mesh(nx, ny, Lx, Ly, seed=seed)
    V, E = P.shape[0], tri.shape[0]
    depth = 4000.0 - 2500.0 * np.exp(-((P[:, 0] - 0.5 * Lx) ** 2) / (2.0 * 200e3 ** 2))
    yc = xy[:, :, 1].mean(axis=1)
    f = 1e-4 + 2e-11 * yc
    taux = -0.1 * np.cos(2.0 * math.pi * yc / Ly)
    R = np.stack([taux / RHO0, np.zeros(E)], axis=1)
    pos = np.concatenate([P, np.zeros((V, 1))], axis=1)
    mesh = _contig(Mesh("channel", tri, xy, pos, depth, f))
    return Case("channel", mesh, Params(tau=tau, M=M, nonlinear_h=nonlinear_h), R,
                np.zeros(V), np.zeros((E, 2)), nsteps)


def sphere_mesh(level=8, land_fraction=0.3, hmin=10.0, hmax=6000.0, seed=20231117):
    """Icosahedral sphere with seeded fractal bathymetry; the shallowest fraction becomes land."""
    X, F = icosphere(level)
    noise = ValueNoise3(seed)
    b = noise.fractal(X, octaves=8, base_freq=1.5, persistence=0.5)
    cut = np.quantile(b, land_fraction)
    wet = b > cut
    keep = wet[F].all(axis=1)
    F = F[keep]
    F, used = _drop_unused(F, X.shape[0])
    X = X[used]
    bw = b[used]
    depth = hmin + (hmax - hmin) * (bw - cut) / (bw.max() - cut)
    Xm = X * R_EARTH
    xy, lat = sphere_element_frames(Xm, F)
    f = 2.0 * OMEGA * np.sin(lat)
    return _contig(Mesh("sphere", F, xy, X, depth, f))


def smooth_element_field(mesh_pos, tri, seed, octaves=4, amp=1.0):
    """Two smooth seeded components per element (centroid samples of value noise), max |v| = amp."""
    Xc = mesh_pos[tri].mean(axis=1)
    Xc = Xc / np.maximum(np.linalg.norm(Xc, axis=1, keepdims=True), 1e-300)
    n1 = ValueNoise3(seed)
    n2 = ValueNoise3(seed + 7919)
    a = np.stack([n1.fractal(Xc, octaves, base_freq=1.0) - 0.5,
                  n2.fractal(Xc, octaves, base_freq=1.0) - 0.5], axis=1)
    m = np.sqrt((a ** 2).sum(axis=1)).max()
    return a * (amp / m)


def sphere_case(level=8, M=50, tau=1800.0, nsteps=50, seed=20231117, forcing_seed=None, nonlinear_h=1):
    """Global-like sphere: fractal bathymetry, 30 % land, f = 2 Omega sin(lat), smooth random forcing."""
    mesh = sphere_mesh(level, seed=seed)
    H0e = mesh.depth[mesh.tri].mean(axis=1)
    a = smooth_element_field(mesh.pos, mesh.tri, seed if forcing_seed is None else forcing_seed, amp=1e-6)
    R = H0e[:, None] * a
    return Case("sphere", mesh, Params(tau=tau, M=M, nonlinear_h=nonlinear_h), R,
                np.zeros(mesh.nv), np.zeros((mesh.ne, 2)), nsteps)


def basin_jittered_mesh(nv_target, aspect, h, seed):
    """Closed basin on a jittered equilateral lattice (boundary vertices left in place)."""
    ny = max(3, int(round(math.sqrt(nv_target / aspect * (2.0 / math.sqrt(3.0))))))
    nx = max(3, int(round(nv_target / ny)))
    P, tri = staggered_lattice(nx, ny, h, periodic_x=False)
    rng = np.random.default_rng(seed)
    jx = rng.uniform(-0.2 * h, 0.2 * h, P.shape[0])
    jy = rng.uniform(-0.2 * h, 0.2 * h, P.shape[0])
    ii = np.arange(P.shape[0]) % nx
    jj = np.arange(P.shape[0]) // nx
    border = (ii == 0) | (ii == nx - 1) | (jj == 0) | (jj == ny - 1)
    jx[border] = 0.0
    jy[border] = 0.0
    P = P + np.stack([jx, jy], axis=1)
    tri = lawson_flip(P, tri)
    xy = P[tri]
    tri, xy = _make_ccw(tri, xy)
    return P, tri, xy


def ensemble_cases(nbasins=64, vmin=2e4, vmax=4e5, h=5e3, M=40, nsteps=50, seed=20231118,
                   f=1e-4, g=G_DEFAULT, theta=THETA_DEFAULT, cfl_fraction=0.8, scale=1.0):
    """Independent closed basins of log-uniform size with smooth random depth and Gaussian bumps.

    Each basin's baroclinic step is tau = M * dt with dt chosen from the gravity-wave
    speed sqrt(g max H) and the lattice spacing so that the substep sits at
    ``cfl_fraction`` of the forward-backward limit 2/sqrt(1+2 theta) for the
    largest lattice wavenumber 4/h (a conservative estimate for jittered lattices).
    ``scale`` shrinks every basin (tests use small ensembles of the same recipe).
    """
    rng = np.random.default_rng(seed)
    cases = []
    for b in range(nbasins):
        nvt = math.exp(rng.uniform(math.log(vmin), math.log(vmax))) * scale
        nvt = max(nvt, 30.0)
        aspect = rng.uniform(1.0, 2.0)
        P, tri, xy = basin_jittered_mesh(nvt, aspect, h, seed=seed * 1000 + b)
        V, E = P.shape[0], tri.shape[0]
        Lx = P[:, 0].max() - P[:, 0].min()
        Ly = P[:, 1].max() - P[:, 1].min()
        dn = ValueNoise3(seed * 1000 + 500 + b)
        Xn = np.stack([P[:, 0] / max(Lx, 1.0), P[:, 1] / max(Lx, 1.0), np.full(V, 0.37 * b)], axis=1)
        d = dn.fractal(Xn, octaves=3, base_freq=2.0)
        d = (d - d.min()) / max(d.max() - d.min(), 1e-12)
        # each basin spans its own seeded sub-range of 1000-5000 m
        dlo = rng.uniform(1000.0, 2500.0)
        dhi = rng.uniform(max(dlo + 500.0, 3000.0), 5000.0)
        depth = dlo + (dhi - dlo) * d
        width = min(Lx, Ly)
        eta0 = np.zeros(V)
        for _ in range(4):
            cx = rng.uniform(P[:, 0].min(), P[:, 0].max())
            cy = rng.uniform(P[:, 1].min(), P[:, 1].max())
            s = rng.uniform(0.05, 0.2) * width
            eta0 += rng.uniform(-1.0, 1.0) * np.exp(-((P[:, 0] - cx) ** 2 + (P[:, 1] - cy) ** 2) / (2 * s * s))
        eta0 *= 0.5 / max(np.abs(eta0).max(), 1e-12)
        cmax = math.sqrt(g * depth.max())
        dt = cfl_fraction * (2.0 / math.sqrt(1.0 + 2.0 * theta)) / (cmax * 4.0 / h)
        pos = np.concatenate([P, np.zeros((V, 1))], axis=1)
        mesh = _contig(Mesh(f"basin{b}", tri, xy, pos, depth, np.full(E, f)))
        cases.append(Case(f"basin{b}", mesh, Params(g=g, theta=theta, tau=M * dt, M=M, nonlinear_h=1),
                          np.zeros((E, 2)), eta0, np.zeros((E, 2)), nsteps))
    return cases


def periodic_square_mesh(n, dx, f=0.0, H=4000.0):
    """Doubly periodic n x n right-triangle mesh (consistent diagonals)."""
    P, tri, xy = rect_right_mesh(n, n, dx, periodic_x=True, periodic_y=True)
    V, E = P.shape[0], tri.shape[0]
    pos = np.concatenate([P, np.zeros((V, 1))], axis=1)
    return _contig(Mesh("periodic", tri, xy, pos, np.full(V, H), np.full(E, f)))


def periodic_wave_case(n=32, dx=10e3, kx=1, ky=0, H=4000.0, M=30, tau=600.0, nsteps=5,
                       theta=THETA_DEFAULT, g=G_DEFAULT):
    """Linear gravity wave: eta0 = cos(2 pi (kx x + ky y) / L) on a periodic mesh, f = 0, U = 0."""
    mesh = periodic_square_mesh(n, dx, f=0.0, H=H)
    L = n * dx
    x, y = mesh.pos[:, 0], mesh.pos[:, 1]
    eta0 = np.cos(2.0 * math.pi * (kx * x + ky * y) / L)
    return Case("periodic_wave", mesh, Params(g=g, theta=theta, tau=tau, M=M, nonlinear_h=0),
                np.zeros((mesh.ne, 2)), eta0, np.zeros((mesh.ne, 2)), nsteps)


def tiny_jittered_case(nx=6, ny=5, h=10e3, seed=1, f=1e-4, H=3000.0, M=4, tau=40.0,
                       nonlinear_h=1, forcing=True):
    """A few dozen vertices: closed jittered basin with random depth, forcing and initial state."""
    rng = np.random.default_rng(seed)
    P, tri, xy = basin_jittered_mesh(nx * ny, nx / ny, h, seed=seed)
    V, E = P.shape[0], tri.shape[0]
    depth = H * (0.6 + 0.8 * rng.random(V))
    pos = np.concatenate([P, np.zeros((V, 1))], axis=1)
    fe = f * (0.5 + rng.random(E))
    mesh = _contig(Mesh("tiny", tri, xy, pos, depth, fe))
    R = (1e-3 * rng.standard_normal((E, 2))) if forcing else np.zeros((E, 2))
    eta0 = 0.3 * rng.standard_normal(V)
    U0 = 5.0 * rng.standard_normal((E, 2))
    return Case("tiny", mesh, Params(tau=tau, M=M, nonlinear_h=nonlinear_h), R, eta0, U0, 3)
