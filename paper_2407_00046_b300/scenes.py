"""Seeded synthetic scene generators: tetrahedral meshes, materials, pins.

This module produces *inputs only*: rest positions, tet connectivity, surface
triangles/edges, per-tet Young's modulus / Poisson ratio / density, pinned
vertices, initial velocities and the time-step parameters. It holds none of the
method's arithmetic (no masses, no D_m^-1, no energies): both the CUDA path and
the FP64 oracle compute those themselves from what is produced here.

The paper's scenes (Table 1, Sec. 6) use meshes that are not available; these
generators stand in for them with lattice bodies of the same kind: stacked
Neo-Hookean cubes, a cube dropped on a slab, and a heterogeneous scene of an
interlocked torus-link chain net (E = 1 GPa) under spiked spherical shells
(E = 5e5 Pa), shaped like the "Puffer Balls on Nets" scene (Table 1: 1.76M tets,
h = 1/30 s, dhat = 1e-3, nu = 0.4, density 1e3).

Hex cells are split into 6 tets along the main diagonal (Kuhn split) with the
local axes taken in global lattice order, so neighbouring cells always agree on
the shared face diagonals and the tet mesh is conforming.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

__all__ = [
    "Scene",
    "lattice_box",
    "torus_link",
    "spiked_shell",
    "merge_bodies",
    "surface_of",
    "two_cubes",
    "cube_stack",
    "chain_net_shells",
    "cube_on_slab",
    "cube_columns",
    "scene_by_name",
]


@dataclasses.dataclass
class Scene:
    """A simulation input. All arrays are host numpy arrays.

    X        [N_v,3] f64  rest positions (also the initial positions x_0)
    V0       [N_v,3] f64  initial velocities
    tets     [N_t,4] i32  positively oriented tetrahedra
    E, nu, rho [N_t] f64  per-tet Young's modulus (Pa), Poisson ratio, density
    pinned   [N_v]   u8   1 = Dirichlet vertex (held at its initial position)
    tris     [N_f,3] i32  boundary triangles
    edges    [N_e,2] i32  boundary edges (i < j)
    surf_verts [N_sv] i32 vertices on the boundary
    body     [N_v]   i32  body id of each vertex
    h, dhat           time step (s) and contact offset (m)
    gravity  [3]     f64  gravitational acceleration (m/s^2)
    """

    name: str
    X: np.ndarray
    V0: np.ndarray
    tets: np.ndarray
    E: np.ndarray
    nu: np.ndarray
    rho: np.ndarray
    pinned: np.ndarray
    tris: np.ndarray
    edges: np.ndarray
    surf_verts: np.ndarray
    body: np.ndarray
    h: float = 1.0 / 30.0
    dhat: float = 1e-3
    gravity: np.ndarray = dataclasses.field(
        default_factory=lambda: np.array([0.0, -9.81, 0.0]))
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def n_verts(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


# --------------------------------------------------------------------------
# Hex -> 6 tets (Kuhn split). Corner c of a hex has bits (bit0, bit1, bit2) =
# offsets along its three local axes. Each tet is a monotone path 000 -> 111.
_KUHN = np.array(
    [[0, 1 << p[0], (1 << p[0]) | (1 << p[1]), 7]
     for p in itertools.permutations(range(3))], dtype=np.int64)


def _kuhn_split(corners: np.ndarray) -> np.ndarray:
    """corners [n_hex, 8] vertex ids indexed by corner bits -> tets [6 n_hex, 4]."""
    return corners[:, _KUHN].reshape(-1, 4)


def _orient(X: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Swap two vertices of every negatively oriented tet (orientation only)."""
    a, b, c, d = (X[tets[:, k]] for k in range(4))
    vol6 = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a)
    if np.any(np.abs(vol6) == 0.0):
        raise ValueError("degenerate tet in generated mesh")
    t = tets.copy()
    neg = vol6 < 0
    t[neg, 2], t[neg, 3] = tets[neg, 3], tets[neg, 2]
    return t


def _rotation(axis: np.ndarray, angle: float) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]],
                  [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def _random_rotation(rng: np.random.Generator, max_deg: float) -> np.ndarray:
    axis = rng.normal(size=3)
    return _rotation(axis, math.radians(rng.uniform(0.0, max_deg)))


# --------------------------------------------------------------------------
# bodies: (X, tets) pairs
def lattice_box(nx: int, ny: int, nz: int, size) -> tuple[np.ndarray, np.ndarray]:
    """Axis-aligned box [0,sx]x[0,sy]x[0,sz], nx*ny*nz cells, 6 tets per cell.

    Vertex (i,j,k) has id i + (nx+1)*(j + (ny+1)*k)."""
    sx, sy, sz = size
    xs = np.linspace(0.0, sx, nx + 1)
    ys = np.linspace(0.0, sy, ny + 1)
    zs = np.linspace(0.0, sz, nz + 1)
    K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1),
                          indexing="ij")
    X = np.stack([xs[I.ravel()], ys[J.ravel()], zs[K.ravel()]], axis=1)
    vid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)  # noqa: E731
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    corners = np.stack([vid(i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1))
                        for c in range(8)], axis=1)
    tets = _orient(X, _kuhn_split(corners))
    return X, tets.astype(np.int32)


def torus_link(R: float, half: float, n_theta: int = 48, n_cross: int = 4):
    """Closed torus link with a square cross-section (side 2*half), centred at
    the origin, ring in the xz-plane (axis y). Hex sweep n_theta x n_cross^2."""
    nc = n_cross + 1
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    off = np.linspace(-half, half, nc)
    T, U, W = np.meshgrid(np.arange(n_theta), np.arange(nc), np.arange(nc),
                          indexing="ij")
    T, U, W = T.ravel(), U.ravel(), W.ravel()
    rad = R + off[U]
    X = np.stack([rad * np.cos(th[T]), off[W], rad * np.sin(th[T])], axis=1)
    vid = lambda t, u, w: (t % n_theta) * nc * nc + u * nc + w  # noqa: E731
    t, u, w = np.meshgrid(np.arange(n_theta), np.arange(n_cross), np.arange(n_cross),
                          indexing="ij")
    t, u, w = t.ravel(), u.ravel(), w.ravel()
    corners = np.stack([vid(t + (c & 1), u + ((c >> 1) & 1), w + ((c >> 2) & 1))
                        for c in range(8)], axis=1)
    tets = _orient(X, _kuhn_split(corners))
    return X, tets.astype(np.int32)


def spiked_shell(radius: float, thickness: float, m: int, layers: int,
                 n_spikes: int, spike_len: float, rng: np.random.Generator):
    """Cubed-sphere shell (outer radius `radius`) of 6*m*m*layers hexes, with
    `n_spikes` tapered spikes of 4 x (2x2) hexes extruded from its outer face."""
    # surface lattice of the cube [0,m]^3
    g = np.arange(m + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    on = (I == 0) | (I == m) | (J == 0) | (J == m) | (K == 0) | (K == m)
    pts = np.stack([I[on], J[on], K[on]], axis=1)
    ns = pts.shape[0]
    lut = -np.ones((m + 1,) * 3, dtype=np.int64)
    lut[pts[:, 0], pts[:, 1], pts[:, 2]] = np.arange(ns)
    q = np.tan((2.0 * pts / m - 1.0) * (np.pi / 4))  # equiangular cube map
    dirs = q / np.linalg.norm(q, axis=1, keepdims=True)
    r_in = radius - thickness
    radii = r_in + thickness * np.arange(layers + 1) / layers
    # vertex id = surface point * (layers+1) + layer
    X = (dirs[:, None, :] * radii[None, :, None]).reshape(-1, 3)
    nl = layers + 1
    corners_all = []
    faces = []  # (normal axis, side)
    for ax in range(3):
        for side in (0, m):
            faces.append((ax, side))
    for ax, side in faces:
        p_ax, q_ax = [a for a in range(3) if a != ax]
        a, b, l = np.meshgrid(np.arange(m), np.arange(m), np.arange(layers), indexing="ij")
        a, b, l = a.ravel(), b.ravel(), l.ravel()
        cs = []
        for c in range(8):
            co = np.zeros((a.size, 3), dtype=np.int64)
            co[:, ax] = side
            co[:, p_ax] = a + (c & 1)
            co[:, q_ax] = b + ((c >> 1) & 1)
            s = lut[co[:, 0], co[:, 1], co[:, 2]]
            cs.append(s * nl + l + ((c >> 2) & 1))
        corners_all.append(np.stack(cs, axis=1))
    corners = np.concatenate(corners_all, axis=0)
    # spikes: 2x2 patches strictly inside a face, not touching each other
    taken = set()
    spikes = []
    tries = 0
    while len(spikes) < n_spikes:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place spikes")
        f = int(rng.integers(6))
        a0 = int(rng.integers(1, m - 2))
        b0 = int(rng.integers(1, m - 2))
        cells = {(f, a0 + da, b0 + db) for da in range(-1, 3) for db in range(-1, 3)}
        if cells & taken:
            continue
        taken |= cells
        spikes.append((f, a0, b0))
    extra_X = []
    extra_corners = []
    next_id = X.shape[0]
    for f, a0, b0 in spikes:
        ax, side = faces[f]
        p_ax, q_ax = [a for a in range(3) if a != ax]
        base = np.zeros((3, 3), dtype=np.int64)
        for da in range(3):
            for db in range(3):
                co = [0, 0, 0]
                co[ax] = side
                co[p_ax] = a0 + da
                co[q_ax] = b0 + db
                base[da, db] = lut[co[0], co[1], co[2]] * nl + layers
        bpos = X[base.ravel()].reshape(3, 3, 3)
        centre = bpos[1, 1]
        normal = centre / np.linalg.norm(centre)
        ids = np.zeros((5, 3, 3), dtype=np.int64)
        ids[0] = base
        for k in range(1, 5):
            taper = 1.0 - 0.125 * k
            pos = centre + (bpos - centre) * taper + normal * (spike_len * k / 4)
            ids[k] = next_id + np.arange(9).reshape(3, 3)
            next_id += 9
            extra_X.append(pos.reshape(9, 3))
        for k in range(4):
            for da in range(2):
                for db in range(2):
                    cs = [ids[k + ((c >> 2) & 1), da + (c & 1), db + ((c >> 1) & 1)]
                          for c in range(8)]
                    extra_corners.append(cs)
    if extra_X:
        X = np.concatenate([X, np.concatenate(extra_X, axis=0)], axis=0)
        corners = np.concatenate([corners, np.array(extra_corners, dtype=np.int64)], axis=0)
    tets = _orient(X, _kuhn_split(corners))
    return X, tets.astype(np.int32)


# --------------------------------------------------------------------------
def surface_of(tets: np.ndarray):
    """Boundary triangles (outward for positive tets), edges, vertices."""
    t = tets.astype(np.int64)
    f = np.concatenate([t[:, [1, 2, 3]], t[:, [0, 3, 2]], t[:, [0, 1, 3]],
                        t[:, [0, 2, 1]]], axis=0)
    key = np.sort(f, axis=1)
    n = int(t.max()) + 1 if t.size else 1
    k = (key[:, 0] * n + key[:, 1]) * n + key[:, 2]
    _, inv, cnt = np.unique(k, return_inverse=True, return_counts=True)
    tris = f[cnt[inv] == 1]
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]], axis=0)
    e = np.sort(e, axis=1)
    edges = np.unique(e, axis=0)
    sv = np.unique(tris.ravel())
    return tris.astype(np.int32), edges.astype(np.int32), sv.astype(np.int32)


def merge_bodies(name, bodies, h=1.0 / 30.0, dhat=1e-3, info=None) -> Scene:
    """bodies: list of dicts with X, tets, E, nu, rho (scalars or per-tet),
    pinned (per-vertex bool, optional) and V0 (3-vector or per-vertex)."""
    Xs, Ts, Es, nus, rhos, pins, vs, bid = [], [], [], [], [], [], [], []
    off = 0
    for b_i, b in enumerate(bodies):
        X, T = b["X"], b["tets"]
        nv, nt = X.shape[0], T.shape[0]
        Xs.append(X)
        Ts.append(T.astype(np.int64) + off)
        Es.append(np.broadcast_to(np.asarray(b["E"], dtype=np.float64), (nt,)))
        nus.append(np.broadcast_to(np.asarray(b.get("nu", 0.4), dtype=np.float64), (nt,)))
        rhos.append(np.broadcast_to(np.asarray(b.get("rho", 1000.0), dtype=np.float64), (nt,)))
        pins.append(np.asarray(b.get("pinned", np.zeros(nv, bool)), dtype=np.uint8))
        vs.append(np.broadcast_to(np.asarray(b.get("V0", np.zeros(3)), dtype=np.float64), (nv, 3)))
        bid.append(np.full(nv, b_i, dtype=np.int32))
        off += nv
    tets = np.concatenate(Ts).astype(np.int32)
    tris, edges, sv = surface_of(tets)
    return Scene(name=name, X=np.ascontiguousarray(np.concatenate(Xs)),
                 V0=np.ascontiguousarray(np.concatenate(vs)), tets=tets,
                 E=np.concatenate(Es).copy(), nu=np.concatenate(nus).copy(),
                 rho=np.concatenate(rhos).copy(), pinned=np.concatenate(pins),
                 tris=tris, edges=edges, surf_verts=sv, body=np.concatenate(bid),
                 h=h, dhat=dhat, info=dict(info or {}))


def _cube(n, L, R=None, lower_corner=(0.0, 0.0, 0.0)):
    X, T = lattice_box(n, n, n, (L, L, L))
    X = X - L / 2
    if R is not None:
        X = X @ R.T
    lo = X.min(axis=0)
    return X - lo + np.asarray(lower_corner), T


# --------------------------------------------------------------------------
# the five workloads
def two_cubes(n: int = 7, L: float = 0.1, gap: float = 0.01, E: float = 1e5) -> Scene:
    """Two stacked lattice cubes (n^3 cells x 6 tets each), `gap` apart; the
    bottom face of the lower cube is pinned."""
    X0, T0 = _cube(n, L, lower_corner=(-L / 2, 0.0, -L / 2))
    X1, T1 = _cube(n, L, lower_corner=(-L / 2, L + gap, -L / 2))
    pin0 = X0[:, 1] <= 1e-12
    return merge_bodies("two_cubes", [
        dict(X=X0, tets=T0, E=E, pinned=pin0),
        dict(X=X1, tets=T1, E=E),
    ], info=dict(n=n, L=L, gap=gap))


def cube_stack(n_cubes: int = 8, n: int = 24, L: float = 0.1, gap: float = 0.01,
               E_range=(1e5, 1e6), seed: int = 2, max_rot_deg: float = 15.0,
               max_offset: float = 0.01) -> Scene:
    """Cubes stacked in y with seeded xz offsets and rotations; AABB gaps of
    `gap`; per-cube E log-uniform in E_range; the lowest cube is unrotated and
    pinned at its base."""
    rng = np.random.default_rng(seed)
    bodies = []
    y = 0.0
    for c in range(n_cubes):
        R = None if c == 0 else _random_rotation(rng, max_rot_deg)
        off = np.zeros(3) if c == 0 else np.array(
            [rng.uniform(-max_offset, max_offset), 0.0, rng.uniform(-max_offset, max_offset)])
        X, T = _cube(n, L, R)
        ext = X.max(axis=0) - X.min(axis=0)
        X = X + np.array([-ext[0] / 2 + off[0], y, -ext[2] / 2 + off[2]])
        E = float(np.exp(rng.uniform(np.log(E_range[0]), np.log(E_range[1]))))
        pin = (X[:, 1] <= y + 1e-12) if c == 0 else None
        d = dict(X=X, tets=T, E=E)
        if pin is not None:
            d["pinned"] = pin
        bodies.append(d)
        y = X[:, 1].max() + gap
    return merge_bodies(f"cube_stack{n_cubes}_n{n}", bodies,
                        info=dict(n_cubes=n_cubes, n=n, seed=seed))


def cube_columns(cols: int = 4, high: int = 4, n: int = 14, L: float = 0.1,
                 gap: float = 0.01, E_range=(1e5, 1e9), seed: int = 5,
                 max_rot_deg: float = 15.0) -> Scene:
    """cols x cols columns of `high` cubes; the bottom layer is unrotated and
    pinned at its base; E log-uniform per cube."""
    rng = np.random.default_rng(seed)
    bodies = []
    pitch = L * 1.3 + gap
    for ci in range(cols):
        for cj in range(cols):
            y = 0.0
            for lev in range(high):
                R = None if lev == 0 else _random_rotation(rng, max_rot_deg)
                X, T = _cube(n, L, R)
                ext = X.max(axis=0) - X.min(axis=0)
                X = X + np.array([ci * pitch - ext[0] / 2, y, cj * pitch - ext[2] / 2])
                E = float(np.exp(rng.uniform(np.log(E_range[0]), np.log(E_range[1]))))
                d = dict(X=X, tets=T, E=E)
                if lev == 0:
                    d["pinned"] = X[:, 1] <= 1e-12
                bodies.append(d)
                y = X[:, 1].max() + gap
    return merge_bodies(f"cube_columns{cols}x{cols}x{high}_n{n}", bodies,
                        info=dict(cols=cols, high=high, n=n, seed=seed))


def cube_on_slab(n_cube: int = 26, L: float = 0.1, slab_cells=(58, 10, 58),
                 slab_size=(0.4, 0.05, 0.4), gap: float = 0.01, seed: int = 4,
                 E_cube: float = 1e5, E_slab: float = 1e6) -> Scene:
    """A lattice cube `gap` above a slab whose bottom face is pinned; the cube
    gets v0 = (0,-1,0) + 0.05 N(0, I). info['target'] is a seeded point near the
    slab top (used by the adjoint loss)."""
    rng = np.random.default_rng(seed)
    Xs, Ts = lattice_box(*slab_cells, slab_size)
    Xs = Xs - np.array([slab_size[0] / 2, 0.0, slab_size[2] / 2])
    Xc, Tc = _cube(n_cube, L, lower_corner=(-L / 2, slab_size[1] + gap, -L / 2))
    v_cube = np.array([0.0, -1.0, 0.0]) + 0.05 * rng.normal(size=3)
    target = np.array([0.0, slab_size[1], 0.0]) + rng.uniform(-0.05, 0.05, size=3)
    return merge_bodies("cube_on_slab", [
        dict(X=Xc, tets=Tc, E=E_cube, V0=v_cube),
        dict(X=Xs, tets=Ts, E=E_slab, pinned=Xs[:, 1] <= 1e-12),
    ], info=dict(target=target, cube_body=0, n_cube=n_cube, seed=seed))


def sliding_cube(n_cube: int = 3, L: float = 0.05, slab_size=(0.3, 0.02, 0.3),
                 gap: float = 5e-4, speed: float = 1.0, E: float = 1e5) -> Scene:
    """A lattice cube resting `gap` (inside dhat) on a fully pinned one-cell
    slab and sliding at `speed` along the slab's top diagonal (the line
    x = z): the friction workload (Sec. 4.1). The cube's vertices stay half a
    cell off that line, so every pair within dhat is an interior PT or EE pair
    with a vertical normal and Coulomb's law fixes the tangential impulse per
    step from the normal one."""
    Xs, Ts = lattice_box(1, 1, 1, slab_size)
    Xs = Xs - np.array([slab_size[0] / 2, slab_size[1], slab_size[2] / 2])
    Xc, Tc = _cube(n_cube, L, lower_corner=(-0.12, gap, -0.12 - L / (2 * n_cube)))
    v0 = speed * np.array([1.0, 0.0, 1.0]) / np.sqrt(2.0)
    return merge_bodies("sliding_cube", [
        dict(X=Xc, tets=Tc, E=E, V0=v0),
        dict(X=Xs, tets=Ts, E=1e6, pinned=np.ones(Xs.shape[0], bool)),
    ], info=dict(n_cube=n_cube, gap=gap, cube_body=0))


def chain_net_shells(nx: int = 9, nz: int = 10, R: float = 0.035, half: float = 0.006,
                     e: float = 0.014, n_shells: int = 4, shell_radius: float = 0.10,
                     shell_thick: float = 0.01, shell_m: int = 32, shell_layers: int = 4,
                     n_spikes: int = 64, spike_len: float = 0.02, drop_gap: float = 0.02,
                     seed: int = 3, E_net: float = 1e9, E_shell: float = 5e5,
                     link_theta: int = 48, link_cross: int = 4) -> Scene:
    """Interlocked torus-link chain net under spiked spherical shells.

    Net: nx*nz flat rings (ring plane xz) at pitch s = 2(R+e), joined by
    vertical connector rings: x-connectors (plane xy) between x-neighbours and
    z-connectors (plane yz) between z-neighbours. Each connector passes through
    the holes of its two flat rings at distance e from their centres, so the
    links interlock without touching (clearance > 1 mm). The cross-section
    (2*half, n_cross cells) keeps the surface cells well above dhat so that no
    surface comes within dhat of itself at rest. Border flat rings are
    pinned. Shells (cubed sphere, outer radius shell_radius, thickness
    shell_thick, 6*m^2*layers hexes, plus tapered spikes) hang in a 2x2 grid
    drop_gap above the net."""
    rng = np.random.default_rng(seed)
    s = 2.0 * (R + e)
    Xl, Tl = torus_link(R, half, link_theta, link_cross)
    bodies = []
    rot_xy = np.array([[1.0, 0, 0], [0, 0, -1.0], [0, 1.0, 0]])   # ring plane xz -> xy
    rot_yz = np.array([[0, 1.0, 0], [-1.0, 0, 0], [0, 0, 1.0]])   # ring plane xz -> yz
    for i in range(nx):
        for k in range(nz):
            border = i in (0, nx - 1) or k in (0, nz - 1)
            X = Xl + np.array([i * s, 0.0, k * s])
            d = dict(X=X, tets=Tl, E=E_net)
            if border:
                d["pinned"] = np.ones(X.shape[0], bool)
            bodies.append(d)
    for k in range(nz):
        for i in range(nx - 1):
            X = Xl @ rot_xy.T + np.array([(i + 0.5) * s, 0.0, k * s])
            bodies.append(dict(X=X, tets=Tl, E=E_net))
    for i in range(nx):
        for k in range(nz - 1):
            X = Xl @ rot_yz.T + np.array([i * s, 0.0, (k + 0.5) * s])
            bodies.append(dict(X=X, tets=Tl, E=E_net))
    net_top = R + half
    cx, cz = (nx - 1) * s / 2, (nz - 1) * s / 2
    sep = 2.0 * (shell_radius + spike_len) + 0.02
    reach = shell_radius + spike_len
    for si in range(n_shells):
        Xs, Ts = spiked_shell(shell_radius, shell_thick, shell_m, shell_layers,
                              n_spikes, spike_len, rng)
        Xs = Xs @ _random_rotation(rng, 180.0).T
        gx, gz = si % 2, si // 2
        centre = np.array([cx + (gx - 0.5) * sep, net_top + drop_gap + reach,
                           cz + (gz - 0.5) * sep])
        bodies.append(dict(X=Xs + centre, tets=Ts, E=E_shell))
    return merge_bodies("chain_net_shells", bodies,
                        info=dict(nx=nx, nz=nz, n_links=nx * nz + nz * (nx - 1) + nx * (nz - 1),
                                  n_shells=n_shells, seed=seed))


def scene_by_name(name: str) -> Scene:
    """The named workloads: 'two_cubes' (4,116 tets), 'cube_stack' (663,552),
    'chain_net_shells' (~1.77M), 'cube_on_slab' (307,296), 'cube_columns'
    (1,053,696), plus a few small variants used by tests."""
    table = {
        "two_cubes": lambda: two_cubes(),
        "two_cubes_small": lambda: two_cubes(n=3),
        "cube_stack": lambda: cube_stack(),
        "cube_stack_small": lambda: cube_stack(n_cubes=3, n=6),
        "chain_net_shells": lambda: chain_net_shells(),
        "chain_net_shells_small": lambda: chain_net_shells(
            nx=3, nz=3, n_shells=1, shell_m=8, shell_layers=2, n_spikes=8,
            link_theta=24, link_cross=2),
        "cube_on_slab": lambda: cube_on_slab(),
        "cube_on_slab_small": lambda: cube_on_slab(n_cube=4, slab_cells=(8, 2, 8)),
        "cube_columns": lambda: cube_columns(),
        "sliding_cube": lambda: sliding_cube(),
    }
    return table[name]()
