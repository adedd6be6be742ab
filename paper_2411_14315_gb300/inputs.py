"""Seeded synthetic inputs: meshes, boundary tags, waveform harmonics, inflow profiles, random states.

This module serves both the CUDA path and the CPU oracle, so it holds none of the harmonic balance
method's arithmetic (no residual, no Jacobian, no spectral operator, no sampling of harmonics onto time
instances).  It only builds the inputs the method is applied to.

Geometry stands in for the paper's patient meshes (Sec. 3: Glenn, cerebral and coronary cases, whose
models come from an external repository): a straight pipe (oscillatory pipe flow), a T-junction of two
inflow tubes and a transverse outflow tube (Glenn-like), a tortuous tube with a saccular bulge
(cerebral-like) and stenosed tubes (coronary-like).  Tetrahedra are linear (P1, Sec. 2.3) and come from
a conforming 6-tetrahedra split of hexahedra.

Face tags: 0 is a no-slip wall; positive tags are caps (inlets or outlets).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# 6-tetrahedra (Kuhn) split of a hexahedron with vertex index v = i + 2 j + 4 k.  Every tetrahedron
# walks the main diagonal 0 -> 7, so two hexahedra that agree on the direction of their in-face axes
# split a shared face along the same diagonal, and the mesh stays conforming.
_KUHN = np.array([(0, 1, 3, 7), (0, 3, 2, 7), (0, 2, 6, 7), (0, 6, 4, 7), (0, 4, 5, 7), (0, 5, 1, 7)],
                 dtype=np.int64)
# local faces of a tetrahedron, opposite local vertex 0, 1, 2, 3
_TET_FACES = np.array([(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)], dtype=np.int64)


@dataclasses.dataclass
class Mesh:
    xyz: np.ndarray          # [n_nodes, 3] float64
    tets: np.ndarray         # [n_tets, 4] int32
    faces: np.ndarray        # [n_faces, 3] int32 boundary triangles
    face_tag: np.ndarray     # [n_faces] int32, 0 = wall
    inlet_tags: tuple
    outlet_tags: tuple
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_faces(self) -> int:
        return int(self.faces.shape[0])


# ----------------------------------------------------------------------------------------------------
# assembly helpers


def _merge_nodes(points: np.ndarray, scale: float):
    """Merge coincident points; returns (unique xyz, inverse index)."""
    key = np.round(points / (scale * 1e-9)).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    return points[first], inv.reshape(-1)


def _signed_volume6(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    x0 = xyz[tets[:, 0]]
    a = xyz[tets[:, 1]] - x0
    b = xyz[tets[:, 2]] - x0
    c = xyz[tets[:, 3]] - x0
    return np.einsum("ij,ij->i", a, np.cross(b, c))


def _orient_positive(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    neg = _signed_volume6(xyz, tets) < 0
    t = tets.copy()
    t[neg, 2], t[neg, 3] = tets[neg, 3], tets[neg, 2]
    return t


def boundary_faces(tets: np.ndarray, n_nodes: int):
    """Triangles that belong to exactly one tetrahedron, in the owning tetrahedron's local order."""
    f = tets[:, _TET_FACES].reshape(-1, 3).astype(np.int64)
    s = np.sort(f, axis=1)
    if n_nodes >= (1 << 21):
        raise ValueError("too many nodes for the face key")
    key = (s[:, 0] << 42) | (s[:, 1] << 21) | s[:, 2]
    _, idx, cnt = np.unique(key, return_index=True, return_counts=True)
    return f[idx[cnt == 1]]


def _finish(xyz, hexes, tag_fn, inlet_tags, outlet_tags, name) -> Mesh:
    tets = hexes[:, _KUHN].reshape(-1, 4)
    tets = _orient_positive(xyz, tets)
    faces = boundary_faces(tets, xyz.shape[0])
    tags = tag_fn(xyz, faces).astype(np.int32)
    return Mesh(xyz=np.ascontiguousarray(xyz, dtype=np.float64),
                tets=np.ascontiguousarray(tets, dtype=np.int32),
                faces=np.ascontiguousarray(faces, dtype=np.int32),
                face_tag=np.ascontiguousarray(tags, dtype=np.int32),
                inlet_tags=tuple(inlet_tags), outlet_tags=tuple(outlet_tags), name=name)


def _structured_hexes(nx: int, ny: int, nz: int) -> np.ndarray:
    """Hexahedra of an (nx+1) x (ny+1) x (nz+1) lattice whose node id is i + (nx+1)(j + (ny+1) k)."""
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    sx, sy = 1, nx + 1
    sz = (nx + 1) * (ny + 1)
    base = i * sx + j * sy + k * sz
    off = np.array([0, sx, sy, sx + sy, sz, sz + sx, sz + sy, sz + sx + sy])
    return base[:, None] + off[None, :]


# ----------------------------------------------------------------------------------------------------
# box


def box_mesh(nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 1.0, lz: float = 1.0,
             origin=(0.0, 0.0, 0.0), jitter: float = 0.0, seed: int = 0) -> Mesh:
    """Box [0,lx]x[0,ly]x[0,lz] + origin split into 6 nx ny nz tetrahedra.

    Tags: 1 x-min, 2 x-max, 3 y-min, 4 y-max, 5 z-min, 6 z-max (no wall tag).  `jitter` moves interior
    nodes by up to that fraction of a cell, to break the lattice's symmetry in tests.
    """
    x = np.linspace(0.0, lx, nx + 1)
    y = np.linspace(0.0, ly, ny + 1)
    z = np.linspace(0.0, lz, nz + 1)
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    xyz = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                    Z.transpose(2, 1, 0).ravel()], axis=1)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        h = np.array([lx / nx, ly / ny, lz / nz])
        interior = ((xyz[:, 0] > 1e-12) & (xyz[:, 0] < lx - 1e-12) & (xyz[:, 1] > 1e-12)
                    & (xyz[:, 1] < ly - 1e-12) & (xyz[:, 2] > 1e-12) & (xyz[:, 2] < lz - 1e-12))
        xyz[interior] += jitter * h * rng.uniform(-1, 1, size=(int(interior.sum()), 3))
    xyz = xyz + np.asarray(origin, dtype=np.float64)
    hexes = _structured_hexes(nx, ny, nz)
    o = np.asarray(origin, dtype=np.float64)
    ext = np.array([lx, ly, lz])

    def tag_fn(p, faces):
        tags = np.zeros(faces.shape[0], dtype=np.int32)
        for axis in range(3):
            for side in range(2):
                val = o[axis] + side * ext[axis]
                on = np.all(np.abs(p[faces, axis] - val) < 1e-9 * max(ext), axis=1)
                tags[on] = 1 + 2 * axis + side
        return tags

    return _finish(xyz, hexes, tag_fn, (), (), f"box{nx}x{ny}x{nz}")


# ----------------------------------------------------------------------------------------------------
# O-grid pipe (straight, or with a radius profile along the axis)


def _ogrid_section(n_core: int, n_rim: int, core_frac: float = 0.5):
    """Quadrilaterals of a unit disc: a square core of n_core^2 cells and 4 rim blocks of n_core x n_rim.

    Returns (points [P,2], quads [Q,4]) with quad corners ordered (i,j), (i+1,j), (i,j+1), (i+1,j+1) in
    block-local axes whose directions agree across every block interface (see _KUHN)."""
    a = core_frac * 0.9                                          # half side of the core square
    s = -a + 2.0 * a * np.arange(n_core + 1) / n_core          # core lattice coordinates
    pts = []
    quads = []

    def add_block(P):  # P [ni+1, nj+1, 2]
        ni, nj = P.shape[0] - 1, P.shape[1] - 1
        base = sum(p.shape[0] for p in pts)
        pts.append(P.reshape(-1, 2))
        idx = base + np.arange((ni + 1) * (nj + 1)).reshape(ni + 1, nj + 1)
        q = np.stack([idx[:-1, :-1], idx[1:, :-1], idx[:-1, 1:], idx[1:, 1:]], axis=-1).reshape(-1, 4)
        quads.append(q)

    X, Y = np.meshgrid(s, s, indexing="ij")
    add_block(np.stack([X, Y], axis=-1))                       # core: i along +x, j along +y

    def arc(m):
        th = -0.75 * math.pi + 0.5 * math.pi * (np.asarray(m) % (4 * n_core)) / n_core
        return np.stack([np.cos(th), np.sin(th)], axis=-1)

    i = np.arange(n_core + 1)
    t = np.arange(n_rim + 1) / n_rim
    sides = [
        (np.stack([s, np.full_like(s, -a)], -1), arc(i)),                    # bottom, s along +x
        (np.stack([np.full_like(s, a), s], -1), arc(n_core + i)),            # right, s along +y
        (np.stack([s, np.full_like(s, a)], -1), arc(3 * n_core - i)),        # top, s along +x
        (np.stack([np.full_like(s, -a), s], -1), arc(4 * n_core - i)),       # left, s along +y
    ]
    for inner, outer in sides:
        P = inner[:, None, :] + (outer - inner)[:, None, :] * t[None, :, None]
        add_block(P)
    return np.concatenate(pts, 0), np.concatenate(quads, 0)


def pipe_mesh(R: float, L: float, n_core: int, n_rim: int, n_axial: int, radius_fn=None,
              name: str = "pipe") -> Mesh:
    """Pipe of radius R along +z from z=0 (inlet, tag 1) to z=L (outlet, tag 2); wall tag 0.

    radius_fn(z) gives the local radius (stenoses); default R everywhere."""
    p2, q = _ogrid_section(n_core, n_rim)
    p2, inv = _merge_nodes(p2, 1.0)
    q = inv[q]
    n2 = p2.shape[0]
    z = L * np.arange(n_axial + 1) / n_axial
    rad = np.full(n_axial + 1, R) if radius_fn is None else np.asarray([radius_fn(zz) for zz in z])
    xyz = np.concatenate([np.concatenate([p2 * rad[k], np.full((n2, 1), z[k])], 1)
                          for k in range(n_axial + 1)], 0)
    k = np.arange(n_axial)
    lo = q[None, :, :] + (k * n2)[:, None, None]
    hexes = np.concatenate([lo, lo + n2], axis=2).reshape(-1, 8)

    def tag_fn(p, faces):
        tags = np.zeros(faces.shape[0], dtype=np.int32)
        tags[np.all(np.abs(p[faces, 2]) < 1e-9 * L, axis=1)] = 1
        tags[np.all(np.abs(p[faces, 2] - L) < 1e-9 * L, axis=1)] = 2
        return tags

    return _finish(xyz, hexes, tag_fn, (1,), (2,), name)


def womersley_mesh(level: int = 1) -> Mesh:
    """Straight pipe R=1, L=5: level 1 is ~3,000 tetrahedra (5x5 core, 4 rims of 5x3, 6 layers);
    each level halves the cell size."""
    f = 2 ** (level - 1)
    return pipe_mesh(1.0, 5.0, 5 * f, 3 * f, 6 * f, name=f"womersley_l{level}")


def stenosed_tube(n_tets_target: int, seed: int, severity=(0.3, 0.7)) -> Mesh:
    """Coronary-like tube: radius U(0.15, 0.25), length 12 radii, one cosine stenosis with a diameter
    reduction drawn from U(severity) (default 30-70 %)."""
    rng = np.random.default_rng(seed)
    R = rng.uniform(0.15, 0.25)
    sev = rng.uniform(*severity)
    L = 12.0 * R
    zc = L * rng.uniform(0.35, 0.6)
    ls = 2.0 * R * rng.uniform(1.0, 2.0)

    def rfun(z):
        if abs(z - zc) < ls:
            return R * (1.0 - 0.5 * sev * (1.0 + math.cos(math.pi * (z - zc) / ls)))
        return R

    # tets ~ 6 * 3 nc^2 * nz with nz ~ L / (R / nc) = 12 nc
    nc = max(3, int(round((n_tets_target / 216.0) ** (1.0 / 3.0))))
    nr = max(2, nc // 2)
    quads = nc * nc + 4 * nc * nr
    nz = max(4, int(round(n_tets_target / (6.0 * quads))))
    return pipe_mesh(R, L, nc, nr, nz, radius_fn=rfun, name=f"stenosis_s{seed}")


def pipe_by_size(n_tets_target: int, seed: int, R: float = 1.0) -> Mesh:
    """Straight pipe, length 5 R, cell count chosen near n_tets_target."""
    nc = max(3, int(round((n_tets_target / 90.0) ** (1.0 / 3.0))))
    nr = max(2, (3 * nc) // 5)
    quads = nc * nc + 4 * nc * nr
    nz = max(3, int(round(n_tets_target / (6.0 * quads))))
    return pipe_mesh(R, 5.0 * R, nc, nr, nz, name=f"pipe_s{seed}")


# ----------------------------------------------------------------------------------------------------
# voxel meshes from a signed inside-test


def _block_tables():
    """For the 256 occupancy patterns of a 2 x 2 x 2 block of cells (bit i + 2 j + 4 k for cell (i, j, k)):
    whether the block is non-manifold at its centre vertex (its inside cells, or its outside cells, form
    more than one face-connected group), and which empty cell to fill to repair it (the first one whose
    filling leaves fewer groups)."""
    cells = [(i, j, k) for k in range(2) for j in range(2) for i in range(2)]
    nbr = [[b for b in range(8) if sum(abs(x - y) for x, y in zip(cells[a], cells[b])) == 1] for a in range(8)]

    def groups(code, want):
        seen, count = set(), 0
        for a in range(8):
            if ((code >> a) & 1) != want or a in seen:
                continue
            count += 1
            stack = [a]
            seen.add(a)
            while stack:
                c = stack.pop()
                for b in nbr[c]:
                    if ((code >> b) & 1) == want and b not in seen:
                        seen.add(b)
                        stack.append(b)
        return count

    bad = np.zeros(256, dtype=bool)
    fill = np.full(256, -1, dtype=np.int64)
    for code in range(256):
        g_in, g_out = groups(code, 1), groups(code, 0)
        if g_in <= 1 and g_out <= 1:
            continue
        bad[code] = True
        for a in range(8):
            if not (code >> a) & 1:
                new = code | (1 << a)
                if groups(new, 1) + groups(new, 0) < g_in + g_out:
                    fill[code] = a
                    break
        if fill[code] < 0:
            fill[code] = next(a for a in range(8) if not (code >> a) & 1)
    return bad, fill, cells


def _manifold_cells(occ: np.ndarray) -> np.ndarray:
    """Add cells to a boolean cell grid until the boundary of the union is a 2-manifold: no two inside
    cells, and no two outside cells, meet only along an edge or at a vertex of a 2 x 2 x 2 block."""
    bad, fill, cells = _block_tables()
    P = np.pad(occ, 1)
    while True:
        code = np.zeros(tuple(d - 1 for d in P.shape), dtype=np.int64)
        for b, (i, j, k) in enumerate(cells):
            code |= P[i:P.shape[0] - 1 + i, j:P.shape[1] - 1 + j, k:P.shape[2] - 1 + k].astype(np.int64) << b
        w = np.nonzero(bad[code])
        if len(w[0]) == 0:
            return P[1:-1, 1:-1, 1:-1]
        f = fill[code[w]]
        off = np.array(cells)[f]
        P[w[0] + off[:, 0], w[1] + off[:, 1], w[2] + off[:, 2]] = True


def voxel_mesh(inside, lo, hi, h: float, cap_planes, inlet_tags, outlet_tags, name: str,
               manifold: bool = False) -> Mesh:
    """Cells of a lattice of spacing ~h over the box [lo, hi] whose centre satisfies inside(points).

    cap_planes: list of (tag, axis, side) -- boundary faces lying on the box face `axis`=lo/hi
    (side 0/1) get that tag; all other boundary faces are walls (tag 0).  manifold: add the cells that
    make the boundary a 2-manifold (cells that would touch the rest only along an edge or at a vertex
    get a face-sharing neighbour)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    n = np.maximum(1, np.round((hi - lo) / h).astype(np.int64))
    hh = (hi - lo) / n
    ci = [lo[d] + hh[d] * (np.arange(n[d]) + 0.5) for d in range(3)]
    keep = []
    for k in range(n[2]):              # slab by slab to bound memory
        # x fastest: cell (x, y, z) has index x + n0 (y + n1 z), the order decoded below
        X, Y = np.meshgrid(ci[0], ci[1], indexing="xy")
        pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, ci[2][k])], 1)
        m = inside(pts)
        ii = np.nonzero(m)[0]
        keep.append(ii + k * n[0] * n[1])
    cells = np.concatenate(keep)
    if manifold:
        occ = np.zeros(int(n[0] * n[1] * n[2]), dtype=bool)
        occ[cells] = True
        occ = _manifold_cells(occ.reshape(int(n[2]), int(n[1]), int(n[0])).transpose(2, 1, 0))
        cells = np.nonzero(occ.transpose(2, 1, 0).ravel())[0]
    ci_x = cells % n[0]
    ci_y = (cells // n[0]) % n[1]
    ci_z = cells // (n[0] * n[1])
    sx, sy, sz = 1, n[0] + 1, (n[0] + 1) * (n[1] + 1)
    base = ci_x * sx + ci_y * sy + ci_z * sz
    off = np.array([0, sx, sy, sx + sy, sz, sz + sx, sz + sy, sz + sx + sy])
    hexes_glob = base[:, None] + off[None, :]
    used, inv = np.unique(hexes_glob, return_inverse=True)
    hexes = inv.reshape(-1, 8)
    gx = used % (n[0] + 1)
    gy = (used // (n[0] + 1)) % (n[1] + 1)
    gz = used // ((n[0] + 1) * (n[1] + 1))
    xyz = np.stack([lo[0] + hh[0] * gx, lo[1] + hh[1] * gy, lo[2] + hh[2] * gz], 1)

    def tag_fn(p, faces):
        tags = np.zeros(faces.shape[0], dtype=np.int32)
        for tag, axis, side in cap_planes:
            val = hi[axis] if side else lo[axis]
            on = np.all(np.abs(p[faces, axis] - val) < 1e-9 * float(np.max(hi - lo)), axis=1)
            tags[on] = tag
        return tags

    return _finish(xyz, hexes, tag_fn, inlet_tags, outlet_tags, name)


def glenn_like(n_tets_target: int = 1_000_000, seed: int = 2000) -> Mesh:
    """Glenn-like T-junction: two inflow tubes of radius 0.6 along z (from z=+Z and z=-Z) meet a
    transverse outflow tube of radius 0.5 along x with outlets at x=-X and x=+X.
    Tags: 1 inlet z=+Z, 2 inlet z=-Z, 3 outlet x=-X, 4 outlet x=+X, 0 wall."""
    rng = np.random.default_rng(seed)
    X = 3.0
    Z = 2.5
    zoff = rng.uniform(-0.05, 0.05, size=2)   # slight offsets of the inflow tubes along x

    def inside(p):
        a = p[:, 1] ** 2 + p[:, 2] ** 2 < 0.5 ** 2
        b = ((p[:, 0] - zoff[0]) ** 2 + p[:, 1] ** 2 < 0.6 ** 2) & (p[:, 2] > 0)
        c = ((p[:, 0] - zoff[1]) ** 2 + p[:, 1] ** 2 < 0.6 ** 2) & (p[:, 2] < 0)
        return a | b | c

    vol = math.pi * 0.25 * 2 * X + 2 * math.pi * 0.36 * Z
    h = (6.0 * vol / n_tets_target) ** (1.0 / 3.0)
    return voxel_mesh(inside, (-X, -0.62, -Z), (X, 0.62, Z), h,
                      [(1, 2, 1), (2, 2, 0), (3, 0, 0), (4, 0, 1)], (1, 2), (3, 4),
                      f"glenn_like_s{seed}")


def cerebral_like(n_tets_target: int = 2_000_000, seed: int = 3000, R: float = 0.2,
                  bulge_R: float = 0.5) -> Mesh:
    """Cerebral-like vessel: a tube of radius R around a seeded cubic-spline centreline from x=0 to
    x=5 (straight near both caps), plus a saccular bulge (sphere of radius bulge_R) on its side.
    Tags: 1 inlet x=0, 2 outlet x=5, 0 wall."""
    from scipy.interpolate import CubicSpline
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    Lx = 5.0
    nctl = int(rng.integers(3, 6))
    xs = np.concatenate([[0.0, 0.6], np.linspace(1.2, Lx - 1.2, nctl), [Lx - 0.6, Lx]])
    ys = np.concatenate([[0.0, 0.0], rng.uniform(-0.6, 0.6, nctl), [0.0, 0.0]])
    zs = np.concatenate([[0.0, 0.0], rng.uniform(-0.6, 0.6, nctl), [0.0, 0.0]])
    cy = CubicSpline(xs, ys, bc_type="clamped")
    cz = CubicSpline(xs, zs, bc_type="clamped")
    tt = np.linspace(0.0, Lx, 4000)
    curve = np.stack([tt, cy(tt), cz(tt)], 1)
    tree = cKDTree(curve)
    # bulge centre: beside the centreline near the middle
    j = len(tt) // 2 + int(rng.integers(-400, 400))
    tang = np.gradient(curve, axis=0)[j]
    tang /= np.linalg.norm(tang)
    side = np.cross(tang, rng.normal(size=3))
    side /= np.linalg.norm(side)
    centre = curve[j] + side * (R + 0.6 * bulge_R)

    def inside(p):
        d, _ = tree.query(p)
        return (d < R) | (np.sum((p - centre) ** 2, axis=1) < bulge_R ** 2)

    lo = np.minimum(curve.min(0) - R, centre - bulge_R) - 0.02
    hi = np.maximum(curve.max(0) + R, centre + bulge_R) + 0.02
    lo[0], hi[0] = 0.0, Lx
    vol = math.pi * R * R * Lx * 1.05 + (4.0 / 3.0) * math.pi * bulge_R ** 3 * 0.8
    h = (6.0 * vol / n_tets_target) ** (1.0 / 3.0)
    return voxel_mesh(inside, lo, hi, h, [(1, 0, 0), (2, 0, 1)], (1,), (2,), f"cerebral_like_s{seed}")


# ----------------------------------------------------------------------------------------------------
# boundary-condition inputs


def tag_nodes(mesh: Mesh, tag: int) -> np.ndarray:
    return np.unique(mesh.faces[mesh.face_tag == tag].ravel())


def parabolic_profile(mesh: Mesh, tag: int) -> np.ndarray:
    """Velocity profile at unit flow on the cap `tag`: (2/(pi R^2)) max(0, 1 - r^2/R^2) along the
    inward normal, where the cap centre is the area-weighted centroid of its faces, the normal the
    area-weighted mean of their unit normals oriented away from the mesh, and R the largest in-plane
    distance of a cap node from the centre.  Zero away from the cap.  Returns [n_nodes, 3]."""
    fa = mesh.faces[mesh.face_tag == tag]
    p = mesh.xyz[fa]
    cr = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    cen = np.sum(p.mean(1) * area[:, None], 0) / area.sum()
    nrm = cr / np.linalg.norm(cr, axis=1, keepdims=True)
    ref = nrm[0]
    nrm = nrm * np.sign(nrm @ ref)[:, None]
    n = np.sum(nrm * area[:, None], 0)
    n /= np.linalg.norm(n)
    mesh_c = mesh.xyz.mean(0)
    if np.dot(cen - mesh_c, n) < 0:
        n = -n
    nodes = np.unique(fa.ravel())
    d = mesh.xyz[nodes] - cen
    d -= np.outer(d @ n, n)
    r2 = np.sum(d * d, 1)
    R2 = r2.max()
    out = np.zeros((mesh.n_nodes, 3))
    out[nodes] = (2.0 / (math.pi * R2)) * np.maximum(0.0, 1.0 - r2 / R2)[:, None] * (-n)[None, :]
    return out


def uniform_profile(mesh: Mesh, tags, vec) -> np.ndarray:
    out = np.zeros((mesh.n_nodes, 3))
    for t in tags:
        out[tag_nodes(mesh, t)] = np.asarray(vec, dtype=np.float64)
    return out


def waveform_harmonics(n_h: int, mean: float, seed: int, amp_lo: float = 0.5, amp_hi: float = 1.0,
                       min_frac: float = 0.2, peak_over_mean: float | None = None):
    """Seeded real harmonics of a periodic waveform q(t) = a[0] + sum_k a[k] cos(k w t) + b[k] sin(k w t).

    Amplitude of harmonic k is mean * U(amp_lo, amp_hi) / k with a uniform random phase.  The
    oscillating part is scaled down until q >= min_frac * mean everywhere, and, if peak_over_mean is
    given, scaled so that max q / mean equals it (when that keeps the minimum).
    Returns (a, b), each of length n_h + 1 (b[0] = 0)."""
    rng = np.random.default_rng(seed)
    a = np.zeros(n_h + 1)
    b = np.zeros(n_h + 1)
    a[0] = mean
    for k in range(1, n_h + 1):
        amp = mean * rng.uniform(amp_lo, amp_hi) / k
        ph = rng.uniform(0.0, 2.0 * math.pi)
        a[k] = amp * math.cos(ph)
        b[k] = amp * math.sin(ph)
    th = np.linspace(0.0, 2.0 * math.pi, 2048, endpoint=False)
    kk = np.arange(1, n_h + 1)
    osc = np.cos(np.outer(th, kk)) @ a[1:] + np.sin(np.outer(th, kk)) @ b[1:]
    s = 1.0
    if peak_over_mean is not None and osc.max() > 0:
        s = (peak_over_mean - 1.0) * mean / osc.max()
    if osc.min() * s < -(1.0 - min_frac) * mean:
        s = (1.0 - min_frac) * mean / -osc.min()
    a[1:] *= s
    b[1:] *= s
    return a, b


def random_state(n_nodes: int, N: int, seed: int, vel: float = 1.0, pres: float = 1.0) -> np.ndarray:
    """O(1) random instance values [n_nodes, 4, N] (u1, u2, u3, p)."""
    rng = np.random.default_rng(seed)
    y = rng.uniform(-1.0, 1.0, size=(n_nodes, 4, N))
    y[:, :3] *= vel
    y[:, 3] *= pres
    return y


def smooth_state(mesh: Mesh, N: int, seed: int, vel: float = 1.0, pres: float = 1.0) -> np.ndarray:
    """Random but spatially smooth instance values [n_nodes, 4, N]: low-order trigonometric fields in
    space times random time samples; avoids the cancellation-free but unphysical extremes of
    random_state when a test wants a flow-like state."""
    rng = np.random.default_rng(seed)
    x = mesh.xyz
    span = np.maximum(x.max(0) - x.min(0), 1e-12)
    xs = (x - x.min(0)) / span
    y = np.zeros((mesh.n_nodes, 4, N))
    for f in range(4):
        for _ in range(3):
            k = rng.integers(0, 3, size=3)
            ph = rng.uniform(0, 2 * math.pi, size=3)
            sp = np.prod(np.cos(math.pi * k[None, :] * xs + ph[None, :]), axis=1)
            tw = rng.uniform(-1, 1, size=N)
            y[:, f, :] += np.outer(sp, tw)
    y[:, :3] *= vel
    y[:, 3] *= pres
    return y
