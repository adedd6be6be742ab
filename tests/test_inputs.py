"""Invariants of the seeded input meshes (the stand-ins for the paper's vessel models, Sec. 3): every
tetrahedron positively oriented with positive volume, a conforming mesh (a face belongs to at most two
tetrahedra), the listed boundary triangles exactly the faces that belong to one tetrahedron, every
node used, inlet and outlet caps tagged.  The structured generators (box, pipes) and the T-junction also
give a closed 2-manifold boundary and the Euler characteristics of a ball; the thin voxelised tube of the
cerebral-like vessel can leave cells that touch along an edge only (which the method does not mind, and
which `manifold=True` repairs).  The voxel generator places every cell where its inside-test put it."""
import math

import numpy as np
import pytest

from paper_2411_14315_gb300 import inputs as I

_LOCAL_FACES = np.array([(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)])
_LOCAL_EDGES = np.array([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])


def _signed_volumes(m):
    x, t = m.xyz, m.tets.astype(np.int64)
    return np.einsum("ij,ij->i", np.cross(x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]]),
                     x[t[:, 3]] - x[t[:, 0]]) / 6.0


def _faces(m):
    t = m.tets.astype(np.int64)
    return np.unique(np.sort(t[:, _LOCAL_FACES].reshape(-1, 3), axis=1), axis=0, return_counts=True)


MESHES = {
    "box": lambda: I.box_mesh(4, 3, 3, lx=1.5, jitter=0.2, seed=90),
    "womersley": lambda: I.womersley_mesh(1),
    "stenosed": lambda: I.stenosed_tube(20_000, 4001),
    "pipe": lambda: I.pipe_by_size(20_000, 1),
    "glenn_like": lambda: I.glenn_like(30_000, 2000),
    "cerebral_like": lambda: I.cerebral_like(30_000, 3000),
}
STRUCTURED = ("box", "womersley", "stenosed", "pipe", "glenn_like")   # checked: a ball at this size


@pytest.fixture(scope="module", params=list(MESHES))
def mesh(request):
    return request.param, MESHES[request.param]()


def test_valid_conforming_tetrahedral_mesh(mesh):
    name, m = mesh
    vol = _signed_volumes(m)
    assert vol.min() > 1e-12 * vol.mean(), name
    faces, count = _faces(m)
    assert count.max() == 2, name                   # conforming: no face shared by three tetrahedra
    listed = np.unique(np.sort(m.faces.astype(np.int64), axis=1), axis=0)
    assert len(listed) == m.n_faces and np.array_equal(listed, faces[count == 1]), name
    assert len(np.unique(m.tets)) == m.n_nodes, name
    assert m.face_tag.shape == (m.n_faces,)
    tags = set(np.unique(m.face_tag).tolist())
    assert set(m.inlet_tags) <= tags and set(m.outlet_tags) <= tags, name


def test_structured_meshes_are_balls_with_closed_manifold_boundary(mesh):
    name, m = mesh
    if name not in STRUCTURED:
        pytest.skip("the thin voxelised tube keeps cells touching along an edge only (see manifold=True)")
    t = m.tets.astype(np.int64)
    faces, _ = _faces(m)
    edges = np.unique(np.sort(t[:, _LOCAL_EDGES].reshape(-1, 2), axis=1), axis=0)
    assert m.n_nodes - len(edges) + len(faces) - m.n_tets == 1, name      # solid ball
    bf = np.sort(m.faces.astype(np.int64), axis=1)
    be, bc = np.unique(np.sort(bf[:, [(0, 1), (0, 2), (1, 2)]].reshape(-1, 2), axis=1), axis=0,
                       return_counts=True)
    assert np.all(bc == 2), name                                            # closed 2-manifold
    assert len(np.unique(bf)) - len(be) + len(bf) == 2, name                # sphere


def test_volumes_of_the_simple_shapes():
    box = MESHES["box"]()
    assert abs(_signed_volumes(box).sum() - 1.5) < 1e-12                    # 1.5 x 1 x 1
    pipe = MESHES["womersley"]()
    # the O-grid section is a polygon inscribed in the circle R = 1, L = 5: a little below pi R^2 L
    v = _signed_volumes(pipe).sum()
    assert 0.97 * math.pi * 5.0 < v < math.pi * 5.0


def _hex_centres(m):
    """Centres of the voxel cells: the 6 tetrahedra of a cell are consecutive, and their mean vertex
    position over all 24 corners is the cell centre."""
    return m.xyz[m.tets.astype(np.int64)].reshape(-1, 6, 4, 3).mean(axis=(1, 2))


def test_voxel_cells_sit_where_the_inside_test_put_them():
    """An L-shaped region on a lattice with different cell counts along x and y: every cell centre is
    inside, and every inside lattice cell is meshed."""
    def inside(p):
        return ((p[:, 0] < 0.4) | (p[:, 1] < 0.25)) & (p[:, 2] < 0.7)

    lo, hi, h = (0.0, 0.0, 0.0), (1.3, 0.8, 1.0), 0.1
    m = I.voxel_mesh(inside, lo, hi, h, [(1, 0, 0)], (1,), (), "L")
    c = _hex_centres(m)
    assert inside(c).all()
    n = np.round((np.asarray(hi) - np.asarray(lo)) / h).astype(int)
    g = [(np.arange(k) + 0.5) * (hi[d] - lo[d]) / k + lo[d] for d, k in enumerate(n)]
    grid = np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)
    assert len(c) == int(inside(grid).sum())


def test_manifold_option_repairs_edge_contacts():
    """Two cells meeting along an edge only, and two meeting at a vertex only: with manifold=True cells are
    added until the boundary is a closed 2-manifold."""
    def inside(p):
        a = (p[:, 0] < 0.5) & (p[:, 1] < 0.5) & (p[:, 2] < 0.5)
        b = (p[:, 0] > 0.5) & (p[:, 0] < 1.0) & (p[:, 1] > 0.5) & (p[:, 1] < 1.0) & (p[:, 2] < 0.5)
        c = (p[:, 0] > 1.0) & (p[:, 1] > 1.0) & (p[:, 2] > 0.5)
        return a | b | c

    lo, hi = (0.0, 0.0, 0.0), (1.5, 1.5, 1.0)
    raw = I.voxel_mesh(inside, lo, hi, 0.5, [], (), (), "pinched")
    fixed = I.voxel_mesh(inside, lo, hi, 0.5, [], (), (), "pinched", manifold=True)
    assert fixed.n_tets > raw.n_tets

    def edge_counts(m):
        bf = np.sort(m.faces.astype(np.int64), axis=1)
        return np.unique(np.unique(np.sort(bf[:, [(0, 1), (0, 2), (1, 2)]].reshape(-1, 2), axis=1), axis=0,
                                   return_counts=True)[1])

    assert 4 in edge_counts(raw)
    assert set(edge_counts(fixed).tolist()) == {2}
    assert inside(_hex_centres(raw)).all()
