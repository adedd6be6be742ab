"""Invariants of the seeded input meshes (the stand-ins for the paper's vessel models, Sec. 3): every
tetrahedron positively oriented with positive volume, a conforming mesh (a face belongs to at most two
tetrahedra), the listed boundary triangles exactly the faces that belong to one tetrahedron, every
node used, inlet and outlet caps tagged.  The structured generators (box, pipes) also give a closed
2-manifold boundary and the Euler characteristics of a ball; the voxel generators (T-junction,
cerebral-like) can leave cells that touch along an edge only, which the method does not mind."""
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
STRUCTURED = ("box", "womersley", "stenosed", "pipe")


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
        pytest.skip("voxel meshes may have cells touching along an edge only")
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
