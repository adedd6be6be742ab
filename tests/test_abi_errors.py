"""Error behaviour of the C ABI that needs no GPU: argument checks that the header documents return
HB_ERR_INVALID_ARG (with a message) before any device work, defaults are filled, and null handles are
handled."""
import ctypes as C

import numpy as np
import pytest

from paper_2411_14315_gb300 import hbgls

INVALID = 1


@pytest.fixture(scope="module")
def lib():
    return hbgls.lib()


def _mesh(n_nodes=4, n_tets=1, n_faces=4, arrays=True):
    xyz = np.zeros((4, 3))
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    faces = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]], dtype=np.int32)
    tags = np.zeros(4, dtype=np.int32)
    m = hbgls.hb_mesh()
    m.n_nodes, m.n_tets, m.n_faces = n_nodes, n_tets, n_faces
    if arrays:
        m.xyz = xyz.ctypes.data_as(C.POINTER(C.c_double))
        m.tets = tets.ctypes.data_as(C.POINTER(C.c_int32))
        m.faces = faces.ctypes.data_as(C.POINTER(C.c_int32))
        m.face_tag = tags.ctypes.data_as(C.POINTER(C.c_int32))
    return m, (xyz, tets, faces, tags)


@pytest.mark.parametrize("case", ["null mesh", "null arrays", "empty", "too many nodes", "rho", "mu", "T",
                                  "n_h negative", "n_h too large"])
def test_create_rejects_bad_arguments(lib, case):
    m, keep = _mesh(arrays=case != "null arrays")
    rho, mu, T, n_h = 1.0, 0.04, 1.0, 2
    if case == "empty":
        m.n_nodes = 0
    elif case == "too many nodes":
        m.n_nodes = 1 << 21
    elif case == "rho":
        rho = 0.0
    elif case == "mu":
        mu = -1.0
    elif case == "T":
        T = float("nan")
    elif case == "n_h negative":
        n_h = -1
    elif case == "n_h too large":
        n_h = 16                               # N = 33 > 31 instances
    out = C.c_void_p()
    arg = None if case == "null mesh" else C.byref(m)
    st = lib.hb_create(arg, rho, mu, T, n_h, 0, None, C.byref(out))
    assert st == INVALID, case
    assert not out.value
    assert len(lib.hb_last_error()) > 0


MESH = 2


@pytest.mark.parametrize("case", ["tet index", "negative tet index", "face index", "negative tag", "flat tet",
                                  "nan coordinate", "infinite coordinate"])
def test_create_rejects_bad_meshes_before_any_device_work(lib, case):
    """Mesh checks run on the host before the device is touched, so they answer HB_ERR_MESH with or
    without a GPU; an inverted (negatively oriented) tetrahedron is not an error."""
    m, (xyz, tets, faces, tags) = _mesh()
    xyz[:] = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    if case == "tet index":
        tets[0, 2] = 4
    elif case == "negative tet index":
        tets[0, 0] = -1
    elif case == "face index":
        faces[1, 1] = 7
    elif case == "negative tag":
        tags[3] = -2
    elif case == "flat tet":
        xyz[3] = [0.3, 0.3, 0.0]                  # the fourth vertex in the plane of the first three
    elif case == "nan coordinate":
        xyz[2, 1] = float("nan")
    elif case == "infinite coordinate":
        xyz[1, 0] = float("inf")
    out = C.c_void_p()
    st = lib.hb_create(C.byref(m), 1.0, 0.04, 1.0, 2, 0, None, C.byref(out))
    assert st == MESH, (case, st, lib.hb_last_error())
    assert not out.value


def test_inverted_tetrahedron_passes_the_mesh_checks(lib):
    m, (xyz, tets, faces, tags) = _mesh()
    xyz[:] = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    tets[0] = [1, 0, 2, 3]                        # negative orientation
    out = C.c_void_p()
    st = lib.hb_create(C.byref(m), 1.0, 0.04, 1.0, 2, 0, None, C.byref(out))
    assert st != MESH, lib.hb_last_error()        # HB_OK on a GPU machine, HB_ERR_CUDA without one
    if out.value:
        assert lib.hb_destroy(out) == 0


def test_defaults_are_filled(lib):
    o = hbgls.hb_solve_opts()
    assert lib.hb_default_opts(C.byref(o)) == 0
    assert o.precision == 1 and 1 <= o.gmres_restart <= 200 and o.rtol > 0 and o.max_steps > 0
    # the paper's settings of Sec. 2.3 where it states them; the extensions default to "unchanged"
    assert o.gmres_rtol_pseudo == 0.03 and o.switch_rtol == 1e-3
    assert o.scatter == 1 and o.backflow_beta < 0 and o.precond == 0 and o.line_search == 1
    mo = hbgls.hb_march_opts()
    assert lib.hb_default_march_opts(C.byref(mo)) == 0
    assert mo.gmres_rtol == 0.03 and mo.newton_rtol == 1e-3 and mo.periods == 4 and mo.rho_inf == 0.5
    assert lib.hb_default_opts(None) == INVALID
    assert lib.hb_default_march_opts(None) == INVALID


def test_null_handles(lib):
    assert lib.hb_destroy(None) == 0
    assert lib.hb_solve(None, None, None) == INVALID
    assert lib.hb_march(None, None, None) == INVALID
    assert lib.hb_set_launch_variant(None, 0) == INVALID
    assert lib.hb_get_launch_variant(None) == -1
    assert lib.hb_launch_count(None) == 0
    assert lib.hb_get_march_samples(None, None) == INVALID
    assert lib.hb_time_residual(None, None, None, None, 0, 0.0, 0.0) == INVALID
    out = C.c_void_p()
    assert lib.hb_batch_create(None, 0, 1, C.byref(out)) == INVALID
    assert lib.hb_batch_destroy(None) == 0


def test_set_stabilization_null_problem(lib):
    """hb_set_stabilization checks its problem before anything else (no device work)."""
    assert lib.hb_set_stabilization(None, 1, 0.0) == INVALID
    assert lib.hb_last_error().decode()


def test_scatter_setting_null_problem(lib):
    """hb_set_scatter / hb_get_scatter check their problem before anything else (no device work)."""
    assert lib.hb_set_scatter(None, 0) == INVALID
    assert lib.hb_get_scatter(None) == -1


def test_batch_grouping_null_batch(lib):
    assert lib.hb_batch_set_grouping(None, 1) == INVALID
