"""GPU parity: the library (through its C ABI) against the CPU oracle, element by element.

FP64 kernels must match to 1e-12 and FP32 kernels to 1e-5, norm-wise relative per field, on seeded
random (non-solution) states; meshes span many element patches and a ragged last patch.
"""
import math

import numpy as np
import pytest

from oracle import hb_oracle as O
from paper_2411_14315_gb300 import inputs as I
from tests import problems as P

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def relerr(a, b):
    """max over fields of ||a_f - b_f|| / ||b_f||."""
    out = 0.0
    for f in range(a.shape[1]):
        d = np.linalg.norm(a[:, f] - b[:, f])
        n = np.linalg.norm(b[:, f])
        out = max(out, d / n if n > 0 else d)
    return out


@pytest.fixture(scope="module")
def box():
    spec = P.box_spec(n=(7, 5, 4), n_h=3)
    return spec, P.oracle_problem(spec), P.gpu_problem(spec)


@pytest.mark.parametrize("precision", [0, 1])
def test_residual_box(box, precision):
    spec, ora, gp = box
    y = I.random_state(spec.mesh.n_nodes, spec.N, 31)
    r_ref = O.residual(ora, y)
    r = gp.residual(y, precision)
    assert relerr(r, r_ref) < TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", [0, 1])
def test_jv_box(box, precision, kind):
    spec, ora, gp = box
    y = I.random_state(spec.mesh.n_nodes, spec.N, 32)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 33)
    shift = 1.7
    ref = (O.jv_paper if kind == 0 else O.jv_exact)(ora, y, v, shift=shift)
    jv = gp.jv(y, v, kind=kind, precision=precision, shift=shift)
    assert relerr(jv, ref) < TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_jacobi_diag_box(box, precision):
    spec, ora, gp = box
    y = I.random_state(spec.mesh.n_nodes, spec.N, 34)
    ref = O.jacobi_diag(ora, y, shift=0.9)
    d = gp.jacobi_diag(y, precision=precision, shift=0.9)
    assert relerr(d, ref) < TOL[precision]


@pytest.mark.parametrize("n_h", [0, 1, 4, 10, 15])
def test_residual_and_jv_across_instance_counts(n_h):
    spec = P.box_spec(seed=40 + n_h, n_h=n_h, n=(5, 4, 3))
    ora = P.oracle_problem(spec)
    gp = P.gpu_problem(spec)
    y = I.random_state(spec.mesh.n_nodes, spec.N, 41)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 42)
    for prec in (0, 1):
        assert relerr(gp.residual(y, prec), O.residual(ora, y)) < TOL[prec]
        assert relerr(gp.jv(y, v, 1, prec, 0.3), O.jv_exact(ora, y, v, shift=0.3)) < TOL[prec]
        assert relerr(gp.jv(y, v, 0, prec, 0.3), O.jv_paper(ora, y, v, shift=0.3)) < TOL[prec]


@pytest.mark.parametrize("n_h", [0, 1, 4, 6, 10, 15])
def test_paper_tangent_launch_variants(n_h):
    """Every launch variant of the FP32 paper-tangent pass (pairs of instances per thread, one instance
    per thread at three block sizes, and the two pipelined variants with a producer warp and bulk copies)
    against the oracle, for compile-time and generic instance counts."""
    spec = P.box_spec(seed=70 + n_h, n_h=n_h, n=(6, 5, 4))
    ora = P.oracle_problem(spec)
    gp = P.gpu_problem(spec)
    y = I.random_state(spec.mesh.n_nodes, spec.N, 71)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 72)
    ref = O.jv_paper(ora, y, v, shift=0.8)
    for var in range(7):
        gp.set_launch_variant(var)
        assert gp.launch_variant() == var
        assert relerr(gp.jv(y, v, 0, 1, 0.8), ref) < TOL[1], var
    with pytest.raises(RuntimeError):
        gp.set_launch_variant(7)


def test_paper_tangent_variants_many_patches_per_block():
    """The persistent and pipelined passes on a T-junction of ~120k tetrahedra (N = 21, several hundred
    patches, so every block of the one-block-per-SM pipelined pass reuses both shared-memory stages
    several times; prescribed velocities and resistance outlets) against the oracle's paper tangent."""
    spec = P.glenn_spec(n_tets=120_000)
    ora = P.oracle_problem(spec)
    gp = P.gpu_problem(spec)
    assert gp.info()["n_patches32"] > 4 * 152
    y = I.random_state(spec.mesh.n_nodes, spec.N, 73)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 74)
    y32 = y.astype(np.float32).astype(np.float64)
    v32 = v.astype(np.float32).astype(np.float64)
    ref = O.jv_paper(ora, y32, v32, shift=300.0)
    for var in (0, 1, 4, 5, 6):
        gp.set_launch_variant(var)
        assert relerr(gp.jv(y32, v32, 0, 1, 300.0), ref) < TOL[1], var
    gp.close()


def test_womersley_pipe_parabolic_profile_and_patches():
    """Womersley pipe (~3,000 tets, N = 9) with the library's own parabolic profile (NULL) against the
    oracle given the input generator's profile: both follow the same definition independently."""
    spec = P.womersley_spec()
    ora = P.oracle_problem(spec)
    gp = P.gpu_problem(spec)
    info = gp.info()
    assert info["n_patches32"] > 4 and info["n_patches64"] > 4
    gp.set_instances(None)
    y0 = gp.instances()
    assert np.allclose(y0, ora.initial_state(), rtol=0, atol=1e-13)
    y = ora.apply_dirichlet(I.smooth_state(spec.mesh, spec.N, 7, vel=2.0))
    for prec in (0, 1):
        assert relerr(gp.residual(y, prec), O.residual(ora, y)) < TOL[prec]
    v = I.random_state(spec.mesh.n_nodes, spec.N, 8)
    for prec in (0, 1):
        assert relerr(gp.jv(y, v, 1, prec), O.jv_exact(ora, y, v)) < TOL[prec]


def test_plug_flow_patch_on_gpu():
    """The exact plug-flow solution (Sec. 2 equations, P1) has zero residual on the GPU too."""
    from tests.test_oracle_pins import _plug_problem
    m, ora, y = _plug_problem(3)
    spec = P.Spec(m, ora.rho, ora.mu, ora.T, ora.n_h, beta=ora.beta_bf)
    for tag, (prof, a, b) in ora.inflow.items():
        spec.inflows.append((tag, prof, a, b))
    for tag, (a, b) in ora.outlet_p.items():
        spec.outlets_p.append((tag, a, b))
    gp = P.gpu_problem(spec)
    r = gp.residual(y, 0)
    scale = np.abs(O.residual(ora, y + 0.01)).max()
    assert np.abs(r).max() < 1e-12 * scale


def test_harmonics_round_trip():
    spec = P.box_spec(n_h=5, n=(3, 3, 3))
    gp = P.gpu_problem(spec)
    ora = P.oracle_problem(spec)
    rng = np.random.default_rng(5)
    coef = rng.normal(size=(spec.mesh.n_nodes, 4, 2 * spec.n_h + 1))
    gp.set_initial(coef)
    y = gp.instances()
    ref = O.harmonics_to_instances(coef, spec.N, spec.T)
    ref = ora.apply_dirichlet(ref)
    assert np.allclose(y, ref, atol=1e-12)
    h = gp.harmonics()
    assert np.allclose(h, O.instances_to_harmonics(y, spec.n_h), atol=1e-12)


def test_device_pointer_entry_points_match_host_ones(box):
    torch = pytest.importorskip("torch")
    spec, ora, gp = box
    y = I.random_state(spec.mesh.n_nodes, spec.N, 51)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 52)
    for prec, dt in ((0, torch.float64), (1, torch.float32)):
        ty = torch.tensor(y, dtype=dt, device="cuda")
        tv = torch.tensor(v, dtype=dt, device="cuda")
        out = torch.empty_like(ty)
        s = torch.cuda.current_stream()
        gp.jv_dev(ty, tv, out, 1, prec, 0.5, stream=s)
        s.synchronize()
        ref = gp.jv(ty.double().cpu().numpy(), tv.double().cpu().numpy(), 1, prec, 0.5)
        assert np.allclose(out.double().cpu().numpy(), ref, rtol=0, atol=1e-12 if prec == 0 else 1e-4)


def _sampled_oracle(spec, y, v, nodes, fn):
    """Oracle value at interior sample nodes from the sub-mesh of their adjacent elements."""
    m = spec.mesh
    adj = np.nonzero(np.isin(m.tets, nodes).any(axis=1))[0]
    sub = m.tets[adj]
    used, inv = np.unique(sub, return_inverse=True)
    tets = inv.reshape(-1, 4)
    pr = O.HBProblem(m.xyz[used], tets, np.zeros((0, 3), dtype=np.int64), np.zeros(0, dtype=np.int64),
                     spec.rho, spec.mu, spec.T, spec.n_h)
    args = [y[used]] + ([v[used]] if v is not None else [])
    out = fn(pr, *args)
    return out[np.searchsorted(used, nodes)]


def test_full_size_cerebral_sampled_parity():
    """Cerebral-like vessel at full size (~2.2M tets, ~405k nodes, N = 21): residual and the paper's
    tangent at 48 sampled interior nodes against the oracle."""
    from paper_2411_14315_gb300 import workloads as W
    spec = W.cerebral_spec()
    gp = P.gpu_problem(spec)
    m = spec.mesh
    n = m.n_nodes
    y = I.random_state(n, spec.N, 64)
    v = I.random_state(n, spec.N, 65)
    v[P.dirichlet_nodes(spec), :3] = 0.0
    interior = np.setdiff1d(np.arange(n), np.unique(m.faces.ravel()))
    nodes = np.sort(np.random.default_rng(66).choice(interior, 48, replace=False))
    checks = [
        (lambda: gp.residual(y, 1), lambda pr, yy: O.residual(pr, yy), None),
        (lambda: gp.jv(y, v, 0, 1, 0.0), lambda pr, yy, vv: O.jv_paper(pr, yy, vv), v),
    ]
    for run, fn, vv in checks:
        got = run()[nodes]
        ref = _sampled_oracle(spec, y, vv, nodes, fn)
        assert relerr(got, ref) < 1e-5
    gp.close()


def test_full_size_glenn_sampled_parity():
    """Glenn-like T-junction at full size (~1M tets, N = 21) in the launch configuration the benchmark
    times: residual and both Jv kinds at 64 sampled interior nodes against the oracle."""
    spec = P.glenn_spec()
    gp = P.gpu_problem(spec)
    m = spec.mesh
    n = m.n_nodes
    y = I.random_state(n, spec.N, 61)
    v = I.random_state(n, spec.N, 62)
    dn = P.dirichlet_nodes(spec)
    v[dn, :3] = 0.0
    bnd = np.unique(m.faces.ravel())
    interior = np.setdiff1d(np.arange(n), bnd)
    rng = np.random.default_rng(63)
    nodes = np.sort(rng.choice(interior, 64, replace=False))
    checks = [
        (lambda: gp.residual(y, 1), lambda pr, yy: O.residual(pr, yy), None),
        (lambda: gp.jv(y, v, 0, 1, 0.0), lambda pr, yy, vv: O.jv_paper(pr, yy, vv), v),
        (lambda: gp.jv(y, v, 1, 1, 0.0), lambda pr, yy, vv: O.jv_exact(pr, yy, vv), v),
    ]
    for run, fn, vv in checks:
        got = run()[nodes]
        ref = _sampled_oracle(spec, y, vv, nodes, fn)
        assert relerr(got, ref) < 1e-5
    # the deterministic summation at full size: bitwise equal on repeat, same sampled values
    gp.set_scatter(0)
    first = gp.jv(y, v, 0, 1, 0.0)
    assert np.array_equal(first, gp.jv(y, v, 0, 1, 0.0))
    assert relerr(first[nodes], _sampled_oracle(spec, y, v, nodes, lambda pr, yy, vv: O.jv_paper(pr, yy, vv))) < 1e-5
    gp.close()


@pytest.mark.parametrize("n_h", [4, 6, 10])
@pytest.mark.parametrize("path", [0, 1, 2])
def test_spectral_pass_paths(n_h, path):
    """The node-level W = shift v + rho H v pass on each implementation (tcgen05 with a TMEM accumulator,
    warp-level mma.sync, FP32 FMAs) inside the paper-tangent Jv, fused and assembled, against the oracle
    (N = 9, 13, 21; a ragged last 128-row tile)."""
    spec = P.box_spec(seed=80 + n_h, n_h=n_h, n=(7, 5, 4))
    ora = P.oracle_problem(spec)
    gp = P.gpu_problem(spec)
    gp.set_spectral_path(path)
    assert gp.spectral_path() == path
    y = I.random_state(spec.mesh.n_nodes, spec.N, 81)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 82)
    ref = O.jv_paper(ora, y, v, shift=0.9)
    assert relerr(gp.jv(y, v, 0, 1, 0.9), ref) < TOL[1]
    assert relerr(gp.jv(y, v, 2, 1, 0.9), ref) < TOL[1]
    gp.close()


def test_spectral_tcgen05_many_tiles():
    """tcgen05 spectral pass over ~65k velocity rows (hundreds of 128-row tiles, several per block, rows of a
    node split across tiles) inside the FP32 paper-tangent Jv, against the oracle."""
    spec = P.glenn_spec(n_tets=120_000)
    ora = P.oracle_problem(spec)
    gp = P.gpu_problem(spec)
    gp.set_spectral_path(0)
    y = I.random_state(spec.mesh.n_nodes, spec.N, 83).astype(np.float32).astype(np.float64)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 84).astype(np.float32).astype(np.float64)
    ref = O.jv_paper(ora, y, v, shift=250.0)
    assert relerr(gp.jv(y, v, 0, 1, 250.0), ref) < TOL[1]
    with pytest.raises(RuntimeError):
        gp.set_spectral_path(3)
    gp.close()


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_fp32_host_buffer_entry_point(box, kind):
    """hb_jv_f32 (FP32 host buffers) against the oracle at the FP32-rounded state and direction."""
    spec, ora, gp = box
    y = I.random_state(spec.mesh.n_nodes, spec.N, 35).astype(np.float32)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 36).astype(np.float32)
    ref = (O.jv_exact if kind == 1 else O.jv_paper)(ora, y.astype(np.float64), v.astype(np.float64), shift=1.1)
    got = gp.jv_f32(y, v, kind=kind, shift=1.1)
    assert got.dtype == np.float32
    assert relerr(got.astype(np.float64), ref) < TOL[1]
