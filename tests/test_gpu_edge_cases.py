"""Degenerate inputs on the GPU: a single triangle, disconnected triangles, zero steps, a state at
rest, and the viscosity and freshwater terms where they reduce to closed forms."""
import numpy as np
import pytest

from oracle import runner as orc
from paper_2311_08241_gb300 import inputs as I
from parity_util import GRAPH, MODES, PERSISTENT, _assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2311_08241_gb300 import sesw

    sesw.load()
    return sesw


def _triangles(n, h=10e3, seed=0):
    """n disconnected right triangles (legs h), random depths, f-plane."""
    rng = np.random.default_rng(seed)
    tri = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    base = np.array([[0.0, 0.0], [h, 0.0], [0.0, h]])
    P = np.concatenate([base + np.array([3 * h * k, 0.0]) for k in range(n)])
    xy = P[tri]
    pos = np.concatenate([P, np.zeros((3 * n, 1))], axis=1)
    depth = 2000.0 + 2000.0 * rng.random(3 * n)
    mesh = I._contig(I.Mesh("triangles", tri, xy, pos, depth, np.full(n, 1e-4)))
    eta0 = 0.2 * rng.standard_normal(3 * n)
    U0 = 3.0 * rng.standard_normal((n, 2))
    R = 1e-3 * rng.standard_normal((n, 2))
    return mesh, eta0, U0, R


@MODES
@pytest.mark.parametrize("ntri,M", [(1, 1), (1, 3), (5, 4)])
def test_single_and_disconnected_triangles(S, mode, ntri, M):
    mesh, eta0, U0, R = _triangles(ntri, seed=ntri + M)
    case = I.Case("triangles", mesh, I.Params(tau=10.0 * M, M=M, nonlinear_h=1), R, eta0, U0, 3)
    got = S.run_case(case, mode=mode)
    _assert_close(case, got, f"{ntri} triangle(s), M={M}, mode={mode}")
    # a lone triangle keeps its volume: its divergence sums to zero over its corners
    om = orc.OracleMesh(mesh)
    av, _ = om.areas()
    assert abs(float(np.sum(av * (got[0] - eta0)))) <= 1e-5 * float(np.sum(av * np.abs(eta0)))


@MODES
def test_zero_steps_and_rest_state(S, mode):
    case = I.tiny_jittered_case(nx=9, ny=7, seed=31)
    with S.Subcycle() as s:
        s.sesw_set_mode(mode)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        before = s.sesw_get_state()
        s.sesw_advance(0)
        after = s.sesw_get_state()
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
        # no forcing, no motion, flat surface: nothing moves
        s.sesw_set_forcing(np.zeros_like(case.R))
        s.sesw_set_state(np.zeros(case.mesh.nv), np.zeros((case.mesh.ne, 2)))
        s.sesw_advance(3)
        eta, U, Um = s.sesw_get_state()
    assert not np.any(eta) and not np.any(U) and not np.any(Um)


def test_viscosity_without_neighbours_and_uniform_freshwater(S):
    """Disconnected triangles have no interior edges, so the viscosity contributes nothing; a
    uniform W from rest lowers every vertex by tau W per step exactly as the oracle does."""
    mesh, eta0, U0, R = _triangles(4, seed=3)
    stiff = S.sesw_mesh_check(mesh)["visc_stiffness"]
    assert stiff == 0.0
    p = I.Params(tau=40.0, M=4, nonlinear_h=1, visc=(1e5, 5.0))
    case = I.Case("triangles", mesh, p, R, eta0, U0, 2)
    with S.Subcycle() as s:
        s.sesw_set_mode(GRAPH)
        s.sesw_mesh_upload(mesh)
        s.sesw_set_params(p)
        s.sesw_set_state(eta0, U0)
        assert np.max(np.abs(s.sesw_viscosity())) == 0.0
        s.sesw_set_forcing(R)
        s.sesw_advance(2)
        got = s.sesw_get_state()
    ref = orc.OracleMesh(mesh).advance(R, p, 2, eta0, U0)[:3]
    for a, b in zip(got, ref):
        assert np.max(np.abs(a - b)) <= 1e-5 * max(1.0, np.max(np.abs(b)))
    for mode in (GRAPH, PERSISTENT):
        with S.Subcycle() as s:
            s.sesw_set_mode(mode)
            s.sesw_mesh_upload(mesh)
            s.sesw_set_params(I.Params(tau=40.0, M=4, nonlinear_h=1))
            s.sesw_set_freshwater(np.full(mesh.nv, 3e-5))
            s.sesw_set_state(np.zeros(mesh.nv), np.zeros((mesh.ne, 2)))
            s.sesw_advance(5)
            eta, U, _ = s.sesw_get_state()
        assert np.max(np.abs(eta + 5 * 40.0 * 3e-5)) <= 1e-6
        assert np.max(np.abs(U)) <= 1e-9


@MODES
def test_upload_with_caller_edges_and_areas(S, mode):
    """A mesh uploaded with the caller's edge connectivity and areas (here the oracle's own tables)
    gives bitwise the result of the same mesh with the tables derived by the library."""
    case = I.basin_case(nsteps=3)
    om = orc.OracleMesh(case.mesh)
    edges, areas = om.edges(), om.areas()
    out = []
    for tables in ((None, None), (edges, areas)):
        with S.Subcycle() as s:
            s.sesw_set_mode(mode)
            s.sesw_mesh_upload(case.mesh, edges=tables[0], areas=tables[1])
            s.sesw_set_params(case.params)
            s.sesw_set_forcing(case.R)
            s.sesw_set_state(case.eta0, case.U0)
            s.sesw_advance(case.nsteps)
            out.append(s.sesw_get_state())
    for k in range(3):
        assert np.array_equal(out[0][k], out[1][k])
    _assert_close(case, out[1], f"basin with caller tables mode={mode}")


@MODES
def test_parameters_changed_between_steps(S, mode):
    """The step coefficients follow every sesw_set_params: the channel advances 3 steps, then 2 with
    another tau (hence dt) and g, then 2 with a third M; against the oracle run through the same
    sequence, within twice the FP32 oracle's drift."""
    import dataclasses

    from parity_util import ENVELOPE_FACTOR, ULP_FLOOR, _maxabs

    case = I.channel_case(nsteps=3)
    p0 = case.params
    seq = [(p0, 3), (dataclasses.replace(p0, tau=0.75 * p0.tau, g=9.7), 2),
           (dataclasses.replace(p0, tau=0.75 * p0.tau, g=9.7, M=30), 2)]
    with S.Subcycle() as s:
        s.sesw_set_mode(mode)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_forcing(case.R)
        for k, (p, n) in enumerate(seq):
            s.sesw_set_params(p)
            if k == 0:
                s.sesw_set_state(case.eta0, case.U0)
            s.sesw_advance(n)
        got = s.sesw_get_state()
    refs = []
    for L in (None, orc.lib_fp32()):
        om = orc.OracleMesh(case.mesh, L) if L is not None else orc.OracleMesh(case.mesh)
        eta, U = case.eta0, case.U0
        for p, n in seq:
            eta, U, Um, _ = om.advance(case.R, p, n, eta, U)
        refs.append((eta, U, Um))
    ref, r32 = refs
    for k, name in enumerate(("eta", "U", "<<U>>")):
        tol = ENVELOPE_FACTOR * _maxabs(r32[k] - ref[k]) + ULP_FLOOR * _maxabs(ref[k])
        assert _maxabs(got[k] - ref[k]) <= tol, f"{name}: {_maxabs(got[k] - ref[k]):.3e} > {tol:.3e}"
