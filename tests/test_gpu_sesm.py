"""SESM substep (AB3-AM4, Eqs. 4.7-4.8) on the GPU against the FP64 oracle, in both execution modes
(graph: one launch per substep; persistent: one launch per step, exchanging the AM4 elevation
between patches), same tolerance rule as the SE path: within twice the drift of the FP32 build of
the oracle, plus a floor of 8 ulp."""
import math

import numpy as np
import pytest

from oracle import closed
from oracle import runner as orc
from paper_2311_08241_gb300 import inputs as I
from parity_util import ENVELOPE_FACTOR, GRAPH, MODES, PERSISTENT, ULP_FLOOR, _maxabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2311_08241_gb300 import sesw

    sesw.load()
    return sesw


def _sesm(case, theta=0.14):
    p = case.params
    case.params = I.Params(g=p.g, theta=theta, tau=p.tau, M=p.M, nonlinear_h=p.nonlinear_h, scheme=1)
    return closed.sesm_params(theta / 2.0)


def _run(S, case, nsteps, mode=GRAPH, bps=None):
    with S.Subcycle() as s:
        s.sesw_set_mode(mode)
        if bps:
            s.sesw_set_blocks_per_sm(bps)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(nsteps)
        info = s.sesw_get_info()
        return s.sesw_get_state(), info


def _check(case, coef, got, nsteps, what):
    ref = orc.OracleMesh(case.mesh).advance_sesm(case.R, case.params, coef, nsteps, case.eta0, case.U0)
    r32 = orc.OracleMesh(case.mesh, orc.lib_fp32()).advance_sesm(case.R, case.params, coef, nsteps, case.eta0,
                                                                   case.U0)
    for k, name in enumerate(("eta", "U", "<<U>>")):
        scale = max(_maxabs(ref[k]), 1e-30)
        err = _maxabs(got[k] - ref[k])
        env = _maxabs(r32[k] - ref[k])
        tol = ENVELOPE_FACTOR * env + ULP_FLOOR * scale
        print(f"{what} {name}: err {err:.3e} env32 {env:.3e} tol {tol:.3e}")
        assert err <= tol, f"{what} {name}: err {err:.3e} > tol {tol:.3e}"
    return ref


@MODES
@pytest.mark.parametrize("name", ["basin", "tiny", "channel", "sphere6"])
def test_sesm_matches_oracle(S, name, mode):
    case = {"basin": lambda: I.basin_case(nsteps=5),
            "tiny": lambda: I.tiny_jittered_case(nx=21, ny=15, seed=5, M=7, tau=70.0),
            "channel": lambda: I.channel_case(nsteps=10),
            "sphere6": lambda: I.sphere_case(level=6, nsteps=5)}[name]()
    coef = _sesm(case)
    (got, info) = _run(S, case, case.nsteps, mode)
    assert info["mode"] == mode
    _check(case, coef, got, case.nsteps, f"{name} mode={mode}")


@MODES
def test_sesm_periodic_wave_closed_form(S, mode):
    case = I.periodic_wave_case(n=32, kx=3, ky=1, nsteps=4, M=30, tau=450.0)
    coef = _sesm(case)
    (eta, U, Um), info = _run(S, case, case.nsteps, mode)
    assert info["mode"] == mode
    p = case.params
    u, e = closed.sesm_mode_amplitude(closed.kappa2_square(32, 10e3, 3, 1), p.g * 4000.0, p.tau / p.M, coef, p.M,
                                      case.nsteps)
    assert np.max(np.abs(eta - e * case.eta0)) < 1e-5


@MODES
def test_sesm_summation_identity_and_volume(S, mode):
    case = I.basin_case(nsteps=1)
    _sesm(case)
    om = orc.OracleMesh(case.mesh)
    av, _ = om.areas()
    with S.Subcycle() as s:
        s.sesw_set_mode(mode)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_state(case.eta0, case.U0)
        prev = s.sesw_get_state()[0]
        for _ in range(6):
            s.sesw_advance(1)
            eta, U, Um = s.sesw_get_state()
            assert np.max(np.abs((eta - prev) + case.params.tau * om.divergence(Um))) < 2e-5
            prev = eta
        vol, _ = s.sesw_diagnostics()
    v0 = float(np.sum(av * case.eta0))
    bound = 4 * 2.0 ** -24 * math.sqrt(6 * case.params.M) * math.sqrt(float(np.sum((av * case.eta0) ** 2)))
    assert abs(vol - v0) <= bound


def test_sesm_rules(S):
    case = I.tiny_jittered_case()
    _sesm(case)
    # the on-chip SESM kernel takes patches of at most 4 x 384 slots: one block per SM on
    # the channel gives patches of ~1300 vertices, whose state the layout then streams
    big = I.channel_case(nsteps=1)
    _sesm(big)
    with S.Subcycle() as s:
        s.sesw_set_mode(PERSISTENT)
        s.sesw_set_blocks_per_sm(1)
        s.sesw_mesh_upload(big.mesh)
        assert s.sesw_get_info()["mode"] == PERSISTENT
        s.sesw_set_params(big.params)
        assert s.sesw_get_info()["streamed"] == 1
    with S.Subcycle() as s:
        s.sesw_set_mode(PERSISTENT)
        s.sesw_mesh_upload(big.mesh)
        s.sesw_set_params(big.params)
        info = s.sesw_get_info()
        assert info["mode"] == PERSISTENT and info["slots_per_thread"] >= 1 and info["block_threads"] <= 384
    with S.Subcycle() as s:
        s.sesw_set_mode(GRAPH)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        lim = s.sesw_get_info()["courant_limit"]
    # the library's limit equals the spectral-radius limit of the per-mode matrix (numpy eigenvalues)
    coef = closed.sesm_params(0.07)
    lo, hi = 0.0, 4.0
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        A = closed.sesm_lattice_matrix(mid * mid, 1.0, 1.0, *coef)
        if np.max(np.abs(np.linalg.eigvals(A))) <= 1 + 1e-9:
            lo = mid
        else:
            hi = mid
    assert abs(lim - lo) < 2e-3, (lim, lo)


def test_sesm_persistent_batch_in_packs(S):
    """A batch of basins with the SESM scheme in persistent mode, more patches than resident blocks
    (several cooperative launches per step, each with its own tag base), matches the oracle per basin."""
    cases = I.ensemble_cases(nbasins=14, scale=0.2, seed=11, nsteps=2)   # ~276k vertices: two packs
    coefs = [_sesm(c) for c in cases]
    with S.Subcycle() as s:
        s.sesw_set_mode(PERSISTENT)
        s.sesw_mesh_upload_batch([c.mesh for c in cases])
        s.sesw_set_params_batch([c.params for c in cases])
        s.sesw_set_forcing(np.concatenate([c.R for c in cases]))
        s.sesw_set_state(np.concatenate([c.eta0 for c in cases]), np.concatenate([c.U0 for c in cases]))
        s.sesw_advance(2)
        info = s.sesw_get_info()
        eta, U, Um = s.sesw_get_state()
    assert info["mode"] == PERSISTENT and info["npack"] > 1, info
    iv = np.cumsum([c.mesh.nv for c in cases])[:-1]
    ie = np.cumsum([c.mesh.ne for c in cases])[:-1]
    for c, coef, e, u, um in zip(cases, coefs, np.split(eta, iv), np.split(U, ie), np.split(Um, ie)):
        _check(c, coef, (e, u, um), 2, f"{c.name} packs={info['npack']}")


def test_sesm_streamed_on_the_sphere_matches_oracle(S):
    """The level-8 sphere's patches are too large for the SESM kernel's on-chip state, so the
    persistent layout streams the transport levels and sums from L2; 2 steps against the oracle."""
    case = I.sphere_case(level=8, nsteps=2)
    coef = _sesm(case)
    (got, info) = _run(S, case, 2, PERSISTENT, bps=2)
    assert info["mode"] == PERSISTENT and info["streamed"] == 1, info
    _check(case, coef, got, 2, "sphere8 SESM streamed")


def test_sesm_streamed_without_the_index_cache(S):
    """Patches that fit the streaming SESM kernel's shared memory only without the slots' corner
    indices (a 704k-vertex channel at the benchmark channel's resolution) read the indices from L2
    every substep; 2 steps against the oracle."""
    case = I.channel_case(nx=1100, ny=640, Lx=4000e3 * 1100 / 588, Ly=2000e3 * 640 / 340, nsteps=2)
    coef = _sesm(case)
    (got, info) = _run(S, case, 2, PERSISTENT)
    assert info["mode"] == PERSISTENT and info["streamed"] == 2, info
    _check(case, coef, got, 2, "channel 704k SESM streamed, indices from L2")


def test_sesm_batch_mixes_streamed_and_cached_packs(S):
    """One SESM step launching different kernels per pack: the level-8 sphere (streamed) batched
    with small basins (on-chip SESM kernel). Every basin against the oracle."""
    sphere = I.sphere_case(level=8, nsteps=2)
    small = I.ensemble_cases(nbasins=3, vmin=5000, vmax=20000, M=sphere.params.M, nsteps=2, seed=5)
    cases = small + [sphere]
    coefs = [_sesm(c) for c in cases]
    with S.Subcycle() as s:
        s.sesw_set_mode(PERSISTENT)
        s.sesw_mesh_upload_batch([c.mesh for c in cases])
        s.sesw_set_params_batch([c.params for c in cases])
        s.sesw_set_forcing(np.concatenate([c.R for c in cases]))
        s.sesw_set_state(np.concatenate([c.eta0 for c in cases]), np.concatenate([c.U0 for c in cases]))
        s.sesw_advance(2)
        info = s.sesw_get_info()
        eta, U, Um = s.sesw_get_state()
    assert info["mode"] == PERSISTENT and info["npack"] >= 2 and info["streamed"] == 0, info
    iv = np.cumsum([c.mesh.nv for c in cases])[:-1]
    ie = np.cumsum([c.mesh.ne for c in cases])[:-1]
    for c, coef, e, u, um in zip(cases, coefs, np.split(eta, iv), np.split(U, ie), np.split(Um, ie)):
        _check(c, coef, (e, u, um), 2, f"{c.name} in a mixed SESM batch")
