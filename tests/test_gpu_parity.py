"""GPU path (through the C-ABI) against the FP64 oracle on the same seeded inputs.

Tolerances. The GPU keeps eta and U in FP32 (geometry derived in FP64, rounded
once). Its drift from the FP64 oracle is compared with the drift of the same
algorithm run in FP32 on the CPU: the oracle source built with float as its working
precision (geometry still derived in double), on the same inputs. For every field,
    max |GPU - FP64 oracle| <= ENVELOPE_FACTOR * max |FP32 oracle - FP64 oracle| + floor,
with ENVELOPE_FACTOR = 2 (the two FP32 programs round in different orders, so their
drifts differ by O(1) factors, not orders of magnitude) and a floor of a few FP32
ulps of the field's scale. On top of that, eta must meet the absolute target
max |d eta| <= 1e-5 m (after 100 baroclinic steps of the channel).
The FP32 drift is large for U in the channel (~8e-5 relative after 4000 substeps):
U is near geostrophic balance there, so FP32 rounding of eta and of the geometry
(about 6e-8 relative) is amplified by g H / (f L).
"""
import math

import numpy as np
import pytest

from oracle import closed
from oracle import runner as orc
from paper_2311_08241_gb300 import inputs as I

pytestmark = pytest.mark.gpu

from parity_util import (ENVELOPE_FACTOR, ETA_ABS_TOL, GRAPH, MODES, PERSISTENT, ULP_FLOOR, _assert_close,
                         _maxabs)


@pytest.fixture(scope="module")
def sesw():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2311_08241_gb300 import sesw as S

    S.load()
    return S


@MODES
def test_basin_matches_oracle(sesw, mode):
    """Closed 1000x500 km basin, Gaussian bump, f-plane, 20 steps of 30 substeps."""
    case = I.basin_case()
    got = sesw.run_case(case, mode=mode)
    _assert_close(case, got, f"basin mode={mode}")


@MODES
def test_channel_matches_oracle_100_steps(sesw, mode):
    """Wind-driven channel (200k vertices), 100 steps; the persistent mode is the benchmark's launch
    configuration."""
    case = I.channel_case(nsteps=100)
    got = sesw.run_case(case, mode=mode)
    _assert_close(case, got, f"channel-100 mode={mode}")


@pytest.mark.parametrize("pv", [32, 100, 777])
@pytest.mark.parametrize("seed", [1, 2])
def test_tiny_meshes_many_patches(sesw, pv, seed):
    """Small jittered basins cut into many ragged patches (guest copies on every border)."""
    case = I.tiny_jittered_case(nx=23, ny=17, seed=seed, M=9, tau=90.0)
    case.nsteps = 4
    got = sesw.run_case(case, patch_vertices=pv, mode=GRAPH)
    _assert_close(case, got, f"tiny pv={pv} seed={seed}")


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiny_meshes_persistent(sesw, seed):
    """Small meshes in the persistent kernel: few patches, ragged slot counts per block."""
    case = I.tiny_jittered_case(nx=23 + seed, ny=17, seed=seed, M=9, tau=90.0)
    case.nsteps = 4
    got = sesw.run_case(case, mode=PERSISTENT)
    _assert_close(case, got, f"tiny persistent seed={seed}")


@MODES
def test_linear_h_and_odd_M(sesw, mode):
    case = I.tiny_jittered_case(nx=30, ny=20, seed=7, M=7, tau=70.0, nonlinear_h=0)
    case.nsteps = 5
    got = sesw.run_case(case, patch_vertices=64, mode=mode)
    _assert_close(case, got, f"linear-H odd M mode={mode}")


@MODES
def test_sphere_matches_oracle(sesw, mode):
    """Icosahedral sphere (level 6 here; level 8 in the next test) with land, forcing and f = 2 Omega sin(lat)."""
    case = I.sphere_case(level=6, nsteps=10)
    got = sesw.run_case(case, mode=mode)
    _assert_close(case, got, f"sphere-l6 mode={mode}")


@MODES
def test_sphere_level8_full_size(sesw, mode):
    """Global-like sphere at full size and length (level 8: ~460k wet vertices), 50 steps of 50
    substeps, the workload's own length."""
    case = I.sphere_case(level=8, nsteps=50)
    got = sesw.run_case(case, mode=mode)
    _assert_close(case, got, f"sphere-l8-50 mode={mode}")


def test_channel_matches_oracle_200_steps(sesw):
    """The channel over its full length of 200 steps (8000 substeps) in the benchmark's launch
    configuration (the other layouts give bitwise the same result, tests/test_gpu_bitwise.py)."""
    case = I.channel_case(nsteps=200)
    got = sesw.run_case(case, mode=PERSISTENT)
    _assert_close(case, got, "channel-200 persistent")


def test_modes_agree(sesw):
    """Graph and persistent execution run the same FP32 arithmetic per triangle and the same
    summation order per vertex: bitwise equal results."""
    case = I.channel_case(nsteps=10)
    a = sesw.run_case(case, mode=GRAPH)
    b = sesw.run_case(case, mode=PERSISTENT)
    for k in range(3):
        assert np.array_equal(a[k], b[k]), f"field {k}: max |diff| {_maxabs(a[k] - b[k]):.3e}"


def test_periodic_wave_closed_form(sesw):
    """A cosine mode on the periodic mesh follows the exact 2x2 recurrence (Eq. 3.7 with kappa^2)."""
    case = I.periodic_wave_case(n=32, kx=3, ky=1, nsteps=4)
    eta, U, Um = sesw.run_case(case)
    p = case.params
    k2 = closed.kappa2_square(32, 10e3, 3, 1)
    u_e = closed.mode_amplitude(k2, p.g * 4000.0, p.tau / p.M, p.theta, case.nsteps * p.M)
    assert np.max(np.abs(eta - u_e[1] * case.eta0)) < 1e-5


def test_summation_identity_and_volume(sesw):
    """Eq. 4.11 per vertex, and volume conservation to FP32 roundoff with FP64 diagnostics."""
    case = I.basin_case(nsteps=1)
    om = orc.OracleMesh(case.mesh)
    av, _ = om.areas()
    with sesw.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_state(case.eta0, case.U0)
        v0, _ = s.sesw_diagnostics()
        eta_prev = s.sesw_get_state()[0]
        vols = []
        for n in range(20):
            s.sesw_advance(1)
            eta, U, Um = s.sesw_get_state()
            resid = (eta - eta_prev) + case.params.tau * om.divergence(Um)
            # FP32: eta carries ~6e-8 relative rounding per substep, Umean the same
            assert np.max(np.abs(resid)) < 2e-5, np.max(np.abs(resid))
            eta_prev = eta
            vols.append(s.sesw_diagnostics()[0])
    assert abs(v0 - float(np.sum(av * case.eta0))) < 1e-6 * float(np.sum(av * np.abs(case.eta0)))
    eps32 = 2.0 ** -24
    bound = 4 * eps32 * math.sqrt(20 * case.params.M) * math.sqrt(float(np.sum((av * case.eta0) ** 2)))
    drift = np.abs(np.array(vols) - v0)
    print("volume drift", drift.max(), "bound", bound)
    assert drift.max() <= bound


def test_diagnostics_match_oracle(sesw):
    case = I.tiny_jittered_case(nx=20, ny=15, seed=4)
    with sesw.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(2)
        eta, U, _ = s.sesw_get_state()
        vol, en = s.sesw_diagnostics()
    om = orc.OracleMesh(case.mesh)
    v_ref, e_ref = om.diagnostics(eta, U, case.params.g, case.params.nonlinear_h)
    assert abs(vol - v_ref) <= 1e-6 * abs(v_ref) + 1e-3
    assert abs(en - e_ref) <= 1e-5 * abs(e_ref)


@MODES
def test_resume_is_bitwise(sesw, mode):
    """Checkpoint/resume: 3 steps, read back, restart in a new context, 2 steps == 5 straight steps."""
    case = I.tiny_jittered_case(nx=25, ny=18, seed=9, M=8, tau=80.0)
    straight = sesw.run_case(case, nsteps=5, mode=mode)
    with sesw.Subcycle() as s:
        s.sesw_set_mode(mode)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(3)
        eta, U, _ = s.sesw_get_state()
    with sesw.Subcycle() as s:
        s.sesw_set_mode(mode)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(eta, U)
        s.sesw_advance(2)
        resumed = s.sesw_get_state()
    for a, b in zip(straight, resumed):
        assert np.array_equal(a, b)


@MODES
def test_deterministic(sesw, mode):
    case = I.channel_case(nsteps=3)
    a = sesw.run_case(case, mode=mode)
    b = sesw.run_case(case, mode=mode)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_device_pointers_match_host(sesw):
    import torch

    case = I.tiny_jittered_case(nx=20, ny=14, seed=6)
    host = sesw.run_case(case, nsteps=2)
    dev = torch.device("cuda", 0)
    with sesw.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(torch.tensor(case.R, device=dev))
        s.sesw_set_state(torch.tensor(case.eta0, device=dev), torch.tensor(case.U0, device=dev))
        s.sesw_advance(2)
        e = torch.empty(case.mesh.nv, dtype=torch.float64, device=dev)
        U = torch.empty((case.mesh.ne, 2), dtype=torch.float64, device=dev)
        Um = torch.empty((case.mesh.ne, 2), dtype=torch.float64, device=dev)
        s.sesw_get_state(e, U, Um)
        torch.cuda.synchronize()
    for a, b in zip(host, (e.cpu().numpy(), U.cpu().numpy(), Um.cpu().numpy())):
        assert np.array_equal(a, b)


def test_errors_are_reported(sesw):
    case = I.tiny_jittered_case()
    with sesw.Subcycle() as s:
        with pytest.raises(sesw.SeswError) as ei:
            s.sesw_advance(1)
        assert ei.value.code == sesw.SESW_ESTATE
        bad = I.Mesh("bad", case.mesh.tri.copy(), case.mesh.xy.copy(), case.mesh.pos, case.mesh.depth,
                      case.mesh.coriolis)
        bad.tri[3, 1] = case.mesh.nv + 5
        with pytest.raises(sesw.SeswError) as ei:
            s.sesw_mesh_upload(bad)
        assert ei.value.code == sesw.SESW_EINVAL and "out of range" in str(ei.value)
        s.sesw_mesh_upload(case.mesh)
        unstable = I.Params(tau=case.params.tau * 20, M=case.params.M)
        with pytest.raises(sesw.SeswError) as ei:
            s.sesw_set_params(unstable)
        assert ei.value.code == sesw.SESW_EINVAL and "stability" in str(ei.value)
        # a blow-up injected from the host (non-finite forcing) is caught on the device
        s.sesw_set_params(case.params)
        R = case.R.copy()
        R[0, 0] = np.nan
        s.sesw_set_forcing(R)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(1)
        assert s.sesw_status() == sesw.SESW_EUNSTABLE
        assert s.sesw_status() == sesw.SESW_OK        # cleared


def test_persistent_wait_gives_up_and_context_stays_usable(sesw):
    """Failure detection without a GPU fault: a patch that never publishes its progress makes
    its neighbours' bounded waits give up (~10 ms budget under the test flag); the step ends,
    the host reads SESW_ETIMEOUT, and the context then runs normal steps again."""
    import time

    case = I.basin_case(nsteps=1)
    with sesw.Subcycle() as s:
        s.sesw_set_mode(PERSISTENT)
        s.sesw_mesh_upload(case.mesh)
        assert s.sesw_get_info()["mode"] == PERSISTENT
        s.sesw_set_params(case.params, flags=sesw.SESW_FLAG_TEST_FORCE_TIMEOUT)
        s.sesw_set_state(case.eta0, case.U0)
        t0 = time.perf_counter()
        s.sesw_advance(1)
        assert s.sesw_status() == sesw.SESW_ETIMEOUT
        assert time.perf_counter() - t0 < 30.0
        assert s.sesw_status() == sesw.SESW_OK
        s.sesw_set_params(case.params)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(1)
        assert s.sesw_status() == sesw.SESW_OK
        got = s.sesw_get_state()
    ref = orc.run_case(case)
    assert _maxabs(got[0] - ref[0]) < 1e-5


def test_persistent_tags_continue_across_launches_with_changing_substep_counts(sesw):
    """The persistent kernel's exchange buffers are never cleared: each launch's tags continue
    from where the previous launch left them, advancing by M + 1. Steps with different M in a
    row, in one context, match the oracle run through the same sequence."""
    case = I.channel_case(nsteps=1)
    p0 = case.params
    dt = p0.tau / p0.M
    seq = [(40, 2), (7, 1), (13, 2), (40, 1)]
    om, om32 = orc.OracleMesh(case.mesh), orc.OracleMesh(case.mesh, orc.lib_fp32())
    ref = (case.eta0, case.U0)
    r32 = (case.eta0, case.U0)
    with sesw.Subcycle() as s:
        s.sesw_set_mode(PERSISTENT)
        s.sesw_mesh_upload(case.mesh)
        assert s.sesw_get_info()["mode"] == PERSISTENT and s.sesw_get_info()["npatch"] > 1
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        for M, n in seq:
            p = I.Params(g=p0.g, theta=p0.theta, tau=dt * M, M=M, nonlinear_h=p0.nonlinear_h)
            s.sesw_set_params(p)
            s.sesw_advance(n)
            assert s.sesw_status() == sesw.SESW_OK
            ref = om.advance(case.R, p, n, ref[0], ref[1])[:3]
            r32 = om32.advance(case.R, p, n, r32[0], r32[1])[:3]
        got = s.sesw_get_state()
    for k, name in enumerate(("eta", "U", "<<U>>")):
        tol = ENVELOPE_FACTOR * _maxabs(r32[k] - ref[k]) + ULP_FLOOR * _maxabs(ref[k])
        assert _maxabs(got[k] - ref[k]) <= tol, name
    assert _maxabs(got[0] - ref[0]) <= ETA_ABS_TOL


def test_streaming_layout_with_freshwater_and_step_mean(sesw):
    """The streaming kernel (the level-8 sphere's patches at two blocks per SM, form streamed): the
    transport, sums and static data stream from L2. Its variant with the per-vertex terms: the
    freshwater flux over 2 steps against the oracle, and the step-mean elevation of one step."""
    case = I.sphere_case(level=8, nsteps=2)
    W = 2e-6 * (0.3 + np.random.default_rng(31).standard_normal(case.mesh.nv))
    with sesw.Subcycle() as s:
        s.sesw_set_blocks_per_sm(2)
        s.sesw_set_persistent_form(sesw.SESW_FORM_STREAM)
        s.sesw_mesh_upload(case.mesh)
        info = s.sesw_get_info()
        assert info["mode"] == PERSISTENT and info["streamed"] == 1, info
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        s.sesw_set_freshwater(W)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(2)
        got = s.sesw_get_state()
        s.sesw_set_freshwater(None)
        s.sesw_set_eta_mean(True)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(1)
        eb = s.sesw_get_eta_mean()
    om = orc.OracleMesh(case.mesh)
    ref = om.advance_ext(case.R, case.params, 2, case.eta0, case.U0, W=W)
    r32 = orc.OracleMesh(case.mesh, orc.lib_fp32()).advance_ext(case.R, case.params, 2, case.eta0, case.U0, W=W)
    for k, name in enumerate(("eta", "U", "<<U>>")):
        tol = ENVELOPE_FACTOR * _maxabs(r32[k] - ref[k]) + ULP_FLOOR * _maxabs(ref[k])
        assert _maxabs(got[k] - ref[k]) <= tol, name
    assert _maxabs(got[0] - ref[0]) <= ETA_ABS_TOL
    *_, eb_ref = om.advance(case.R, case.params, 1, case.eta0, case.U0, want_eta_mean=True)
    assert _maxabs(eb - eb_ref) <= ETA_ABS_TOL


def test_streaming_without_the_index_cache(sesw):
    """Patches that fit the streaming kernel's shared memory only without the slots' corner indices
    (an 816k-vertex channel at the benchmark channel's resolution, one patch per block) read the
    indices from L2 every substep; 2 steps against the oracle."""
    case = I.channel_case(nx=1200, ny=680, Lx=4000e3 * 1200 / 588, Ly=2000e3 * 680 / 340, nsteps=2)
    with sesw.Subcycle() as s:
        s.sesw_set_mode(PERSISTENT)
        s.sesw_mesh_upload(case.mesh)
        info = s.sesw_get_info()
        assert info["streamed"] == 2, info
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(2)
        assert s.sesw_status() == sesw.SESW_OK
        got = s.sesw_get_state()
    ref = orc.OracleMesh(case.mesh).advance(case.R, case.params, 2, case.eta0, case.U0)[:3]
    r32 = orc.OracleMesh(case.mesh, orc.lib_fp32()).advance(case.R, case.params, 2, case.eta0, case.U0)[:3]
    for k, name in enumerate(("eta", "U", "<<U>>")):
        tol = ENVELOPE_FACTOR * _maxabs(r32[k] - ref[k]) + ULP_FLOOR * _maxabs(ref[k])
        assert _maxabs(got[k] - ref[k]) <= tol, name
    assert _maxabs(got[0] - ref[0]) <= ETA_ABS_TOL


def test_contexts_with_different_layouts_coexist(sesw):
    """Kernel attributes are process-wide: a context with large patches keeps working after a
    context with small patches has been set up (and the other way round)."""
    big = I.channel_case(nsteps=2)
    small = I.tiny_jittered_case(nx=20, ny=14, seed=3)
    with sesw.Subcycle() as a, sesw.Subcycle() as b:
        for s, c in ((a, big), (b, small)):
            s.sesw_set_mode(PERSISTENT)
            s.sesw_mesh_upload(c.mesh)
            s.sesw_set_params(c.params)
            s.sesw_set_forcing(c.R)
            s.sesw_set_state(c.eta0, c.U0)
        a.sesw_advance(2)
        b.sesw_advance(2)
        ra, rb = a.sesw_get_state(), b.sesw_get_state()
    assert np.array_equal(ra[0], sesw.run_case(big, nsteps=2, mode=PERSISTENT)[0])
    assert np.array_equal(rb[0], sesw.run_case(small, nsteps=2, mode=PERSISTENT)[0])


@MODES
def test_async_host_transfers_match_the_synchronous_path(sesw, mode):
    """Pipelined steps through sesw_set_forcing_async / sesw_get_state_async (double-buffered,
    waited on two steps later) give bitwise the results of the synchronous calls."""
    import torch

    case = I.tiny_jittered_case(nx=12, ny=9, seed=41, M=6, tau=60.0)
    rng = np.random.default_rng(3)
    forcings = [case.R * (1.0 + 0.5 * rng.standard_normal()) for _ in range(6)]
    ref = []
    with sesw.Subcycle() as s:
        s.sesw_set_mode(mode)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_state(case.eta0, case.U0)
        for R in forcings:
            s.sesw_set_forcing(R)
            s.sesw_advance(1)
            ref.append(s.sesw_get_state())
    pin = lambda shape: torch.empty(shape, dtype=torch.float64).pin_memory()
    Rh = [pin((case.mesh.ne, 2)) for _ in range(2)]
    outs = [(pin(case.mesh.nv), pin((case.mesh.ne, 2)), pin((case.mesh.ne, 2))) for _ in range(2)]
    tickets = [0, 0]
    got = []
    with sesw.Subcycle() as s:
        s.sesw_set_mode(mode)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_state(case.eta0, case.U0)
        for n, R in enumerate(forcings):
            k = n & 1
            if n >= 2:
                s.sesw_wait(tickets[k])
                got.append(tuple(x.numpy().copy() for x in outs[k]))
            Rh[k].copy_(torch.from_numpy(R))
            s.sesw_set_forcing_async(Rh[k])
            s.sesw_advance(1)
            tickets[k] = s.sesw_get_state_async(*outs[k])
        for n in (len(forcings) - 2, len(forcings) - 1):
            s.sesw_wait(tickets[n & 1])
            got.append(tuple(x.numpy().copy() for x in outs[n & 1]))
        s.sesw_wait(0)
        with pytest.raises(sesw.SeswError, match="ticket"):
            s.sesw_wait(tickets[1] + 5)
    assert len(got) == len(ref)
    for a, b in zip(ref, got):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
