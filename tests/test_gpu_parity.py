"""GPU path (through the C-ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (FP32 state on the GPU, FP64 in the oracle):
  eta    max |d eta| <= ETA_TOL m. 1e-5 m after 100 channel steps (4000 substeps) is
         the stated target; with FP32 rounding (2^-24 relative) per substep on
         |eta| <~ 1 m, an unbiased random walk over 4000 substeps stays near
         6e-8 * sqrt(4000) ~ 4e-6 m.
  U, <<U>>  max |dU| <= U_REL * max |U_ref| (+ a floor of 1e-6 m^2/s for fields at rest),
         the same per-substep rounding argument applied to the transport.
"""
import math

import numpy as np
import pytest

from oracle import closed
from oracle import runner as orc
from paper_2311_08241_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ETA_TOL = 1e-5
U_REL = 2e-5


@pytest.fixture(scope="module")
def sesw():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2311_08241_gb300 import sesw as S

    S.load()
    return S


def _errs(ref, got):
    e_ref, U_ref, M_ref = ref[:3]
    e, U, Um = got
    de = float(np.max(np.abs(e - e_ref)))
    su = max(float(np.max(np.abs(U_ref))), 1e-300)
    sm = max(float(np.max(np.abs(M_ref))), 1e-300)
    du = float(np.max(np.abs(U - U_ref)))
    dm = float(np.max(np.abs(Um - M_ref)))
    return de, du, su, dm, sm


def _assert_close(ref, got, what, eta_tol=ETA_TOL, u_rel=U_REL):
    de, du, su, dm, sm = _errs(ref, got)
    print(f"{what}: max|d eta| = {de:.3e}, max|dU| = {du:.3e} (rel {du / su:.2e}), "
          f"max|d<<U>>| = {dm:.3e} (rel {dm / sm:.2e})")
    assert de <= eta_tol, f"{what}: eta error {de:.3e}"
    assert du <= u_rel * su + 1e-6, f"{what}: U error {du:.3e} vs scale {su:.3e}"
    assert dm <= u_rel * sm + 1e-6, f"{what}: <<U>> error {dm:.3e} vs scale {sm:.3e}"


def test_basin_matches_oracle(sesw):
    """Closed 1000x500 km basin, Gaussian bump, f-plane, 20 steps of 30 substeps."""
    case = I.basin_case()
    ref = orc.run_case(case)
    got = sesw.run_case(case)
    _assert_close(ref, got, "basin")


def test_channel_matches_oracle_100_steps(sesw):
    """Wind-driven channel (200k vertices) in the benchmark's launch configuration, 100 steps."""
    case = I.channel_case(nsteps=100)
    ref = orc.run_case(case)
    got = sesw.run_case(case)
    _assert_close(ref, got, "channel-100")


@pytest.mark.parametrize("pv", [32, 100, 777])
@pytest.mark.parametrize("seed", [1, 2])
def test_tiny_meshes_many_patches(sesw, pv, seed):
    """Small jittered basins cut into many ragged patches (guest copies on every border)."""
    case = I.tiny_jittered_case(nx=23, ny=17, seed=seed, M=9, tau=90.0)
    case.nsteps = 4
    ref = orc.run_case(case)
    got = sesw.run_case(case, patch_vertices=pv)
    _assert_close(ref, got, f"tiny pv={pv} seed={seed}")


def test_linear_h_and_odd_M(sesw):
    case = I.tiny_jittered_case(nx=30, ny=20, seed=7, M=7, tau=70.0, nonlinear_h=0)
    case.nsteps = 5
    ref = orc.run_case(case)
    got = sesw.run_case(case, patch_vertices=64)
    _assert_close(ref, got, "linear-H odd M")


def test_sphere_matches_oracle(sesw):
    """Icosahedral sphere (level 6 here; level 8 in the next test) with land, forcing and f = 2 Omega sin(lat)."""
    case = I.sphere_case(level=6, nsteps=10)
    ref = orc.run_case(case)
    got = sesw.run_case(case)
    _assert_close(ref, got, "sphere-l6")


def test_sphere_level8_full_size(sesw):
    """Global-like sphere at full size (level 8: ~460k wet vertices), 5 steps of 50 substeps."""
    case = I.sphere_case(level=8, nsteps=5)
    ref = orc.run_case(case)
    got = sesw.run_case(case)
    _assert_close(ref, got, "sphere-l8")


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
    bound = 4 * eps32 * math.sqrt(20 * case.params.M) * math.sqrt(float(np.sum((av * case.eta0) ** 2))) * 10
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


def test_resume_is_bitwise(sesw):
    """Checkpoint/resume: 3 steps, read back, restart in a new context, 2 steps == 5 straight steps."""
    case = I.tiny_jittered_case(nx=25, ny=18, seed=9, M=8, tau=80.0)
    straight = sesw.run_case(case, nsteps=5)
    with sesw.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(3)
        eta, U, _ = s.sesw_get_state()
    with sesw.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(eta, U)
        s.sesw_advance(2)
        resumed = s.sesw_get_state()
    for a, b in zip(straight, resumed):
        assert np.array_equal(a, b)


def test_deterministic(sesw):
    case = I.channel_case(nsteps=3)
    a = sesw.run_case(case)
    b = sesw.run_case(case)
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
