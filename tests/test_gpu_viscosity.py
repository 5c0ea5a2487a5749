"""Barotropic viscous regularisation (Eq. viscosity_BT) and freshwater flux W (Eq. 4.5) on the GPU
against the FP64 oracle. Same tolerance rule as the other parity tests: the GPU error is within
twice the drift of the oracle's FP32 build plus 8 ulp of the field's scale."""
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


CASES = {
    "tiny": lambda: I.tiny_jittered_case(nx=21, ny=15, seed=5, M=7, tau=70.0),
    "basin": lambda: I.basin_case(nsteps=5),
    "channel": lambda: I.channel_case(nsteps=4),
    "sphere6": lambda: I.sphere_case(level=6, nsteps=4),
}


def _h(mesh):
    xy = np.asarray(mesh.xy)
    a = 0.5 * np.abs((xy[:, 1, 0] - xy[:, 0, 0]) * (xy[:, 2, 1] - xy[:, 0, 1])
                     - (xy[:, 2, 0] - xy[:, 0, 0]) * (xy[:, 1, 1] - xy[:, 0, 1]))
    return math.sqrt(2.0 * float(np.mean(a)))


def _with_visc(S, case, target=0.2, u_ref=0.05):
    """Coefficients with a viscous number of `target` and a flow part of about half the background
    at the velocity scale u_ref (m/s)."""
    stiff = S.sesw_mesh_check(case.mesh)["visc_stiffness"]
    dt = case.params.tau / case.params.M
    A = target / (dt * stiff)
    Cv = 0.5 * A / (u_ref * _h(case.mesh))
    p = case.params
    case.params = I.Params(g=p.g, theta=p.theta, tau=p.tau, M=p.M, nonlinear_h=p.nonlinear_h, visc=(A, Cv))
    return A, Cv


def _freshwater(case, seed=3, amp=2e-6):
    """Smooth-ish random W (m/s): evaporation and precipitation of a few tenths of a metre per day."""
    rng = np.random.default_rng(seed)
    return amp * (0.3 + rng.standard_normal(case.mesh.nv))


def _envelope_check(ref, r32, got, what, names=("eta", "U", "<<U>>")):
    report = []
    for k, name in enumerate(names):
        scale = max(_maxabs(ref[k]), 1e-30)
        err = _maxabs(got[k] - ref[k])
        env = _maxabs(r32[k] - ref[k])
        tol = ENVELOPE_FACTOR * env + ULP_FLOOR * scale
        report.append(f"{name}: err {err:.3e} env32 {env:.3e} tol {tol:.3e}")
        assert err <= tol, f"{what}: {report[-1]}"
    print(what, "; ".join(report))


def _run(S, case, nsteps, mode=GRAPH, W=None):
    with S.Subcycle() as s:
        s.sesw_set_mode(mode)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        if W is not None:
            s.sesw_set_freshwater(W)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(nsteps)
        info = s.sesw_get_info()
        return s.sesw_get_state(), info


# ---------------------------------------------------------------- the operator


@pytest.mark.parametrize("name", sorted(CASES))
def test_viscosity_operator_matches_oracle(S, name):
    case = CASES[name]()
    A, Cv = _with_visc(S, case)
    m = case.mesh
    rng = np.random.default_rng(11)
    He = m.depth[m.tri].mean(axis=1)
    U = He[:, None] * 0.05 * rng.standard_normal((m.ne, 2))
    eta = 0.5 * rng.standard_normal(m.nv)
    with S.Subcycle() as s:
        s.sesw_set_mode(GRAPH)
        s.sesw_mesh_upload(m)
        s.sesw_set_params(case.params)
        s.sesw_set_state(eta, U)
        got = s.sesw_viscosity()
    nl = case.params.nonlinear_h
    ref = orc.OracleMesh(m).viscosity(U, eta, nl, A, Cv)
    r32 = orc.OracleMesh(m, orc.lib_fp32()).viscosity(U, eta, nl, A, Cv)
    _envelope_check((ref,), (r32,), (got,), f"R_hV {name}", names=("R_hV",))


# ---------------------------------------------------------------- the step


@pytest.mark.parametrize("name", sorted(CASES))
def test_step_with_viscosity_and_freshwater_matches_oracle(S, name):
    case = CASES[name]()
    A, Cv = _with_visc(S, case)
    W = _freshwater(case)
    got, info = _run(S, case, case.nsteps, W=W)
    assert 0.15 < info["visc_number"] < 0.25
    om = orc.OracleMesh(case.mesh)
    ref = om.advance_ext(case.R, case.params, case.nsteps, case.eta0, case.U0, W=W, visc=(A, Cv))
    r32 = orc.OracleMesh(case.mesh, orc.lib_fp32()).advance_ext(case.R, case.params, case.nsteps, case.eta0,
                                                                  case.U0, W=W, visc=(A, Cv))
    _envelope_check(ref, r32, got, f"SE+visc+W {name}")
    # the terms are exercised: without them the result is far outside the tolerance
    plain = om.advance(case.R, case.params, case.nsteps, case.eta0, case.U0)[:3]
    for k in range(3):
        assert _maxabs(plain[k] - ref[k]) > 20 * (ENVELOPE_FACTOR * _maxabs(r32[k] - ref[k])
                                                  + ULP_FLOOR * _maxabs(ref[k]))


@MODES
@pytest.mark.parametrize("name", ["tiny", "channel"])
def test_freshwater_matches_oracle_in_both_modes(S, name, mode):
    case = CASES[name]()
    W = _freshwater(case, seed=4)
    got, info = _run(S, case, case.nsteps, mode=mode, W=W)
    assert info["mode"] == mode
    om = orc.OracleMesh(case.mesh)
    ref = om.advance_ext(case.R, case.params, case.nsteps, case.eta0, case.U0, W=W)
    r32 = orc.OracleMesh(case.mesh, orc.lib_fp32()).advance_ext(case.R, case.params, case.nsteps, case.eta0,
                                                                  case.U0, W=W)
    _envelope_check(ref, r32, got, f"SE+W {name} mode {mode}")


@MODES
@pytest.mark.parametrize("name", ["tiny", "basin"])
def test_sesm_freshwater_matches_oracle(S, name, mode):
    case = CASES[name]()
    p = case.params
    case.params = I.Params(g=p.g, theta=0.14, tau=p.tau, M=p.M, nonlinear_h=p.nonlinear_h, scheme=1)
    coef = closed.sesm_params(0.07)
    W = _freshwater(case, seed=5)
    got, info = _run(S, case, case.nsteps, mode=mode, W=W)
    assert info["mode"] == mode
    ref = orc.OracleMesh(case.mesh).advance_sesm(case.R, case.params, coef, case.nsteps, case.eta0, case.U0, W=W)
    r32 = orc.OracleMesh(case.mesh, orc.lib_fp32()).advance_sesm(case.R, case.params, coef, case.nsteps,
                                                                   case.eta0, case.U0, W=W)
    _envelope_check(ref, r32, got, f"SESM+W {name}")


@MODES
def test_freshwater_volume_and_eq_4_11(S, mode):
    """On a closed basin each step changes the volume by -tau sum A_v W, and
    eta^{n+1} - eta^n = -tau (div <<U>> + W), on the GPU's own outputs."""
    case = I.basin_case(nsteps=1)
    om = orc.OracleMesh(case.mesh)
    av, _ = om.areas()
    W = _freshwater(case, seed=6, amp=1e-5)
    tau = case.params.tau
    with S.Subcycle() as s:
        s.sesw_set_mode(mode)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_freshwater(W)
        s.sesw_set_state(case.eta0, case.U0)
        vol0, _ = s.sesw_diagnostics()
        prev = s.sesw_get_state()[0]
        for n in range(4):
            s.sesw_advance(1)
            eta, U, Um = s.sesw_get_state()
            r = (eta - prev) + tau * (om.divergence(Um) + W)
            assert np.max(np.abs(r)) < 2e-5, n
            prev = eta
        vol, _ = s.sesw_diagnostics()
    want = vol0 - 4 * tau * float(np.sum(av * W))
    scale = float(np.sum(av * np.abs(case.eta0)))
    assert abs(vol - want) <= 1e-5 * scale, (vol, want)


# ---------------------------------------------------------------- rules


def test_setting_and_clearing_the_terms(S):
    """Clearing W (NULL) and turning the viscosity off give back the plain path bit for bit; a
    viscosity with a viscous number above 1 is refused unless the stability check is off."""
    case = CASES["tiny"]()
    plain, _ = _run(S, case, 3)
    A, Cv = _with_visc(S, CASES["tiny"]())
    with S.Subcycle() as s:
        s.sesw_set_mode(GRAPH)
        s.sesw_mesh_upload(case.mesh)
        p0 = case.params
        pv = I.Params(g=p0.g, theta=p0.theta, tau=p0.tau, M=p0.M, nonlinear_h=p0.nonlinear_h, visc=(A, Cv))
        s.sesw_set_params(pv)
        s.sesw_set_forcing(case.R)
        s.sesw_set_freshwater(_freshwater(case))
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(2)
        s.sesw_set_freshwater(None)
        s.sesw_set_params(p0)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(3)
        got = s.sesw_get_state()
        for a, b in zip(plain, got):
            assert np.array_equal(a, b)
        big = I.Params(g=p0.g, theta=p0.theta, tau=p0.tau, M=p0.M, nonlinear_h=p0.nonlinear_h, visc=(20 * A, 0.0))
        with pytest.raises(S.SeswError, match="viscous number"):
            s.sesw_set_params(big)
        s.sesw_set_params(big, flags=1)
        assert s.sesw_get_info()["visc_number"] > 1.0


def test_viscosity_rules(S):
    case = CASES["tiny"]()
    _with_visc(S, case)
    with S.Subcycle() as s:
        s.sesw_set_mode(PERSISTENT)
        s.sesw_mesh_upload(case.mesh)
        with pytest.raises(S.SeswError, match="SESW_MODE_GRAPH"):
            s.sesw_set_params(case.params)
        s.sesw_set_params(I.Params(tau=case.params.tau, M=case.params.M))
        with pytest.raises(S.SeswError, match="SESW_MODE_GRAPH"):
            s.sesw_viscosity()
    with S.Subcycle() as s:
        s.sesw_set_mode(GRAPH)
        s.sesw_mesh_upload(case.mesh)
        p = case.params
        with pytest.raises(S.SeswError, match="SE scheme"):
            s.sesw_set_params(I.Params(tau=p.tau, M=p.M, scheme=1, visc=p.visc))
        with pytest.raises(S.SeswError, match=">= 0"):
            s.sesw_set_params(I.Params(tau=p.tau, M=p.M, visc=(-1.0, 0.0)))
        # zero coefficients: the operator is zero
        s.sesw_set_params(I.Params(tau=p.tau, M=p.M))
        s.sesw_set_state(case.eta0, case.U0)
        assert np.max(np.abs(s.sesw_viscosity())) == 0.0
        s.sesw_set_params(p)
        s.sesw_surrogate_init(1)
        with pytest.raises(S.SeswError, match="freshwater"):
            s.sesw_surrogate_advance(1, 1e30)


def test_batch_basins_bitwise_as_single_uploads(S):
    """A batch with viscosity and W gives every basin exactly what its own upload gives."""
    cases = I.ensemble_cases(nbasins=3, vmin=2000, vmax=6000, nsteps=3, seed=41)
    for c in cases:
        c.U0 = np.random.default_rng(1).standard_normal((c.mesh.ne, 2)) * 20.0
    stiff = max(S.sesw_mesh_check(c.mesh)["visc_stiffness"] for c in cases)
    p0 = cases[0].params
    dts = [c.params.tau / c.params.M for c in cases]
    A = 0.2 / (max(dts) * stiff)
    for c in cases:
        q = c.params
        c.params = I.Params(g=q.g, theta=q.theta, tau=q.tau, M=q.M, nonlinear_h=q.nonlinear_h, visc=(A, 2.0))
    Ws = [_freshwater(c, seed=10 + k) for k, c in enumerate(cases)]
    single = []
    for c, W in zip(cases, Ws):
        single.append(_run(S, c, 3, W=W)[0])
    with S.Subcycle() as s:
        s.sesw_set_mode(GRAPH)
        s.sesw_mesh_upload_batch([c.mesh for c in cases])
        s.sesw_set_params_batch([c.params for c in cases])
        s.sesw_set_forcing(np.concatenate([c.R for c in cases]))
        s.sesw_set_freshwater(np.concatenate(Ws))
        s.sesw_set_state(np.concatenate([c.eta0 for c in cases]), np.concatenate([c.U0 for c in cases]))
        s.sesw_advance(3)
        eta, U, Um = s.sesw_get_state()
    vo = eo = 0
    for c, (se, sU, sUm) in zip(cases, single):
        nv, ne = c.mesh.nv, c.mesh.ne
        assert np.array_equal(eta[vo:vo + nv], se)
        assert np.array_equal(U[eo:eo + ne], sU)
        assert np.array_equal(Um[eo:eo + ne], sUm)
        vo += nv
        eo += ne
