"""Learned surrogate on the GPU: forward and gradient against the FP64 numpy reference of the same
network, training, and the physical guarantees of a surrogate step (exact volume, Eq. 4.11, fallback)."""
import numpy as np
import pytest

from oracle import mpnn
from oracle import runner as orc
from paper_2311_08241_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SCALES = [0.3, 3000.0, 5.0, 1e-3, 1e-4, 1e4, 1.0, 0.1]


@pytest.fixture(scope="module")
def S():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2311_08241_gb300 import sesw

    sesw.load()
    return sesw


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def test_forward_and_gradient_match_fp64_reference(S):
    case = I.tiny_jittered_case(nx=10, ny=8, seed=4)
    m = case.mesh
    rng = np.random.default_rng(5)
    eta, U, R = _f32(case.eta0), _f32(case.U0), _f32(case.R)
    dum = _f32(0.5 * rng.standard_normal((m.ne, 2)))
    duM = _f32(0.5 * rng.standard_normal((m.ne, 2)))
    deb = _f32(0.05 * rng.standard_normal(m.nv))
    with S.Subcycle() as s:
        s.sesw_mesh_upload(m)
        s.sesw_set_params(case.params)
        s.sesw_surrogate_init(2, seed=3)
        s.sesw_surrogate_scales(set=SCALES)
        w = (0.3 * rng.standard_normal(s.sesw_surrogate_nparam())).astype(np.float32)
        s.sesw_surrogate_weights(set=w)
        s.sesw_surrogate_set_sample(0, eta, U, R, dum, duM, deb)
        loss, g = s.sesw_surrogate_gradient(0)
        oe, ov = s.sesw_surrogate_predict(0)
    sc = dict(zip(("eta", "H", "U", "R", "f", "L", "out_U", "out_eta"), SCALES))
    G = mpnn.Graph(m)
    xv, xe = mpnn.features(G, eta, U, R, sc)
    wq = mpnn.quantise(w.astype(np.float64))
    te = np.concatenate([dum, duM], axis=1) / sc["out_U"]
    tv = (deb / sc["out_eta"])[:, None]
    # the message layers take BF16 inputs on the tensor cores; the reference rounds the same values
    L_ref, g_ref = mpnn.loss_and_grad(G, wq, xv, xe, te, tv, sc, bf16_msgs=True)
    oe_ref, ov_ref = mpnn.forward(G, wq, xv, xe, sc, bf16_msgs=True)
    print("loss", loss, L_ref, "max|g|", np.abs(g_ref).max(), "max|dg|", np.abs(g - g_ref).max(),
          "max|doe|", np.abs(oe - oe_ref).max(), "max|oe|", np.abs(oe_ref).max())
    # The GPU forms the message inputs in FP32 and the reference in FP64; where a value sits on
    # a bfloat16 rounding boundary the two round it to neighbouring values (2^-8 apart in
    # relative terms), which moves outputs by about 1e-4 of their scale. The bound below is
    # ten times that; a wrong operand layout or accumulation gives errors of order one.
    assert abs(loss - L_ref) <= 1e-3 * abs(L_ref)
    assert np.max(np.abs(oe - oe_ref)) <= 1e-3 * np.max(np.abs(oe_ref)) + 1e-6
    assert np.max(np.abs(ov - ov_ref[:, 0])) <= 1e-3 * np.max(np.abs(ov_ref)) + 1e-6
    assert np.max(np.abs(g - g_ref)) <= 1e-3 * np.max(np.abs(g_ref))
    # most outputs agree to FP32 accumulation order
    assert np.median(np.abs(oe - oe_ref)) <= 1e-5 * np.max(np.abs(oe_ref))


def _record(s, case, nsamples, nsteps_between=1):
    s.sesw_set_eta_mean(True)
    s.sesw_set_forcing(case.R)
    s.sesw_set_state(case.eta0, case.U0)
    for i in range(nsamples):
        s.sesw_surrogate_record_input(i)
        s.sesw_advance(1)
        s.sesw_surrogate_record_target(i)


def test_training_reduces_loss(S):
    case = I.tiny_jittered_case(nx=16, ny=12, seed=7, M=10, tau=100.0)
    with S.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_surrogate_init(8, seed=1)
        _record(s, case, 8)
        s.sesw_surrogate_fit_scales(8, 1e4)
        idx = np.arange(6)
        before = s.sesw_surrogate_loss(idx)
        for _ in range(60):
            s.sesw_surrogate_train(idx, 2e-3)
        after = s.sesw_surrogate_loss(idx)
    print("loss before", before, "after", after)
    assert after < 0.3 * before


def test_surrogate_step_keeps_volume_and_eq_4_11(S):
    """An accepted surrogate step sets eta^{n+1} = eta^n - tau div <<U>>: volume is conserved and
    Eq. 4.11 holds whatever the network predicts."""
    case = I.tiny_jittered_case(nx=16, ny=12, seed=9, M=10, tau=100.0)
    om = orc.OracleMesh(case.mesh)
    av, _ = om.areas()
    with S.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_surrogate_init(1, seed=2)
        s.sesw_surrogate_scales(set=SCALES)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        eta0 = s.sesw_get_state()[0]
        nfb, resid = s.sesw_surrogate_advance(1, 1e30)
        assert nfb == 0 and np.isfinite(resid)
        eta1, U1, Um = s.sesw_get_state()
    assert np.max(np.abs((eta1 - eta0) + case.params.tau * om.divergence(Um))) < 2e-5 * max(1.0, np.max(np.abs(eta0)))
    v0, v1 = float(np.sum(av * eta0)), float(np.sum(av * eta1))
    assert abs(v1 - v0) <= 1e-5 * float(np.sum(av * np.abs(eta0)))


def test_rejected_step_is_the_plain_step(S):
    case = I.tiny_jittered_case(nx=16, ny=12, seed=10, M=10, tau=100.0)
    plain = S.run_case(case, nsteps=2)
    with S.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_surrogate_init(1, seed=2)
        s.sesw_surrogate_scales(set=SCALES)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        nfb, _ = s.sesw_surrogate_advance(2, -1.0)
        got = s.sesw_get_state()
    assert nfb == 2
    for a, b in zip(plain, got):
        assert np.array_equal(a, b)


def test_step_mean_elevation_matches_oracle_and_summed_momentum(S):
    """The plain path's eta_bar (training target) against the oracle, and the exactly summed momentum
    equation that the surrogate's residual check uses, on the GPU outputs (linear H)."""
    case = I.tiny_jittered_case(nx=14, ny=10, seed=12, nonlinear_h=0, M=9, tau=90.0)
    with S.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_eta_mean(True)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(1)
        eta1, U1, Um = s.sesw_get_state()
        eb = s.sesw_get_eta_mean()
    om = orc.OracleMesh(case.mesh)
    *_, eb_ref = om.advance(case.R, case.params, 1, case.eta0, case.U0, want_eta_mean=True)
    assert np.max(np.abs(eb - eb_ref)) < 1e-5
    p = case.params
    Sp = Um - p.theta / p.M * (U1 - case.U0) + (case.U0 - U1) / (2 * p.M)
    cor = np.stack([-Sp[:, 1], Sp[:, 0]], axis=1) * case.mesh.coriolis[:, None]
    H0e = case.mesh.depth[case.mesh.tri].mean(axis=1)[:, None]
    r = U1 - case.U0 + p.tau * (cor + p.g * H0e * om.gradient(eb) - case.R)
    assert np.max(np.abs(r)) < 1e-4 * np.max(np.abs(U1 - case.U0))


def test_trained_surrogate_gains_over_persistence_on_held_out_data(S):
    """What training buys: on held-out trajectories of a small sphere, the trained network's loss is
    well below that of persistence (zero increments, the prediction without the network)."""
    from paper_2311_08241_gb300 import surrogate as SG

    case = I.sphere_case(level=4, nsteps=10)
    forcing = lambda k: SG.sphere_forcing(case, 500 + k)
    ntraj, nst = 10, 10
    with S.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_surrogate_init(ntraj * nst, seed=1)
        SG.generate(s, case.mesh, forcing, ntraj, nst)
        sp = SG.split(ntraj, nst, test_fraction=0.2)
        s.sesw_surrogate_fit_scales(ntraj * nst, 2e5)
        base = SG.persistence_loss(s, sp.test)
        SG.train(s, sp.train, 12, lr=3e-3)
        test = s.sesw_surrogate_loss(sp.test)
    print("held-out loss", test, "persistence", base)
    assert test < 0.5 * base


def test_surrogate_against_plain_and_reduced_M_on_held_out_forcing(S):
    """The three ways to take a baroclinic step, on a held-out forcing of a small sphere after
    training: the surrogate with its fallback, the plain subcycle at M (the reference) and the
    plain subcycle at M/2. Each reports its time per step and its SSH error against the
    reference; the test checks that the numbers are produced and consistent, and states them
    (a surrogate slower or less accurate than halving M is a valid outcome)."""
    from paper_2311_08241_gb300 import surrogate as SG

    case = I.sphere_case(level=4, nsteps=10)
    forcing = lambda k: SG.sphere_forcing(case, 700 + k)
    ntraj, nst = 10, 10
    with S.Subcycle() as s:
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_surrogate_init(ntraj * nst, seed=1)
        SG.generate(s, case.mesh, forcing, ntraj, nst)
        sp = SG.split(ntraj, nst, test_fraction=0.2)
        s.sesw_surrogate_fit_scales(ntraj * nst, 2e5)
        SG.train(s, sp.train, 12, lr=3e-3)
        weights = s.sesw_surrogate_weights()
        scales = s.sesw_surrogate_scales()
    held_out = forcing(ntraj - 1)      # the last trajectory's forcing is in the test split
    M = case.params.M
    roll = SG.rollout_error(case, held_out, case.params, weights, scales, nst, 0.1, coarse_M=(M // 2,))
    gain = SG.gain_summary(roll)
    print("gain over the plain subcycle:", gain)
    for form in ("plain", f"plain_M{M // 2}", "surrogate", "surrogate_no_fallback"):
        assert roll[form]["ms_per_step"] > 0 and np.isfinite(roll[form]["max_ssh_error_m"]), form
    assert roll["plain"]["max_ssh_error_m"] == 0.0
    assert roll[f"plain_M{M // 2}"]["max_ssh_error_m"] > 0.0
    sur = roll["surrogate"]
    assert 0 <= sur["fallback_steps"] <= nst
    if sur["fallback_steps"] == nst:
        # every step rejected: the fallback is the plain step itself, bit for bit
        assert sur["max_ssh_error_m"] == 0.0
    assert set(gain) >= {"surrogate", f"plain_M{M // 2}"}
    for v in gain.values():
        assert v["speedup_vs_plain"] > 0
