"""Batched ensembles (one upload, one advance for many basins of uneven size) on the GPU."""
import numpy as np
import pytest

from oracle import runner as orc
from paper_2311_08241_gb300 import inputs as I
from parity_util import GRAPH, PERSISTENT, _assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2311_08241_gb300 import sesw

    sesw.load()
    return sesw


def _ensemble(n=6, scale=0.02, seed=20231118):
    return I.ensemble_cases(nbasins=n, scale=scale, seed=seed, nsteps=3)


def _run_batch(S, cases, mode, nsteps, patch_vertices=None, large_form=None):
    with S.Subcycle() as s:
        s.sesw_set_mode(mode)
        if patch_vertices:
            s.sesw_set_patch_vertices(patch_vertices)
        if large_form is not None:
            s.sesw_set_large_basins(0, large_form)
        s.sesw_mesh_upload_batch([c.mesh for c in cases])
        s.sesw_set_params_batch([c.params for c in cases])
        s.sesw_set_forcing(np.concatenate([c.R for c in cases]))
        s.sesw_set_state(np.concatenate([c.eta0 for c in cases]), np.concatenate([c.U0 for c in cases]))
        s.sesw_advance(nsteps)
        info = s.sesw_get_info()
        out = s.sesw_get_state()
        diag = s.sesw_diagnostics_batch()
    return out, info, diag


def _split(cases, arr, per):
    sizes = [c.mesh.nv if per == "v" else c.mesh.ne for c in cases]
    return np.split(arr, np.cumsum(sizes)[:-1])


def test_batch_graph_is_bitwise_the_single_runs(S):
    """Each basin of a graph-mode batch equals its own upload with the same patch size, bit for bit."""
    cases = _ensemble()
    assert len({c.params.tau for c in cases}) > 1          # basins differ in dt
    (eta, U, Um), info, _ = _run_batch(S, cases, GRAPH, 3, patch_vertices=128)
    assert info["nbasin"] == len(cases)
    for c, e, u, um in zip(cases, _split(cases, eta, "v"), _split(cases, U, "e"), _split(cases, Um, "e")):
        single = S.run_case(c, nsteps=3, patch_vertices=128, mode=GRAPH)
        assert np.array_equal(single[0], e) and np.array_equal(single[1], u) and np.array_equal(single[2], um)


@pytest.mark.parametrize("mode", [GRAPH, PERSISTENT], ids=["graph", "persistent"])
def test_batch_matches_oracle_per_basin(S, mode):
    cases = _ensemble(n=5, seed=7)
    (eta, U, Um), info, (vol, en) = _run_batch(S, cases, mode, 3)
    if mode == PERSISTENT:
        assert info["mode"] == PERSISTENT
    for c, e, u, um, v, en_b in zip(cases, _split(cases, eta, "v"), _split(cases, U, "e"), _split(cases, Um, "e"),
                                   vol, en):
        _assert_close(c, (e, u, um), f"{c.name} mode={mode}", nsteps=3)
        om = orc.OracleMesh(c.mesh)
        v_ref, e_ref = om.diagnostics(e, u, c.params.g, c.params.nonlinear_h)
        av, _ = om.areas()
        assert abs(v - v_ref) <= 1e-6 * float(np.sum(av * np.abs(e))) + 1e-3
        assert abs(en_b - e_ref) <= 1e-5 * abs(e_ref)
        # each basin conserves its own volume (FP32 state, FP64 sums)
        v0 = float(np.sum(av * c.eta0))
        assert abs(v - v0) <= 1e-5 * float(np.sum(av * np.abs(c.eta0)))


def test_batch_persistent_packs(S):
    """More patches than resident blocks: the batch runs as several cooperative launches per step."""
    cases = I.ensemble_cases(nbasins=14, scale=0.2, seed=11, nsteps=2)   # ~276k vertices: two packs
    (eta, U, Um), info, _ = _run_batch(S, cases, PERSISTENT, 2)
    assert info["mode"] == PERSISTENT and info["npack"] > 1, info
    for c, e, u, um in zip(cases, _split(cases, eta, "v"), _split(cases, U, "e"), _split(cases, Um, "e")):
        _assert_close(c, (e, u, um), f"{c.name} packs={info['npack']}", nsteps=2)


def test_batch_parameter_rules(S):
    cases = _ensemble(n=3)
    with S.Subcycle() as s:
        s.sesw_mesh_upload_batch([c.mesh for c in cases])
        bad = [c.params for c in cases]
        bad[1] = I.Params(g=bad[1].g, theta=bad[1].theta, tau=bad[1].tau, M=bad[1].M + 1)
        with pytest.raises(S.SeswError, match="differ only in tau"):
            s.sesw_set_params_batch(bad)
        with pytest.raises(S.SeswError, match="one parameter set per"):
            s.sesw_set_params_batch([c.params for c in cases[:2]])
        unstable = [c.params for c in cases]
        p = unstable[2]
        unstable[2] = I.Params(g=p.g, theta=p.theta, tau=p.tau * 8, M=p.M)
        with pytest.raises(S.SeswError, match="basin 2"):
            s.sesw_set_params_batch(unstable)


@pytest.fixture(scope="module")
def full_ensemble():
    """The batched configuration at full size (64 basins, log-uniform 2e4-4e5 vertices, 8.6 M in
    total; the benchmark's seed) with its FP64 and FP32 oracle results after 3 steps."""
    cases = I.ensemble_cases(nbasins=64, scale=1.0, seed=20231118, nsteps=3)
    ref = [orc.run_case(c, nsteps=3) for c in cases]
    r32 = [orc.run_case(c, nsteps=3, L=orc.lib_fp32()) for c in cases]
    return cases, ref, r32


@pytest.mark.parametrize("bps", [1, 2, 3, 4])
def test_full_size_ensemble_matches_oracle(S, full_ensemble, bps):
    """Every basin of the full-size ensemble, advanced as one batch in persistent packs (the layouts
    the benchmark's autotuner chooses among), against the oracle: within twice the FP32 oracle's
    drift plus 8 ulp, and |eta error| <= 1e-5 m."""
    from parity_util import ENVELOPE_FACTOR, ETA_ABS_TOL, ULP_FLOOR, _maxabs

    cases, ref, r32 = full_ensemble
    with S.Subcycle() as s:
        s.sesw_set_mode(PERSISTENT)
        s.sesw_set_blocks_per_sm(bps)
        s.sesw_mesh_upload_batch([c.mesh for c in cases])
        s.sesw_set_params_batch([c.params for c in cases])
        s.sesw_set_forcing(np.concatenate([c.R for c in cases]))
        s.sesw_set_state(np.concatenate([c.eta0 for c in cases]), np.concatenate([c.U0 for c in cases]))
        s.sesw_advance(3)
        info = s.sesw_get_info()
        eta, U, Um = s.sesw_get_state()
    assert info["mode"] == PERSISTENT and info["nbasin"] == 64 and info["npack"] > 1, info
    worst = 0.0
    for b, (c, e, u, um) in enumerate(zip(cases, _split(cases, eta, "v"), _split(cases, U, "e"),
                                          _split(cases, Um, "e"))):
        for k, got in enumerate((e, u, um)):
            err = _maxabs(got - ref[b][k])
            tol = ENVELOPE_FACTOR * _maxabs(r32[b][k] - ref[b][k]) + ULP_FLOOR * _maxabs(ref[b][k])
            assert err <= tol, f"basin {b} ({c.mesh.nv} vertices) field {k}: {err:.3e} > {tol:.3e}"
        worst = max(worst, _maxabs(e - ref[b][0]))
    assert worst <= ETA_ABS_TOL


def test_batch_mixes_streamed_and_cached_packs(S):
    """One step launching different kernels per pack: the level-8 sphere (a large basin whose pack
    streams its state from L2) batched with small basins (cached packs). Every basin against the
    oracle."""
    sphere = I.sphere_case(level=8, nsteps=2)
    small = I.ensemble_cases(nbasins=3, vmin=5000, vmax=20000, M=sphere.params.M, nsteps=2, seed=5)
    cases = small + [sphere]
    (eta, U, Um), info, _ = _run_batch(S, cases, PERSISTENT, 2, large_form=S.SESW_FORM_STREAM)
    assert info["mode"] == PERSISTENT and info["npack"] >= 2, info
    assert info["streamed"] == 0 and info["cached"] == 1, info     # the first pack: the small basins
    for c, e, u, um in zip(cases, _split(cases, eta, "v"), _split(cases, U, "e"), _split(cases, Um, "e")):
        _assert_close(c, (e, u, um), f"{c.name} in a mixed batch", nsteps=2)
