"""Bitwise agreement of every execution layout on the GPU.

Each triangle's update is one fixed sequence of FP32 roundings (the same device function in
every kernel), and each vertex adds its triangles' corner fluxes in the order of the caller's
triangle ids, whatever the patch layout. So the graph and persistent modes, every patch size,
every persistent kernel form (registers, streamed with or without the corner-index cache),
every number of blocks per SM and every batch in which a mesh is uploaded must give exactly the
same eta, U and <<U>>. The oracle comparisons of the other GPU tests then hold for all of them
at once.
"""
import numpy as np
import pytest

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


def _run(S, case, nsteps, mode, pv=None, form=None, bps=None, sesm=False):
    with S.Subcycle() as s:
        s.sesw_set_mode(mode)
        if pv:
            s.sesw_set_patch_vertices(pv)
        if form is not None:
            s.sesw_set_persistent_form(form)
        if bps:
            s.sesw_set_blocks_per_sm(bps)
        s.sesw_mesh_upload(case.mesh)
        p = case.params
        if sesm:
            p = I.Params(g=p.g, theta=p.theta, tau=p.tau, M=p.M, nonlinear_h=p.nonlinear_h, scheme=1)
        s.sesw_set_params(p)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(nsteps)
        return s.sesw_get_state(), s.sesw_get_info()


def _same(a, b, what):
    for k, name in enumerate(("eta", "U", "<<U>>")):
        d = np.max(np.abs(a[k] - b[k])) if a[k].size else 0.0
        assert np.array_equal(a[k], b[k]), f"{what}: {name} differs (max |diff| {d:.3e})"


LAYOUTS = [
    ("graph pv=256", dict(mode=GRAPH)),
    ("graph pv=1000", dict(mode=GRAPH, pv=1000)),
    ("persistent auto", dict(mode=PERSISTENT)),
    ("persistent bps=1", dict(mode=PERSISTENT, bps=1)),
    ("persistent bps=4", dict(mode=PERSISTENT, bps=4)),
    ("persistent registers", dict(mode=PERSISTENT, form=1)),
    ("persistent streamed", dict(mode=PERSISTENT, form=2)),
    ("persistent streamed, indices from L2", dict(mode=PERSISTENT, form=3)),
]


@pytest.mark.parametrize("sesm", [False, True], ids=["SE", "SESM"])
def test_channel_every_layout_is_bitwise_the_same(S, sesm):
    """The benchmark channel (200k vertices, 10 steps) in eight layouts, including both streaming
    kernels with and without their corner-index cache on a mesh that also fits the cached form."""
    case = I.channel_case(nsteps=10)
    ref, _ = _run(S, case, 10, sesm=sesm, **LAYOUTS[0][1])
    seen = set()
    for name, kw in LAYOUTS[1:]:
        got, info = _run(S, case, 10, sesm=sesm, **kw)
        if kw["mode"] == PERSISTENT:
            assert info["mode"] == PERSISTENT, (name, info)
            seen.add(info["streamed"])
            if kw.get("form") == 3:
                assert info["streamed"] == 2, (name, info)
        _same(ref, got, f"{'SESM' if sesm else 'SE'} {name}")
    assert seen == {0, 1, 2}, seen


@pytest.mark.parametrize("seed", [1, 2])
def test_ragged_patches_are_bitwise_the_same(S, seed):
    """Small jittered basins cut into many ragged patches (guest copies on every border): patch
    sizes 32, 100 and 777 in graph mode and the persistent layout agree bit for bit, with linear
    and nonlinear H, and with the result against the oracle once."""
    for nl in (1, 0):
        case = I.tiny_jittered_case(nx=23, ny=17, seed=seed, M=9, tau=90.0, nonlinear_h=nl)
        ref, _ = _run(S, case, 4, GRAPH, pv=32)
        _assert_close(case, ref, f"ragged seed={seed} nonlinear={nl}", nsteps=4)
        for pv in (100, 777):
            _same(ref, _run(S, case, 4, GRAPH, pv=pv)[0], f"seed={seed} pv={pv}")
        _same(ref, _run(S, case, 4, PERSISTENT)[0], f"seed={seed} persistent")


def _split(cases, arr, per):
    sizes = [c.mesh.nv if per == "v" else c.mesh.ne for c in cases]
    return np.split(arr, np.cumsum(sizes)[:-1])


def test_persistent_batch_in_packs_is_bitwise_the_single_runs(S):
    """Each basin of a persistent batch that needs several packs (one cooperative launch each, with
    its own patch sizes) equals its own single upload, bit for bit, in both modes."""
    cases = I.ensemble_cases(nbasins=14, scale=0.2, seed=11, nsteps=2)
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
    parts = zip(cases, _split(cases, eta, "v"), _split(cases, U, "e"), _split(cases, Um, "e"))
    for b, (c, e, u, um) in enumerate(parts):
        single, sinfo = _run(S, c, 2, PERSISTENT)
        assert sinfo["mode"] == PERSISTENT
        _same(single, (e, u, um), f"basin {b} persistent")
        if b % 5 == 0:
            _same(_run(S, c, 2, GRAPH)[0], (e, u, um), f"basin {b} graph")


def test_batch_with_large_basins_on_their_own_residency(S):
    """A batch whose large basins (above one grid of 1280-vertex patches) run at two blocks per SM,
    streamed or in registers, next to small basins at one block per SM with cached static data:
    every basin bitwise equals its own single upload."""
    big = I.ensemble_cases(nbasins=2, vmin=2.1e5, vmax=2.4e5, seed=31, nsteps=2)
    small = I.ensemble_cases(nbasins=3, vmin=5e3, vmax=2e4, seed=32, nsteps=2, M=big[0].params.M)
    cases = small + big
    singles = [_run(S, c, 2, PERSISTENT)[0] for c in cases]
    for lform in (S.SESW_FORM_AUTO, S.SESW_FORM_STREAM):
        with S.Subcycle() as s:
            s.sesw_set_mode(PERSISTENT)
            s.sesw_set_blocks_per_sm(1)
            s.sesw_set_large_basins(2, lform)
            s.sesw_mesh_upload_batch([c.mesh for c in cases])
            s.sesw_set_params_batch([c.params for c in cases])
            s.sesw_set_forcing(np.concatenate([c.R for c in cases]))
            s.sesw_set_state(np.concatenate([c.eta0 for c in cases]), np.concatenate([c.U0 for c in cases]))
            s.sesw_advance(2)
            info = s.sesw_get_info()
            eta, U, Um = s.sesw_get_state()
        assert info["mode"] == PERSISTENT and info["npack"] >= 3, info
        parts = zip(cases, singles, _split(cases, eta, "v"), _split(cases, U, "e"), _split(cases, Um, "e"))
        for b, (c, single, e, u, um) in enumerate(parts):
            _same(single, (e, u, um), f"basin {b} large form {lform}")


def test_sphere_register_and_streamed_layouts_are_bitwise_the_same(S):
    """The level-8 sphere in automatic mode runs the register kernel at one block per SM with 7
    slots per thread, its vertices' data and compensation terms in shared memory; the streaming
    kernel at two blocks per SM gives bitwise the same 3 steps."""
    case = I.sphere_case(level=8, nsteps=3)
    got, info = _run(S, case, 3, PERSISTENT)
    assert info["mode"] == PERSISTENT and info["streamed"] == 0 and info["cached"] == 2, info
    assert info["blocks_per_sm"] == 1 and info["slots_per_thread"] == 7, info
    ref, info2 = _run(S, case, 3, PERSISTENT, form=2, bps=2)
    assert info2["streamed"] == 1, info2
    _same(ref, got, "sphere8 registers vs streamed")
