"""The allocation-free diagnostics entry point against the context-based one (GPU).

sesw_diagnostics_noalloc is for callers that cannot allocate device memory where
they need the volume and energy of a state (inside another framework's memory pool,
or in a loop that must stay out of the CUDA allocator): it takes only caller buffers
and keeps its scratch in a fixed device array of the library. This file is named so
that pytest collects it last.

Both entry points sum the same FP64 terms (the context keeps its element areas and rest
depths in FP64 too), only in a different order, so they agree to about 1e-13 relative.
"""
import math

import numpy as np
import pytest

from paper_2311_08241_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REL = 1e-12


def _areas(m):
    """Element areas and median-dual areas in FP64, each vertex's sum in element order."""
    xy = m.xy
    area_e = 0.5 * ((xy[:, 1, 0] - xy[:, 0, 0]) * (xy[:, 2, 1] - xy[:, 0, 1])
                    - (xy[:, 2, 0] - xy[:, 0, 0]) * (xy[:, 1, 1] - xy[:, 0, 1]))
    area_v = np.zeros(m.nv)
    third = area_e / 3.0
    for e in range(m.ne):
        for k in range(3):
            area_v[m.tri[e, k]] += third[e]
    return area_v, area_e


def test_noalloc_diagnostics_match_context_diagnostics_on_two_calls():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2311_08241_gb300 import sesw as S

    case = I.basin_case(nsteps=2)
    m = case.mesh
    dev = torch.device("cuda", 0)
    with S.Subcycle(0) as s:
        s.sesw_mesh_upload(m)
        s.sesw_set_params(case.params)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(case.nsteps)
        vol_ref, en_ref = s.sesw_diagnostics()
        eta = torch.empty(m.nv, dtype=torch.float64, device=dev)
        U = torch.empty((m.ne, 2), dtype=torch.float64, device=dev)
        s.sesw_get_state(eta, U, None)
        torch.cuda.synchronize()

    # the caller's own mesh weights, in FP64
    area_v, area_e = _areas(m)
    eta_h = eta.cpu().numpy()
    h_e = m.depth[m.tri].mean(axis=1) + eta_h[m.tri].mean(axis=1)
    t = {k: torch.tensor(v, device=dev) for k, v in dict(area_v=area_v, area_e=area_e, h_e=h_e).items()}
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    scale_v = float(np.sum(area_v * np.abs(eta_h)))
    for call in range(2):
        out.fill_(float("nan"))
        rc = S.sesw_diagnostics_noalloc(m.nv, m.ne, t["area_v"], eta, t["area_e"], t["h_e"], U,
                                        case.params.g, out, stream)
        assert rc == S.SESW_OK, f"call {call}: status {rc}"
        torch.cuda.synchronize()
        vol, en = out.tolist()
        assert abs(vol - vol_ref) <= REL * scale_v, (call, vol, vol_ref)
        assert abs(en - en_ref) <= REL * abs(en_ref), (call, en, en_ref)

    # sizes beyond the scratch are refused before anything is launched (called through the C-ABI
    # directly: the binding would already refuse buffers shorter than the sizes)
    L = S.load()
    ptrs = [t["area_v"].data_ptr(), eta.data_ptr(), t["area_e"].data_ptr(), t["h_e"].data_ptr(), U.data_ptr()]
    rc = L.sesw_diagnostics_noalloc(S.SESW_NOALLOC_MAX_ITEMS + 1, m.ne, *ptrs, case.params.g, out.data_ptr(), None)
    assert rc == S.SESW_EINVAL
    # so is a gravity that is not positive
    for g in (0.0, -9.81, float("nan")):
        rc = S.sesw_diagnostics_noalloc(m.nv, m.ne, t["area_v"], eta, t["area_e"], t["h_e"], U, g, out, stream)
        assert rc == S.SESW_EINVAL, g
    # the binding refuses buffers the library would misread
    with pytest.raises(TypeError):
        S.sesw_diagnostics_noalloc(m.nv, m.ne, t["area_v"], eta.float(), t["area_e"], t["h_e"], U,
                                   case.params.g, out, stream)
    with pytest.raises(TypeError):
        S.sesw_diagnostics_noalloc(m.nv, m.ne, t["area_v"], eta, t["area_e"], t["h_e"], U.t(),
                                   case.params.g, out, stream)


def test_noalloc_diagnostics_many_chunks():
    """More than 256 chunks of 4096 items (the final kernel's thread stride), two calls in a row,
    against an exactly rounded host sum."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2311_08241_gb300 import sesw as S

    rng = np.random.default_rng(3)
    nv, ne = 1_500_001, 3_000_017          # 367 and 733 chunks
    area_v = rng.uniform(1e6, 3e6, nv)
    eta = rng.normal(0.0, 0.5, nv)
    area_e = rng.uniform(5e5, 1.5e6, ne)
    h_e = rng.uniform(100.0, 5000.0, ne)
    U = rng.normal(0.0, 20.0, (ne, 2))
    g = 9.81
    vol_ref = math.fsum(area_v * eta)
    en_ref = math.fsum(np.concatenate([area_v * 0.5 * g * eta * eta,
                                       area_e * (U[:, 0] ** 2 + U[:, 1] ** 2) / (2.0 * h_e)]))
    dev = torch.device("cuda", 0)
    t = {k: torch.tensor(v, device=dev) for k, v in dict(area_v=area_v, eta=eta, area_e=area_e, h_e=h_e, U=U).items()}
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        out.fill_(float("nan"))
        rc = S.sesw_diagnostics_noalloc(nv, ne, t["area_v"], t["eta"], t["area_e"], t["h_e"], t["U"], g, out, stream)
        assert rc == S.SESW_OK
        torch.cuda.synchronize()
        vol, en = out.tolist()
        assert abs(vol - vol_ref) <= REL * float(np.sum(np.abs(area_v * eta))), (call, vol, vol_ref)
        assert abs(en - en_ref) <= REL * en_ref, (call, en, en_ref)
