"""The allocation-free diagnostics entry point against the context-based one (GPU).

sesw_diagnostics_noalloc is for callers that cannot allocate device memory where
they need the volume and energy of a state (inside another framework's memory pool,
or in a loop that must stay out of the CUDA allocator): it takes only caller buffers
and keeps its scratch in a fixed device array of the library. This file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2311_08241_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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
    xy = m.xy
    area_e = 0.5 * ((xy[:, 1, 0] - xy[:, 0, 0]) * (xy[:, 2, 1] - xy[:, 0, 1])
                    - (xy[:, 2, 0] - xy[:, 0, 0]) * (xy[:, 1, 1] - xy[:, 0, 1]))
    area_v = np.zeros(m.nv)
    for k in range(3):
        np.add.at(area_v, m.tri[:, k], area_e / 3.0)
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
        # the tolerance of the context diagnostics test: 1e-6 relative on volume, 1e-5 on energy
        assert abs(vol - vol_ref) <= 1e-6 * max(abs(vol_ref), scale_v) + 1e-3, (call, vol, vol_ref)
        assert abs(en - en_ref) <= 1e-5 * abs(en_ref), (call, en, en_ref)

    # sizes beyond the scratch are refused before anything is launched
    rc = S.sesw_diagnostics_noalloc(S.SESW_NOALLOC_MAX_ITEMS + 1, m.ne, t["area_v"], eta, t["area_e"],
                                    t["h_e"], U, case.params.g, out, stream)
    assert rc == S.SESW_EINVAL
