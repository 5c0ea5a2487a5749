"""Shared parity helpers of the GPU tests (see tests/test_gpu_parity.py for the tolerance rule)."""
import numpy as np
import pytest

from oracle import runner as orc

ETA_ABS_TOL = 1e-5
ENVELOPE_FACTOR = 2.0
ULP_FLOOR = 8 * 2.0 ** -24
GRAPH, PERSISTENT = 1, 2          # SESW_MODE_GRAPH, SESW_MODE_PERSISTENT
MODES = pytest.mark.parametrize("mode", [GRAPH, PERSISTENT], ids=["graph", "persistent"])


def _maxabs(x):
    return float(np.max(np.abs(x))) if np.size(x) else 0.0


def _assert_close(case, got, what, nsteps=None):
    """GPU result vs the FP64 oracle, within twice the FP32 oracle's drift (see module docstring)."""
    ref = orc.run_case(case, nsteps=nsteps)
    r32 = orc.run_case(case, nsteps=nsteps, L=orc.lib_fp32())
    names = ("eta", "U", "<<U>>")
    report = []
    for k, name in enumerate(names):
        scale = max(_maxabs(ref[k]), 1e-30)
        err = _maxabs(got[k] - ref[k])
        env = _maxabs(r32[k] - ref[k])
        tol = ENVELOPE_FACTOR * env + ULP_FLOOR * scale
        report.append(f"{name}: err {err:.3e} env32 {env:.3e} tol {tol:.3e} (scale {scale:.3e})")
        assert err <= tol, f"{what}: {report[-1]}"
    print(f"{what}: " + "; ".join(report))
    assert _maxabs(got[0] - ref[0]) <= ETA_ABS_TOL, f"{what}: eta above the absolute target"
    return ref
