"""Build and call the C oracle (oracle.c) through ctypes.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP, no floating-point contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path):
    """Load a compiled oracle and declare its C signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    L.oracle_mesh_new.restype = P
    L.oracle_mesh_new.argtypes = [I, I, P, P, P, P, ctypes.POINTER(I)]
    L.oracle_mesh_free.restype = None
    L.oracle_mesh_free.argtypes = [P]
    L.oracle_mesh_info.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
    L.oracle_areas.argtypes = [P, P, P]
    L.oracle_edges.argtypes = [P, P, P]
    L.oracle_gradient.argtypes = [P, P, P]
    L.oracle_divergence.argtypes = [P, P, P]
    L.oracle_diagnostics.argtypes = [P, P, P, D, I, ctypes.POINTER(D), ctypes.POINTER(D)]
    L.oracle_advance.argtypes = [P, P, D, D, D, I, I, I, P, P, P, P, P]
    L.oracle_set_threads.argtypes = [I]
    L.oracle_advance_sesm.argtypes = [P, P, D, D, D, D, D, D, I, I, I, P, P, P]
    L.oracle_advance_sesm.restype = I
    L.oracle_advance_sesm_w.argtypes = [P, P, P, D, D, D, D, D, D, I, I, I, P, P, P]
    L.oracle_advance_sesm_w.restype = I
    L.oracle_viscosity.argtypes = [P, P, P, P, I, D, D, P]
    L.oracle_viscosity.restype = I
    L.oracle_advance_ext.argtypes = [P, P, P, P, D, D, D, I, I, D, D, I, P, P, P]
    L.oracle_advance_ext.restype = I
    for f in ("oracle_mesh_info", "oracle_areas", "oracle_edges", "oracle_gradient",
              "oracle_divergence", "oracle_diagnostics", "oracle_advance",
              "oracle_set_threads"):
        getattr(L, f).restype = I
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


_lib32 = None


def lib_fp32():
    """The same oracle source built with float as its working precision. Used only to
    measure how far FP32 arithmetic of the algorithm drifts from FP64."""
    global _lib32
    with _lock:
        if _lib32 is None:
            path = os.path.join(_BUILD, "liboracle_fp32.so")
            if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
                os.makedirs(_BUILD, exist_ok=True)
                tmp = path + f".tmp{os.getpid()}"
                subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                                "-fno-fast-math", "-DORACLE_REAL=float", "-o", tmp, _SRC, "-lm"], check=True)
                os.replace(tmp, path)
            _lib32 = _bind(path)
    return _lib32


def build_variant(source_text: str, tag: str):
    """Compile a modified copy of oracle.c (used only to show that the pins catch
    planted mistakes) and return its bound library."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_BUILD, f"variant_{tag}.c")
    so = os.path.join(_BUILD, f"libvariant_{tag}_{os.getpid()}.so")
    with open(src, "w") as fh:
        fh.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-o", so, src, "-lm"], check=True)
    return _bind(so)


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 keeps it); returns the count in use."""
    return lib().oracle_set_threads(int(n))


class OracleMesh:
    """The oracle's own view of a mesh (edges, median-dual areas, segment normals)."""

    def __init__(self, mesh, L=None):
        L = lib() if L is None else L
        self._L = L
        self.nv = mesh.nv
        self.ne = mesh.ne
        self._tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        self._xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
        self._depth = np.ascontiguousarray(mesh.depth, dtype=np.float64)
        self._f = np.ascontiguousarray(mesh.coriolis, dtype=np.float64)
        st = ctypes.c_int(0)
        h = L.oracle_mesh_new(self.nv, self.ne, _p(self._tri), _p(self._xy), _p(self._depth),
                              _p(self._f), ctypes.byref(st))
        if not h:
            raise ValueError(f"oracle rejected the mesh (status {st.value})")
        self._h = ctypes.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            self._L.oracle_mesh_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        self._L.oracle_mesh_info(self._h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def areas(self):
        av = np.empty(self.nv)
        ae = np.empty(self.ne)
        self._L.oracle_areas(self._h, _p(av), _p(ae))
        return av, ae

    def edges(self):
        ned, _ = self.info()
        ev = np.empty((ned, 2), dtype=np.int32)
        ee = np.empty((ned, 2), dtype=np.int32)
        self._L.oracle_edges(self._h, _p(ev), _p(ee))
        return ev, ee

    def gradient(self, eta):
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        out = np.empty((self.ne, 2))
        self._L.oracle_gradient(self._h, _p(eta), _p(out))
        return out

    def divergence(self, F):
        F = np.ascontiguousarray(F, dtype=np.float64)
        out = np.empty(self.nv)
        rc = self._L.oracle_divergence(self._h, _p(F), _p(out))
        if rc:
            raise MemoryError("oracle_divergence")
        return out

    def diagnostics(self, eta, U, g, nonlinear_h):
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        U = np.ascontiguousarray(U, dtype=np.float64)
        v, e = ctypes.c_double(), ctypes.c_double()
        self._L.oracle_diagnostics(self._h, _p(eta), _p(U), float(g), int(nonlinear_h),
                                 ctypes.byref(v), ctypes.byref(e))
        return v.value, e.value

    def advance(self, R, params, nsteps, eta, U, want_diag=False, want_eta_mean=False):
        """Advance nsteps baroclinic steps. Returns (eta, U, Umean, diag or None) and, with
        want_eta_mean, the step-mean elevation of the last step as a fifth item; inputs untouched."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        eta = np.array(eta, dtype=np.float64, copy=True)
        U = np.array(U, dtype=np.float64, copy=True)
        Umean = np.zeros((self.ne, 2))
        diag = np.zeros((max(nsteps, 1), 2)) if want_diag else None
        emean = np.zeros(self.nv) if want_eta_mean else None
        rc = self._L.oracle_advance(self._h, _p(R), float(params.g), float(params.theta),
                                  float(params.tau), int(params.M), int(params.nonlinear_h),
                                  int(nsteps), _p(eta), _p(U), _p(Umean),
                                  _p(diag) if diag is not None else None,
                                  _p(emean) if emean is not None else None)
        if rc:
            raise RuntimeError(f"oracle_advance failed ({rc})")
        if want_eta_mean:
            return eta, U, Umean, diag, emean
        return eta, U, Umean, diag


    def viscosity(self, U, eta, nonlinear_h, Abg, Cv):
        """R_hV of Eq. (viscosity_BT) per element (element frames), at transport U and elevation eta."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        out = np.zeros((self.ne, 2))
        rc = self._L.oracle_viscosity(self._h, _p(self._xy), _p(U), _p(eta), int(nonlinear_h), float(Abg),
                                      float(Cv), _p(out))
        if rc:
            raise RuntimeError(f"oracle_viscosity failed ({rc})")
        return out

    def advance_ext(self, R, params, nsteps, eta, U, W=None, visc=None):
        """SE steps with the freshwater flux W ([V] m/s, positive out of the ocean) and/or the
        viscous regularisation visc = (A_bg, C_v); either may be None."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        Wc = None if W is None else np.ascontiguousarray(W, dtype=np.float64)
        Abg, Cv = (0.0, 0.0) if visc is None else (float(visc[0]), float(visc[1]))
        eta = np.array(eta, dtype=np.float64, copy=True)
        U = np.array(U, dtype=np.float64, copy=True)
        Umean = np.zeros((self.ne, 2))
        rc = self._L.oracle_advance_ext(self._h, _p(self._xy) if visc is not None else None, _p(R),
                                        _p(Wc) if Wc is not None else None, float(params.g), float(params.theta),
                                        float(params.tau), int(params.M), int(params.nonlinear_h), Abg, Cv,
                                        int(nsteps), _p(eta), _p(U), _p(Umean))
        if rc:
            raise RuntimeError(f"oracle_advance_ext failed ({rc})")
        return eta, U, Umean

    def advance_sesm(self, R, params, coef, nsteps, eta, U, W=None):
        """SESM steps (Eqs. 4.7-4.8); coef = (beta, delta, gamma, zeta); W: optional freshwater
        flux [V]. Returns (eta, U, Umean)."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        eta = np.array(eta, dtype=np.float64, copy=True)
        U = np.array(U, dtype=np.float64, copy=True)
        Umean = np.zeros((self.ne, 2))
        b, d, g, z = (float(x) for x in coef)
        if W is None:
            rc = self._L.oracle_advance_sesm(self._h, _p(R), float(params.g), b, d, g, z, float(params.tau),
                                             int(params.M), int(params.nonlinear_h), int(nsteps), _p(eta), _p(U),
                                             _p(Umean))
        else:
            Wc = np.ascontiguousarray(W, dtype=np.float64)
            rc = self._L.oracle_advance_sesm_w(self._h, _p(R), _p(Wc), float(params.g), b, d, g, z,
                                               float(params.tau), int(params.M), int(params.nonlinear_h),
                                               int(nsteps), _p(eta), _p(U), _p(Umean))
        if rc:
            raise RuntimeError(f"oracle_advance_sesm failed ({rc})")
        return eta, U, Umean


def run_case(case, nsteps=None, want_diag=False, L=None):
    """Convenience: run a ``inputs.Case`` from its initial state."""
    om = OracleMesh(case.mesh, L)
    try:
        return om.advance(case.R, case.params, case.nsteps if nsteps is None else nsteps,
                          case.eta0, case.U0, want_diag=want_diag)
    finally:
        om.close()
