"""Python binding of libsesw (include/sesw.h) through ctypes.

The functions below carry the C names and only marshal arguments: every step of
the barotropic subcycle runs in the library's CUDA kernels. PyTorch supplies the
device memory (its caching allocator, through the library's allocator callback)
and the stream. There is no CPU fallback: if the library cannot be loaded, or no
CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SESW_OK = 0
SESW_EINVAL = -1
SESW_ECUDA = -2
SESW_ESTATE = -3
SESW_ETIMEOUT = -4
SESW_EUNSTABLE = -5
SESW_ENOMEM = -6
SESW_HOST = 0
SESW_DEVICE = 1
SESW_FLAG_NO_STABILITY_CHECK = 1
SESW_FLAG_TEST_FORCE_TIMEOUT = 2
SESW_PRECISION_FP32 = 0
SESW_MODE_AUTO = 0
SESW_MODE_GRAPH = 1
SESW_MODE_PERSISTENT = 2
SESW_FORM_AUTO = 0
SESW_FORM_REGISTERS = 1
SESW_FORM_STREAM = 2
SESW_FORM_STREAM_UNCACHED = 3

_NAMES = {0: "SESW_OK", -1: "SESW_EINVAL", -2: "SESW_ECUDA", -3: "SESW_ESTATE", -4: "SESW_ETIMEOUT",
          -5: "SESW_EUNSTABLE", -6: "SESW_ENOMEM"}

# every symbol include/sesw.h declares
EXPORTS = ("sesw_create", "sesw_set_stream", "sesw_set_mode", "sesw_set_persistent_form", "sesw_set_large_basins",
           "sesw_set_blocks_per_sm",
           "sesw_set_patch_vertices",
           "sesw_set_block_threads",
           "sesw_mesh_upload", "sesw_mesh_upload_batch", "sesw_set_params_batch", "sesw_diagnostics_batch",
           "sesw_set_params", "sesw_set_state", "sesw_set_forcing", "sesw_set_freshwater", "sesw_viscosity",
           "sesw_set_forcing_async", "sesw_get_state_async", "sesw_wait",
           "sesw_advance", "sesw_get_state",
           "sesw_diagnostics", "sesw_diagnostics_noalloc", "sesw_set_eta_mean", "sesw_get_eta_mean", "sesw_status", "sesw_mesh_check",
           "sesw_get_info", "sesw_last_error", "sesw_destroy",
           "sesw_surrogate_init", "sesw_surrogate_nparam", "sesw_surrogate_weights", "sesw_surrogate_scales",
           "sesw_surrogate_set_sample", "sesw_surrogate_record_input", "sesw_surrogate_record_target",
           "sesw_surrogate_fit_scales", "sesw_surrogate_train", "sesw_surrogate_loss", "sesw_surrogate_gradient",
           "sesw_surrogate_predict", "sesw_surrogate_advance")
SESW_NOALLOC_MAX_CHUNKS = 8192
SESW_NOALLOC_MAX_ITEMS = SESW_NOALLOC_MAX_CHUNKS * 4096


class SeswError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class sesw_mesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("ne", ctypes.c_int32), ("tri", ctypes.c_void_p),
                ("xy", ctypes.c_void_p), ("pos", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("coriolis", ctypes.c_void_p), ("ned", ctypes.c_int32), ("edge_v", ctypes.c_void_p),
                ("edge_e", ctypes.c_void_p), ("area_v", ctypes.c_void_p), ("area_e", ctypes.c_void_p)]


class sesw_params(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("theta", ctypes.c_double), ("tau", ctypes.c_double),
                ("M", ctypes.c_int32), ("nonlinear_h", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("eta_bound", ctypes.c_double), ("sesm_beta", ctypes.c_double),
                ("sesm_delta", ctypes.c_double), ("sesm_gamma", ctypes.c_double), ("sesm_zeta", ctypes.c_double),
                ("visc_background", ctypes.c_double), ("visc_flow", ctypes.c_double),
                ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class sesw_info(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("ne", ctypes.c_int32), ("npatch", ctypes.c_int32),
                ("nslot", ctypes.c_int32), ("max_patch_slots", ctypes.c_int32),
                ("patch_vertices", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("slots_per_thread", ctypes.c_int32),
                ("cached", ctypes.c_int32), ("nbasin", ctypes.c_int32), ("courant_max", ctypes.c_double),
                ("courant_limit", ctypes.c_double), ("stiffness_bound", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("npack", ctypes.c_int32), ("streamed", ctypes.c_int32),
                ("visc_number", ctypes.c_double), ("visc_stiffness", ctypes.c_double),
                ("step_graph", ctypes.c_int32), ("launches", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsesw.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libsesw not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.sesw_create.argtypes = [ctypes.POINTER(P), I, P, ALLOC_FN, FREE_FN, P]
        L.sesw_set_stream.argtypes = [P, P]
        L.sesw_set_patch_vertices.argtypes = [P, ctypes.c_int32]
        L.sesw_set_block_threads.argtypes = [P, ctypes.c_int32]
        L.sesw_set_mode.argtypes = [P, ctypes.c_int32]
        L.sesw_set_blocks_per_sm.argtypes = [P, ctypes.c_int32]
        L.sesw_set_persistent_form.argtypes = [P, ctypes.c_int32]
        L.sesw_set_large_basins.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
        L.sesw_mesh_upload.argtypes = [P, ctypes.POINTER(sesw_mesh)]
        L.sesw_set_params.argtypes = [P, ctypes.POINTER(sesw_params)]
        L.sesw_mesh_upload_batch.argtypes = [P, ctypes.c_int32, ctypes.POINTER(sesw_mesh)]
        L.sesw_set_params_batch.argtypes = [P, ctypes.c_int32, ctypes.POINTER(sesw_params)]
        L.sesw_diagnostics_batch.argtypes = [P, P, P]
        L.sesw_set_state.argtypes = [P, P, P, I]
        L.sesw_set_forcing.argtypes = [P, P, I]
        L.sesw_set_freshwater.argtypes = [P, P, I]
        L.sesw_set_forcing_async.argtypes = [P, P]
        L.sesw_get_state_async.argtypes = [P, P, P, P, ctypes.POINTER(ctypes.c_uint64)]
        L.sesw_wait.argtypes = [P, ctypes.c_uint64]
        L.sesw_viscosity.argtypes = [P, P, I]
        L.sesw_advance.argtypes = [P, ctypes.c_int32]
        L.sesw_get_state.argtypes = [P, P, P, P, I]
        L.sesw_diagnostics.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(D)]
        L.sesw_status.argtypes = [P]
        L.sesw_set_eta_mean.argtypes = [P, ctypes.c_int32]
        L.sesw_get_eta_mean.argtypes = [P, P, I]
        L.sesw_diagnostics_noalloc.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, D, P, P]
        L.sesw_get_info.argtypes = [P, ctypes.POINTER(sesw_info)]
        L.sesw_mesh_check.argtypes = [ctypes.POINTER(sesw_mesh), ctypes.c_int32, ctypes.POINTER(sesw_info),
                                      ctypes.c_char_p, ctypes.c_size_t]
        I64 = ctypes.c_int64
        L.sesw_surrogate_init.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
        L.sesw_surrogate_nparam.argtypes = [P, ctypes.POINTER(I64)]
        L.sesw_surrogate_weights.argtypes = [P, P, P]
        L.sesw_surrogate_scales.argtypes = [P, P, P]
        L.sesw_surrogate_set_sample.argtypes = [P, I64, P, P, P, P, P, P, I]
        L.sesw_surrogate_record_input.argtypes = [P, I64]
        L.sesw_surrogate_record_target.argtypes = [P, I64]
        L.sesw_surrogate_fit_scales.argtypes = [P, I64, D]
        L.sesw_surrogate_train.argtypes = [P, P, ctypes.c_int32, D, ctypes.POINTER(D)]
        L.sesw_surrogate_loss.argtypes = [P, P, ctypes.c_int32, ctypes.POINTER(D)]
        L.sesw_surrogate_gradient.argtypes = [P, I64, P, ctypes.POINTER(D)]
        L.sesw_surrogate_predict.argtypes = [P, I64, P, P]
        L.sesw_surrogate_advance.argtypes = [P, ctypes.c_int32, D, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(D)]
        L.sesw_last_error.argtypes = [P]
        L.sesw_last_error.restype = ctypes.c_char_p
        L.sesw_destroy.argtypes = [P]
        L.sesw_destroy.restype = None
        for n in EXPORTS:
            if n not in ("sesw_last_error", "sesw_destroy"):
                getattr(L, n).restype = I
        _lib = L
        return L


def _ptr(x):
    """Address of a numpy array (host) or a torch tensor (device or host)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(x.data_ptr())


def _where(x):
    if x is None or isinstance(x, np.ndarray):
        return SESW_HOST
    return SESW_DEVICE if x.is_cuda else SESW_HOST


class Subcycle:
    """One libsesw context: a mesh, parameters, forcing and state on one GPU.

    Methods map one to one onto the C calls (sesw_mesh_upload, sesw_set_params, ...).
    Host arrays are numpy float64 (int32 for indices); device arrays are torch
    float64 CUDA tensors, passed by address.
    """

    def __init__(self, device: int = 0, stream=None, use_torch_allocator: bool = True):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libsesw needs a CUDA device; none is available")
        self._L = load()
        self.device = device
        self._stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._alloc_cb = ALLOC_FN(0)
        self._free_cb = FREE_FN(0)
        if use_torch_allocator:
            dev, strm = device, self._stream

            def _alloc(nbytes, _user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm)
                except Exception:
                    return None

            def _free(ptr, _user):
                try:
                    torch.cuda.caching_allocator_delete(ptr)
                except Exception:
                    pass

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
        h = ctypes.c_void_p()
        rc = self._L.sesw_create(ctypes.byref(h), device, ctypes.c_void_p(self._stream.cuda_stream),
                                 self._alloc_cb, self._free_cb, None)
        if rc != SESW_OK:
            raise SeswError(rc, "sesw_create failed")
        self._h = h
        self.nv = self.ne = 0
        self.params = None

    # -- helpers
    def _check(self, rc):
        if rc != SESW_OK:
            raise SeswError(rc, self._L.sesw_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._L.sesw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- the C calls
    def sesw_set_patch_vertices(self, n: int):
        return self._check(self._L.sesw_set_patch_vertices(self._h, int(n)))

    def sesw_set_mode(self, mode: int):
        return self._check(self._L.sesw_set_mode(self._h, int(mode)))

    def sesw_set_blocks_per_sm(self, k: int):
        return self._check(self._L.sesw_set_blocks_per_sm(self._h, int(k)))

    def sesw_set_persistent_form(self, form: int):
        return self._check(self._L.sesw_set_persistent_form(self._h, int(form)))

    def sesw_set_large_basins(self, blocks_per_sm: int = 0, form: int = -1):
        return self._check(self._L.sesw_set_large_basins(self._h, int(blocks_per_sm), int(form)))

    def sesw_set_block_threads(self, n: int):
        return self._check(self._L.sesw_set_block_threads(self._h, int(n)))

    def sesw_mesh_upload(self, mesh, edges=None, areas=None):
        m, keep = _mesh_struct(mesh, edges, areas)
        rc = self._check(self._L.sesw_mesh_upload(self._h, ctypes.byref(m)))
        del keep
        self.nv, self.ne = int(mesh.nv), int(mesh.ne)
        return rc

    def sesw_set_params(self, p, flags: int = 0, eta_bound: float = 0.0):
        cp = _params_struct(p, flags, eta_bound)
        self.params = p
        return self._check(self._L.sesw_set_params(self._h, ctypes.byref(cp)))

    def sesw_mesh_upload_batch(self, meshes):
        structs, keeps = zip(*[_mesh_struct(m) for m in meshes])
        arr = (sesw_mesh * len(structs))(*structs)
        rc = self._check(self._L.sesw_mesh_upload_batch(self._h, len(structs), arr))
        del keeps
        self.nv = sum(int(m.nv) for m in meshes)
        self.ne = sum(int(m.ne) for m in meshes)
        self.nbasin = len(structs)
        return rc

    def sesw_set_params_batch(self, params, flags: int = 0, eta_bound: float = 0.0):
        arr = (sesw_params * len(params))(*[_params_struct(p, flags, eta_bound) for p in params])
        self.params = params[0]
        return self._check(self._L.sesw_set_params_batch(self._h, len(params), arr))

    def sesw_diagnostics_batch(self):
        n = self.sesw_get_info()["nbasin"]
        vol = np.empty(n)
        en = np.empty(n)
        self._check(self._L.sesw_diagnostics_batch(self._h, _ptr(vol), _ptr(en)))
        return vol, en

    def sesw_set_state(self, eta, U):
        eta = _as_f64(eta)
        U = _as_f64(U)
        return self._check(self._L.sesw_set_state(self._h, _ptr(eta), _ptr(U), _where(eta if eta is not None else U)))

    def sesw_set_forcing(self, R):
        R = _as_f64(R)
        return self._check(self._L.sesw_set_forcing(self._h, _ptr(R), _where(R)))

    def sesw_set_forcing_async(self, R):
        """Forcing from a host buffer (pinned for overlap); keep R unchanged until a later ticket's wait."""
        R = _as_f64(R)
        if _where(R) != SESW_HOST:
            raise ValueError("sesw_set_forcing_async takes a host buffer")
        return self._check(self._L.sesw_set_forcing_async(self._h, _ptr(R)))

    def sesw_get_state_async(self, eta=None, U=None, Umean=None):
        """Start reading the state into host buffers; returns the ticket for sesw_wait."""
        for x in (eta, U, Umean):
            if x is not None and _where(x) != SESW_HOST:
                raise ValueError("sesw_get_state_async fills host buffers")
        t = ctypes.c_uint64()
        self._check(self._L.sesw_get_state_async(self._h, _ptr(eta), _ptr(U), _ptr(Umean), ctypes.byref(t)))
        return t.value

    def sesw_wait(self, ticket: int = 0):
        return self._check(self._L.sesw_wait(self._h, int(ticket)))

    def sesw_set_freshwater(self, W):
        """Freshwater flux [nv] (m/s, positive out of the ocean); None removes it."""
        W = _as_f64(W)
        where = SESW_HOST if W is None else _where(W)
        return self._check(self._L.sesw_set_freshwater(self._h, _ptr(W), where))

    def sesw_viscosity(self, out=None):
        """The barotropic viscous regularisation at the current state, [ne][2] in caller order."""
        if out is None:
            out = np.empty((self.ne, 2))
        self._check(self._L.sesw_viscosity(self._h, _ptr(out), _where(out)))
        return out

    def sesw_advance(self, nsteps: int):
        return self._check(self._L.sesw_advance(self._h, int(nsteps)))

    def sesw_get_state(self, eta=None, U=None, Umean=None):
        """Fill the given buffers (numpy or torch float64); with no buffers, return new numpy arrays."""
        if eta is None and U is None and Umean is None:
            eta = np.empty(self.nv)
            U = np.empty((self.ne, 2))
            Umean = np.empty((self.ne, 2))
        where = _where(next(x for x in (eta, U, Umean) if x is not None))
        self._check(self._L.sesw_get_state(self._h, _ptr(eta), _ptr(U), _ptr(Umean), where))
        return eta, U, Umean

    def sesw_set_eta_mean(self, enable: bool = True):
        return self._check(self._L.sesw_set_eta_mean(self._h, int(bool(enable))))

    def sesw_get_eta_mean(self, out=None):
        if out is None:
            out = np.empty(self.nv)
        self._check(self._L.sesw_get_eta_mean(self._h, _ptr(out), _where(out)))
        return out

    # -- surrogate
    def sesw_surrogate_init(self, capacity: int, seed: int = 0):
        return self._check(self._L.sesw_surrogate_init(self._h, int(capacity), int(seed)))

    def sesw_surrogate_nparam(self):
        n = ctypes.c_int64()
        self._check(self._L.sesw_surrogate_nparam(self._h, ctypes.byref(n)))
        return n.value

    def sesw_surrogate_weights(self, set=None):
        w = np.empty(self.sesw_surrogate_nparam(), dtype=np.float32)
        s = None if set is None else np.ascontiguousarray(set, dtype=np.float32)
        self._check(self._L.sesw_surrogate_weights(self._h, _ptr(w), _ptr(s)))
        return w

    def sesw_surrogate_scales(self, set=None):
        g = np.empty(8)
        s = None if set is None else np.ascontiguousarray(set, dtype=np.float64)
        self._check(self._L.sesw_surrogate_scales(self._h, _ptr(g), _ptr(s)))
        return g

    def sesw_surrogate_set_sample(self, index, eta, U, R, d_umean, d_um, d_etabar):
        arrs = [_as_f64(x) for x in (eta, U, R, d_umean, d_um, d_etabar)]
        return self._check(self._L.sesw_surrogate_set_sample(self._h, int(index), *[_ptr(a) for a in arrs],
                                                             _where(arrs[0])))

    def sesw_surrogate_record_input(self, index):
        return self._check(self._L.sesw_surrogate_record_input(self._h, int(index)))

    def sesw_surrogate_record_target(self, index):
        return self._check(self._L.sesw_surrogate_record_target(self._h, int(index)))

    def sesw_surrogate_fit_scales(self, nsamples, length_scale):
        return self._check(self._L.sesw_surrogate_fit_scales(self._h, int(nsamples), float(length_scale)))

    def sesw_surrogate_train(self, indices, learning_rate):
        idx = np.ascontiguousarray(indices, dtype=np.int64)
        loss = ctypes.c_double()
        self._check(self._L.sesw_surrogate_train(self._h, _ptr(idx), len(idx), float(learning_rate),
                                                 ctypes.byref(loss)))
        return loss.value

    def sesw_surrogate_loss(self, indices):
        idx = np.ascontiguousarray(indices, dtype=np.int64)
        loss = ctypes.c_double()
        self._check(self._L.sesw_surrogate_loss(self._h, _ptr(idx), len(idx), ctypes.byref(loss)))
        return loss.value

    def sesw_surrogate_gradient(self, index):
        g = np.empty(self.sesw_surrogate_nparam(), dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self._L.sesw_surrogate_gradient(self._h, int(index), _ptr(g), ctypes.byref(loss)))
        return loss.value, g

    def sesw_surrogate_predict(self, index):
        oe = np.empty((self.ne, 4))
        ov = np.empty(self.nv)
        self._check(self._L.sesw_surrogate_predict(self._h, int(index), _ptr(oe), _ptr(ov)))
        return oe, ov

    def sesw_surrogate_advance(self, nsteps, resid_tol):
        nf = ctypes.c_int32()
        r = ctypes.c_double()
        self._check(self._L.sesw_surrogate_advance(self._h, int(nsteps), float(resid_tol), ctypes.byref(nf),
                                                   ctypes.byref(r)))
        return nf.value, r.value

    def sesw_diagnostics(self):
        v, e = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.sesw_diagnostics(self._h, ctypes.byref(v), ctypes.byref(e)))
        return v.value, e.value

    def sesw_status(self):
        return self._L.sesw_status(self._h)

    def sesw_get_info(self):
        info = sesw_info()
        self._check(self._L.sesw_get_info(self._h, ctypes.byref(info)))
        return {k: getattr(info, k) for k, _ in sesw_info._fields_}


def _params_struct(p, flags=0, eta_bound=0.0):
    coef = getattr(p, "sesm", None) or (0.0, 0.0, 0.0, 0.0)
    visc = getattr(p, "visc", None) or (0.0, 0.0)
    return sesw_params(float(p.g), float(p.theta), float(p.tau), int(p.M), int(p.nonlinear_h),
                       int(getattr(p, "scheme", 0)), int(flags), float(eta_bound), *(float(x) for x in coef),
                       *(float(x) for x in visc), int(getattr(p, "precision", SESW_PRECISION_FP32)), 0)


def _mesh_struct(mesh, edges=None, areas=None):
    """The C mesh description; edges = (edge_v [ned][2], edge_e [ned][2]) and areas = (area_v, area_e)
    are the optional caller tables (None: the library derives them)."""
    def opt(x, dt):
        return None if x is None else np.ascontiguousarray(x, dtype=dt)

    ev, ee = edges if edges is not None else (None, None)
    av, ae = areas if areas is not None else (None, None)
    keep = [np.ascontiguousarray(mesh.tri, dtype=np.int32),
            np.ascontiguousarray(mesh.xy, dtype=np.float64),
            None if mesh.pos is None else np.ascontiguousarray(mesh.pos, dtype=np.float64),
            np.ascontiguousarray(mesh.depth, dtype=np.float64),
            np.ascontiguousarray(mesh.coriolis, dtype=np.float64),
            opt(ev, np.int32), opt(ee, np.int32), opt(av, np.float64), opt(ae, np.float64)]
    t, xy, pos, d, f, kv, ke, kav, kae = keep
    ned = 0 if kv is None else int(kv.shape[0])
    m = sesw_mesh(int(mesh.nv), int(t.shape[0]), _ptr(t), _ptr(xy), _ptr(pos), _ptr(d), _ptr(f), ned, _ptr(kv),
                  _ptr(ke), _ptr(kav), _ptr(kae))
    return m, keep


def sesw_mesh_check(mesh, patch_vertices: int = 512, edges=None, areas=None):
    """Host-only validation and layout of a mesh (no GPU needed). Returns the layout facts."""
    L = load()
    m, keep = _mesh_struct(mesh, edges, areas)
    info = sesw_info()
    buf = ctypes.create_string_buffer(512)
    rc = L.sesw_mesh_check(ctypes.byref(m), int(patch_vertices), ctypes.byref(info), buf, 512)
    del keep
    if rc != SESW_OK:
        raise SeswError(rc, buf.value.decode())
    return {k: getattr(info, k) for k, _ in sesw_info._fields_}


def sesw_diagnostics_noalloc(nv, ne, area_v, eta, area_e, h_e, U, g, out, stream=None):
    """Allocation-free volume/energy of caller-held device arrays (torch float64 CUDA
    tensors); writes out[0:2] on the stream and returns the status code."""
    import torch

    L = load()
    dev = torch.cuda.current_device()
    need = {"area_v": (area_v, int(nv)), "eta": (eta, int(nv)), "area_e": (area_e, int(ne)),
            "h_e": (h_e, int(ne)), "U": (U, 2 * int(ne)), "out": (out, 2)}
    for name, (t, n) in need.items():
        if not (isinstance(t, torch.Tensor) and t.dtype == torch.float64 and t.is_contiguous()
                and t.is_cuda and t.device.index == dev and t.numel() >= n):
            raise TypeError(f"{name} must be a contiguous torch.float64 tensor on cuda:{dev} "
                            f"with at least {n} elements")
    sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    return L.sesw_diagnostics_noalloc(int(nv), int(ne), _ptr(area_v), _ptr(eta), _ptr(area_e), _ptr(h_e),
                                      _ptr(U), float(g), _ptr(out), sp)


def _as_f64(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return np.ascontiguousarray(x, dtype=np.float64)
    import torch

    if x.dtype != torch.float64 or not x.is_contiguous():
        raise TypeError("device buffers must be contiguous torch.float64 tensors")
    return x


def run_case(case, nsteps=None, device=0, patch_vertices=None, mode=None, form=None, blocks_per_sm=None):
    """Upload a case, advance it and return (eta, U, Umean) as numpy arrays."""
    with Subcycle(device) as s:
        if mode is not None:
            s.sesw_set_mode(mode)
        if form is not None:
            s.sesw_set_persistent_form(form)
        if blocks_per_sm is not None:
            s.sesw_set_blocks_per_sm(blocks_per_sm)
        if patch_vertices:
            s.sesw_set_patch_vertices(patch_vertices)
        s.sesw_mesh_upload(case.mesh)
        s.sesw_set_params(case.params)
        s.sesw_set_forcing(case.R)
        s.sesw_set_state(case.eta0, case.U0)
        s.sesw_advance(case.nsteps if nsteps is None else nsteps)
        return s.sesw_get_state()
