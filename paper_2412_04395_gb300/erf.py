"""Thin Python binding of the C ABI in include/erf.h (argument marshalling only).

Every step of the dycore runs in the CUDA library ``liberf_gb300.so`` built in-tree; there is no
Python or CPU fallback.  PyTorch is used for the device workspace and the CUDA stream only.
Function names are those of the ABI; ``Dycore`` bundles one handle with its workspace.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liberf_gb300.so")

ERF_OK, ERF_EINVAL, ERF_ENOSPACE, ERF_ECUDA, ERF_ENONFINITE, ERF_ESTATE, ERF_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "ERF_OK", -1: "ERF_EINVAL", -2: "ERF_ENOSPACE", -3: "ERF_ECUDA", -4: "ERF_ENONFINITE",
                -5: "ERF_ESTATE", -6: "ERF_EUNSUPPORTED"}
FIELDS = {"rho": 0, "rhotheta": 1, "rhou": 2, "rhov": 3, "rhow": 4,
          "base_rho": 5, "base_p": 6, "base_theta": 7, "rhophi": 8, "rhotke": 9,
          "rhoqv": 10, "rhoqc": 11, "rhoqr": 12, "precip": 13, "base_qv": 14, "p_anelastic": 15}
ERF_F64, ERF_F32 = 0, 1
ERF_OPT_TMA_STENCILS = 1
ERF_OPT_COLUMN_FUSION = 2
ERF_OPT_WARP_COLUMNS = 3

# symbols the library must export (checked by the CPU tests)
EXPORTS = ["erf_workspace_bytes", "erf_init_grid", "erf_set_initial", "erf_set_state", "erf_rk3_step",
           "erf_get_state", "erf_diagnostics", "erf_profile_steps", "erf_last_error", "erf_destroy",
           "erf_reduce_state_noalloc", "erf_train_scratch_bytes", "erf_train_closure", "erf_closure_grad",
           "erf_column_stats", "erf_standardise", "erf_set_closure_weights", "erf_closure_features",
           "erf_closure_fields", "erf_filter_state", "erf_set_tracer_initial", "erf_set_option",
           "erf_get_option", "erf_selftest_wait_timeout", "erf_selftest_tensor_cores",
           "erf_column_block_bytes", "erf_pack_columns", "erf_unpack_columns", "erf_set_initial_moist",
           "erf_capture_reference"]


class ErfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double),
                ("z_faces", C.POINTER(C.c_double)), ("terrain_nodes", C.POINTER(C.c_double)),
                ("terrain_beta", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("dt", C.c_double), ("n_substeps", C.c_int32), ("substep_mode", C.c_int32),
                ("beta_s", C.c_double), ("beta_d", C.c_double),
                ("scal_adv", C.c_int32), ("closure", C.c_int32),
                ("Cs", C.c_double), ("Pr_t", C.c_double), ("nu", C.c_double),
                ("precision", C.c_int32), ("gravity", C.c_double),
                ("f_cor", C.c_double), ("u_g", C.c_double), ("v_g", C.c_double),
                ("surface", C.c_int32), ("z0", C.c_double), ("sfc_theta_flux", C.c_double),
                ("theta_s", C.c_double), ("brunt_N", C.c_double), ("p_s", C.c_double),
                ("n_knots", C.c_int32), ("knot_z", C.POINTER(C.c_double)),
                ("knot_theta", C.POINTER(C.c_double)), ("tracer", C.c_int32), ("mom_adv", C.c_int32),
                ("ray_tau", C.c_double), ("ray_zd", C.c_double), ("ray_fields", C.c_int32),
                ("moist", C.c_int32), ("n_qknots", C.c_int32), ("qknot_z", C.POINTER(C.c_double)),
                ("qknot_v", C.POINTER(C.c_double)), ("relax_tau", C.c_double), ("relax_width", C.c_double),
                ("anelastic", C.c_int32)]


class Diag(C.Structure):
    _fields_ = [("mass", C.c_double), ("max_abs_w", C.c_double), ("theta_min", C.c_double),
                ("theta_max", C.c_double), ("cfl_acoustic", C.c_double), ("nonfinite", C.c_int32),
                ("steps_done", C.c_int64), ("kernels_per_step", C.c_int32)]


class TrainCfg(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float)]


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("total_ms", C.c_double), ("launches", C.c_int32)]


_LIB = None


def load_library(path: str = LIB_PATH):
    """Loads the in-tree CUDA library; raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    vp = C.c_void_p
    L.erf_workspace_bytes.argtypes = [C.POINTER(GridDesc), C.POINTER(Config), C.POINTER(C.c_size_t)]
    L.erf_init_grid.argtypes = [C.POINTER(GridDesc), C.POINTER(Config), vp, C.c_size_t, vp, C.POINTER(vp)]
    L.erf_set_initial.argtypes = [vp, vp, vp, vp, vp, C.c_int32]
    L.erf_set_tracer_initial.argtypes = [vp, vp, C.c_int32]
    L.erf_set_option.argtypes = [vp, C.c_int32, C.c_int64]
    L.erf_selftest_wait_timeout.argtypes = [C.c_int32, vp, vp, C.POINTER(C.c_int32)]
    L.erf_selftest_tensor_cores.argtypes = [vp, vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.erf_get_option.argtypes = [vp, C.c_int32, C.POINTER(C.c_int64)]
    L.erf_set_state.argtypes = [vp, C.c_int32, vp, C.c_int32, C.c_int32]
    L.erf_rk3_step.argtypes = [vp, C.c_int32]
    L.erf_get_state.argtypes = [vp, C.c_int32, vp, C.c_int32, C.c_int32]
    L.erf_diagnostics.argtypes = [vp, C.POINTER(Diag)]
    L.erf_profile_steps.argtypes = [vp, C.c_int32, C.POINTER(KernelTime), C.c_int32, C.POINTER(C.c_int32)]
    L.erf_train_scratch_bytes.argtypes = [C.c_int32]
    L.erf_train_scratch_bytes.restype = C.c_size_t
    L.erf_train_closure.argtypes = [C.POINTER(TrainCfg), vp, vp, C.c_int64, vp, vp, vp, C.c_size_t, vp]
    L.erf_closure_grad.argtypes = [vp, vp, C.c_int32, vp, vp, vp, vp, C.c_size_t, vp]
    L.erf_column_stats.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, vp]
    L.erf_standardise.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, vp, vp]
    L.erf_set_closure_weights.argtypes = [vp, C.c_char_p, C.c_size_t]
    L.erf_closure_features.argtypes = [vp, vp]
    L.erf_closure_fields.argtypes = [vp, vp, C.POINTER(C.c_uint32)]
    L.erf_filter_state.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp, vp]
    L.erf_set_initial_moist.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int32]
    L.erf_capture_reference.argtypes = [vp]
    L.erf_column_block_bytes.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]
    L.erf_pack_columns.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp]
    L.erf_unpack_columns.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp]
    L.erf_last_error.argtypes = [vp]
    L.erf_last_error.restype = C.c_char_p
    L.erf_destroy.argtypes = [vp]
    for name in ("erf_workspace_bytes", "erf_init_grid", "erf_set_initial", "erf_set_state", "erf_rk3_step",
                 "erf_get_state", "erf_diagnostics", "erf_profile_steps", "erf_train_closure", "erf_closure_grad",
                 "erf_column_stats", "erf_standardise", "erf_set_closure_weights", "erf_closure_features",
                 "erf_closure_fields", "erf_filter_state", "erf_set_tracer_initial", "erf_set_option",
                 "erf_get_option", "erf_selftest_wait_timeout", "erf_selftest_tensor_cores",
                 "erf_column_block_bytes", "erf_pack_columns", "erf_unpack_columns", "erf_set_initial_moist",
                 "erf_capture_reference"):
        getattr(L, name).restype = C.c_int
    _LIB = L
    return L


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class _Keep:
    """Host buffers referenced by the C structs stay alive while the structs are used."""

    def __init__(self):
        self.bufs = []

    def __call__(self, a):
        a = _f64(a)
        if a is not None:
            self.bufs.append(a)
        return a


def make_structs(wl):
    """GridDesc + Config for a workload (see workloads.Workload)."""
    keep = _Keep()
    zeta = keep(wl.zeta)
    ter = keep(wl.terrain) if wl.terrain is not None else None
    g = GridDesc(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, _dp(zeta), _dp(ter), wl.terrain_beta)
    kz = kt = None
    nk = 0
    if wl.knots is not None:
        kz, kt = keep(wl.knots[0]), keep(wl.knots[1])
        nk = len(kz)
    qz = qk = None
    nq = 0
    if getattr(wl, "qv_knots", None) is not None:
        qz, qk = keep(wl.qv_knots[0]), keep(wl.qv_knots[1])
        nq = len(qz)
    c = Config(dt=wl.dt, n_substeps=wl.n_substeps, substep_mode=getattr(wl, "substep_mode", 0),
               beta_s=wl.beta_s, beta_d=wl.beta_d, scal_adv=wl.scal_adv, closure=wl.closure, Cs=wl.Cs,
               Pr_t=wl.Pr_t, nu=wl.nu, precision=wl.precision, gravity=wl.gravity, f_cor=wl.f_cor,
               u_g=wl.u_g, v_g=wl.v_g, surface=wl.surface, z0=wl.z0, sfc_theta_flux=wl.sfc_theta_flux,
               theta_s=wl.theta_s, brunt_N=wl.brunt_N, p_s=wl.p_s, n_knots=nk, knot_z=_dp(kz),
               knot_theta=_dp(kt), tracer=getattr(wl, "tracer", 0), mom_adv=wl.mom_adv,
               ray_tau=wl.ray_tau, ray_zd=wl.ray_zd, ray_fields=wl.ray_fields, moist=wl.moist, n_qknots=nq,
               qknot_z=_dp(qz), qknot_v=_dp(qk), relax_tau=wl.relax_tau, relax_width=wl.relax_width,
               anelastic=getattr(wl, "anelastic", 0))
    return g, c, keep


def _check(L, h, status):
    if status != ERF_OK:
        msg = L.erf_last_error(h)
        raise ErfError(status, msg.decode() if msg else "")


def erf_workspace_bytes(grid, cfg) -> int:
    L = load_library()
    n = C.c_size_t()
    _check(L, None, L.erf_workspace_bytes(C.byref(grid), C.byref(cfg), C.byref(n)))
    return n.value


def erf_init_grid(grid, cfg, workspace_ptr: int, nbytes: int, stream_ptr: int):
    L = load_library()
    h = C.c_void_p()
    _check(L, None, L.erf_init_grid(C.byref(grid), C.byref(cfg), C.c_void_p(workspace_ptr), nbytes,
                                    C.c_void_p(stream_ptr), C.byref(h)))
    return h


class Dycore:
    """One handle of the CUDA dycore with its torch-owned device workspace.

    ``wl`` is a workloads.Workload; the stream is torch's current CUDA stream at construction.
    """

    def __init__(self, wl, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the GB300 dycore needs a CUDA device; there is no CPU path")
        self.L = load_library()
        self.wl = wl
        self.device = torch.device(device or "cuda")
        self.grid, self.cfg, self._keep = make_structs(wl)
        nbytes = erf_workspace_bytes(self.grid, self.cfg)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        ptr = self.workspace.data_ptr()
        ptr = (ptr + 255) & ~255
        self.stream = torch.cuda.current_stream(self.device)
        self.h = erf_init_grid(self.grid, self.cfg, ptr, nbytes, self.stream.cuda_stream)
        self.shape_c = (wl.nz, wl.ny, wl.nx)
        self.shape_w = (wl.nz + 1, wl.ny, wl.nx)
        self.terrain = wl.terrain is not None and bool(np.any(np.asarray(wl.terrain) != 0.0))

    def close(self):
        if getattr(self, "h", None):
            self.L.erf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self, name):
        if name == "rhow":
            return self.shape_w
        if name == "precip":
            return (self.wl.ny, self.wl.nx)
        if name.startswith("base_") and not self.terrain:
            return (self.wl.nz,)
        return self.shape_c

    # -- ABI calls
    def erf_set_initial(self, dtheta=None, u=None, v=None, w=None):
        arrs = [_f64(a) for a in (dtheta, u, v, w)]
        ptrs = [None if a is None else a.ctypes.data for a in arrs]
        _check(self.L, self.h, self.L.erf_set_initial(self.h, *ptrs, 0))

    def erf_set_initial_moist(self, dtheta=None, qv=None, u=None, v=None, w=None):
        arrs = [_f64(a) for a in (dtheta, qv, u, v, w)]
        ptrs = [None if a is None else a.ctypes.data for a in arrs]
        _check(self.L, self.h, self.L.erf_set_initial_moist(self.h, *ptrs, 0))

    def erf_capture_reference(self):
        _check(self.L, self.h, self.L.erf_capture_reference(self.h))

    def erf_set_initial_device(self, dtheta=None, u=None, v=None, w=None):
        ptrs = [None if t is None else t.data_ptr() for t in (dtheta, u, v, w)]
        _check(self.L, self.h, self.L.erf_set_initial(self.h, *ptrs, 1))

    def erf_set_option(self, option, value):
        _check(self.L, self.h, self.L.erf_set_option(self.h, int(option), int(value)))

    def erf_get_option(self, option):
        v = C.c_int64()
        _check(self.L, self.h, self.L.erf_get_option(self.h, int(option), C.byref(v)))
        return v.value

    def erf_set_tracer_initial(self, phi):
        a = _f64(phi)
        assert a.shape == self.shape_c
        _check(self.L, self.h, self.L.erf_set_tracer_initial(self.h, a.ctypes.data, 0))

    def erf_set_state(self, name, arr):
        import torch
        if isinstance(arr, torch.Tensor):
            assert arr.is_cuda and arr.is_contiguous() and tuple(arr.shape) == self._shape(name)
            dt = ERF_F64 if arr.dtype == torch.float64 else ERF_F32
            _check(self.L, self.h, self.L.erf_set_state(self.h, FIELDS[name], arr.data_ptr(), 1, dt))
        else:
            a = np.ascontiguousarray(arr)
            assert a.shape == self._shape(name)
            dt = ERF_F64 if a.dtype == np.float64 else ERF_F32
            if dt == ERF_F32:
                a = a.astype(np.float32, copy=False)
            _check(self.L, self.h, self.L.erf_set_state(self.h, FIELDS[name], a.ctypes.data, 0, dt))

    def erf_rk3_step(self, nsteps=1):
        _check(self.L, self.h, self.L.erf_rk3_step(self.h, int(nsteps)))

    def erf_get_state(self, name, out=None, dtype=np.float64):
        import torch
        if out is not None and isinstance(out, torch.Tensor):
            dt = ERF_F64 if out.dtype == torch.float64 else ERF_F32
            _check(self.L, self.h, self.L.erf_get_state(self.h, FIELDS[name], out.data_ptr(), 1, dt))
            return out
        a = out if out is not None else np.empty(self._shape(name), dtype=dtype)
        dt = ERF_F64 if a.dtype == np.float64 else ERF_F32
        _check(self.L, self.h, self.L.erf_get_state(self.h, FIELDS[name], a.ctypes.data, 0, dt))
        return a

    def erf_diagnostics(self):
        d = Diag()
        st = self.L.erf_diagnostics(self.h, C.byref(d))
        out = {f: getattr(d, f) for f, _ in Diag._fields_}
        out["status"] = st
        return out

    def erf_profile_steps(self, nsteps=1):
        """Per-kernel device time of nsteps directly launched, event-bracketed steps."""
        buf = (KernelTime * 64)()
        n = C.c_int32()
        _check(self.L, self.h, self.L.erf_profile_steps(self.h, int(nsteps), buf, 64, C.byref(n)))
        return {buf[i].name.decode(): (buf[i].total_ms, buf[i].launches) for i in range(n.value)}

    def state(self):
        out = {k: self.erf_get_state(k) for k in ("rho", "rhotheta", "rhou", "rhov", "rhow")}
        if getattr(self.wl, "moist", 0):
            out.update({k: self.erf_get_state(k) for k in ("rhoqv", "rhoqc", "rhoqr")})
        return out

    # -- x-y pencil decomposition: column blocks of the prognostic state (device buffers)
    def erf_column_block_bytes(self, ni, nj):
        n = C.c_size_t()
        _check(self.L, self.h, self.L.erf_column_block_bytes(self.h, int(ni), int(nj), C.byref(n)))
        return n.value

    def empty(self, ni, nj):
        """A device buffer for one column block (the path's storage type)."""
        import torch
        dt = torch.float32 if self.wl.precision == 1 else torch.float64
        n = self.erf_column_block_bytes(ni, nj) // (4 if dt == torch.float32 else 8)
        return torch.empty(n, dtype=dt, device=self.device)

    def pack(self, i0, ni, j0, nj, out=None):
        buf = self.empty(ni, nj) if out is None else out
        _check(self.L, self.h, self.L.erf_pack_columns(self.h, int(i0), int(ni), int(j0), int(nj), buf.data_ptr()))
        return buf

    def unpack(self, i0, ni, j0, nj, buf):
        assert buf.is_cuda and buf.is_contiguous()
        assert buf.numel() * buf.element_size() >= self.erf_column_block_bytes(ni, nj)
        _check(self.L, self.h, self.L.erf_unpack_columns(self.h, int(i0), int(ni), int(j0), int(nj), buf.data_ptr()))

    # -- learned closure
    def erf_set_closure_weights(self, blob: bytes):
        _check(self.L, self.h, self.L.erf_set_closure_weights(self.h, blob, len(blob)))

    def erf_closure_features(self):
        import torch
        out = torch.empty((self.wl.ncell, 12), dtype=torch.float32, device=self.device)
        _check(self.L, self.h, self.L.erf_closure_features(self.h, out.data_ptr()))
        return out

    def erf_closure_fields(self):
        import torch
        out = torch.empty((9,) + self.shape_c, dtype=torch.float32, device=self.device)
        nfb = C.c_uint32()
        _check(self.L, self.h, self.L.erf_closure_fields(self.h, out.data_ptr(), C.byref(nfb)))
        return out, nfb.value

    def erf_filter_state(self, r=4):
        """Coarse FP64 C-grid state (dict of torch tensors) and SGS targets [Nc, 9]."""
        import torch
        nz, ny, nx = self.shape_c
        Nz, Ny, Nx = nz // r, ny // r, nx // r
        dev = self.device
        f = {k: torch.empty((Nz, Ny, Nx), dtype=torch.float64, device=dev) for k in ("rho", "rhotheta", "rhou", "rhov")}
        f["rhow"] = torch.empty((Nz + 1, Ny, Nx), dtype=torch.float64, device=dev)
        T = torch.empty((Nz * Ny * Nx, 9), dtype=torch.float32, device=dev)
        _check(self.L, self.h, self.L.erf_filter_state(self.h, r, f["rho"].data_ptr(), f["rhotheta"].data_ptr(),
                                                       f["rhou"].data_ptr(), f["rhov"].data_ptr(),
                                                       f["rhow"].data_ptr(), T.data_ptr()))
        return f, T


def erf_selftest_wait_timeout(max_polls=1000):
    """1 if a bounded device-side wait on an mbarrier that never completes gives up and reports it."""
    import torch
    L = load_library()
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = C.c_int32()
    _check(L, None, L.erf_selftest_wait_timeout(int(max_polls), C.c_void_p(flag.data_ptr()),
                                                C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(out)))
    return out.value


def erf_selftest_tensor_cores():
    """(mismatching outputs, timed out) of the tcgen05 self-test: MMAs of the closure network's
    operand shapes on exact integer data, checked against integer loops on the device."""
    import torch
    L = load_library()
    words = torch.zeros(2, dtype=torch.int32, device="cuda")
    bad, to = C.c_int32(), C.c_int32()
    _check(L, None, L.erf_selftest_tensor_cores(C.c_void_p(words.data_ptr()),
                                                C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                                C.byref(bad), C.byref(to)))
    return bad.value, to.value


# ---------------------------------------------------------------- learned closure (training)
def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def erf_train_scratch_bytes(batch: int) -> int:
    return load_library().erf_train_scratch_bytes(int(batch))


def erf_closure_grad(X, T, params, stream=None):
    """Loss and gradient of one batch (torch CUDA float32 tensors X [n,12], T [n,9], params [9737])."""
    import torch
    L = load_library()
    n = X.shape[0]
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    nb = erf_train_scratch_bytes(n)
    scratch = torch.empty(nb, dtype=torch.uint8, device=params.device)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(L, None, L.erf_closure_grad(_ptr(X), _ptr(T), n, _ptr(params), _ptr(grad), _ptr(loss),
                                       _ptr(scratch), nb, C.c_void_p(st)))
    return loss, grad


def erf_train_closure(X, T, params, epochs, batch, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """Adam training in place on params; returns the per-batch losses (torch CUDA tensor)."""
    import torch
    L = load_library()
    n = X.shape[0]
    steps = epochs * ((n + batch - 1) // batch)
    losses = torch.empty(max(steps, 1), dtype=torch.float32, device=params.device)
    nb = erf_train_scratch_bytes(batch)
    scratch = torch.empty(nb, dtype=torch.uint8, device=params.device)
    cfg = TrainCfg(epochs, batch, lr, beta1, beta2, eps)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(L, None, L.erf_train_closure(C.byref(cfg), _ptr(X), _ptr(T), n, _ptr(params), _ptr(losses),
                                        _ptr(scratch), nb, C.c_void_p(st)))
    return losses[:steps]


def erf_column_stats(A, stream=None):
    import torch
    L = load_library()
    mean = torch.empty(A.shape[1], dtype=torch.float32, device=A.device)
    sd = torch.empty_like(mean)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(L, None, L.erf_column_stats(_ptr(A), A.shape[0], A.shape[1], _ptr(mean), _ptr(sd), C.c_void_p(st)))
    return mean, sd


def erf_standardise(A, mean, sd, stream=None):
    import torch
    L = load_library()
    out = torch.empty_like(A)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(L, None, L.erf_standardise(_ptr(A), A.shape[0], A.shape[1], _ptr(mean), _ptr(sd), _ptr(out),
                                      C.c_void_p(st)))
    return out
