"""ctypes wrapper of the FP64 C oracle (``erf_oracle.c``).

Test infrastructure only.  Configuration fields, their meaning and the readings they encode are
documented in ``erf_oracle.c``; this module only marshals arguments.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "erf_oracle.c")


def lib_path() -> str:
    return os.path.join(_HERE, "liberf_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, OpenMP for the pointwise passes)."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


class _Cfg(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double),
        ("terrain_beta", C.c_int32),
        ("dt", C.c_double),
        ("n_substeps", C.c_int32), ("substep_mode", C.c_int32), ("acoustic_off", C.c_int32),
        ("beta_s", C.c_double), ("beta_d", C.c_double),
        ("mom_adv", C.c_int32), ("scal_adv", C.c_int32), ("closure", C.c_int32),
        ("Cs", C.c_double), ("Pr_t", C.c_double), ("nu", C.c_double),
        ("gravity", C.c_double),
        ("f_cor", C.c_double), ("u_g", C.c_double), ("v_g", C.c_double),
        ("surface", C.c_int32), ("z0", C.c_double), ("sfc_theta_flux", C.c_double),
        ("theta_s", C.c_double), ("brunt_N", C.c_double), ("p_s", C.c_double),
        ("tracer", C.c_int32),
        ("ray_tau", C.c_double), ("ray_zd", C.c_double), ("ray_fields", C.c_int32),
        ("moist", C.c_int32), ("relax_tau", C.c_double), ("relax_width", C.c_double),
        ("anelastic", C.c_int32),
    ]


@dataclass
class OracleConfig:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    terrain_beta: int = 1
    dt: float = 0.25
    n_substeps: int = 6
    substep_mode: int = 0
    acoustic_off: int = 0
    beta_s: float = 0.1
    beta_d: float = 0.1
    mom_adv: int = 5
    scal_adv: int = 0
    closure: int = 0
    Cs: float = 0.17
    Pr_t: float = 1.0 / 3.0
    nu: float = 0.0
    gravity: float = 9.81
    f_cor: float = 0.0
    u_g: float = 0.0
    v_g: float = 0.0
    surface: int = 0
    z0: float = 0.1
    sfc_theta_flux: float = 0.0
    theta_s: float = 300.0
    brunt_N: float = 0.0
    p_s: float = 1.0e5
    tracer: int = 0
    ray_tau: float = 0.0
    ray_zd: float = 0.0
    ray_fields: int = 0
    moist: int = 0
    relax_tau: float = 0.0
    relax_width: float = 0.0
    anelastic: int = 0


_LIB = None
# model of the learned closure: (user, rho, rho theta, rho u, rho v, rho w, planes out)
_SGS_FN = C.CFUNCTYPE(None, C.c_void_p, *([C.POINTER(C.c_double)] * 6))


def _lib():
    global _LIB
    if _LIB is None:
        path = build_oracle()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Cfg), dp, dp, C.c_int, dp, dp]
        L.orc_create2.restype = C.c_void_p
        L.orc_create2.argtypes = [C.POINTER(_Cfg), dp, dp, C.c_int, dp, dp, C.c_int, dp, dp]
        L.orc_set_initial_q.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        L.orc_capture_reference.argtypes = [C.c_void_p]
        L.orc_get_precip.argtypes = [C.c_void_p, dp]
        L.orc_kessler.argtypes = [C.c_void_p]
        L.orc_qvs.restype = C.c_double
        L.orc_qvs.argtypes = [C.c_double, C.c_double]
        L.orc_rain_speed.restype = C.c_double
        L.orc_rain_speed.argtypes = [C.c_double] * 3
        L.orc_rain_evap.restype = C.c_double
        L.orc_rain_evap.argtypes = [C.c_double] * 5
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_initial.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.orc_get_field.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_set_field.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_set_tracer_initial.argtypes = [C.c_void_p, dp]
        L.orc_get_geom.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_slow_rhs.argtypes = [C.c_void_p] + [dp] * 8
        L.orc_get_mu.argtypes = [C.c_void_p, dp]
        L.orc_get_aux.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_set_sgs_model.argtypes = [C.c_void_p, _SGS_FN, C.c_void_p]
        L.orc_substep_once.argtypes = [C.c_void_p, C.c_double] + [dp] * 10
        L.orc_mass.restype = C.c_double
        L.orc_mass.argtypes = [C.c_void_p]
        L.orc_interp.restype = C.c_double
        L.orc_interp.argtypes = [dp, C.c_double, C.c_int]
        L.orc_weno5.restype = C.c_double
        L.orc_weno5.argtypes = [dp, C.c_double, C.c_int]
        L.orc_eos.argtypes = [C.c_double, dp, dp]
        L.orc_thomas.argtypes = [C.c_int, dp, dp, dp, dp, dp]
        L.orc_hse_column.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double, C.c_double, dp, dp]
        L.orc_ustar.restype = C.c_double
        L.orc_ustar.argtypes = [C.c_double] * 6
        L.orc_psi_m.restype = C.c_double
        L.orc_psi_m.argtypes = [C.c_double]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        L.orc_sizeof_cfg.restype = C.c_int
        assert L.orc_sizeof_cfg() == C.sizeof(_Cfg), "oracle config struct layout mismatch"
        _LIB = L
    return _LIB


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


FIELDS = {"rho": 0, "rhotheta": 1, "rhou": 2, "rhov": 3, "rhow": 4,
          "base_rho": 5, "base_p": 6, "base_theta": 7, "rhophi": 8, "rhotke": 9,
          "rhoqv": 10, "rhoqc": 11, "rhoqr": 12, "base_qv": 13, "p_anelastic": 14}
GEOM = {"zc": 0, "Hc": 1, "Hx": 2, "Hy": 3, "hxi_x": 4, "heta_y": 5,
        "zw": 6, "hxi_w": 7, "heta_w": 8, "zn": 9}


class Oracle:
    """One grid + configuration of the oracle; fields are numpy arrays [k][j][i]."""

    def __init__(self, cfg: OracleConfig, zeta, terrain=None, knots=None, qv_knots=None):
        L = _lib()
        self.cfg = cfg
        c = _Cfg(**{f.name: getattr(cfg, f.name) for f in fields(cfg)})
        self._zeta = _f64(zeta)
        assert self._zeta.shape == (cfg.nz + 1,)
        self._ter = _f64(terrain)
        if self._ter is not None:
            assert self._ter.shape == (cfg.ny, cfg.nx)
        kz = kt = None
        nk = 0
        if knots is not None:
            kz = _f64(knots[0]); kt = _f64(knots[1]); nk = len(kz)
        self._kz, self._kt = kz, kt
        qz = qv = None
        nq = 0
        if qv_knots is not None:
            qz = _f64(qv_knots[0]); qv = _f64(qv_knots[1]); nq = len(qz)
        self._qz, self._qv = qz, qv
        self._h = L.orc_create2(C.byref(c), _p(self._zeta), _p(self._ter), nk, _p(kz), _p(kt), nq, _p(qz), _p(qv))
        self.shape_c = (cfg.nz, cfg.ny, cfg.nx)
        self.shape_w = (cfg.nz + 1, cfg.ny, cfg.nx)

    def close(self):
        if self._h:
            _lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self, f):
        return self.shape_w if f == "rhow" else self.shape_c

    def set_initial(self, dtheta=None, u=None, v=None, w=None, qv=None):
        """Initial state at unchanged pressure; moist configurations take the water vapour q_v
        at cells (None: the base state's)."""
        a = [_f64(x) for x in (dtheta, qv, u, v, w)]
        _lib().orc_set_initial_q(self._h, *[_p(x) for x in a])

    def capture_reference(self):
        """The current state becomes the reference of the lateral relaxation zones."""
        _lib().orc_capture_reference(self._h)

    def precip(self):
        out = np.empty((self.cfg.ny, self.cfg.nx))
        _lib().orc_get_precip(self._h, _p(out))
        return out

    def kessler(self):
        """One Kessler microphysics step on the current state (test hook)."""
        _lib().orc_kessler(self._h)

    def set_tracer_initial(self, phi):
        """rho phi = rho phi0 with the current rho (configuration with tracer = 1)."""
        a = _f64(phi)
        assert a.shape == self.shape_c
        _lib().orc_set_tracer_initial(self._h, _p(a))

    def get(self, name):
        out = np.empty(self._shape(name), dtype=np.float64)
        rc = _lib().orc_get_field(self._h, FIELDS[name], _p(out))
        assert rc == 0
        return out

    def set(self, name, arr):
        a = _f64(arr)
        assert a.shape == self._shape(name)
        rc = _lib().orc_set_field(self._h, FIELDS[name], _p(a))
        assert rc == 0

    def geom(self, name):
        shp = self.shape_c if GEOM[name] < 6 else self.shape_w
        out = np.empty(shp, dtype=np.float64)
        _lib().orc_get_geom(self._h, GEOM[name], _p(out))
        return out

    def set_sgs_model(self, model):
        """Model of the learned closure (configuration closure = 3): model(rho, rho theta, rho u,
        rho v, rho w) -> array [9][nz][ny][nx] of the density-weighted cell-centre stresses
        rho t11, t22, t33, t12, t13, t23 and heat fluxes rho h1, h2, h3, evaluated on every
        stage state."""
        sc, sw = self.shape_c, self.shape_w
        n, nw = int(np.prod(sc)), int(np.prod(sw))

        def call(_user, r, rt, ru, rv, rw, out):
            a = [np.ctypeslib.as_array(q, shape=(nw if q is rw else n,)) for q in (r, rt, ru, rv, rw)]
            planes = model(a[0].reshape(sc), a[1].reshape(sc), a[2].reshape(sc), a[3].reshape(sc),
                           a[4].reshape(sw))
            np.ctypeslib.as_array(out, shape=(9 * n,))[:] = np.asarray(planes, dtype=np.float64).reshape(-1)

        self._sgs_cb = _SGS_FN(call)   # kept alive as long as the oracle
        _lib().orc_set_sgs_model(self._h, self._sgs_cb, None)

    def step(self, n=1):
        rc = _lib().orc_step(self._h, int(n))
        assert rc == 0, rc

    def slow_rhs(self):
        sc, sw = self.shape_c, self.shape_w
        out = [np.empty(sc), np.empty(sc), np.empty(sc), np.empty(sc), np.empty(sw),
               np.empty(sc), np.empty(sc), np.empty(sc)]
        rc = _lib().orc_slow_rhs(self._h, *[_p(x) for x in out])
        assert rc == 0, rc
        keys = ["R_rho", "R_rhotheta", "R_rhou", "R_rhov", "R_rhow", "pp", "pi", "theta"]
        return dict(zip(keys, out))

    def substep_once(self, dtau, X, R=None):
        """One acoustic substep about the current (stage) state; X, R: dicts keyed
        rho, rhotheta, rhou, rhov, rhow of perturbations / slow tendencies."""
        keys = ("rho", "rhotheta", "rhou", "rhov", "rhow")
        xs = [np.array(X[k], dtype=np.float64, copy=True) for k in keys]
        rs = [None if R is None else _f64(R[k]) for k in keys]
        _lib().orc_substep_once(self._h, float(dtau), *[_p(x) for x in xs], *[_p(r) for r in rs])
        return dict(zip(keys, xs))

    def mu(self):
        out = np.empty(self.shape_c)
        _lib().orc_get_mu(self._h, _p(out))
        return out

    def aux(self, name):
        """Cell arrays of the last slow-RHS evaluation: "mu" (rho K_m), "muh" (rho K_h) and
        "tke_src" (the SGS-energy source) of the Deardorff closure."""
        out = np.empty(self.shape_c)
        rc = _lib().orc_get_aux(self._h, {"mu": 0, "muh": 1, "tke_src": 2}[name], _p(out))
        assert rc == 0
        return out

    def mass(self):
        return _lib().orc_mass(self._h)

    def state(self):
        out = {k: self.get(k) for k in ("rho", "rhotheta", "rhou", "rhov", "rhow")}
        if self.cfg.moist:
            out.update({k: self.get(k) for k in ("rhoqv", "rhoqc", "rhoqr")})
        return out


def set_threads(n: int) -> int:
    """Sets the OpenMP thread count of the oracle; returns the count now in effect."""
    L = _lib()
    L.orc_set_threads(int(n))
    return L.orc_get_threads()


def interp(q, s, order):
    q = _f64(q)
    return _lib().orc_interp(_p(q), float(s), int(order))


def weno5(q, s, z=False):
    q = _f64(q)
    return _lib().orc_weno5(_p(q), float(s), int(bool(z)))


def thomas(a, b, c, d):
    a, b, c, d = (_f64(x) for x in (a, b, c, d))
    x = np.empty_like(d)
    _lib().orc_thomas(len(d), _p(a), _p(b), _p(c), _p(d), _p(x))
    return x


def eos(rt):
    p = C.c_double()
    pi = C.c_double()
    _lib().orc_eos(float(rt), C.byref(p), C.byref(pi))
    return p.value, pi.value


def hse_column(zc, theta, p_s=1.0e5, theta_surf=None, g=9.81):
    zc = _f64(zc); th = _f64(theta)
    n = len(zc)
    rho = np.empty(n); p = np.empty(n)
    _lib().orc_hse_column(n, _p(zc), _p(th), float(p_s),
                          float(th[0] if theta_surf is None else theta_surf), float(g), _p(rho), _p(p))
    return rho, p


def psi_m(zeta):
    return _lib().orc_psi_m(float(zeta))


def ustar(U, z1, z0, Q=0.0, theta=300.0, g=9.81):
    return _lib().orc_ustar(float(U), float(z1), float(z0), float(Q), float(theta), float(g))


def qvs(T, p):
    """Saturation mixing ratio (Tetens) of the oracle's Kessler scheme."""
    return _lib().orc_qvs(float(T), float(p))


def rain_speed(rho, qr, rho_sfc):
    """Rain terminal velocity [m/s] of the oracle's Kessler scheme."""
    return _lib().orc_rain_speed(float(rho), float(qr), float(rho_sfc))


def rain_evap(rho, qv, qr, qvs_, p):
    """Rain evaporation rate [1/s] of the oracle's Kessler scheme."""
    return _lib().orc_rain_evap(float(rho), float(qv), float(qr), float(qvs_), float(p))


def config_from(wl, **over) -> OracleConfig:
    """The oracle configuration of a workload (paper_2412_04395_gb300.workloads.Workload, the seeded
    input description both implementations read), optionally with fields overridden."""
    cfg = OracleConfig(nx=wl.nx, ny=wl.ny, nz=wl.nz, dx=wl.dx, dy=wl.dy,
                       terrain_beta=wl.terrain_beta, dt=wl.dt, n_substeps=wl.n_substeps,
                       beta_s=wl.beta_s, beta_d=wl.beta_d, mom_adv=wl.mom_adv,
                       scal_adv=wl.scal_adv, closure=wl.closure, Cs=wl.Cs, Pr_t=wl.Pr_t,
                       nu=wl.nu, gravity=wl.gravity, f_cor=wl.f_cor, u_g=wl.u_g, v_g=wl.v_g,
                       surface=wl.surface, z0=wl.z0, sfc_theta_flux=wl.sfc_theta_flux,
                       theta_s=wl.theta_s, brunt_N=wl.brunt_N, p_s=wl.p_s, tracer=wl.tracer,
                       ray_tau=wl.ray_tau, ray_zd=wl.ray_zd, ray_fields=wl.ray_fields,
                       moist=wl.moist, relax_tau=wl.relax_tau, relax_width=wl.relax_width,
                       anelastic=wl.anelastic)
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


def from_workload(wl, init=True, **over) -> Oracle:
    """An oracle of a workload with its initial state set (passive scalar, SGS energy and water
    species included)."""
    o = Oracle(config_from(wl, **over), wl.zeta, wl.terrain, wl.knots, wl.qv_knots)
    if init:
        o.set_initial(wl.dtheta, wl.u, wl.v, wl.w, qv=wl.qv)
        if wl.tracer and wl.phi is not None:
            o.set_tracer_initial(wl.phi)
        if wl.closure == 4 and wl.tke is not None:
            o.set("rhotke", o.get("rho") * wl.tke)
        if wl.moist and (wl.qc is not None or wl.qr is not None):
            rho = o.get("rho")
            if wl.qc is not None:
                o.set("rhoqc", rho * wl.qc)
            if wl.qr is not None:
                o.set("rhoqr", rho * wl.qr)
            o.capture_reference()
    return o
