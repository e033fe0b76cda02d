import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU validation")


def oracle_config_from(wl, **over):
    from oracle import OracleConfig
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


def make_oracle(wl, init=True, **over):
    """Oracle for a workload (optionally overriding configuration fields), initial state set."""
    from oracle import Oracle
    o = Oracle(oracle_config_from(wl, **over), wl.zeta, wl.terrain, wl.knots, wl.qv_knots)
    if init:
        o.set_initial(wl.dtheta, wl.u, wl.v, wl.w, qv=wl.qv)
        if wl.moist and (wl.qc is not None or wl.qr is not None):
            rho = o.get("rho")
            if wl.qc is not None:
                o.set("rhoqc", rho * wl.qc)
            if wl.qr is not None:
                o.set("rhoqr", rho * wl.qr)
            o.capture_reference()
        if wl.tracer and wl.phi is not None:
            o.set_tracer_initial(wl.phi)
        if wl.closure == 4 and wl.tke is not None:
            o.set("rhotke", o.get("rho") * wl.tke)
    return o


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    return oracle.build_oracle()
