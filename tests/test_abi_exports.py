"""CPU checks of the boundary: the CUDA library builds for sm_103a, loads, and exports every
entry point include/erf.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*(erf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_04395_gb300.build import build_library
    path = build_library()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("erf_init_grid", "erf_set_state", "erf_rk3_step", "erf_get_state"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2412_04395_gb300 import erf
    assert sorted(erf.EXPORTS) == sorted(n for n in _declared() if n in erf.EXPORTS)
    assert set(_declared()) <= set(erf.EXPORTS) | {"erf_set_initial"}


def test_workspace_bytes_and_validation_without_gpu(lib):
    """Host-side argument checks run without a device."""
    from paper_2412_04395_gb300 import erf, workloads as W
    wl = W.density_current(nx=32, ny=4, nz=16, dx=400.0)
    g, c, keep = erf.make_structs(wl)
    n = erf.erf_workspace_bytes(g, c)
    assert n > 30 * 8 * wl.ncell
    c.n_substeps = 3
    with pytest.raises(erf.ErfError) as e:
        erf.erf_workspace_bytes(g, c)
    assert e.value.status == erf.ERF_EINVAL
    c.n_substeps = 6
    wl2 = W.hill_bubble(nx=16, ny=16, nz=8, dx=200.0).with_(closure=W.CLOSURE_SMAGORINSKY)
    g2, c2, keep2 = erf.make_structs(wl2)
    with pytest.raises(erf.ErfError) as e:
        erf.erf_workspace_bytes(g2, c2)
    assert e.value.status == erf.ERF_EUNSUPPORTED


def test_advection_orders_are_validated_without_gpu(lib):
    """mom_adv takes 0/5 (upwind-5) or 3 (upwind-3); scal_adv 0, 1 (WENO5-JS/Z) or 3 (upwind-3)."""
    from paper_2412_04395_gb300 import erf, workloads as W
    wl = W.density_current(nx=32, ny=4, nz=16, dx=400.0)
    for mom, scal in ((5, 0), (3, 3), (0, 1), (3, 0)):
        g, c, keep = erf.make_structs(wl.with_(mom_adv=mom, scal_adv=scal))
        assert erf.erf_workspace_bytes(g, c) > 0
    for mom, scal in ((4, 0), (6, 0), (5, 2), (5, 5)):
        g, c, keep = erf.make_structs(wl.with_(mom_adv=mom, scal_adv=scal))
        with pytest.raises(erf.ErfError) as e:
            erf.erf_workspace_bytes(g, c)
        assert e.value.status == erf.ERF_EINVAL
