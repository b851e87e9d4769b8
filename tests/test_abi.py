"""The C-ABI library builds, loads and exports every symbol include/lbm.h
declares (no compute calls: this runs without a GPU)."""
import os
import re

import pytest

from tests.conftest import ROOT


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ["lbm_create", "lbm_set_geometry", "lbm_step", "lbm_moments", "lbm_destroy",
                     "lbm_init_equilibrium", "lbm_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import shutil

    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1710_09472_gb300 import _lib
    from paper_1710_09472_gb300.build import build

    build()
    lib = _lib.load()
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding names the same entry points
    assert set(_lib.SIGNATURES) >= set(_declared_symbols())
    assert lib.lbm_status_string(0) == b"ok"


@pytest.mark.parametrize("D,fname", [(2, "constants_2d.txt"), (3, "constants_3d.txt")])
def test_library_weight_integrals_host_only(D, fname):
    """The library's own FP64 weight integrals (host-only entry point) give the
    printed thetabar = I2/I0 and c0 = I0^-1/2, c1 = I2^-1/2, c2 = I4^-1/2."""
    import shutil

    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1710_09472_gb300.build import build
    from paper_1710_09472_gb300.lbm import weight_integrals
    from tests.conftest import load_golden

    build()
    g = load_golden(fname)
    I = weight_integrals(D)
    assert abs(I[1] / I[0] / g["thetabar"] - 1) < 1e-14
    assert abs(I[0] ** -0.5 / g["c0"] - 1) < 1e-14
    assert abs(I[1] ** -0.5 / g["c1"] - 1) < 1e-14
    assert abs(I[2] ** -0.5 / g["c2"] - 1) < 1e-14


def _enum_values(name):
    """{enumerator: value} of the typedef enum `name` in include/lbm.h."""
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef enum\s*\{([^}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    return {k: int(v) for k, v in re.findall(r"(LBM_[A-Z0-9_]+)\s*=\s*(\d+)", m.group(1))}


def test_binding_enums_match_header():
    """The binding's name -> value tables use the header's enumerator values."""
    from paper_1710_09472_gb300 import _lib

    vel = _enum_values("lbm_velset")
    assert {f"LBM_{k}": v for k, v in _lib.VEL.items()} == vel
    stat = _enum_values("lbm_stat")
    assert {f"LBM_{k.upper()}": v for k, v in _lib.STAT.items()} == stat
    force = _enum_values("lbm_force")
    assert {f"LBM_FORCE_{k.upper()}": v for k, v in _lib.FORCE.items()} == force
