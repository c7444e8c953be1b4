"""Host-side checks of the C ABI library (no GPU needed): it builds, loads,
exports every symbol include/kin.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def kin():
    from paper_2212_11010_gb300 import build
    build.build()
    import paper_2212_11010_gb300 as kin
    kin.load_library()
    return kin


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "kin.h")).read()
    return sorted(set(re.findall(r"\b(kin_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["kin_create", "kin_set_state", "kin_step", "kin_get_state", "kin_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(kin):
    lib = ctypes.CDLL(kin.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(kin.EXPORTED) == declared_symbols()


BAD = [
    dict(dim=4), dict(degree=0), dict(degree=4), dict(system=7), dict(lam=-1.0), dict(dt=0.0),
    dict(omega=2.5), dict(omega=0.5), dict(iters=0), dict(precision=9), dict(tiles=(3, 1)),
    dict(block=(3, 1)), dict(velset=1), dict(gamma=1.0), dict(system=2), dict(inflow=(2, 0)),
    dict(inflow=(0, 0, 1)), dict(inflow=(1, 0), velset=4),
]


@pytest.mark.parametrize("bad", BAD, ids=[str(b) for b in BAD])
def test_create_rejects_bad_arguments(kin, bad):
    args = dict(dim=2, n=(8, 8), lo=(0, 0), hi=(1, 1), system=kin.KIN_EULER, lam=5.0, omega=2.0,
                gamma=1.4, tiles=(2, 2), iters=3, precision=kin.KIN_FP32, block=(0, 0))
    degree, dt, velset = 2, 0.01, 2
    degree = bad.pop("degree", degree)
    dt = bad.pop("dt", dt)
    velset = bad.pop("velset", velset)
    args.update(bad)
    if args["dim"] > 3:
        args["n"], args["lo"], args["hi"] = (8, 8, 8), (0, 0, 0), (1, 1, 1)
    mesh, model, opts = kin.make_args(**args)
    model.velset = velset
    with pytest.raises(kin.KinError) as ei:
        kin.kin_create(mesh, model, degree, dt, opts)
    assert ei.value.status == kin.KIN_EINVAL
    assert len(kin.kin_last_error(None)) > 0


@pytest.mark.parametrize("bad", [dict(sigma=-1.0), dict(sigma=float("nan")), dict(velset=5)],
                         ids=["sigma<0", "sigma=nan", "D3Q4"])
def test_create_rejects_bad_maxwell_arguments(kin, bad):
    # Maxwell's equations run in 3D on the six axis velocities with sigma >= 0
    velset = bad.pop("velset", 3)
    mesh, model, opts = kin.make_args(dim=3, n=(4, 4, 4), lo=(0, 0, 0), hi=(1, 1, 1),
                                      system=kin.KIN_MAXWELL, lam=3.3, omega=2.0, gamma=1.4,
                                      tiles=(1, 1, 1), iters=3, precision=kin.KIN_FP64,
                                      block=(0, 0, 0), **bad)
    model.velset = velset
    with pytest.raises(kin.KinError) as ei:
        kin.kin_create(mesh, model, 1, 0.01, opts)
    assert ei.value.status == kin.KIN_EINVAL


def test_null_context_calls_are_rejected(kin):
    lib = kin.load_library()
    assert lib.kin_step(None, 1) == kin.KIN_EINVAL
    assert lib.kin_sync(None) == kin.KIN_EINVAL
    assert lib.kin_destroy(None) == kin.KIN_OK
    assert lib.kin_last_error(None)
