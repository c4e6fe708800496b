"""The C-ABI library builds, loads on a machine without a GPU, and exports
every entry point that include/smr.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "smr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(smr_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libsmr():
    from paper_2407_21724_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("smr_create", "smr_set_scene", "smr_matvec", "smr_solve", "smr_far_field",
                 "smr_near_field", "smr_precond", "smr_rhs_plane_waves"):
        assert must in names


def test_library_exports_every_declared_symbol(libsmr):
    missing = [n for n in _declared() if not hasattr(libsmr, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2407_21724_gb300 import smr
    assert set(smr.exported_symbols()) == set(_declared())


def test_default_opts_without_gpu(libsmr):
    from paper_2407_21724_gb300 import smr
    o = smr.smr_default_opts()
    assert (o.L0, o.n_theta, o.n_phi, o.pitch) == (10, 16, 32, 0.5)
    so = smr.smr_default_solve_opts()
    assert so.tol == 1e-4 and so.precond == smr.SMR_PRECOND_BLOCKDIAG


def test_create_fails_cleanly_without_gpu(libsmr):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2407_21724_gb300 import smr
    with pytest.raises(smr.SmrError):
        smr.smr_create()
