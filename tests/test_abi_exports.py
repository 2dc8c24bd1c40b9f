"""The C-ABI library builds for sm_103a and exports every symbol that
include/grom.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2311_03694_gb300 as grom

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "grom.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grom_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return grom.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("grom_create", "grom_nonlinear", "grom_step", "grom_destroy", "grom_traj_create",
                     "grom_get_state", "grom_set_state", "grom_upload_tensor_slab"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (grom_[a-z0-9_]+)", out))
    assert set(_declared()) <= exported


def test_binding_covers_every_declared_symbol():
    assert set(_declared()) <= set(grom.EXPORTS)


def test_build_targets_sm103a_only():
    assert grom._build_mod.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
