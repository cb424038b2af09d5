"""CPU-only checks of the C ABI library: it builds for sm_103a, loads, and
exports every entry point that include/*.h declares (no compute calls)."""
import os
import re
import subprocess

import pytest

from paper_2404_10223_gb300 import build as B
from paper_2404_10223_gb300 import tnqe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib_path():
    if not os.path.exists(B.LIB):
        B.build()
    return B.LIB


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(tnqe_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["tnqe_create", "tnqe_add_mps", "tnqe_rotate", "tnqe_matrix_elements", "tnqe_solve",
              "tnqe_last_error", "tnqe_destroy", "tnqe_mlp_create", "tnqe_mlp_forward", "tnqe_mlp_gradient",
              "tnqe_mlp_adam_step"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tnqe_[a-z_0-9]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_resolves(lib_path):
    lib = tnqe.load(lib_path)
    for n in declared_functions():
        assert getattr(lib, n) is not None
    assert set(tnqe.EXPORTED) <= set(declared_functions())
    from paper_2404_10223_gb300 import mlp
    assert set(mlp.EXPORTED) <= set(declared_functions())
    mlp.load(lib_path)


def test_default_options_without_gpu(lib_path):
    o = tnqe.tnqe_default_options()
    assert o.precision == 0 and o.cutoff == 1e-14 and o.solve_eps == 1e-10 and o.max_jacobi_sweeps == 60

