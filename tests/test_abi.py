"""The C ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/*.h declares (no compute calls here)."""
import os
import re

import pytest

import paper_1308_2864_gb300 as ks
from paper_1308_2864_gb300 import build as kbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:ks_status|size_t|void|int|unsigned long long|const char\s*\*)\s*\**\s*(ks_\w+)\s*\(", re.M)


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            names |= set(DECL.findall(open(os.path.join(inc, f)).read()))
    return names


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("ks_problem_create", "ks_energy_grad", "ks_retract", "ks_minimize"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = kbuild.build()
    assert os.path.exists(path)
    lib = ks.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared but not exported"
    bound = {s[0] for s in ks.SIGNATURES}
    assert declared_functions() == bound


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1308_2864_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_error_string_without_gpu():
    lib = ks.load_library()
    assert lib.ks_last_error_string() is not None
