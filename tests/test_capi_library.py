"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/*.h declares (CPU only: no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(ouu_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2305_20053_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ouu_create_problem", "ouu_sample_fields", "ouu_pde_solve_batch", "ouu_adjoint_batch",
                     "ouu_risk_and_grad"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(lib):
    from paper_2305_20053_gb300 import capi
    missing = [n for n in declared_functions() if n not in capi.SIGNATURES]
    assert not missing, missing


def test_default_desc_without_gpu(lib):
    from paper_2305_20053_gb300 import capi
    d = capi.problem_desc()
    assert d.n == 129 and d.lattice_L == 10 and d.max_samples == 4096
    assert d.newton_rtol == 1e-10 and d.reaction_r == 1.0


def test_invalid_problem_is_rejected_on_the_host(lib):
    """Argument checks run before any device work, so this needs no GPU."""
    from paper_2305_20053_gb300 import capi
    L = capi.load()
    h = ctypes.c_void_p()
    for bad in (dict(n=6), dict(n=1025 * 2 + 1), dict(lattice_L=0), dict(bump_width=-1.0), dict(max_samples=0),
                dict(cg_rtol=2.0)):
        d = capi.problem_desc(**bad)
        assert L.ouu_create_problem(ctypes.byref(d), None, ctypes.byref(h)) == 1
        assert capi.last_error()
