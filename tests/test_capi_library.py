"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/*.h declares; the host-side argument checks of the library and of the binding
reject bad descriptors, null handles and short buffers (CPU only: no compute call is made)."""
import ctypes
import glob
import os
import re

import numpy as np
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


def test_invalid_network_is_rejected_on_the_host(lib):
    """ouu_dino_create checks its descriptor before any device work."""
    from paper_2305_20053_gb300 import capi
    L = capi.load()
    h = ctypes.c_void_p()
    for bad in (dict(n=6), dict(n=2049), dict(lattice_L=0), dict(r_u=300), dict(r_m=0), dict(r_m=241), dict(width=12),
                dict(max_batch=4), dict(max_eval=0), dict(gamma=0.0), dict(jac_weight=-1.0)):
        d = capi.dino_desc(**bad)
        assert L.ouu_dino_create(ctypes.byref(d), None, ctypes.byref(h)) == capi.OUU_ERR_INVALID_ARG, bad
        assert capi.last_error() and h.value is None


def test_null_handles_are_rejected(lib):
    from paper_2305_20053_gb300 import capi
    L = capi.load()
    bad = capi.OUU_ERR_INVALID_ARG
    x = ctypes.c_double(0.0)
    r = capi.risk_desc(capi.RISK_MEAN_VAR)
    assert L.ouu_sample_fields(None, 1, 0, 4, None) == bad
    assert L.ouu_pde_solve_batch(None, None, 4, None, 0, None, None, None) == bad
    assert L.ouu_adjoint_batch(None, None, None, 4, None, None) == bad
    assert L.ouu_risk_and_grad(None, 0, None, None, 4, ctypes.byref(r), 1, ctypes.byref(x), ctypes.byref(x),
                               ctypes.byref(x), ctypes.byref(x), None, None) == bad
    assert L.ouu_dino_set_params(None, None, 0) == bad
    assert L.ouu_dino_set_fused_network(None, 0) == bad
    assert L.ouu_dino_set_graphs(None, 1) == bad
    out = ctypes.c_void_p()
    assert L.ouu_batch_create(None, 0, 0, ctypes.byref(out)) == bad
    assert "problem is null" in (L.ouu_sample_fields(None, 1, 0, 4, None) and capi.last_error())
    z4 = (ctypes.c_double * 4)()
    assert L.ouu_dino_validate(None, None, None, 4, ctypes.byref(r), 1, z4, 1, 0.01, 0.05, None, None, None) == bad
    assert L.ouu_last_backend(None) == -1
    assert L.ouu_dino_save(None, b"x") == bad and L.ouu_dino_load(None, b"x") == bad
    # destroying nothing succeeds; queries on nothing give zero
    assert L.ouu_destroy_problem(None) == capi.OUU_OK and L.ouu_dino_destroy(None) == capi.OUU_OK
    assert L.ouu_problem_slots(None) == 0 and L.ouu_dino_num_params(None) == 0


def test_last_error_is_thread_local_and_truncates(lib):
    import threading
    from paper_2305_20053_gb300 import capi
    L = capi.load()
    assert L.ouu_dino_set_graphs(None, 1) == capi.OUU_ERR_INVALID_ARG
    mine = capi.last_error()
    seen = {}

    def other():
        seen["before"] = capi.last_error()
        L.ouu_sample_fields(None, 1, 0, 4, None)
        seen["after"] = capi.last_error()

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["before"] == "" and "problem is null" in seen["after"]
    assert capi.last_error() == mine
    buf = ctypes.create_string_buffer(8)
    full = L.ouu_last_error(buf, 5)
    assert full == len(mine.encode()) and buf.value == mine.encode()[:4]


def test_binding_refuses_short_buffers():
    """Sizes are checked in the binding before anything reaches the library (CPU only: the
    handles below are never created, the checks raise first)."""
    import torch
    from paper_2305_20053_gb300 import capi
    capi.need(None, 10, "x")
    capi.need(np.zeros(10), 10, "x")
    with pytest.raises(ValueError, match="x: 9 elements"):
        capi.need(torch.zeros(3, 3), 10, "x")
    P = object.__new__(capi.Problem)
    P.n, P.d_z = 9, 4
    with pytest.raises(ValueError, match="m_dev"):
        P.ouu_sample_fields(1, 0, 3, torch.zeros(2, 9, 9, dtype=torch.float64))
    m3 = torch.zeros(3, 9, 9, dtype=torch.float64)
    q3, s3 = torch.zeros(3, dtype=torch.float64), torch.zeros(3, dtype=torch.int32)
    with pytest.raises(ValueError, match="u_dev"):
        P.ouu_pde_solve_batch(m3, 3, torch.zeros(4), 0, m3[:2], q3, s3)
    with pytest.raises(ValueError, match="z_dev: 11 elements, the call needs 12"):   # 4 (3 - 1) + 4
        P.ouu_pde_solve_batch(m3, 3, torch.zeros(11), 4, None, q3, s3)
    with pytest.raises(ValueError, match="status_dev"):
        P.ouu_pde_solve_batch(m3, 3, torch.zeros(4), 0, None, q3, s3[:2])
    with pytest.raises(ValueError, match="gradq_dev"):
        P.ouu_adjoint_batch(m3, m3, 3, None, torch.zeros(3, 3, dtype=torch.float64))
    with pytest.raises(ValueError, match="m_dev"):
        P.ouu_risk_and_grad(capi.BACKEND_PDE, None, m3, 4, [capi.risk_desc(capi.RISK_MEAN_VAR)], np.zeros(4))
    D = object.__new__(capi.Dino)
    D.desc, D.d_z = capi.dino_desc(n=9, lattice_L=2, r_m=8, r_u=5, width=16), 4
    with pytest.raises(ValueError, match="output scale"):
        D.ouu_dino_set_output_scale(np.ones(4))
    with pytest.raises(ValueError, match="z: 3 entries"):
        D.ouu_dino_eval(torch.zeros(2, 9, 9, dtype=torch.float64), 2, np.zeros(3))
    with pytest.raises(ValueError, match="gradq_dev"):
        D.ouu_dino_eval(torch.zeros(2, 9, 9, dtype=torch.float64), 2, np.zeros(4), None, None, None,
                        torch.zeros(2, 3, dtype=torch.float64))
    with pytest.raises(ValueError, match="xi"):
        D.ouu_kernel_dino_network(torch.zeros(2, 7), 2, np.zeros(4), 2)
    with pytest.raises(ValueError, match="zs"):
        D.ouu_dino_validate(P, m3, 3, [capi.risk_desc(capi.RISK_MEAN_VAR)], np.zeros((2, 5)))
    with pytest.raises(ValueError, match="m_dev"):
        D.ouu_dino_validate(P, m3, 4, [capi.risk_desc(capi.RISK_MEAN_VAR)], np.zeros((2, 4)))


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "ouu.h"
int main(void) {
  ouu_problem_desc d;
  ouu_default_problem_desc(&d);
  if (d.n != 129 || d.lattice_L != 10) return 2;
  d.n = 6;
  ouu_problem_t p = NULL;
  ouu_status st = ouu_create_problem(&d, NULL, &p);
  char msg[256];
  ouu_last_error(msg, sizeof msg);
  printf("%d %s\n", (int)st, msg);
  return (st == OUU_ERR_INVALID_ARG && p == NULL && strlen(msg) > 0 && ouu_last_backend(NULL) == -1) ? 0 : 1;
}
"""


def test_headers_compile_as_c_and_a_c_program_links(lib, tmp_path):
    """The boundary is a C ABI: both headers compile as C99 and C++17, and a plain C program
    links against libouu.so and calls it (host-side calls only)."""
    import shutil
    import subprocess
    gcc, gxx = shutil.which("gcc"), shutil.which("g++")
    if not gcc or not gxx:
        pytest.skip("gcc/g++ not available")
    inc = os.path.join(ROOT, "include")
    for h in glob.glob(os.path.join(inc, "*.h")):
        for cmd in ([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c"],
                    [gxx, "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-x", "c++"]):
            r = subprocess.run(cmd + ["-I", inc, h], capture_output=True, text=True)
            assert r.returncode == 0, r.stderr
    src, exe = tmp_path / "t.c", tmp_path / "t"
    src.write_text(C_PROGRAM)
    libdir = os.path.dirname(lib._name)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-L", libdir, "-louu",
                        "-Wl,-rpath," + libdir, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.stdout, r.stderr)
    assert r.stdout.startswith("1 ")
