"""The C-ABI library builds, loads and exports every function include/gdwd.h declares;
argument checks that need no GPU reject bad input with GDWD_EINVAL."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_12019_gb300 import build, gdwd
    build.build()
    return gdwd.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "gdwd.h")).read()
    # function declarations: a return type at the start of a line, then the name and "("
    return sorted(set(re.findall(r"^(?:gdwd_status|const char\s*\*)\s*(gdwd_\w+)\s*\(", txt, re.M)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "gdwd_create" in names and "gdwd_solve" in names and "gdwd_free" in names
    for name in names:
        assert hasattr(lib, name), name


def test_struct_sizes_match_header():
    from paper_2305_12019_gb300 import gdwd
    # sizes implied by the header's field lists (LP64)
    assert ctypes.sizeof(gdwd.Options) == 5 * 8 + 4 * 4 + 8 + 8 * 8
    assert ctypes.sizeof(gdwd.Result) == 12 * 8 + 2 * 4 + 4 * 8
    assert ctypes.sizeof(gdwd.Info) == 2 * 8 + 4 * 4 + 2 * 8 + 2 * 8 + 3 * 8 + 4 * 4


def test_default_options(lib):
    from paper_2305_12019_gb300 import gdwd
    o = gdwd.default_options()
    assert o.mu == 1.0 and o.tau == 1.618 and o.tol == 1e-6 and o.max_iter == 20000 and o.store == gdwd.F32
    assert lib.gdwd_default_options(None) == 1


def _create(lib, Z, y, q=1.0, C=1.0, zdt=0, d=None, n=None, ldz=None, opts=None):
    from paper_2305_12019_gb300 import gdwd
    h = ctypes.c_void_p()
    d = Z.shape[0] if d is None else d
    n = Z.shape[1] if n is None else n
    ldz = d if ldz is None else ldz
    yy = np.ascontiguousarray(y, dtype=np.float64)
    return lib.gdwd_create(ctypes.c_void_p(Z.ctypes.data), zdt, d, n, ldz, 0,
                           yy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), q, C,
                           None if opts is None else ctypes.byref(opts), ctypes.byref(h)), h


def test_invalid_arguments_rejected(lib):
    from paper_2305_12019_gb300 import gdwd
    Z = np.asfortranarray(np.ones((5, 4)))
    y = np.array([1.0, -1.0, 1.0, -1.0])
    cases = [
        dict(d=0), dict(n=1), dict(ldz=3), dict(q=0.0), dict(q=-1.0), dict(C=0.0), dict(C=float("nan")),
        dict(zdt=7),
    ]
    for kw in cases:
        st, h = _create(lib, Z, y, **kw)
        assert st == 1, kw
        assert h.value is None
    st, h = _create(lib, Z, np.array([1.0, 1.0, 1.0, 1.0]))
    assert st == 1 and b"both classes" in lib.gdwd_last_error(None)
    st, h = _create(lib, Z, np.array([1.0, 0.0, 1.0, -1.0]))
    assert st == 1 and b"labels" in lib.gdwd_last_error(None)
    o = gdwd.default_options()
    o.tau = 1.7
    assert _create(lib, Z, y, opts=o)[0] == 1
    o = gdwd.default_options()
    o.store = 9
    assert _create(lib, Z, y, opts=o)[0] == 1
    # option values and combinations checked before any device work
    for field, val in (("kernelized", 2), ("kernelized", -2), ("solver", 3), ("gram_path", 2), ("stop_rule", 3),
                       ("dots_every", -1)):
        o = gdwd.default_options()
        setattr(o, field, val)
        assert _create(lib, Z, y, opts=o)[0] == 1, field
    for kw in ({"refine": 1}, {"kernelized": 1}, {"store": gdwd.DTYPES["bf16"]}):
        o = gdwd.default_options()
        o.solver = 1
        for k, v in kw.items():
            setattr(o, k, v)
        st, h = _create(lib, Z, y, opts=o)
        assert st == 8 and h.value is None, kw          # GDWD_EUNSUPPORTED
        assert b"direct solver" in lib.gdwd_last_error(None)
    for kw in ({"refine": 1}, {"kernelized": 1}, {"store": gdwd.DTYPES["e4m3"]}):
        o = gdwd.default_options()
        o.solver = 2
        for k, v in kw.items():
            setattr(o, k, v)
        st, h = _create(lib, Z, y, opts=o)
        assert st == 8 and h.value is None, kw          # GDWD_EUNSUPPORTED
        assert b"inexact solver" in lib.gdwd_last_error(None)
    assert lib.gdwd_free(None) == 0
    assert lib.gdwd_solve(None, None, 0, None, 0, None, None) == 1
    assert lib.gdwd_prox(None, None, None, 1.0, -1.0, 4, None, None) == 1


def test_request_struct_size():
    from paper_2305_12019_gb300 import gdwd
    # void* + 2 int32 + 3 int64 + ptr + 2 double + gdwd_options + 2 ptr (LP64)
    assert ctypes.sizeof(gdwd.Request) == 8 + 8 + 24 + 8 + 16 + ctypes.sizeof(gdwd.Options) + 16


def test_server_arguments_rejected(lib):
    from paper_2305_12019_gb300 import gdwd
    s = ctypes.c_void_p()
    assert lib.gdwd_server_create(0, 0, ctypes.byref(s)) == 1
    assert lib.gdwd_server_create(65, 0, ctypes.byref(s)) == 1
    assert lib.gdwd_server_submit(None, None, None) == 1
    assert lib.gdwd_server_destroy(None) == 0
    assert lib.gdwd_solve_batch(None, -1, 1, None, None) == 1
    assert lib.gdwd_solve_batch(None, 0, 1, None, None) == 0


def test_header_is_c_and_links_from_c(tmp_path, lib):
    """include/gdwd.h compiles as C99 and a C program links against libgdwd.so and
    calls it (the calls that need no GPU)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include "gdwd.h"
int main(void) {
  gdwd_options o;
  if (gdwd_default_options(&o) != GDWD_OK) return 1;
  if (gdwd_default_options(NULL) != GDWD_EINVAL) return 2;
  if (o.max_iter != 20000 || o.store != GDWD_F32 || o.solver != 0 || o.kernelized != 0) return 3;
  if (gdwd_free(NULL) != GDWD_OK) return 4;
  gdwd_handle* h = 0;
  double y[2] = {1.0, 1.0};
  float z[2] = {1.0f, 1.0f};
  if (gdwd_create(z, GDWD_F32, 1, 2, 1, 0, y, 1.0, 1.0, &o, &h) != GDWD_EINVAL || h) return 5;
  printf("ok %zu %zu\n", sizeof(gdwd_options), sizeof(gdwd_info));
  return 0;
}
''')
    libdir = os.path.join(ROOT, "paper_2305_12019_gb300")
    exe = tmp_path / "abi"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", libdir, "-lgdwd", "-Wl,-rpath," + libdir, "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0 and "cannot find -lgdwd" in r.stderr:
        # the library file is libgdwd.so in the package directory: link it by path
        r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                            os.path.join(libdir, "libgdwd.so"), "-Wl,-rpath," + libdir, "-o", str(exe)],
                           capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    from paper_2305_12019_gb300 import gdwd
    assert out.stdout.split() == ["ok", str(ctypes.sizeof(gdwd.Options)), str(ctypes.sizeof(gdwd.Info))]


def test_gram_noalloc_refuses_host_tensors(lib):
    """The binding of gdwd_gram_noalloc checks device, dtype and the output's size
    before it calls the library (no GPU needed for the refusal)."""
    import torch
    from paper_2305_12019_gb300 import gdwd
    Z = torch.as_strided(torch.ones(8 * 4, dtype=torch.float32), (8, 4), (1, 8))
    K = torch.zeros(16, dtype=torch.float64)
    with pytest.raises(ValueError):
        gdwd.gram_noalloc(Z, K)
    Zh = torch.as_strided(torch.ones(8 * 4, dtype=torch.float16), (8, 4), (1, 8))
    with pytest.raises(ValueError):
        gdwd.gram_noalloc(Zh, K)
