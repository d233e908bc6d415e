"""The C-ABI library loads and exports every entry point include/fep3m.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "fep3m.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fep3m_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1503_08509_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_header_declares_the_api():
    syms = declared_symbols()
    for s in ("fep3m_create", "fep3m_set_particles", "fep3m_compute", "fep3m_vjp", "fep3m_destroy"):
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    from paper_1503_08509_gb300 import _lib
    for s in declared_symbols():
        assert hasattr(lib, s), s
        assert s in _lib.SIGNATURES, s


def test_status_strings(lib):
    for st in range(0, -8, -1):
        assert lib.fep3m_strerror(st)


def test_create_rejects_bad_config_before_touching_the_gpu(lib):
    import ctypes
    from paper_1503_08509_gb300 import _lib
    h = ctypes.c_void_p()
    for kw in (dict(L=-1.0, n_el=16), dict(L=1.0, n_el=6), dict(L=1.0, n_el=16, q=5), dict(L=1.0, n_el=16, q=0),
               dict(L=1.0, n_el=16, q=1, flags=_lib.FEP3M_ONE_ELEMENT),
               dict(L=1.0, n_el=16, q=2, flags=_lib.FEP3M_MULTIGRID), dict(L=1.0, n_el=300, q=2),
               dict(L=1.0, n_el=16, precision=5), dict(L=float("nan"), n_el=16),
               dict(L=1.0, n_el=16, q=2, flags=_lib.FEP3M_DIRICHLET),
               dict(L=1.0, n_el=16, flags=_lib.FEP3M_DIRICHLET | _lib.FEP3M_MULTIGRID),
               dict(L=1.0, n_el=16, flags=_lib.FEP3M_DIRICHLET | _lib.FEP3M_NEUTRALIZE),
               dict(L=1.0, n_el=6, flags=_lib.FEP3M_DIRICHLET)):
        base = dict(L=1.0, n_el=16, q=1, n_sr=3, precision=0)
        base.update(kw)
        cfg = _lib.Config(**base)
        assert lib.fep3m_create(ctypes.byref(cfg), None, ctypes.byref(h)) == _lib.FEP3M_EINVAL
        assert not h.value


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of fep3m_config and fep3m_stats have the header's size and field offsets
    (a C program built against include/fep3m.h prints them)."""
    import ctypes
    import shutil
    import subprocess
    from paper_1503_08509_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fep3m.h"', "int main(void) {"]
    for cname, py in (("fep3m_config", _lib.Config), ("fep3m_stats", _lib.Stats)):
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            name, field, val = ln.split()
            got[(name, field)] = int(val)
    for cname, py in (("fep3m_config", _lib.Config), ("fep3m_stats", _lib.Stats)):
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
