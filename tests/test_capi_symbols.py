"""The C-ABI library builds, loads and exports every symbol include/spd.h
declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "spd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1405_4644_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["spd_create", "spd_destroy", "spd_factor", "spd_solve_ir", "spd_cg", "spd_residual"]:
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_lists_match_header(libpath):
    import paper_1405_4644_gb300 as spd
    assert sorted(spd.EXPORTED) == declared_symbols()
    spd.lib()  # loads and binds every signature


def test_opts_defaults_without_gpu(libpath):
    import paper_1405_4644_gb300 as spd
    o = spd.spd_opts_default()
    assert o.tol == 1e-14 and o.crit == 0 and o.maxit == 50 and o.band == -1


def test_header_compiles_as_c(tmp_path):
    import subprocess
    src = tmp_path / "t.c"
    src.write_text('#include "spd.h"\nint main(void){spd_opts o; spd_opts_default(&o); return 0;}\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o",
                        str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_missing_library_fails_loudly(monkeypatch):
    """No fallback: with libspd.so absent every entry point raises instead of
    computing anything elsewhere."""
    import paper_1405_4644_gb300 as spd
    monkeypatch.setattr(spd, "_lib", None)
    monkeypatch.setattr(spd, "_LIB_PATH", os.path.join(os.path.dirname(spd.__file__), "_absent", "libspd.so"))
    with pytest.raises(spd.SpdError, match="not built"):
        spd.lib()
    with pytest.raises(spd.SpdError, match="not built"):
        spd.spd_create(None)
