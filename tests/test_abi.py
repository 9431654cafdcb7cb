"""The C-ABI library builds, loads and exports every entry point that
include/gprox.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gprox.h")).read()
    return re.findall(r"^GP_API\s+[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M)


@pytest.fixture(scope="module")
def libpath():
    from paper_1805_09453_gb300 import build

    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for required in ("dct2_poisson", "rof_solve", "emd_solve", "pd_step"):
        assert required in names
    assert len(names) == len(set(names))


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(L, name), name
    L.gp_abi_version.restype = ctypes.c_int
    src = open(os.path.join(ROOT, "include", "gprox.h")).read()
    want = int(re.search(r"#define GP_ABI_VERSION (\d+)", src).group(1))
    assert L.gp_abi_version() == want
    from paper_1805_09453_gb300 import gprox

    assert gprox.ABI_VERSION == want


def test_binding_lists_every_symbol():
    from paper_1805_09453_gb300 import gprox

    assert sorted(gprox.EXPORTS) == sorted(_declared())


def test_default_opts_without_gpu(libpath):
    from paper_1805_09453_gb300 import gprox

    o = gprox.default_opts(max_iters=7)
    assert o.max_iters == 7 and o.gap_every == 10 and abs(o.tol_rel_gap - 1e-5) < 1e-20


def test_no_fallback_when_library_missing(monkeypatch, tmp_path):
    from paper_1805_09453_gb300 import gprox

    monkeypatch.setattr(gprox, "_lib", None)
    monkeypatch.setattr(gprox, "_LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        gprox.lib()
