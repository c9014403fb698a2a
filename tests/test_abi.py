"""The C ABI library builds, loads and exports every function include/*.h declares (no GPU).

Only host-side argument checks that return before any CUDA call are exercised here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mhd_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_10816_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mhd_create", "mhd_step", "mhd_divb", "mhd_destroy", "mhd_max_dt", "mhd_stats",
                     "mhd_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_rejects_bad_boxes_before_touching_the_device(lib):
    from paper_2609_10816_gb300 import mhd

    L = mhd.lib()
    out = ctypes.c_void_p()
    for cfg in (mhd._Config(0, 4, 4, 0.1, 0.1, 0.1, 5 / 3, 3), mhd._Config(4, 4, 4, -0.1, 0.1, 0.1, 5 / 3, 3),
                mhd._Config(4, 4, 4, 0.1, 0.1, 0.1, 1.0, 3)):
        rc = L.mhd_create(ctypes.byref(cfg), None, ctypes.byref(out))
        assert rc == mhd.ERR_ARG
        assert out.value is None
        assert L.mhd_create_error()
    assert L.mhd_create(None, None, ctypes.byref(out)) == mhd.ERR_ARG
    assert L.mhd_step(None, None, 1.0, 0, 0.0) == mhd.ERR_ARG
    L.mhd_destroy(None)


def test_scheme_bits_match_header():
    from paper_2609_10816_gb300 import mhd

    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    vals = dict(re.findall(r"(MHD_\w+)\s*=\s*([^,\n/]+)", src))

    def ev(s):
        return eval(s.strip(), {}, {})

    assert mhd.RECON["ppm"] == ev(vals["MHD_RECON_PPM"])
    assert mhd.RIEMANN["hlld"] == ev(vals["MHD_RIEMANN_HLLD"])
    assert mhd.EMF["b25a"] == ev(vals["MHD_EMF_B25A"])
    assert mhd.FOFC_OFF == ev(vals["MHD_FOFC_OFF"])


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2609_10816_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
    for f in glob.glob(os.path.join(pkg, "csrc", "*")):
        assert "oracle" not in open(f).read().lower(), f
