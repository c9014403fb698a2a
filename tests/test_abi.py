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
    assert L.mhd_step_cfl(None, None, 0.3, 0, 0.0) == mhd.ERR_ARG
    assert L.mhd_last_dt(None, None) == mhd.ERR_ARG
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


def test_batch_and_noalloc_reject_bad_arguments_before_touching_the_device(lib):
    from paper_2609_10816_gb300 import mhd

    L = mhd.lib()
    out = ctypes.c_void_p()
    for dims in ([4, 4, 0], [4, -1, 4], [2048, 2048, 1024]):  # empty, negative, >= 2^31 cells
        arr = (ctypes.c_int * 3)(*dims)
        assert L.mhd_batch_create(arr, 1, 0.1, 5 / 3, None, ctypes.byref(out)) == mhd.ERR_ARG
        assert out.value is None
        assert L.mhd_batch_last_error(None)
    arr = (ctypes.c_int * 3)(4, 4, 4)
    assert L.mhd_batch_create(arr, 0, 0.1, 5 / 3, None, ctypes.byref(out)) == mhd.ERR_ARG
    assert L.mhd_batch_create(arr, 1, -0.1, 5 / 3, None, ctypes.byref(out)) == mhd.ERR_ARG
    assert L.mhd_batch_step(None, None, 0.3, 0, 0.0) == mhd.ERR_ARG
    assert L.mhd_batch_set_schedule(None, 64, 1, 0, 1) == mhd.ERR_ARG
    ms = (ctypes.c_double * 12)()
    assert L.mhd_batch_phase_ms(None, ms) == mhd.ERR_ARG
    # the allocation-free step refuses boxes above its fixed array before any device work
    cfg = mhd._Config(64, 64, 64, 0.1, 0.1, 0.1, 5 / 3, 3)
    fake = ctypes.c_double(0.0)  # never dereferenced: the size check comes first
    ptr = ctypes.addressof(fake)
    state = mhd._State(ptr, ptr, ptr, ptr)
    rc = L.mhd_step_noalloc(ctypes.byref(cfg), ctypes.byref(state), ctypes.c_double(0.1), 0, ctypes.c_double(0.0),
                            None)
    assert rc == mhd.ERR_ARG and b"exceeds" in L.mhd_create_error()
