"""The C ABI library builds, loads without a GPU and exports every function
that include/*.h declares; argument checks that happen on the host reject
bad input without touching a device."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1608_01125_gb300 import binding, build_ext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return binding.lib()


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(trilens_\w+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)  # resolvable through the loader


def test_status_strings(lib):
    for code in range(0, -7, -1):
        s = binding.status_str(code)
        assert s and s != "unknown status"
    assert binding.status_str(-99) == "unknown status"
    assert b"sm_103a" in lib.trilens_version()


def test_invalid_arguments_rejected_on_host(lib):
    h = ctypes.c_void_p()
    ok = binding.Params(10.0, 1e16, binding.FP64, 0, 0, 0, 0)
    empty = binding.Beam(0, *([None] * 8))
    bad_n = binding.Beam(-1, *([None] * 8))
    missing = binding.Beam(5, *([None] * 8))
    huge = binding.Beam(1 << 27, *([None] * 8))
    for A, B, P in ((bad_n, empty, ok), (missing, empty, ok), (huge, empty, ok)):
        assert lib.trilens_create(ctypes.byref(h), ctypes.byref(A), ctypes.byref(B),
                                  ctypes.byref(P), None) == binding.ERR_INVALID
    for P in (binding.Params(0.0, 1e16, 0, 0, 0, 0, 0), binding.Params(10.0, -1.0, 0, 0, 0, 0, 0),
              binding.Params(10.0, 1e16, 7, 0, 0, 0, 0), binding.Params(10.0, 1e16, 0, 33, 0, 0, 0),
              binding.Params(10.0, 1e16, 0, 0, 8, 0, 0), binding.Params(10.0, 1e16, 0, 0, 0, 17, 0), binding.Params(10.0, 1e16, 0, 0, 0, 9, 0),
              binding.Params(10.0, 1e16, 0, 0, 0, 0, -5)):
        assert lib.trilens_create(ctypes.byref(h), ctypes.byref(empty), ctypes.byref(empty),
                                  ctypes.byref(P), None) == binding.ERR_INVALID
    assert lib.trilens_create(None, ctypes.byref(empty), ctypes.byref(empty), ctypes.byref(ok),
                              None) == binding.ERR_INVALID
    assert lib.trilens_build(None, 0) == binding.ERR_INVALID
    assert lib.trilens_collide_step(None, 0, None, 0, None) == binding.ERR_INVALID
    assert lib.trilens_debug_eval64(None, None, -1, 0, None) == binding.ERR_INVALID
    assert lib.trilens_run(None, 0, 1, None) == binding.ERR_INVALID
    assert lib.trilens_debug_set_parts(None, 2) == binding.ERR_INVALID
    for name in ("trilens_debug_set_cut_cap", "trilens_debug_set_key_bits"):
        assert getattr(lib, name)(None, 8) == binding.ERR_INVALID
    assert lib.trilens_debug_shrink_buffers(None, 64) == binding.ERR_INVALID
    # pair products: argument checks before any device work; no hits is a no-op
    pp = lib.trilens_pair_products
    assert pp(None, ctypes.byref(empty), None, 0, 0, None, None) == binding.ERR_INVALID
    assert pp(ctypes.byref(empty), ctypes.byref(bad_n), None, 0, 0, None, None) == binding.ERR_INVALID
    assert pp(ctypes.byref(empty), ctypes.byref(empty), None, -1, 0, None, None) == binding.ERR_INVALID
    assert pp(ctypes.byref(empty), ctypes.byref(empty), None, 0, 0, None, None) == 0
    assert pp(ctypes.byref(empty), ctypes.byref(empty), None, 3, 0, None, None) == binding.ERR_INVALID
    # depletion: a context is required; nothing runs without one
    n = ctypes.c_int64(-5)
    x = ctypes.c_double(-5.0)
    assert lib.trilens_deplete_step(None, 0, None, 0, None, None, None, ctypes.byref(n),
                                    ctypes.byref(x)) == binding.ERR_INVALID
    assert lib.trilens_deplete_rounds(None, ctypes.byref(n)) == binding.ERR_INVALID
    rec = (ctypes.c_int64 * 5)()
    da = lib.trilens_deplete_step_async
    assert da(None, 0, None, 0, None, None, None, None) == binding.ERR_INVALID
    assert da(None, 0, None, 0, None, None, None, ctypes.addressof(rec)) == binding.ERR_INVALID
    assert da(None, 0, None, 0, None, None, None, ctypes.addressof(rec) + 4) == binding.ERR_INVALID
    # swarm split (IP regime): bad beams, sizes or parameters never reach the device
    P = binding.Params(10.0, 1e16, 0, 0, 0, 0, 0)
    sm = lib.trilens_swarm_mark
    assert sm(None, ctypes.byref(empty), 0.1, 0.1, ctypes.byref(P), 0, 1, None, None,
              None) == binding.ERR_INVALID
    assert sm(ctypes.byref(empty), ctypes.byref(empty), -0.1, 0.1, ctypes.byref(P), 0, 1, None,
              None, None) == binding.ERR_INVALID
    assert sm(ctypes.byref(empty), ctypes.byref(empty), 0.1, 0.1, ctypes.byref(P), 0, 0, None,
              None, None) == binding.ERR_INVALID
    assert sm(ctypes.byref(missing), ctypes.byref(empty), 0.1, 0.1, ctypes.byref(P), 0, 1, None,
              None, None) == binding.ERR_INVALID
    assert lib.trilens_swarm_count(ctypes.byref(bad_n), None, None, ctypes.byref(n),
                                   None) == binding.ERR_INVALID
    assert lib.trilens_swarm_count(ctypes.byref(empty), None, None, ctypes.byref(n),
                                   None) == binding.ERR_INVALID
    assert lib.trilens_swarm_expand(ctypes.byref(empty), -1.0, None, 0, None, None, None,
                                    None) == binding.ERR_INVALID
    assert lib.trilens_swarm_expand(ctypes.byref(empty), 0.5, None, 0, None, None, None,
                                    None) == binding.ERR_INVALID
    # band stress: sizes and constants are checked before anything is launched
    bs = lib.trilens_debug_band_stress
    dummy = ctypes.c_void_p(256)
    assert bs(1, -1, 5.0, 1e14, dummy, None, 0, None) == binding.ERR_INVALID
    assert bs(1, 10, 5.0, 1e14, None, None, 0, None) == binding.ERR_INVALID
    assert bs(1, 10, 0.0, 1e14, dummy, None, 0, None) == binding.ERR_INVALID
    assert bs(1, 10, 5.0, -1.0, dummy, None, 0, None) == binding.ERR_INVALID
    assert bs(1, 10, 5.0, 1e14, dummy, None, 4, None) == binding.ERR_INVALID
    assert bs(1, 10, 5.0, 1e14, dummy, dummy, 11, None) == binding.ERR_INVALID
    lib.trilens_destroy(None)
