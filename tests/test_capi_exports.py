"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/skis.h declares (no compute calls here)."""
import ctypes
import os
import re

import paper_1709_03565_gb300 as skis

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(skis_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_entry_point():
    path = skis.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name
    # the Python binding names the same entry points
    for name in names:
        assert hasattr(skis, name), name


def test_last_error_is_callable_without_gpu():
    skis.build()
    assert isinstance(skis.skis_last_error(), str)


def test_bad_arguments_are_rejected_before_any_device_work():
    skis.build()
    import numpy as np

    lib = skis.lib()
    out = ctypes.c_void_p()
    # n = 0 is rejected on the host, with a message
    rc = lib.skis_load_graph(ctypes.byref(out), 0, 0, None, None, None, skis.SKIS_W_WC, 0, skis.SKIS_MEM_HOST, None)
    assert rc == skis.SKIS_EINVAL and "n must be" in skis.skis_last_error()
    # unknown weight model
    src = np.array([1], np.int32)
    dst = np.array([0], np.int32)
    rc = lib.skis_load_graph(ctypes.byref(out), 2, 1, ctypes.c_void_p(src.ctypes.data),
                             ctypes.c_void_p(dst.ctypes.data), None, 9, 0, skis.SKIS_MEM_HOST, None)
    assert rc == skis.SKIS_EINVAL
    assert lib.skis_sketch_set_option(None, 0, 1) == skis.SKIS_EINVAL
