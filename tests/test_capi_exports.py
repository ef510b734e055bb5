"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/skis.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

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
    # the coin-generator probe checks its sizes and form on the host: no thread or block, a third
    # form, 2^32 blocks in all, more than 2^31 blocks a thread
    for args in ((1, 0, 1, 0), (1, 1, 0, 0), (1, 1, 1, 2), (1, 1 << 20, 1 << 12, 0), (1, 1, (1 << 31) + 1, 0)):
        with pytest.raises(skis.SkisError):
            skis.skis_philox_rate(*args)


_CTYPES = {"int32_t": ctypes.c_int32, "uint32_t": ctypes.c_uint32, "int64_t": ctypes.c_int64,
           "uint64_t": ctypes.c_uint64, "double": ctypes.c_double, "int": ctypes.c_int}


def _header_text():
    text = open(os.path.join(ROOT, "include", "skis.h")).read()
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def test_binding_structs_match_the_header():
    """Every struct the binding passes by pointer has the header's fields, in
    order, with the same C types (a drifted layout would corrupt results)."""
    text = _header_text()
    for name in ("skis_graph_info", "skis_stats", "skis_dssa_result"):
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), text, flags=re.S).group(1)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            ctype, names = decl.split(None, 1)
            for f in names.split(","):
                fields.append((f.strip(), _CTYPES[ctype]))
        ours = getattr(skis._binding, name)._fields_
        assert [(f, t) for f, t in ours] == fields, name
        hsize = sum(ctypes.sizeof(t) for _, t in fields)
        assert ctypes.sizeof(getattr(skis._binding, name)) >= hsize


def test_binding_constants_match_the_header():
    """Status codes, weight models, memory spaces, diffusion models and
    sketch options carry the header's values."""
    text = _header_text()
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(SKIS_[A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert len(consts) >= 25
    for k, v in consts.items():
        assert getattr(skis, k) == v, k
