"""The ctypes mirrors of the header's structs and enums match include/km.h
field for field (names, order, C types), so the binding and the library
agree on every byte; checked on the CPU by parsing the header."""
import ctypes
import os
import re

import paper_2405_12052_gb300 as km

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "km.h")
CTYPES = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double,
          "float": ctypes.c_float, "void*": ctypes.c_void_p}


def _strip_comments(s):
    return re.sub(r"/\*.*?\*/", "", s, flags=re.S)


def _struct_fields(name):
    src = _strip_comments(open(HEADER).read())
    m = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, flags=re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        ty, rest = decl.split(" ", 1)
        if rest.startswith("*"):
            ty, rest = ty + "*", rest[1:]
        for var in rest.split(","):
            var = var.strip()
            arr = re.match(r"(\w+)\[(\d+)\]", var)
            fields.append((arr.group(1), CTYPES[ty] * int(arr.group(2))) if arr else (var, CTYPES[ty]))
    return fields


def _enum_values():
    src = _strip_comments(open(HEADER).read())
    return {name: int(v) for name, v in re.findall(r"\b(KM_\w+)\s*=\s*(-?\d+)", src)}


def _same(py_struct, header_fields):
    assert [f for f, _ in py_struct._fields_] == [f for f, _ in header_fields]
    for (f, t_py), (_, t_h) in zip(py_struct._fields_, header_fields):
        assert ctypes.sizeof(t_py) == ctypes.sizeof(t_h) and ctypes.alignment(t_py) == ctypes.alignment(t_h), f


def test_options_stats_and_batch_info_match_the_header():
    _same(km._Options, _struct_fields("km_options"))
    _same(km._Stats, _struct_fields("km_stats"))
    _same(km._BatchInfo, _struct_fields("km_batch_info"))


def test_option_names_map_to_the_header_enums():
    e = _enum_values()
    assert km.E_MODES == {"norm": e["KM_E_NORM"], "squared": e["KM_E_SQUARED"]}
    assert km.LABEL_POLICIES == {"every_step": e["KM_LABELS_EVERY_STEP"], "final": e["KM_LABELS_FINAL"]}
    assert km.DIST_PATHS == {"auto": e["KM_DIST_AUTO"], "simt": e["KM_DIST_SIMT"], "tensor": e["KM_DIST_TENSOR"]}
    assert km.TC_OPERANDS == {"bf16": e["KM_TC_BF16"], "f16": e["KM_TC_F16"]}
    assert (km.KM_SOA_DxN, km.KM_AOS_NxD) == (e["KM_SOA_DxN"], e["KM_AOS_NxD"])
    assert (km.KM_HOST, km.KM_DEVICE_COPY, km.KM_DEVICE_BORROW) == (e["KM_HOST"], e["KM_DEVICE_COPY"],
                                                                   e["KM_DEVICE_BORROW"])


def test_status_names_match_the_header():
    e = _enum_values()
    statuses = {v: k for k, v in e.items() if k in ("KM_OK", "KM_NOT_CONVERGED") or k.startswith("KM_E")
                and k not in ("KM_E_NORM", "KM_E_SQUARED")}
    assert km.STATUS == statuses
