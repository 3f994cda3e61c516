"""Host-side checks of the C ABI (no GPU needed, no compute calls)."""
import ctypes as C
import re

import numpy as np
import pytest

from paper_1811_11481_b300 import binding, config


@pytest.fixture(scope="module")
def lib():
    from paper_1811_11481_b300 import build
    build.build()
    return binding.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = binding.declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # and the binding describes every declared entry point
    assert set(names) <= set(binding._PROTOS), set(names) - set(binding._PROTOS)


def test_default_params_agree_with_python_defaults(lib):
    p = binding.default_params_struct()
    d = config.default_params()
    for name, _ in binding.tpc_params._fields_:
        v = getattr(p, name)
        if name in ("c0t", "c0r"):
            np.testing.assert_array_equal(np.array(list(v), np.float32), np.float32(d[name]))
        else:
            assert np.float32(v) == np.float32(d[name]), name


def test_struct_layouts_match_header(lib):
    # sizes implied by the header (natural alignment, x86-64)
    assert C.sizeof(binding.tpc_geometry) == 4 + 4 + 8 + 4 * 3 + 4 + 3 * 8
    assert C.sizeof(binding.tpc_clusters) == 8 + 4 + 4 + 8 + 7 * 8 + 4 + 4
    assert C.sizeof(binding.tpc_tracks) == 8 + 8 + 4 * 8
    assert C.sizeof(binding.tpc_calib) == 8 + 8 + 8 + 4 + 4
    src = open(binding.HEADER).read()
    body = src[:src.index("} tpc_params;")].rsplit("typedef struct {", 1)[1]
    fields = re.findall(r"(?:float|int32_t)\s+([\w, \[\]0-9]+);", body)
    names = []
    for f in fields:
        names += [x.strip().split("[")[0] for x in f.split(",")]
    assert names == [n for n, _ in binding.tpc_params._fields_]


def test_create_rejects_bad_geometry_without_touching_the_device(lib):
    h = C.c_void_p()
    assert lib.tpc_create(None, None, None, C.byref(h)) == 1
    rx = np.array([85.0, 84.0, 86.0], np.float32)  # not increasing
    g = binding.tpc_geometry(3, rx.ctypes.data_as(C.POINTER(C.c_float)), 0.17, 250.0, 0.5)
    assert lib.tpc_create(C.byref(g), None, None, C.byref(h)) == 1
    g2 = binding.tpc_geometry(1000, rx.ctypes.data_as(C.POINTER(C.c_float)), 0.17, 250.0, 0.5)
    assert lib.tpc_create(C.byref(g2), None, None, C.byref(h)) == 1
    assert not h.value
    assert lib.tpc_last_error(None) == b"null context"
    lib.tpc_destroy(None)


def test_every_struct_field_offset_matches_the_compiled_header(tmp_path):
    """Compile a C program against include/tpc.h that prints sizeof and
    offsetof of every field the ctypes binding declares, and compare."""
    import os
    import subprocess
    structs = [binding.tpc_geometry, binding.tpc_params, binding.tpc_calib,
               binding.tpc_clusters, binding.tpc_kernel_stat, binding.tpc_tuning,
               binding.tpc_tracks]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "tpc.h"',
             "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'  printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        parts = line.split()
        got[tuple(parts[:-1])] = int(parts[-1])
    for st in structs:
        n = st.__name__
        assert got[(n, "size")] == C.sizeof(st), n
        for f, _ in st._fields_:
            assert got[(n, f)] == getattr(st, f).offset, (n, f)
