"""The C-ABI library builds, loads and exports every entry point of include/dp.h.

CPU only: no call here launches device work (argument checks that fail
before any CUDA call, option defaults and the version string only).
"""
import ctypes as C
import os
import re

import numpy as np

from paper_2201_01446_gb300 import build, dp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dp_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 15
    lib = C.CDLL(build.LIB)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(dp.EXPORTS)


def test_library_is_built_for_sm_103a_only():
    # the one -gencode every translation unit and the link are given
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_defaults_and_version():
    o = dp.dp_options_default()
    assert o.tabulated == 1 and o.fit_precision == 0
    assert abs(o.table_step - 0.01) < 1e-15 and o.s_max == 2.0
    assert o.skin == 2.0 and o.rebuild_every == 10
    assert o.embed_precision == 0 and o.tanh_table == 0 and o.md_graphs == 1
    assert o.s_ext == 0.0 and o.ext_stride == 10
    assert "sm_103a" in dp.dp_version()


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of dp_options and dp_thermo against the C compiler's
    # layout of include/dp.h (size and every field offset)
    structs = {"dp_options": dp.dp_options, "dp_thermo": dp.dp_thermo}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dp.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    assert os.system(f"gcc -std=c11 -I {inc} {src} -o {exe}") == 0
    got = dict(line.split() for line in os.popen(str(exe)).read().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)


def test_create_rejects_bad_arguments_before_touching_the_device(tmp_path, cu_model_path):
    for kw in [dict(rc=0.5, rcs=1.0), dict(rc=-1.0, rcs=0.5), dict(ntypes=0)]:
        args = dict(model_path=cu_model_path, ntypes=1, rc=8.0, rcs=0.5, sel=[256])
        args.update(kw)
        try:
            dp.dp_create(**args, stream=None)
            raise AssertionError("expected DPError")
        except dp.DPError as e:
            assert e.code == 1
    for field, value in [("table_step", 0.0), ("ext_stride", 0), ("s_ext", -1.0)]:
        o = dp.dp_options_default()
        setattr(o, field, value)
        try:
            dp.dp_create(cu_model_path, 1, 8.0, 0.5, [256], options=o, stream=None)
            raise AssertionError("expected DPError")
        except dp.DPError as e:
            assert e.code == 1, field
    bad = tmp_path / "bad.model"
    bad.write_bytes(b"NOTAMODEL" + bytes(64))
    try:
        dp.dp_create(str(bad), 1, 8.0, 0.5, [256], stream=None)
        raise AssertionError("expected DPError")
    except dp.DPError as e:
        assert e.code == 2
        assert "model" in str(e)
