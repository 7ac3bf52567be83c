"""The C-ABI library builds, loads and exports every function include/lt.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2310_02043_gb300 import _build, lighttrace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header, prefix="lt"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(" + prefix + r"_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return lighttrace.load_library()


def test_every_declared_function_is_exported(lib):
    names = _declared("lt.h")
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(lighttrace.EXPORTED) <= set(names)


def test_every_surrogate_function_is_exported(lib):
    from paper_2310_02043_gb300 import surrogate
    names = _declared("sg.h", "sg")
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(surrogate.EXPORTED) == set(names)
    assert lib.sg_create(None, 0, None) == lighttrace.LT_ERR_ARG


def test_every_header_is_checked():
    assert sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")) == ["lt.h", "sg.h"]


def test_version_and_argument_checks(lib):
    assert lib.lt_version() == 2
    assert lib.lt_create(None, 0, None) == lighttrace.LT_ERR_ARG
    assert lib.lt_destroy(None) == lighttrace.LT_OK
    assert lib.lt_last_error(None) == b"null context"


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the size and field offsets the C
    compiler gives the header's structs."""
    structs = {"lt_light": lighttrace.lt_light, "lt_stats": lighttrace.lt_stats, "lt_bvh_node": lighttrace.lt_bvh_node,
               "lt_bvh_cnode": lighttrace.lt_bvh_cnode}
    lines = ['#include "lt.h"', "#include <stdio.h>", "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        name, key, value = line.split()
        cls = structs[name]
        want = ctypes.sizeof(cls) if key == "size" else getattr(cls, key).offset
        assert int(value) == want, (name, key, value, want)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())
    assert ctypes.sizeof(lighttrace.lt_light) == 36


def test_every_declaration_is_documented():
    """Each exported function of the headers sits directly under a comment
    that states what it does."""
    for header in ("lt.h", "sg.h"):
        lines = open(os.path.join(ROOT, "include", header)).read().split("\n")
        for i, line in enumerate(lines):
            m = re.match(r"^(LT_API|SG_API)\b.*?\b((lt|sg)_[a-z_0-9]+)\(", line)
            if not m:
                continue
            prev = lines[i - 1]
            assert prev.rstrip().endswith("*/") or prev.startswith("#define"), (header, m.group(2))
