"""The C-ABI library builds, loads and exports every function include/lt.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

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
    assert lib.lt_version() == 1
    assert lib.lt_create(None, 0, None) == lighttrace.LT_ERR_ARG
    assert lib.lt_destroy(None) == lighttrace.LT_OK
    assert lib.lt_last_error(None) == b"null context"


def test_struct_layouts_match_the_header():
    assert ctypes.sizeof(lighttrace.lt_light) == 36
    assert ctypes.sizeof(lighttrace.lt_stats) == 8 * 5 + 4 * 4 + 8 + 4 * 2


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
