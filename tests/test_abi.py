"""The C-ABI library loads and exports every entry point of include/dtsort.h
(no GPU needed, no compute calls)."""
import os
import re

import pytest

import paper_2401_00710_gb300 as dts

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "dtsort.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"DTSORT_API\s+[\w\s\*]*?\b(dtsort_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    dts.build()
    return dts.lib()


def test_header_declares_the_entry_points():
    syms = declared_symbols()
    for name in ("dtsort_u32", "dtsort_u32_kv", "dtsort_u64", "dtsort_u64_kv",
                 "dtsort_segmented_u32_kv", "dtsort_workspace_bytes",
                 "dtsort_create", "dtsort_last_device_error"):
        assert name in syms
    assert set(syms) <= set(dts.EXPORTED) | {"dtsort_status_string"}


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(7):
        s = dts.status_string(code)
        assert s.startswith("DTSORT_")
    assert "TIMEOUT" in dts.status_string(dts.DTSORT_ERR_DEVICE_TIMEOUT)


def test_default_options(lib):
    o = dts.dtsort_default_options()
    assert o.gamma_max == 9 and o.heavy_detection == 1 and o.seed == 1
    assert o.wait_limit_ms == 2000 and o.debug_fault == 0


def test_null_handle_is_rejected(lib):
    assert lib.dtsort_u32(None, None, 10, None, 0, None) == dts.DTSORT_ERR_INVALID_ARG
    assert lib.dtsort_destroy(None) == dts.DTSORT_ERR_INVALID_ARG


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(dts._build_ext, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(dts, "_lib", None)
    with pytest.raises(RuntimeError):
        dts.lib()


@pytest.mark.parametrize("cls,cname", [(dts.dtsort_options, "dtsort_options"),
                                       (dts.dtsort_stats, "dtsort_stats")])
def test_binding_structs_match_the_header(cls, cname, tmp_path):
    # the ctypes mirrors of the header's structs: every field at the C
    # compiler's offset, and the same total size (a field added to or dropped
    # from one side only would shift the ones after it)
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dtsort.h"',
             "int main(void) {",
             '  printf("size %%zu\\n", sizeof(%s));' % cname]
    for name, _ in cls._fields_:
        lines.append('  printf("%s %%zu\\n", offsetof(%s, %s));' % (name, cname, name))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = dict(line.split() for line in out.strip().splitlines())
    assert int(got["size"]) == ctypes.sizeof(cls)
    for name, _ in cls._fields_:
        assert int(got[name]) == getattr(cls, name).offset, name
