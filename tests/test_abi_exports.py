"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/etale.h (no GPU needed, no compute call made)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "etale.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(etale_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2607_02543_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("etale_create", "etale_insert", "etale_delete", "etale_search", "etale_reclaim"):
        assert must in names


def test_every_declared_symbol_is_exported(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (etale_[a-z_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_declares_all(lib_path):
    import paper_2607_02543_gb300 as pkg
    lib = pkg.load()
    assert sorted(pkg.EXPORTS) == declared_functions()
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_has_no_cpu_fallback(tmp_path):
    from paper_2607_02543_gb300 import binding
    with pytest.raises(ImportError):
        binding.load.__wrapped__ if hasattr(binding.load, "__wrapped__") else None
        saved = binding._lib
        binding._lib = None
        try:
            binding.load(str(tmp_path / "missing.so"))
        finally:
            binding._lib = saved


def test_build_targets_sm103a():
    from paper_2607_02543_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the size and field offsets that a
    C compiler gives the structures of include/etale.h."""
    from paper_2607_02543_gb300 import binding
    pairs = [("etale_config", binding.Config), ("etale_tuning", binding.Tuning), ("etale_stats_t", binding.Stats)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "etale.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    import ctypes
    for cname, py in pairs:
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
