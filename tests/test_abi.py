"""The C ABI library builds, loads, and exports every entry point that
include/kpp.h declares (no GPU needed: only host-side functions are called)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"KPP_API\s+[\w\s\*]+?\b(kpp_\w+)\s*\(", txt)
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_1908_02136_gb300 as kpp

    return kpp.load_library()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ["kpp_seed", "kpp_workspace_size", "kpp_read_status", "kpp_quantize",
                     "kpp_seed_host", "kpp_status_string", "kpp_version", "kpp_describe",
                     "kpp_seed_batched", "kpp_batch_workspace_size", "kpp_seed_noalloc",
                     "kpp_tune", "kpp_tune_workspace_size", "kpp_tune_clear",
                     "kpp_lloyd_workspace_size", "kpp_lloyd_prepare", "kpp_lloyd_step",
                     "kpp_lloyd_assign", "kpp_kmeans_par_workspace_size", "kpp_kmeans_par",
                     "kpp_shard_exchange_words", "kpp_shard_workspace_size", "kpp_shard_first",
                     "kpp_shard_pass", "kpp_shard_pick", "kpp_shard_phi", "kpp_measure_read"]:
        assert required in names


@pytest.mark.parametrize("debug", [False, True])
def test_every_declared_symbol_is_exported(lib, debug):
    from paper_1908_02136_gb300 import build

    out = subprocess.run(["nm", "-D", "--defined-only", build.lib_path(debug)],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)", out))
    for name in declared_entry_points():
        assert name in exported, name
        assert hasattr(lib, name)
    # nothing but the declared C names leaks out of the library
    ours = {n for n in exported if n.startswith("kpp")}
    assert ours == set(declared_entry_points())


def test_host_only_entry_points(lib):
    import paper_1908_02136_gb300 as kpp

    assert kpp.kpp_version() >= 100
    for code in range(10):
        s = kpp.kpp_status_string(code)
        assert isinstance(s, str) and s and s != "unknown status"
    assert kpp.kpp_status_string(99) == "unknown status"
    kpp.kpp_tune_clear()  # host-side table only


def test_invalid_arguments_fail_synchronously(lib):
    import paper_1908_02136_gb300 as kpp

    # NULL points / K > N / bad dtype are rejected before any CUDA call
    assert kpp.kpp_seed(None, None, 10, 2, 3, 0, 1, 0, None, 0, None, None, None,
                        None, 0, None) == kpp.ERR_INVALID_ARG
    assert kpp.kpp_workspace_size(10, 2, 11, 0) == 0
    assert kpp.kpp_workspace_size(10, 0, 1, 0) == 0
    assert kpp.kpp_workspace_size(10, 2, 1, 7) == 0
    assert kpp.kpp_quantize(None, 4, 4, kpp.BF16, None, None, None) == kpp.ERR_INVALID_ARG
    assert kpp.kpp_kmeans_par_workspace_size(10, 129, 5) == 0
    assert kpp.kpp_kmeans_par_workspace_size(10, 4, 0) == 0
    import ctypes

    nc = ctypes.c_int64(-1)
    assert kpp.kpp_kmeans_par(None, 10, 4, 2, 4.0, 2, 1, 0, 5, None, None, ctypes.addressof(nc),
                              None, None, None, None, None, 0, None) == kpp.ERR_INVALID_ARG


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's struct mirrors follow the C layout field by field."""
    import ctypes

    import paper_1908_02136_gb300 as kpp

    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "kpp.h"', "int main(void){"]
    for cname, py in (("kpp_options", kpp.Options), ("kpp_plan", kpp.Plan),
                      ("kpp_problem", kpp.Problem), ("kpp_shard", kpp.Shard)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in (("kpp_options", kpp.Options), ("kpp_plan", kpp.Plan),
                      ("kpp_problem", kpp.Problem), ("kpp_shard", kpp.Shard)):
        assert got[(cname, "size")] == ctypes.sizeof(py)
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
    with pytest.raises(KeyError):
        kpp._opts_ptr({"no_such_option": 1})
