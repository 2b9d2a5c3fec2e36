"""The C ABI library loads on a machine without a GPU and exports every entry
point include/lhr.h declares; the Python binding carries the same names. No
compute call is made here."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lhr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lhr_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lhr_build_db", "lhr_query", "lhr_query_window", "lhr_aggregate_2d", "lhr_free_db",
                     "lhr_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    be = __graft_entry__._build_ext()
    be.build()
    lib = ctypes.CDLL(be.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_uses_the_abi_names():
    import __graft_entry__
    __graft_entry__._build_ext().build()
    import paper_2006_08861_gb300 as lhr
    for n in declared_functions():
        if n in ("lhr_free_db", "lhr_db_info"):
            continue  # reached through Database
        assert hasattr(lhr, n), n


def test_circle_limit_host_rule_matches_paper_constants():
    # The host computes the integer circle limit the kernel uses; 3 m over
    # 30 cm tiles must give 10 tiles, squared 100 (§3.2).
    from oracle.aggregate import circle_r2_limit
    assert circle_r2_limit(3.0, 0.3) == 100


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of the ABI structs have the C compiler's sizes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "lhr.h"\nint main(void) { printf("%zu %zu %zu %zu %zu", '
                   'sizeof(lhr_db_config), sizeof(lhr_query_params), sizeof(lhr_agg_params), '
                   'sizeof(lhr_server_config), sizeof(lhr_server_result)); return 0; }\n')
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    import __graft_entry__
    __graft_entry__._build_ext().build()
    import paper_2006_08861_gb300 as lhr
    want = [ctypes.sizeof(c) for c in (lhr.DbConfig, lhr.QueryParams, lhr.AggParams, lhr.ServerConfig,
                                       lhr.ServerResult)]
    assert got == want
