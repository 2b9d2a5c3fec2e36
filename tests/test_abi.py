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
