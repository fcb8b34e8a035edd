"""The C ABI library loads and exports every function include/idet.h declares
(no GPU needed: nothing is computed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "idet.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(idet_[a-z0-9_]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["idet_int_det", "idet_largest_invariant_factor", "idet_det_mod_primes",
              "idet_lu_mod_prime", "idet_dixon_digits", "idet_crt_symmetric"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_idet_build", os.path.join(ROOT, "paper_cs_0511066_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    lib = ctypes.CDLL(mod.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_imports_and_defaults():
    import paper_cs_0511066_b300 as idet
    o = idet.default_opts()
    assert o.log2_epsilon == -64.0 and o.lif == 1 and o.certify == 0
    assert idet.launch_count() >= 0
