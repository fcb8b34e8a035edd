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


def test_orders_above_the_limit_are_rejected_before_any_device_work():
    """n > IDET_MAX_ORDER returns IDET_ERR_ARG from the argument checks,
    which run before any CUDA call (so this needs no GPU): the byte counts of
    such orders would overflow."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_idet_build", os.path.join(ROOT, "paper_cs_0511066_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    lib = ctypes.CDLL(mod.build())
    lib.idet_last_error.restype = ctypes.c_char_p
    hdr = open(os.path.join(ROOT, "include", "idet.h")).read()
    limit = int(re.search(r"#define IDET_MAX_ORDER (\d+)", hdr).group(1))
    assert limit == 65536
    big = ctypes.c_int64(limit + 1)
    dummy = ctypes.c_void_p(64)          # never dereferenced: the checks fail first
    i64, i32, u32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
    calls = {
        "idet_int_det": lambda: lib.idet_int_det(dummy, big, big, i32(0), None, None, dummy, None),
        "idet_largest_invariant_factor": lambda: lib.idet_largest_invariant_factor(
            dummy, big, big, dummy, i32(0), None, None, dummy),
        "idet_det_mod_primes": lambda: lib.idet_det_mod_primes(
            dummy, big, big, i32(0), dummy, i32(1), None, None, dummy),
        "idet_lu_mod_prime": lambda: lib.idet_lu_mod_prime(
            dummy, big, big, i32(0), u32(2147483629), None, None, dummy, dummy),
        "idet_dixon_digits": lambda: lib.idet_dixon_digits(
            dummy, big, big, dummy, u32(2147483629), i32(1), i32(0), None, dummy, dummy),
        "idet_int_det_mp": lambda: lib.idet_int_det_mp(
            dummy, dummy, big, i32(2), i32(0), None, None, dummy, None),
    }
    for name, call in calls.items():
        assert call() == 1, name
    ns = (i64 * 2)(3, limit + 1)
    ldas = (i64 * 2)(3, limit + 1)
    ptrs = (ctypes.c_void_p * 2)(64, 64)
    assert lib.idet_int_det_batch(i32(2), ptrs, ns, ldas, i32(0), None, None, dummy, None) == 1
    assert b"invalid matrix 1" in lib.idet_last_error()


def test_crt_rejects_repeated_primes_on_the_host():
    """A repeated prime has no inverse modulo the product of the others, so
    Garner's method would return a wrong value; the call refuses it before
    any device work."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_idet_build", os.path.join(ROOT, "paper_cs_0511066_b300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    lib = ctypes.CDLL(mod.build())
    lib.idet_last_error.restype = ctypes.c_char_p
    res = (ctypes.c_uint32 * 3)(1, 2, 3)
    pr = (ctypes.c_uint32 * 3)(1048583, 1048589, 1048583)
    out = ctypes.c_void_p(64)            # never dereferenced: the check fails first
    assert lib.idet_crt_symmetric(res, pr, ctypes.c_int32(3), None, out, None) == 1
    assert b"distinct" in lib.idet_last_error()


def test_empty_inputs_return_before_any_device_work():
    """The 0 x 0 matrix has determinant 1 (and largest invariant factor 1),
    det mod p of it is 1 for every prime, and the empty Chinese remaindering
    gives 0 with no agreements; these answers come from the argument checks,
    before any CUDA call, so no GPU is needed."""
    import paper_cs_0511066_b300 as idet
    lib = idet._lib

    def big(fn):
        buf = (ctypes.c_uint32 * 4)(7, 7, 7, 7)
        out = idet.idet_int(5, 9, 4, buf)
        rc = fn(ctypes.byref(out))
        assert rc == 0, idet._lib.idet_last_error()
        return idet._to_int(out, buf)

    assert big(lambda o: lib.idet_int_det(None, 0, 0, 0, None, None, o, None)) == 1
    assert big(lambda o: lib.idet_largest_invariant_factor(None, 0, 0, None, 0, None, None, o)) == 1
    assert big(lambda o: lib.idet_int_det_mp(None, None, 0, 1, 0, None, None, o, None)) == 1
    trailing = ctypes.c_int32(-1)
    assert big(lambda o: lib.idet_crt_symmetric(None, None, 0, None, o, ctypes.byref(trailing))) == 0
    assert trailing.value == 0
    primes = (ctypes.c_uint32 * 3)(1048583, 1048589, 1048601)
    out = (ctypes.c_uint32 * 3)(0, 0, 0)
    assert lib.idet_det_mod_primes(None, 0, 0, 0, primes, 3, None, None, out) == 0
    assert list(out) == [1, 1, 1]


def test_binding_refuses_matrices_it_would_have_to_change():
    """Float input is accepted only when every entry is an integer: a silent
    truncation would change the matrix and so the determinant. The checks run
    in the binding, before any device work."""
    import numpy as np
    import pytest
    import paper_cs_0511066_b300 as idet
    with pytest.raises(ValueError):
        idet.int_det(np.array([[1.5, 0.0], [0.0, 1.0]]))
    with pytest.raises(ValueError):
        idet.int_det(np.array([[np.inf, 0.0], [0.0, 1.0]]))
    with pytest.raises(ValueError):
        idet.int_det(np.array([["a", "b"], ["c", "d"]]))
    with pytest.raises(ValueError):
        idet.int_det(np.zeros((2, 3), dtype=np.int64))
    assert idet._as_int64(np.array([[2.0, -3.0]])).tolist() == [[2, -3]]
    assert idet._as_int64([[1, 2], [3, 4]]).dtype == np.int64
    # values that numpy's cast would wrap are refused, not wrapped
    with pytest.raises(ValueError):
        idet.int_det(np.array([[1e19, 0.0], [0.0, 1.0]]))
    with pytest.raises(ValueError):
        idet.int_det(np.array([[2.0 ** 63, 0.0], [0.0, 1.0]]))
    with pytest.raises(ValueError):
        idet.int_det(np.array([[2 ** 64 - 1, 0], [0, 1]], dtype=np.uint64))
    with pytest.raises(ValueError):
        idet.int_det(np.array([[1 << 70, 0], [0, 1]], dtype=object))
    assert idet._as_int64(np.array([[-(2.0 ** 63)]])).tolist() == [[-(1 << 63)]]
    assert idet._as_int64(np.array([[2 ** 63 - 1]], dtype=np.uint64)).tolist() == [[2 ** 63 - 1]]


def test_early_termination_scan_refuses_bad_streams_on_the_host():
    """idet_cra_early_termination checks its primes (odd, prime, distinct,
    below 2^31) and parameters before any device work."""
    import paper_cs_0511066_b300 as idet
    lib = idet._lib
    lib.idet_last_error.restype = ctypes.c_char_p
    out = ctypes.byref(idet.idet_int(0, 0, 0, None))   # not written: the checks fail first
    stop, why = ctypes.c_int32(7), ctypes.c_int32(7)
    f = lib.idet_cra_early_termination
    res = (ctypes.c_uint32 * 2)(1, 2)
    same = (ctypes.c_uint32 * 2)(1048583, 1048583)
    assert f(res, same, 2, 100.0, -64.0, 20.0, 73586.0, 0, None, out,
             ctypes.byref(stop), ctypes.byref(why)) == 1
    composite = (ctypes.c_uint32 * 2)(1048583, 1048583 * 3)
    assert f(res, composite, 2, 100.0, -64.0, 20.0, 73586.0, 0, None, out,
             ctypes.byref(stop), ctypes.byref(why)) == 1
    good = (ctypes.c_uint32 * 2)(1048583, 1048589)
    assert f(res, good, 2, 100.0, 0.5, 20.0, 73586.0, 0, None, out,
             ctypes.byref(stop), ctypes.byref(why)) == 1      # epsilon must be < 1
