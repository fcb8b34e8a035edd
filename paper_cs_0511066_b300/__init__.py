"""Python binding of libidet (the C ABI in include/idet.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libidet.so. Matrices may be numpy int64 arrays (host) or torch
int64 CUDA tensors (device). Workspace is drawn from torch's CUDA caching
allocator and calls run on torch's current stream.

The library must have been built (python -m paper_cs_0511066_b300.build, or
__graft_entry__.build()); importing this module without libidet.so raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libidet.so")

IDET_OK = 0
IDET_ERR_ARG = 1
IDET_ERR_BUFFER = 2
IDET_ERR_SINGULAR = 3
IDET_ERR_NOMEM = 4
IDET_ERR_TIMEOUT = 5
IDET_ERR_CUDA = 6
IDET_ERR_INTERNAL = 7

PATH_AUTO, PATH_INT64, PATH_I8, PATH_F64, PATH_BF16 = 0, 1, 2, 3, 4


class IdetError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libidet error {code}: {msg}")
        self.code = code


class idet_int(ctypes.Structure):
    _fields_ = [("sign", ctypes.c_int32), ("nlimbs", ctypes.c_uint32),
                ("cap", ctypes.c_uint32), ("limbs", ctypes.POINTER(ctypes.c_uint32))]


class idet_opts(ctypes.Structure):
    _fields_ = [("log2_epsilon", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("certify", ctypes.c_int32), ("update_path", ctypes.c_int32),
                ("nb", ctypes.c_int32), ("wave", ctypes.c_int32),
                ("lif", ctypes.c_int32), ("prime_bits", ctypes.c_int32),
                ("inject_fault", ctypes.c_int32), ("i_max", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class idet_stats(ctypes.Structure):
    _fields_ = [("primes_used", ctypes.c_int32), ("primes_in_cra", ctypes.c_int32),
                ("et_stop", ctypes.c_int32), ("lift_iters", ctypes.c_int32),
                ("lift_timed_out", ctypes.c_int32), ("log2_K", ctypes.c_int32),
                ("log2_H", ctypes.c_double), ("ms_lu", ctypes.c_double),
                ("ms_lift", ctypes.c_double), ("ms_cra", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("launches", ctypes.c_uint64),
                ("ms_lift_kernel", ctypes.c_double), ("lift_bytes", ctypes.c_double),
                ("lu_macs", ctypes.c_double), ("ms_inverse", ctypes.c_double),
                ("ms_rr", ctypes.c_double), ("inverse_macs", ctypes.c_double),
                ("ms_lift_setup", ctypes.c_double), ("lift_path", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_cs_0511066_b300.build`")

_lib = ctypes.CDLL(LIB_PATH)
_P = ctypes.c_void_p
_i64, _i32, _u32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
_lib.idet_default_opts.argtypes = [ctypes.POINTER(idet_opts)]
_lib.idet_default_opts.restype = None
_lib.idet_last_error.restype = ctypes.c_char_p
_lib.idet_launch_count.restype = ctypes.c_uint64
_lib.idet_int_det.argtypes = [_P, _i64, _i64, _i32, ctypes.POINTER(idet_opts), _P,
                              ctypes.POINTER(idet_int), ctypes.POINTER(idet_stats)]
_lib.idet_largest_invariant_factor.argtypes = [_P, _i64, _i64, _P, _i32,
                                               ctypes.POINTER(idet_opts), _P,
                                               ctypes.POINTER(idet_int)]
_lib.idet_det_mod_primes.argtypes = [_P, _i64, _i64, _i32, _P, _i32,
                                     ctypes.POINTER(idet_opts), _P, _P]
_lib.idet_lu_mod_prime.argtypes = [_P, _i64, _i64, _i32, _u32, ctypes.POINTER(idet_opts),
                                   _P, _P, _P]
_lib.idet_dixon_digits.argtypes = [_P, _i64, _i64, _P, _u32, _i32, _i32, _P, _P, _P]
_lib.idet_crt_symmetric.argtypes = [_P, _P, _i32, _P, ctypes.POINTER(idet_int),
                                    ctypes.POINTER(ctypes.c_int32)]
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_lib.idet_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, ctypes.c_void_p]
_lib.idet_set_allocator.restype = None

_torch = None
_allocator_installed = False
_cb_refs = []


def _get_torch():
    global _torch
    if _torch is None:
        try:
            import torch  # noqa: F401
            _torch = torch
        except Exception:  # pragma: no cover
            _torch = False
    return _torch or None


def use_torch_allocator() -> bool:
    """Route libidet's device workspace through torch's caching allocator."""
    global _allocator_installed
    if _allocator_installed:
        return True
    torch = _get_torch()
    if torch is None or not torch.cuda.is_available():
        return False

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    a, f = _ALLOC_FN(_alloc), _FREE_FN(_free)
    _cb_refs[:] = [a, f]
    _lib.idet_set_allocator(a, f, None)
    _allocator_installed = True
    return True


def _stream_ptr(stream=None) -> int:
    torch = _get_torch()
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if torch is not None and torch.cuda.is_available():
        return int(torch.cuda.current_stream().cuda_stream)
    return 0


def _check(rc: int):
    if rc != IDET_OK:
        raise IdetError(rc, _lib.idet_last_error().decode(errors="replace"))


def default_opts(**kw) -> idet_opts:
    o = idet_opts()
    _lib.idet_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def _matrix(A):
    """(pointer, n, lda, on_device, keepalive) for a numpy or torch matrix."""
    torch = _get_torch()
    if torch is not None and isinstance(A, torch.Tensor):
        if A.dtype != torch.int64 or A.dim() != 2 or A.shape[0] != A.shape[1]:
            raise ValueError("square int64 tensor expected")
        if A.stride(1) != 1:
            A = A.contiguous()
        return A.data_ptr(), A.shape[0], A.stride(0), 1 if A.is_cuda else 0, A
    a = np.ascontiguousarray(_as_int64(A))
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("square matrix expected")
    return a.ctypes.data, a.shape[0], a.shape[1], 0, a


def _as_int64(x):
    """int64 array of x, refusing input that the conversion would change: float
    input must hold integers exactly (a silent truncation would change the
    matrix), and float, unsigned or arbitrary-precision values must lie in
    [-2^63, 2^63) (numpy would wrap them); other kinds are refused."""
    arr = np.asarray(x)
    if arr.dtype.kind == "f":
        if not (np.all(np.isfinite(arr)) and np.all(arr == np.trunc(arr))):
            raise ValueError("integer entries expected (got non-integral floats)")
        # 2^63 is exact in every float type; values at or above it, or below
        # -2^63, do not fit int64
        if arr.size and (np.any(arr >= 2.0 ** 63) or np.any(arr < -(2.0 ** 63))):
            raise ValueError("entries out of the int64 range")
    elif arr.dtype.kind == "u":
        if arr.size and arr.max() > np.iinfo(np.int64).max:
            raise ValueError("entries out of the int64 range")
    elif arr.dtype == object:
        flat = arr.ravel()
        if any(not isinstance(v, (int, np.integer)) or not (-(1 << 63) <= int(v) < (1 << 63))
               for v in flat):
            raise ValueError("integer entries in the int64 range expected")
    elif arr.dtype.kind not in "ib":
        raise ValueError(f"integer entries expected (got dtype {arr.dtype})")
    return np.asarray(arr, dtype=np.int64)


def _vector(b, on_device):
    torch = _get_torch()
    if torch is not None and isinstance(b, torch.Tensor):
        b = b.to(torch.int64)
        if on_device and not b.is_cuda:
            b = b.cuda()
        return b.contiguous().data_ptr(), b
    v = np.ascontiguousarray(_as_int64(b))
    if on_device:
        t = torch.from_numpy(v).cuda()
        return t.data_ptr(), t
    return v.ctypes.data, v


def _to_int(x: idet_int, buf) -> int:
    v = 0
    for i in range(x.nlimbs - 1, -1, -1):
        v = (v << 32) | int(buf[i])
    return -v if x.sign < 0 else v


def _call_int(fn, *args, cap: int = 1 << 12):
    while True:
        buf = (ctypes.c_uint32 * cap)()
        out = idet_int(0, 0, cap, buf)
        rc = fn(*args, ctypes.byref(out))
        if rc == IDET_ERR_BUFFER and out.nlimbs > cap:
            cap = int(out.nlimbs) + 8
            continue
        _check(rc)
        return _to_int(out, buf)


def int_det(A, *, certify: bool = False, seed: int | None = None, lif: bool | int = True,
            update_path: int | None = None, nb: int | None = None, wave: int | None = None,
            log2_epsilon: float | None = None, prime_bits: int | None = None, stream=None,
            inject_fault: int | None = None, i_max: int | None = None,
            return_stats: bool = False):
    """det(A) as a Python int (idet_int_det). inject_fault (tests of failure
    detection only): 1-based index of a CRA prime whose modular determinant
    is made wrong on the host."""
    use_torch_allocator()
    ptr, n, lda, dev, keep = _matrix(A)
    o = default_opts(certify=int(certify), seed=seed, lif=int(lif), update_path=update_path,
                     nb=nb, wave=wave, log2_epsilon=log2_epsilon, prime_bits=prime_bits,
                     inject_fault=inject_fault, i_max=i_max)
    st = idet_stats()
    cap = max(64, int(n * 40 // 32) + 64)
    while True:
        buf = (ctypes.c_uint32 * cap)()
        out = idet_int(0, 0, cap, buf)
        rc = _lib.idet_int_det(ptr, n, lda, dev, ctypes.byref(o), _stream_ptr(stream),
                               ctypes.byref(out), ctypes.byref(st))
        if rc == IDET_ERR_BUFFER and out.nlimbs > cap:
            cap = int(out.nlimbs) + 8
            continue
        if rc != IDET_OK:
            err = IdetError(rc, _lib.idet_last_error().decode(errors="replace"))
            err.stats = st.as_dict()
            raise err
        break
    d = _to_int(out, buf)
    del keep
    return (d, st.as_dict()) if return_stats else d


def largest_invariant_factor(A, b, *, seed: int | None = None, stream=None) -> int:
    """lcm of the denominators of A^{-1} b (idet_largest_invariant_factor)."""
    use_torch_allocator()
    ptr, n, lda, dev, keep = _matrix(A)
    bp, bkeep = _vector(b, dev)
    o = default_opts(seed=seed)
    return _call_int(lambda *a: _lib.idet_largest_invariant_factor(*a), ptr, n, lda, bp, dev,
                     ctypes.byref(o), _stream_ptr(stream), cap=max(64, n * 40 // 32 + 64))


def det_mod_primes(A, primes, *, update_path: int | None = None, nb: int | None = None,
                   stream=None) -> np.ndarray:
    use_torch_allocator()
    ptr, n, lda, dev, keep = _matrix(A)
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    out = np.zeros(len(pr), dtype=np.uint32)
    o = default_opts(update_path=update_path, nb=nb)
    _check(_lib.idet_det_mod_primes(ptr, n, lda, dev, pr.ctypes.data, len(pr), ctypes.byref(o),
                                    _stream_ptr(stream), out.ctypes.data))
    return out


def lu_mod_prime(A, p: int, *, nb: int | None = None, update_path: int | None = None,
                 stream=None):
    """(LU residues in [0,p), perm, singular flag)."""
    use_torch_allocator()
    ptr, n, lda, dev, keep = _matrix(A)
    lu = np.zeros((n, n), dtype=np.uint32)
    perm = np.zeros(n, dtype=np.int32)
    o = default_opts(nb=nb, update_path=update_path)
    rc = _lib.idet_lu_mod_prime(ptr, n, lda, dev, p, ctypes.byref(o), _stream_ptr(stream),
                                lu.ctypes.data, perm.ctypes.data)
    if rc == IDET_ERR_SINGULAR:
        return lu, perm, True
    _check(rc)
    return lu, perm, False


def dixon_digits(A, b, p: int, m: int, *, stream=None):
    """(digits [m][n] int32, residual r_m [n] int64)."""
    use_torch_allocator()
    ptr, n, lda, dev, keep = _matrix(A)
    bp, bkeep = _vector(b, dev)
    digits = np.zeros((m, n), dtype=np.int32)
    res = np.zeros(n, dtype=np.int64)
    _check(_lib.idet_dixon_digits(ptr, n, lda, bp, p, m, dev, _stream_ptr(stream),
                                  digits.ctypes.data, res.ctypes.data))
    return digits, res


_lib.idet_dixon_digits_block.argtypes = [_P, _i64, _i64, _P, _i32, _u32, _i32, _i32, _P, _P, _P,
                                         ctypes.POINTER(idet_stats)]


def dixon_digits_block(A, B, p: int, m: int, *, stream=None, return_stats: bool = False):
    """Block lift of the rows of B (1 or 2 right-hand sides) in one pass
    (idet_dixon_digits_block): (digits [k][m][n] int32, residuals [k][n]
    int64)."""
    use_torch_allocator()
    ptr, n, lda, dev, keep = _matrix(A)
    torch = _get_torch()
    if torch is not None and isinstance(B, torch.Tensor):
        Bt = B.to(torch.int64).contiguous()
        if dev and not Bt.is_cuda:
            Bt = Bt.cuda()
        k = Bt.shape[0] if Bt.dim() == 2 else 1
        bp, bkeep = Bt.data_ptr(), Bt
    else:
        Bh = np.ascontiguousarray(_as_int64(B))
        k = Bh.shape[0] if Bh.ndim == 2 else 1
        bp, bkeep = _vector(Bh.reshape(-1), dev)
    digits = np.zeros((k, m, n), dtype=np.int32)
    res = np.zeros((k, n), dtype=np.int64)
    st = idet_stats()
    _check(_lib.idet_dixon_digits_block(ptr, n, lda, bp, k, p, m, dev, _stream_ptr(stream),
                                        digits.ctypes.data, res.ctypes.data, ctypes.byref(st)))
    return (digits, res, st.as_dict()) if return_stats else (digits, res)


def crt_symmetric(residues, primes, *, stream=None):
    """(r, trailing agreements) (idet_crt_symmetric)."""
    use_torch_allocator()
    res = np.ascontiguousarray(np.asarray(residues, dtype=np.uint32))
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    tr = ctypes.c_int32(0)
    v = _call_int(lambda *a: _lib.idet_crt_symmetric(res.ctypes.data, pr.ctypes.data, len(pr),
                                                     _stream_ptr(stream), a[0], ctypes.byref(tr)),
                  cap=len(pr) + 8)
    return v, int(tr.value)


_lib.idet_extended_bonus.argtypes = [_P, _i64, _i64, _P, _P, _i32, ctypes.POINTER(idet_opts), _P,
                                     ctypes.POINTER(idet_int), ctypes.POINTER(idet_int)]


def extended_bonus(A, B, R, *, seed: int | None = None, stream=None):
    """(pi~_2, s~) of Section 3.2 for two right-hand sides B (2 x n) and a
    2 x n matrix R (idet_extended_bonus)."""
    use_torch_allocator()
    ptr, n, lda, dev, keep = _matrix(A)
    Bh = np.ascontiguousarray(_as_int64(B)).reshape(2, n)
    Rh = np.ascontiguousarray(_as_int64(R)).reshape(2, n)
    o = default_opts(seed=seed)
    cap = max(64, int(n * 80 // 32) + 64)
    while True:
        b1 = (ctypes.c_uint32 * cap)()
        b2 = (ctypes.c_uint32 * cap)()
        pi = idet_int(0, 0, cap, b1)
        st = idet_int(0, 0, cap, b2)
        rc = _lib.idet_extended_bonus(ptr, n, lda, Bh.ctypes.data, Rh.ctypes.data, dev,
                                      ctypes.byref(o), _stream_ptr(stream), ctypes.byref(pi),
                                      ctypes.byref(st))
        if rc == IDET_ERR_BUFFER:
            cap = max(int(pi.nlimbs), int(st.nlimbs)) + 8
            continue
        _check(rc)
        return _to_int(pi, b1), _to_int(st, b2)


_lib.idet_cra_early_termination.argtypes = [_P, _P, _i32, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, _i32, _P,
                                            ctypes.POINTER(idet_int),
                                            ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]


def cra_early_termination(residues, primes, log2_H: float, log2_epsilon: float, log2_l: float,
                          pool_size: int, *, certify: bool = False, stream=None):
    """(r, stop index or -1, reason) of Alg. 2.1's loop over the given stream
    (idet_cra_early_termination)."""
    use_torch_allocator()
    res = np.ascontiguousarray(np.asarray(residues, dtype=np.uint32))
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    stop, why = ctypes.c_int32(0), ctypes.c_int32(0)
    v = _call_int(lambda *a: _lib.idet_cra_early_termination(
        res.ctypes.data, pr.ctypes.data, len(pr), float(log2_H), float(log2_epsilon),
        float(log2_l), float(pool_size), int(certify), _stream_ptr(stream), a[0],
        ctypes.byref(stop), ctypes.byref(why)), cap=len(pr) + 8)
    return v, int(stop.value), int(why.value)


_lib.idet_int_det_batch.argtypes = [_i32, _P, _P, _P, _i32, ctypes.POINTER(idet_opts), _P, _P,
                                    ctypes.POINTER(idet_stats)]


def int_det_batch(mats, *, seed: int | None = None, update_path: int | None = None,
                  stream=None, return_stats: bool = False):
    """[det(A_i)] for a list of square matrices (numpy int64, or torch int64
    CUDA tensors), through idet_int_det_batch."""
    use_torch_allocator()
    count = len(mats)
    infos = [_matrix(A) for A in mats]
    devs = {d for (_, _, _, d, _) in infos}
    if len(devs) > 1:
        raise ValueError("all matrices must be on the host or all on the device")
    dev = devs.pop() if devs else 0
    ptrs = (ctypes.c_void_p * max(count, 1))(*[p for (p, _, _, _, _) in infos])
    ns = (ctypes.c_int64 * max(count, 1))(*[nn for (_, nn, _, _, _) in infos])
    lds = (ctypes.c_int64 * max(count, 1))(*[ld for (_, _, ld, _, _) in infos])
    caps = [max(64, int(nn * 40 // 32) + 64) for (_, nn, _, _, _) in infos]
    bufs = [(ctypes.c_uint32 * c)() for c in caps]
    outs = (idet_int * max(count, 1))()
    for i in range(count):
        outs[i] = idet_int(0, 0, caps[i], bufs[i])
    o = default_opts(seed=seed, update_path=update_path)
    st = idet_stats()
    _check(_lib.idet_int_det_batch(count, ptrs, ns, lds, dev, ctypes.byref(o),
                                   _stream_ptr(stream), outs, ctypes.byref(st)))
    res = [_to_int(outs[i], bufs[i]) for i in range(count)]
    del infos
    return (res, st.as_dict()) if return_stats else res


_lib.idet_det_mod_primes_noalloc.argtypes = [_P, _i64, _i64, _i32, _P, _i32, _P, _P]


def det_mod_primes_noalloc(A, primes, *, stream=None) -> np.ndarray:
    """det(A) mod p_k through idet_det_mod_primes_noalloc: no device memory is
    allocated (n <= 128, at most 32 primes); see include/idet.h."""
    ptr, n, lda, dev, keep = _matrix(A)
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    out = np.zeros(len(pr), dtype=np.uint32)
    _check(_lib.idet_det_mod_primes_noalloc(ptr, n, lda, dev, pr.ctypes.data, len(pr),
                                            _stream_ptr(stream), out.ctypes.data))
    return out


def launch_count() -> int:
    return int(_lib.idet_launch_count())


_lib.idet_set_wait_limit.argtypes = [_i64]
_lib.idet_set_wait_limit.restype = None


def set_wait_limit(cycles: int) -> None:
    """Cycle limit of the lifting kernels' bounded waits (failure-detection
    tests; 0 restores the default), idet_set_wait_limit."""
    _lib.idet_set_wait_limit(int(cycles))


__all__ = ["int_det", "largest_invariant_factor", "det_mod_primes", "lu_mod_prime",
           "dixon_digits", "dixon_digits_block", "crt_symmetric", "cra_early_termination",
           "extended_bonus",
           "launch_count", "default_opts", "IdetError",
           "use_torch_allocator", "LIB_PATH"]


_lib.idet_int_det_mp.argtypes = [_P, _P, _i64, _i32, _i32, ctypes.POINTER(idet_opts), _P,
                                 ctypes.POINTER(idet_int), ctypes.POINTER(idet_stats)]


def int_det_mp(mag, sgn, *, certify: bool = False, seed: int | None = None, lif: bool = True,
               prime_bits: int | None = None, stream=None, inject_fault: int | None = None,
               return_stats: bool = False):
    """det(A) for multi-word entries (idet_int_det_mp): mag is uint32
    [n][n][L] (little-endian base-2^32 magnitudes), sgn int8 [n][n] in
    {-1, 0, 1}; numpy arrays or CUDA tensors (both on the same side)."""
    use_torch_allocator()
    torch = _get_torch()
    if torch is not None and isinstance(mag, torch.Tensor):
        if not isinstance(sgn, torch.Tensor) or mag.is_cuda != sgn.is_cuda:
            raise ValueError("mag and sgn must both be host arrays or both CUDA tensors")
        if mag.dtype not in (torch.int32, torch.uint32) or sgn.dtype != torch.int8:
            raise ValueError("mag must be 32-bit, sgn int8")
        mag, sgn = mag.contiguous(), sgn.contiguous()
        n, L, dev = mag.shape[0], mag.shape[2], 1 if mag.is_cuda else 0
        mp, sp, keep = mag.data_ptr(), sgn.data_ptr(), (mag, sgn)
    else:
        m = np.ascontiguousarray(np.asarray(mag, dtype=np.uint32))
        g = np.ascontiguousarray(np.asarray(sgn, dtype=np.int8))
        n, L, dev = m.shape[0], m.shape[2], 0
        mp, sp, keep = m.ctypes.data, g.ctypes.data, (m, g)
    if mag.shape[:2] != (n, n) or tuple(sgn.shape) != (n, n):
        raise ValueError("mag must be [n][n][L] and sgn [n][n]")
    o = default_opts(certify=int(certify), seed=seed, lif=int(lif), prime_bits=prime_bits,
                     inject_fault=inject_fault)
    st = idet_stats()
    cap = max(64, int(n * (32 * L + 16) // 32) + 64)
    buf = (ctypes.c_uint32 * cap)()
    out = idet_int(0, 0, cap, buf)
    _check(_lib.idet_int_det_mp(mp, sp, n, L, dev, ctypes.byref(o), _stream_ptr(stream),
                                ctypes.byref(out), ctypes.byref(st)))
    d = _to_int(out, buf)
    del keep
    return (d, st.as_dict()) if return_stats else d


class idet_job_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batched", ctypes.c_int32),
                ("worker", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("ms_queue", ctypes.c_double), ("ms_run", ctypes.c_double),
                ("ms_latency", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_end_ms", ctypes.c_double), ("stats", idet_stats)]


class idet_server_stats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int32), ("running", ctypes.c_int32),
                ("max_running", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("bytes_in_use", ctypes.c_uint64), ("budget", ctypes.c_uint64),
                ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("groups", ctypes.c_uint64)]


_lib.idet_server_create.argtypes = [ctypes.c_size_t, _i32, _i32, _i32, ctypes.POINTER(idet_opts)]
_lib.idet_server_create.restype = _P
_lib.idet_submit.argtypes = [_P, _P, _i64, _i64, ctypes.POINTER(ctypes.c_uint64)]
_lib.idet_poll.argtypes = [_P, ctypes.c_uint64, _i32, ctypes.POINTER(idet_int),
                           ctypes.POINTER(idet_job_info)]
_lib.idet_server_info.argtypes = [_P, ctypes.POINTER(idet_server_stats)]
_lib.idet_server_info.restype = None
_lib.idet_server_destroy.argtypes = [_P]
_lib.idet_server_destroy.restype = None


class Server:
    """Determinant server with continuous batching (idet_server_*): submit
    host matrices, poll for exact determinants. See include/idet.h."""

    def __init__(self, hbm_budget: int = 0, slots: int = 4, small_n: int = 512,
                 max_batch: int = 64, **opts):
        _get_torch()  # the CUDA context is the one torch uses
        o = default_opts(**opts)
        self._srv = _lib.idet_server_create(int(hbm_budget), slots, small_n, max_batch,
                                            ctypes.byref(o))
        if not self._srv:
            raise IdetError(IDET_ERR_ARG, _lib.idet_last_error().decode(errors="replace"))
        self._cap = {}

    def submit(self, A) -> int:
        a = np.ascontiguousarray(_as_int64(A))
        if a.ndim != 2 or a.shape[0] != a.shape[1]:
            raise ValueError("square matrix expected")
        t = ctypes.c_uint64(0)
        _check(_lib.idet_submit(self._srv, a.ctypes.data, a.shape[0], a.shape[0], ctypes.byref(t)))
        n = a.shape[0]
        amax = int(np.abs(a).max()) if n else 0
        self._cap[t.value] = int(n * (amax.bit_length() + 0.5 * math.log2(n + 1)) / 32) + 16
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """(det, info dict), or None if not finished within timeout_ms."""
        info = idet_job_info()
        cap = self._cap.get(ticket, 64)
        while True:
            buf = (ctypes.c_uint32 * cap)()
            out = idet_int(0, 0, cap, buf)
            rc = _lib.idet_poll(self._srv, ticket, timeout_ms, ctypes.byref(out), ctypes.byref(info))
            if rc == IDET_ERR_BUFFER:
                cap = int(out.nlimbs) + 8
                continue
            if rc == IDET_ERR_TIMEOUT:
                return None
            self._cap.pop(ticket, None)
            _check(rc)
            d = {f: getattr(info, f) for f, _ in info._fields_ if f not in ("pad", "stats")}
            d["stats"] = info.stats.as_dict()
            return _to_int(out, buf), d

    def info(self) -> dict:
        s = idet_server_stats()
        _lib.idet_server_info(self._srv, ctypes.byref(s))
        return {f: getattr(s, f) for f, _ in s._fields_ if f != "pad"}

    def close(self):
        if self._srv:
            _lib.idet_server_destroy(self._srv)
            self._srv = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class idet_tuned(ctypes.Structure):
    _fields_ = [("update_path", ctypes.c_int32), ("nb", ctypes.c_int32),
                ("wave", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("ms_per_prime", ctypes.c_double)]


_lib.idet_autotune.argtypes = [_i64, _i32, _i32, _P, ctypes.POINTER(idet_tuned)]
_lib.idet_tuning_save.argtypes = [ctypes.c_char_p]
_lib.idet_tuning_load.argtypes = [ctypes.c_char_p]
_lib.idet_tuning_clear.restype = None


def autotune(n: int, prime_bits: int = 21, entry_bits: int = 21, stream=None) -> dict:
    """Times the LU variants for order n (idet_autotune) and records the
    fastest in the library's table; returns the winner."""
    use_torch_allocator()
    t = idet_tuned()
    _check(_lib.idet_autotune(n, prime_bits, entry_bits, _stream_ptr(stream), ctypes.byref(t)))
    return {"update_path": t.update_path, "nb": t.nb, "wave": t.wave,
            "ms_per_prime": t.ms_per_prime}


def tuning_save(path: str) -> None:
    _check(_lib.idet_tuning_save(os.fsencode(path)))


def tuning_load(path: str) -> None:
    _check(_lib.idet_tuning_load(os.fsencode(path)))


def tuning_clear() -> None:
    _lib.idet_tuning_clear()


# The tuning table measured on B300 ships with the package; IDET_TUNING
# names another file, or "none" to start untuned.
_TUNING = os.environ.get("IDET_TUNING",
                         os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_b300.json"))
if _TUNING != "none" and os.path.exists(_TUNING):
    tuning_load(_TUNING)
