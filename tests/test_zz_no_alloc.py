"""The allocation-free entry point (idet_det_mod_primes_noalloc) agrees with
the oracle and with idet_det_mod_primes on two calls in a row, and allocates
no device memory.

It exists for callers that cannot allocate device memory (a framework that
owns all device memory through its own pool, a context that forbids
allocation); it works in a fixed scratch area compiled into the library. This
file is collected last so that a run stopping at the first failure has run
every other test first; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import workloads
from oracle import modular

pytestmark = pytest.mark.gpu

idet = pytest.importorskip("paper_cs_0511066_b300")

P21 = [1048583, 1048589, 1048601, 1048609, 1048613, 1048627, 1048633, 1048661]
P31 = [2147483629, 2147483587, 2147483579, 2147483563]


def test_noalloc_matches_oracle_and_det_mod_primes_twice_in_a_row():
    A1 = workloads.dense_pm100(100, seed=21)
    A2 = workloads.dense_uniform(128, -(1 << 20), 1 << 20, seed=22)
    got1 = idet.det_mod_primes_noalloc(A1, P21)
    got2 = idet.det_mod_primes_noalloc(A2, P21[:5])
    assert list(got1) == list(modular.det_mod_primes(A1, P21))
    assert list(got2) == list(modular.det_mod_primes(A2, P21[:5]))
    assert list(got1) == list(idet.det_mod_primes(A1, P21))
    assert list(got2) == list(idet.det_mod_primes(A2, P21[:5]))


def test_noalloc_full_scratch_n128_32_primes():
    """The documented limits together: n = 128 and 32 primes fill the residue
    area and the reduction's shared parameter array."""
    pool = modular.primes_in(1 << 20, 1 << 21)
    primes = pool[100:132]
    A = workloads.dense_uniform(128, -(1 << 40), 1 << 40, seed=24)
    want = list(modular.det_mod_primes(A, primes))
    assert list(idet.det_mod_primes_noalloc(A, primes)) == want
    assert list(idet.det_mod_primes_noalloc(A, primes)) == want


def test_noalloc_device_input_and_wide_primes():
    torch = pytest.importorskip("torch")
    A = workloads.dense_pm2p20(77, seed=23)
    Ad = torch.from_numpy(A).cuda()
    first = idet.det_mod_primes_noalloc(Ad, P31)
    second = idet.det_mod_primes_noalloc(A, P31)
    want = list(modular.det_mod_primes(A, P31))
    assert list(first) == want and list(second) == want


def test_noalloc_allocates_no_device_memory():
    """After a first call (which loads the library's module and its static
    scratch array on this device), further calls leave the device's free
    memory and torch's allocator statistics unchanged."""
    torch = pytest.importorskip("torch")
    A = workloads.dense_pm100(90, seed=25)
    Ad = torch.from_numpy(A).cuda()
    want = list(modular.det_mod_primes(A, P21))
    idet.det_mod_primes_noalloc(Ad, P21)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st0 = torch.cuda.memory_stats()
    for _ in range(3):
        assert list(idet.det_mod_primes_noalloc(Ad, P21)) == want
        assert list(idet.det_mod_primes_noalloc(A, P21)) == want
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    st1 = torch.cuda.memory_stats()
    assert free1 == free0
    for k in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert st1.get(k, 0) == st0.get(k, 0), k


def test_noalloc_rejects_sizes_entries_and_primes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    with pytest.raises(idet.IdetError) as e:
        idet.det_mod_primes_noalloc(np.eye(129, dtype=np.int64), P21[:1])
    assert e.value.code == 1
    with pytest.raises(idet.IdetError):
        idet.det_mod_primes_noalloc(np.eye(8, dtype=np.int64), P21 * 5)
    with pytest.raises(idet.IdetError):          # mixed prime classes
        idet.det_mod_primes_noalloc(np.eye(8, dtype=np.int64), P21[:2] + P31[:1])
    big = np.eye(8, dtype=np.int64)
    big[2, 3] = np.iinfo(np.int64).min          # |a| >= 2^62: residues would wrap
    for M in (big, torch.from_numpy(big).cuda()):
        with pytest.raises(idet.IdetError) as e:
            idet.det_mod_primes_noalloc(M, P21[:2])
        assert e.value.code == 1
    ok = np.eye(8, dtype=np.int64)
    ok[2, 3] = (1 << 62) - 1
    assert list(idet.det_mod_primes_noalloc(ok, P21[:2])) == list(modular.det_mod_primes(ok, P21[:2]))
