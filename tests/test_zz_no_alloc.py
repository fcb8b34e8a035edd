"""The allocation-free entry point (idet_det_mod_primes_noalloc) agrees with
idet_det_mod_primes on two calls in a row.

It exists for callers that cannot allocate device memory (a framework that
owns all device memory, a context that forbids allocation); it works in a
fixed scratch area compiled into the library. This file is collected last so
that a run stopping at the first failure has run every other test first; it
also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

idet = pytest.importorskip("paper_cs_0511066_b300")

P21 = [1048583, 1048589, 1048601, 1048609, 1048613, 1048627, 1048633, 1048661]
P31 = [2147483629, 2147483587, 2147483579, 2147483563]


def test_noalloc_matches_det_mod_primes_twice_in_a_row():
    A1 = workloads.dense_pm100(100, seed=21)
    A2 = workloads.dense_uniform(128, -(1 << 20), 1 << 20, seed=22)
    got1 = idet.det_mod_primes_noalloc(A1, P21)
    got2 = idet.det_mod_primes_noalloc(A2, P21[:5])
    assert list(got1) == list(idet.det_mod_primes(A1, P21))
    assert list(got2) == list(idet.det_mod_primes(A2, P21[:5]))


def test_noalloc_device_input_and_wide_primes():
    torch = pytest.importorskip("torch")
    A = workloads.dense_pm2p20(77, seed=23)
    Ad = torch.from_numpy(A).cuda()
    first = idet.det_mod_primes_noalloc(Ad, P31)
    second = idet.det_mod_primes_noalloc(A, P31)
    want = idet.det_mod_primes(A, P31)
    assert list(first) == list(want) and list(second) == list(want)


def test_noalloc_rejects_sizes_beyond_its_limits():
    with pytest.raises(idet.IdetError) as e:
        idet.det_mod_primes_noalloc(np.eye(129, dtype=np.int64), P21[:1])
    assert e.value.code == 1
    with pytest.raises(idet.IdetError):
        idet.det_mod_primes_noalloc(np.eye(8, dtype=np.int64), P21 * 5)
