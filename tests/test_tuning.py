"""The autotuner's table: JSON save/load round trip and rejection of bad
files (host only), and on the GPU that tuning records a valid choice and the
tuned LU still gives the oracle's residues."""
import json
import random

import pytest

import workloads
from oracle import modular

idet = pytest.importorskip("paper_cs_0511066_b300")


def test_tuning_json_round_trip(tmp_path):
    src = tmp_path / "t.json"
    entries = [{"bucket": 36, "n": 512, "prime_bits": 21, "update_path": 5, "nb": 32,
                "wave": 16, "ms_per_prime": 0.25},
               {"bucket": 47, "n": 3444, "prime_bits": 31, "update_path": 1, "nb": 16,
                "wave": 8, "ms_per_prime": 9.5}]
    src.write_text(json.dumps({"version": 1, "entries": entries}))
    idet.tuning_clear()
    idet.tuning_load(str(src))
    out = tmp_path / "out.json"
    idet.tuning_save(str(out))
    got = json.loads(out.read_text())["entries"]
    key = lambda e: (e["bucket"], e["prime_bits"])
    for a, b in zip(sorted(entries, key=key), sorted(got, key=key)):
        for k in ("bucket", "prime_bits", "update_path", "nb", "wave"):
            assert a[k] == b[k]
        assert abs(a["ms_per_prime"] - b["ms_per_prime"]) < 1e-6
    idet.tuning_clear()


@pytest.mark.parametrize("bad", ['{"entries": [{"bucket": 3}]}', "not json",
                                 '{"entries": [{"bucket": 3, "prime_bits": 22, "update_path": 1, '
                                 '"nb": 32, "wave": 4, "ms_per_prime": 1}]}'])
def test_tuning_rejects_bad_files(tmp_path, bad):
    p = tmp_path / "bad.json"
    p.write_text(bad)
    with pytest.raises(idet.IdetError):
        idet.tuning_load(str(p))


@pytest.mark.gpu
def test_autotune_records_a_valid_choice(tmp_path):
    idet.tuning_clear()
    t = idet.autotune(300, prime_bits=21, entry_bits=21)
    assert t["update_path"] in (1, 2, 4, 5) and t["nb"] in (16, 32) and t["wave"] in (4, 8, 16)
    assert t["ms_per_prime"] > 0
    A = workloads.dense_pm2p20(300, seed=4)
    P21 = modular.primes_in(1 << 20, 1 << 21)
    primes = random.Random(2).sample(P21, 6)
    assert list(idet.det_mod_primes(A, primes)) == list(modular.det_mod_primes(A, primes))
    t31 = idet.autotune(257, prime_bits=31, entry_bits=16)
    assert t31["update_path"] in (1, 5)
    p = tmp_path / "t.json"
    idet.tuning_save(str(p))
    ent = json.loads(p.read_text())["entries"]
    assert {e["prime_bits"] for e in ent} == {21, 31}
    idet.tuning_clear()
