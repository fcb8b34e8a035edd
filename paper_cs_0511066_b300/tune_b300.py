"""Builds the LU tuning table for this GPU: runs idet_autotune over a range of
orders for both prime classes and writes the JSON table (by default next to
this file, where the binding loads it at import).

    python paper_cs_0511066_b300/tune_b300.py [--out PATH]
"""
import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_cs_0511066_b300 as idet  # noqa: E402

SIZES = [128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "tuning_b300.json"))
    args = ap.parse_args()
    idet.tuning_clear()
    for bits, entry_bits in ((21, 21), (31, 16)):
        for n in SIZES:
            t = idet.autotune(n, prime_bits=bits, entry_bits=entry_bits)
            print(json.dumps({"n": n, "prime_bits": bits, **t}), flush=True)
    idet.tuning_save(args.out)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
