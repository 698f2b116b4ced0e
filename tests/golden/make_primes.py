"""Writes tests/golden/primes.json: seed-generated NTT-friendly primes per width.

Two tables: moduli of W-4 bits (Barrett contexts) and full-width moduli of W bits
(Montgomery contexts).  Calls only the oracle (gen_prime, gen_prime_full, two_adicity).
Run from the repository root:
    python tests/golden/make_primes.py
"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import gen_prime, gen_prime_full, two_adicity  # noqa: E402

WIDTHS = (64, 128, 256, 384, 512, 768, 1024)
SEEDS = (0, 1, 2, 3)


def main():
    out = {"comment": "q = c*2^32 + 1 with exactly W-4 bits (paper Sec. 5.2); c from "
                      "random.Random('moma:<W>:<seed>'); Miller-Rabin accepted; written by "
                      "tests/golden/make_primes.py from oracle.gen_prime",
           "primes": []}
    for w in WIDTHS:
        for s in SEEDS:
            q = gen_prime(w, s)
            out["primes"].append({"width": w, "seed": s, "q": hex(q), "bits": q.bit_length(),
                                  "two_adicity": two_adicity(q)})
    out["full_comment"] = ("q = c*2^32 + 1 with exactly W bits (full-width modulus); c from "
                           "random.Random('moma-full:<W>:<seed>'); Miller-Rabin accepted; oracle.gen_prime_full")
    out["full_primes"] = []
    for w in WIDTHS:
        for s in SEEDS[:2]:
            q = gen_prime_full(w, s)
            out["full_primes"].append({"width": w, "seed": s, "q": hex(q), "bits": q.bit_length(),
                                       "two_adicity": two_adicity(q)})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "primes.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
