"""Writes paper_2501_07535_gb300/primes.json: seed-generated NTT-friendly primes per width.

The table is input data for the library's users (moduli of the benchmark and test workloads);
it is kept in the package so that the library does not depend on the test directory.

Two tables: moduli of W-4 bits (Barrett contexts) and full-width moduli of W bits
(Montgomery contexts).  Calls only the oracle (gen_prime, gen_prime_full, two_adicity).
Run from the repository root:
    python tests/golden/make_primes.py           (write the table)
    python tests/golden/make_primes.py --check   (exit 1 if the committed table differs)
"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import gen_prime, gen_prime_full, two_adicity  # noqa: E402

WIDTHS = (64, 128, 256, 384, 512, 768, 1024)
SEEDS = (0, 1, 2, 3)


ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
TABLE = os.path.join(ROOT, "paper_2501_07535_gb300", "primes.json")


def table():
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
    return json.dumps(out, indent=1) + "\n"


def main(argv):
    text = table()
    if "--check" in argv:
        with open(TABLE) as f:
            return 0 if f.read() == text else 1
    with open(TABLE, "w") as f:
        f.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
