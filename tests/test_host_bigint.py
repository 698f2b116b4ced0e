"""The library's host-side big integers (csrc/moma_bigint.hpp: every per-modulus constant --
Barrett mu, twiddle companions, roots of unity, R^2 mod q, the primality check -- is computed with
them) against Python integers and sympy, through a small C++ harness compiled here with g++.
No GPU involved."""
import os
import random
import shutil
import subprocess

import pytest

from paper_2501_07535_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sympy = pytest.importorskip("sympy")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("bigint") / "bigint_harness")
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_2501_07535_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "bigint_harness.cpp"), "-o", exe], check=True)

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return out.stdout.split("\n")[:len(lines)]
    return run


def _hex(v):
    return format(v, "x")


def _values(rng, count, max_bits):
    vals = [0, 1, 2, (1 << 32) - 1, 1 << 32, (1 << 64) - 1, (1 << max_bits) - 1, 1 << (max_bits - 1)]
    vals += [rng.getrandbits(rng.randrange(1, max_bits + 1)) for _ in range(count)]
    return vals


def test_arithmetic_matches_python(harness):
    rng = random.Random(1)
    cases, want = [], []
    xs = _values(rng, 150, 2100)
    for a in xs:
        b = rng.choice(xs)
        cases += [f"add {_hex(a)} {_hex(b)}", f"mul {_hex(a)} {_hex(b)}", f"cmp {_hex(a)} {_hex(b)}"]
        want += [_hex(a + b), _hex(a * b), str((a > b) - (a < b))]
        hi, lo = max(a, b), min(a, b)
        cases.append(f"sub {_hex(hi)} {_hex(lo)}")
        want.append(_hex(hi - lo))
        s = rng.randrange(0, 300)
        cases += [f"shl {_hex(a)} {_hex(s)}", f"shr {_hex(a)} {_hex(s)}"]
        want += [_hex(a << s), _hex(a >> s)]
        if b:
            cases.append(f"divmod {_hex(a)} {_hex(b)}")
            want.append(f"{_hex(a // b)} {_hex(a % b)}")
        nw = (a.bit_length() + 31) // 32 + rng.randrange(0, 3)
        cases.append(f"words {_hex(a)} {_hex(max(nw, 1))}")
        want.append(_hex(a))
    assert harness(cases) == want


def test_reducer_matches_python(harness):
    """The fixed-modulus reduction used for powers, companions and roots: quotient and remainder
    for every x below its 2^(2 bits(m) + 8) range, modular products and powers, at the library's
    moduli and at random odd ones."""
    rng = random.Random(2)
    mods = [inputs.prime(w).q for w in (64, 128, 256, 384, 512, 768, 1024)]
    mods += [inputs.prime_full(w).q for w in (256, 1024)] + [rng.getrandbits(300) | 1 for _ in range(5)]
    cases, want = [], []
    for m in mods:
        k = 2 * m.bit_length() + 8
        for x in [0, 1, m - 1, m, m + 1, (1 << k) - 1, m * m - 1] + [rng.randrange(1 << k) for _ in range(20)]:
            cases.append(f"red_divmod {_hex(x)} {_hex(m)}")
            want.append(f"{_hex(x // m)} {_hex(x % m)}")
        for _ in range(10):
            a, b, e = rng.randrange(m), rng.randrange(m), rng.getrandbits(rng.randrange(1, 1100))
            cases += [f"mulmod {_hex(a)} {_hex(b)} {_hex(m)}", f"powmod {_hex(a)} {_hex(e)} {_hex(m)}"]
            want += [_hex(a * b % m), _hex(pow(a, e, m))]
    assert harness(cases) == want


def test_primality_matches_sympy(harness):
    rng = random.Random(3)
    ns = [2, 3, 4, 5, 9, 89, 91, 97, 561, 1105, 1729, 2465, 2821, 6601, 8911, 41041, 825265,  # Carmichael
          (1 << 61) - 1, (1 << 89) - 1, (1 << 127) - 1, (1 << 127) + 1]
    ns += [inputs.prime(w).q for w in (64, 128, 256, 384, 512, 768, 1024)]
    ns += [rng.getrandbits(rng.randrange(8, 200)) | 1 for _ in range(300)]
    got = harness([f"prime {_hex(n)}" for n in ns])
    assert got == [str(int(sympy.isprime(n))) for n in ns]
