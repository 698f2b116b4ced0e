"""Pins for the CPU oracle: checks against things other than itself.

Each test fixes the oracle to a value the paper prints, a closed form, an invariant,
a special case that reduces to a library routine (sympy), or brute force on tiny
inputs, so that a dropped term, a wrong sign/index or a transposed operand in the
oracle fails at least one of them.
"""
import json
import os
import random

import numpy as np
import pytest

import oracle
from paper_2501_07535_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sympy = pytest.importorskip("sympy")

# NTT-friendly small/medium primes whose q-1 sympy can factor (so primitive_root works)
SMALL_PRIMES = [17, 97, 257, 7681, 12289, 65537, 998244353, 2**64 - 2**32 + 1]


def _rand_vec(rng, n, q):
    return [rng.randrange(q) for _ in range(n)]


# ------------------------------------------------------------------ primes / moduli

def test_primes_table_is_prime_and_shaped():
    table = inputs.load_primes()
    assert len(table) == 28
    for (w, s), p in table.items():
        assert sympy.isprime(p.q), (w, s)
        assert p.q.bit_length() == w - 4 == p.bits          # Sec. 5.2: W-4 bit modulus
        assert (p.q - 1) % (1 << 32) == 0 and p.two_adicity >= 32
        assert oracle.two_adicity(p.q) == p.two_adicity


def test_primes_table_regenerates_from_oracle():
    table = inputs.load_primes()
    for w in (64, 128, 256, 384, 512, 768, 1024):
        assert oracle.gen_prime(w, 0) == table[(w, 0)].q


def test_package_prime_table_is_the_oracle_scripts_output():
    """The library's table (paper_2501_07535_gb300/primes.json) is exactly what the oracle-only
    script writes: every entry, both tables."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_primes", os.path.join(os.path.dirname(__file__), "golden",
                                                                             "make_primes.py"))
    mp = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mp)
    assert mp.TABLE == inputs.PRIMES_JSON
    assert mp.main(["--check"]) == 0


def test_miller_rabin_matches_sympy():
    rng = random.Random(7)
    for _ in range(300):
        n = rng.randrange(3, 1 << 80) | 1
        assert oracle.is_probable_prime(n, rng) == sympy.isprime(n)
    # Carmichael numbers and prime powers
    for n in (561, 1105, 1729, 2465, 2821, 6601, 8911, 3 ** 20, 7 ** 11, 2 ** 61 - 1, 2 ** 89 - 1):
        assert oracle.is_probable_prime(n, rng) == sympy.isprime(n)


# ------------------------------------------------------------------ roots of unity

@pytest.mark.parametrize("width", [64, 128, 256, 384, 512, 768, 1024])
def test_root_is_primitive_for_all_supported_sizes(width):
    q = inputs.prime(width).q
    for lg in range(1, 25):
        n = 1 << lg
        w = oracle.root_of_unity(q, n)
        assert pow(w, n, q) == 1
        assert pow(w, n // 2, q) == q - 1          # hence order exactly n
    # consistency across sizes: w_{n/2} = w_n^2
    assert pow(oracle.root_of_unity(q, 1 << 20), 2, q) == oracle.root_of_unity(q, 1 << 19)


@pytest.mark.parametrize("width", [64, 128, 256, 384, 512, 768, 1024])
def test_generator_is_smallest_nonresidue(width):
    q = inputs.prime(width).q
    g = oracle.smallest_nonresidue(q)
    assert sympy.legendre_symbol(g, q) == -1
    for h in range(2, g):
        assert sympy.legendre_symbol(h, q) == 1


# ------------------------------------------------------------------ the NTT sum

def test_golden_hand_example():
    d = json.load(open(os.path.join(GOLDEN, "ntt_q17_n4.json")))
    assert oracle.dft_naive(d["x"], d["w"], d["q"]) == d["y"]
    assert oracle.ntt_radix2(d["x"], d["w"], d["q"]) == d["y"]
    assert oracle.ntt_inv(d["y"], d["q"], d["w"]) == d["x"]


@pytest.mark.parametrize("q", SMALL_PRIMES)
def test_ntt_matches_sympy(q):
    rng = random.Random(q)
    for lg in range(0, 9):
        n = 1 << lg
        if (q - 1) % n:
            continue
        x = _rand_vec(rng, n, q)
        ref = sympy.discrete.transforms.ntt(x, q)
        pr = sympy.primitive_root(q)
        w = pow(pr, (q - 1) // n, q)
        assert oracle.dft_naive(x, w, q) == ref
        assert oracle.ntt_radix2(x, w, q) == ref
        assert oracle.ntt_inv(ref, q, w) == [v % q for v in x]
        assert oracle.ntt_inv(ref, q, w) == sympy.discrete.transforms.intt(ref, q)


@pytest.mark.parametrize("width", [64, 128, 256, 384, 512, 768, 1024])
def test_fast_ntt_matches_brute_force(width):
    q = inputs.prime(width).q
    rng = random.Random(width)
    for lg in (1, 2, 3, 5, 7):
        n = 1 << lg
        x = _rand_vec(rng, n, q)
        w = oracle.root_of_unity(q, n)
        assert oracle.ntt_fwd(x, q) == oracle.dft_naive(x, w, q)


@pytest.mark.parametrize("width", [128, 256])
def test_ntt_special_inputs(width):
    q = inputs.prime(width).q
    n = 64
    w = oracle.root_of_unity(q, n)
    e0 = [1] + [0] * (n - 1)
    e1 = [0, 1] + [0] * (n - 2)
    ones = [1] * n
    assert oracle.ntt_fwd(e0, q) == ones
    assert oracle.ntt_fwd(ones, q) == [n] + [0] * (n - 1)
    assert oracle.ntt_fwd(e1, q) == [pow(w, k, q) for k in range(n)]
    # a shifted delta picks out the row w^(jk) of Eq. ntt
    e5 = [0] * n
    e5[5] = 1
    assert oracle.ntt_fwd(e5, q) == [pow(w, 5 * k, q) for k in range(n)]


def test_ntt_linearity_and_roundtrip():
    q = inputs.prime(256).q
    rng = random.Random(3)
    n = 1 << 10
    a, b = _rand_vec(rng, n, q), _rand_vec(rng, n, q)
    c = rng.randrange(q)
    fa, fb = oracle.ntt_fwd(a, q), oracle.ntt_fwd(b, q)
    lhs = oracle.ntt_fwd([(c * u + v) % q for u, v in zip(a, b)], q)
    assert lhs == [(c * u + v) % q for u, v in zip(fa, fb)]
    assert oracle.ntt_inv(fa, q) == a


def test_horner_sample_matches_transform():
    q = inputs.prime(384).q
    rng = random.Random(5)
    n = 256
    x = _rand_vec(rng, n, q)
    w = oracle.root_of_unity(q, n)
    y = oracle.ntt_fwd(x, q)
    for k in (0, 1, 2, 77, 128, 255):
        assert oracle.ntt_eval_at(x, q, k, w) == y[k]


# ------------------------------------------------------------------ polynomial products

def test_convolution_theorem():
    q = inputs.prime(256).q
    rng = random.Random(11)
    for n in (2, 8, 64, 256):
        a, b = _rand_vec(rng, n, q), _rand_vec(rng, n, q)
        naive = oracle.cyclic_convolution_naive(a, b, q)
        assert oracle.polymul_cyclic(a, b, q) == naive
        # numpy's exact object-dtype convolution, folded mod x^n - 1
        full = np.convolve(np.array(a, dtype=object), np.array(b, dtype=object))
        folded = [0] * n
        for i, v in enumerate(full):
            folded[i % n] += int(v)
        assert naive == [v % q for v in folded]


def test_polymul_naive_matches_sympy_poly():
    rng = random.Random(13)
    a = [rng.randrange(1 << 100) for _ in range(9)]
    b = [rng.randrange(1 << 100) for _ in range(6)]
    X = sympy.symbols("X")
    pa = sympy.Poly(list(reversed(a)), X)
    pb = sympy.Poly(list(reversed(b)), X)
    assert oracle.polymul_naive(a, b) == [int(c) for c in reversed((pa * pb).all_coeffs())]


# ------------------------------------------------------------------ negacyclic transforms

@pytest.mark.parametrize("width", [128, 256, 384, 768])
def test_negacyclic_transform_evaluates_at_odd_powers(width):
    q = inputs.prime(width).q
    rng = random.Random(width + 9)
    for lg in (1, 3, 6):
        n = 1 << lg
        x = _rand_vec(rng, n, q)
        psi = oracle.psi_root(q, n)
        assert pow(psi, 2 * n, q) == 1 and pow(psi, n, q) == q - 1
        y = oracle.ntt_fwd_negacyclic(x, q)
        for k in range(n):
            assert y[k] == oracle.ntt_eval_at(x, q, 1, pow(psi, 2 * k + 1, q))  # f(psi^(2k+1))
        assert oracle.ntt_inv_negacyclic(y, q) == x


def test_negacyclic_convolution():
    q = inputs.prime(256).q
    rng = random.Random(21)
    for n in (2, 8, 64):
        a, b = _rand_vec(rng, n, q), _rand_vec(rng, n, q)
        naive = oracle.negacyclic_convolution_naive(a, b, q)
        assert oracle.polymul_negacyclic(a, b, q) == naive
        # the full product over the integers, reduced with x^n = -1
        full = oracle.polymul_naive(a, b)
        red = [0] * n
        for i, v in enumerate(full):
            red[i % n] += v if i < n else -v
        assert naive == [v % q for v in red]
    # x^(n-1) * x = x^n = -1
    n = 8
    e = [0] * n
    e[n - 1] = 1
    x1 = [0, 1] + [0] * (n - 2)
    assert oracle.polymul_negacyclic(e, x1, q) == [q - 1] + [0] * (n - 1)


# ------------------------------------------------------------------ elementwise ops

@pytest.mark.parametrize("width", [128, 256, 384, 768])
def test_elementwise_ops_invariants(width):
    q = inputs.prime(width).q
    rng = random.Random(width + 1)
    edge = [0, 1, 2, q - 1, q - 2, q // 2, (q + 1) // 2, (1 << 32) - 1, (1 << 64) - 1]
    vals = edge + _rand_vec(rng, 40, q)
    for a in vals:
        inv = int(sympy.mod_inverse(a, q)) if a else None
        if inv is not None:
            assert oracle.mulmod(a, inv, q) == 1
        # a + (q - a) = 0 and the tie a + b == q must not return q (addmod reading)
        assert oracle.addmod(a, (q - a) % q, q) == 0
        assert oracle.addmod_by_compare(a, (q - a) % q, q) == 0
        for b in vals[:12]:
            s = oracle.addmod(a, b, q)
            assert 0 <= s < q and oracle.submod(s, b, q) == a
            assert oracle.addmod_by_compare(a, b, q) == s
            assert oracle.submod_by_compare(a, b, q) == oracle.submod(a, b, q)
            assert oracle.submod(a, b, q) == oracle.addmod(a, (q - b) % q, q)
            assert oracle.axpy(a, b, s, q) == oracle.addmod(oracle.mulmod(a, b, q), s, q)
    # Fermat: a^(q-1) = 1 by square-and-multiply over the oracle's mulmod
    for a in vals[1:6]:
        r, base, e = 1, a, q - 1
        while e:
            if e & 1:
                r = oracle.mulmod(r, base, q)
            base = oracle.mulmod(base, base, q)
            e >>= 1
        assert r == 1
    # distributivity ties mulmod to addmod
    for _ in range(50):
        a, b, c = _rand_vec(rng, 3, q)
        assert oracle.mulmod(a, oracle.addmod(b, c, q), q) == \
            oracle.addmod(oracle.mulmod(a, b, q), oracle.mulmod(a, c, q), q)


def test_vector_forms_match_scalar_forms():
    q = inputs.prime(256).q
    rng = random.Random(17)
    a, b = _rand_vec(rng, 33, q), _rand_vec(rng, 33, q)
    al = rng.randrange(q)
    assert oracle.vec_addmod(a, b, q) == [oracle.addmod(x, y, q) for x, y in zip(a, b)]
    assert oracle.vec_submod(a, b, q) == [oracle.submod(x, y, q) for x, y in zip(a, b)]
    assert oracle.vec_mulmod(a, b, q) == [oracle.mulmod(x, y, q) for x, y in zip(a, b)]
    assert oracle.vec_axpy(al, a, b, q) == [oracle.axpy(al, x, y, q) for x, y in zip(a, b)]


# ------------------------------------------------------------------ Barrett (Sec. 3.1)

@pytest.mark.parametrize("width", [64, 128, 256, 384, 512, 768, 1024])
def test_barrett_steps_exact_and_one_correction(width):
    B = width - 4
    rng = random.Random(width)
    qs = [rng.randrange(1 << (B - 1), 1 << B) | 1 for _ in range(8)]
    qs.append(inputs.prime(width).q)
    for q in qs:
        mu = oracle.barrett_mu(q, B)
        assert mu < (1 << width)                # mu fits the W-bit container
        for _ in range(400):
            a, b = rng.randrange(q), rng.randrange(q)
            c, t = oracle.barrett_mulmod_steps(a, b, q, B, mu)
            assert c == a * b % q
            assert 0 <= t < 2 * q               # one conditional subtraction suffices
        for a, b in ((q - 1, q - 1), (0, q - 1), (1, 1)):
            c, t = oracle.barrett_mulmod_steps(a, b, q, B, mu)
            assert c == a * b % q and 0 <= t < 2 * q


def test_barrett_needs_full_bit_length():
    # With q two bits shorter than MBITS the estimate can be off by two (reading of Sec. 5.2:
    # q must have exactly MBITS bits for the single correction of Listing 1).
    B = 60
    rng = random.Random(1)
    worst = 0
    for _ in range(20):
        q = rng.randrange(1 << (B - 3), 1 << (B - 2)) | 1
        for _ in range(2000):
            a, b = rng.randrange(q), rng.randrange(q)
            _, t = oracle.barrett_mulmod_steps(a, b, q, B)
            worst = max(worst, t // q)
    assert worst >= 2


# ------------------------------------------------------------------ full-width moduli (Montgomery)

def test_full_width_primes_table():
    table = inputs.load_full_primes()
    assert len(table) == 14
    for (w, s), p in table.items():
        assert sympy.isprime(p.q), (w, s)
        assert p.q.bit_length() == w == p.bits                 # fills the container
        assert (p.q - 1) % (1 << 32) == 0 and p.two_adicity >= 32
        assert oracle.gen_prime_full(w, s) == p.q


@pytest.mark.parametrize("width", [64, 128, 256, 384, 512, 768, 1024])
def test_montgomery_redc_is_multiplication_by_r_inverse(width):
    """REDC(T) = T R^-1 mod q (sympy's modular inverse), below 2q before its correction."""
    R = 1 << width
    rng = random.Random(width)
    for q in (inputs.prime_full(width).q, inputs.prime_full(width, 1).q, inputs.prime(width).q):
        rinv = int(sympy.mod_inverse(R, q))
        qi = oracle.montgomery_qinv_word(q)
        assert (q * qi + 1) % (1 << 32) == 0
        for T in [0, 1, q - 1, q, q * R - 1, (q - 1) * (q - 1)] + [rng.randrange(q * R) for _ in range(200)]:
            raw = oracle.montgomery_redc_words(T, q, width, final=False)
            assert 0 <= raw < 2 * q
            r = oracle.montgomery_redc_words(T, q, width)
            assert r == T * rinv % q
            assert (r * R - T) % q == 0


@pytest.mark.parametrize("width", [128, 256, 384, 768])
def test_mulmod_via_montgomery_is_the_product(width):
    rng = random.Random(3 * width)
    q = inputs.prime_full(width).q
    edge = [0, 1, 2, q - 1, q - 2, (1 << (width - 1)) % q, q // 2]
    pairs = [(a, b) for a in edge for b in edge] + [(rng.randrange(q), rng.randrange(q)) for _ in range(300)]
    for a, b in pairs:
        assert oracle.mulmod_via_montgomery(a, b, q, width) == a * b % q
        assert oracle.montgomery_mul(a, b, q, width) == a * b * int(sympy.mod_inverse(1 << width, q)) % q


@pytest.mark.parametrize("width,step", [(6, 1), (8, 7)])
def test_barrett_fixed_exhaustive_on_small_widths(width, step):
    """The fixed-multiplicand reading on every a < 2^W and w < q for odd q < 2^W (every
    `step`-th): a w mod q, a quotient estimate at most one below floor(a w / q), hence a value
    below 2q before the subtractions (the kernels' truncated estimate may take one more)."""
    worst = 0
    for q in range(3, 1 << width, 2 * step):
        for w in range(q):
            for a in range(1 << width):
                c, r, s = oracle.barrett_fixed_steps(a, w, q, width)
                Q = a * w // q
                assert c == a * w % q and Q - 1 <= s <= Q and 0 <= r < 2 * q, (q, w, a)
                worst = max(worst, Q - s)
    assert worst == 1


@pytest.mark.parametrize("width", [64, 128, 256, 384, 512, 768, 1024])
def test_barrett_fixed_at_machine_words(width):
    """(W-4)-bit test primes, multiplicands w < q (edge and random), operands a over all of
    [0, 2^W) as in the transforms' lazy values."""
    rng = random.Random(width + 29)
    q = inputs.prime(width).q
    ws = [0, 1, q - 1, q // 2] + [rng.randrange(q) for _ in range(20)]
    As = [0, 1, q - 1, 4 * q - 1, (1 << width) - 1] + [rng.randrange(1 << width) for _ in range(40)]
    for w in ws:
        for a in As:
            c, r, s = oracle.barrett_fixed_steps(a, w, q, width)
            Q = a * w // q
            assert c == a * w % q and Q - 1 <= s <= Q and 0 <= r < 2 * q


@pytest.mark.parametrize("word_bits,limbs,step", [(3, 2, 1), (4, 2, 7), (3, 3, 23)])
def test_barrett_full_exhaustive_on_small_words(word_bits, limbs, step):
    """The whole-word Barrett reading on every a, b < q for odd moduli of `limbs` words of
    `word_bits` bits with a nonzero top word (every `step`-th such modulus): the exact product,
    a quotient estimate within 2 below floor(a b / q), hence a value below 3q before the
    subtractions.  (For a b < q^2 these sizes never show an estimate 2 short: the bound is not
    tight here.)"""
    base = 1 << word_bits
    worst = 0
    for q in range(base ** (limbs - 1) + 1, base ** limbs, 2 * step):
        for a in range(q):
            for b in range(a, q):
                c, r, s = oracle.barrett_full_steps(a, b, q, limbs, word_bits)
                Q = a * b // q
                assert c == a * b % q and Q - 2 <= s <= Q and 0 <= r < 3 * q, (q, a, b)
                worst = max(worst, Q - s)
    assert worst >= 1  # the estimate does fall short: the subtractions are needed


@pytest.mark.parametrize("width", [64, 128, 256, 384, 512, 768, 1024])
def test_barrett_full_at_machine_words(width):
    """32-bit words at every container width: moduli with top word 1, 2^W - 1 and the full-width
    test prime; edge and random operands."""
    rng = random.Random(width + 17)
    L = width // 32
    for q in ((1 << (width - 32)) + 12345, (1 << width) - 1, inputs.prime_full(width).q):
        edge = [0, 1, q - 1, q - 2, q // 2, (1 << (width - 32)) - 1, (1 << (width - 1)) % q]
        pairs = [(a, b) for a in edge for b in edge] + [(rng.randrange(q), rng.randrange(q)) for _ in range(200)]
        for a, b in pairs:
            c, r, s = oracle.barrett_full_steps(a, b, q, L)
            Q = a * b // q
            assert c == a * b % q and Q - 2 <= s <= Q and 0 <= r < 3 * q


def test_full_width_transform_roots():
    for w in (64, 128, 256, 384, 512, 768, 1024):
        q = inputs.prime_full(w).q
        for lg in (1, 12, 24):
            n = 1 << lg
            wn = oracle.root_of_unity(q, n)
            assert pow(wn, n, q) == 1 and pow(wn, n // 2, q) == q - 1


# ------------------------------------------------------------------ representation

def test_digit_order_fixture():
    d = json.load(open(os.path.join(GOLDEN, "digits.json")))
    digits, z = d["digits_msb_first"], d["z"]
    n = len(digits)
    assert sum(x * z ** (n - 1 - i) for i, x in enumerate(digits)) == d["value"]
    # the same reading with z = 2^32: paper order is most significant first, memory is LSW first
    x0, x1 = 0xDEADBEEF, 0x01234567
    assert inputs.limbs_to_int([x1, x0]) == x0 * 2 ** 32 + x1


def test_inputs_residues_uniform_and_deterministic():
    q = inputs.prime(256).q
    a = inputs.residues(q, 8, 4096, seed=1)
    b = inputs.residues(q, 8, 4096, seed=1)
    assert np.array_equal(a, b)
    vals = inputs.to_ints(a)
    assert all(0 <= v < q for v in vals)
    assert inputs.to_ints(inputs.from_ints(vals, 8)) == vals
    mean = sum(vals) / len(vals)
    assert abs(mean / q - 0.5) < 0.03
    # top bits are exercised (values above q/2 and near q appear)
    assert max(vals) > q * 0.99
