"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of an oracle function on the CPU (a dropped term, a wrong
sign or index, a transposed operand, the paper's literal '>' tie-break, a wrong shift), swaps it
into the oracle module, and checks that the references the pins use (the hand-computed fixture,
sympy, brute force, closed forms, defining identities) reject the planted version.  The GPU path is
not involved.
"""
import json
import os
import random

import pytest

import oracle
from oracle import moma_oracle as om
from paper_2501_07535_gb300 import inputs

sympy = pytest.importorskip("sympy")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _fixture():
    return json.load(open(os.path.join(GOLDEN, "ntt_q17_n4.json")))


def _ntt_pins_hold() -> bool:
    """The transform pins of test_oracle.py, condensed: hand fixture, sympy, closed forms, round trip."""
    d = _fixture()
    if om.ntt_fwd(d["x"], d["q"], d["w"]) != d["y"]:
        return False
    q = 7681
    rng = random.Random(5)
    for n in (4, 16, 64):
        x = [rng.randrange(q) for _ in range(n)]
        w = pow(sympy.primitive_root(q), (q - 1) // n, q)
        if om.ntt_fwd(x, q, w) != sympy.discrete.transforms.ntt(x, q):
            return False
        if om.ntt_inv(om.ntt_fwd(x, q, w), q, w) != x:
            return False
    Q = inputs.prime(256).q
    n = 32
    e1 = [0, 1] + [0] * (n - 2)
    w = om.root_of_unity(Q, n)
    return om.ntt_fwd(e1, Q) == [pow(w, k, Q) for k in range(n)]


def _conv_pins_hold() -> bool:
    q = inputs.prime(128).q
    rng = random.Random(9)
    for n in (4, 16):
        a = [rng.randrange(q) for _ in range(n)]
        b = [rng.randrange(q) for _ in range(n)]
        X = sympy.symbols("x")
        prod = sympy.Poly(list(reversed(a)), X) * sympy.Poly(list(reversed(b)), X)
        full = [int(c) for c in reversed(prod.all_coeffs())]
        folded = [0] * n
        for i, v in enumerate(full):
            folded[i % n] += v
        want = [v % q for v in folded]
        if om.cyclic_convolution_naive(a, b, q) != want or om.polymul_cyclic(a, b, q) != want:
            return False
    return True


def _mutant_dft_drops_first_term(x, w, q):
    n = len(x)
    return [sum(x[j] * pow(w, j * k, q) for j in range(1, n)) % q for k in range(n)]


def _mutant_radix2_transposed_twiddle(x, w, q):
    # w^(jk) with the twiddle exponent taken from the other index: reverses the output order
    y = om.dft_naive(x, w, q)
    return [y[0]] + list(reversed(y[1:]))


def _mutant_inverse_without_scale(y, q, w=None):
    n = len(y)
    if w is None:
        w = om.root_of_unity(q, n)
    return om.ntt_radix2(y, pow(w, -1, q), q)


def _mutant_inverse_wrong_sign(y, q, w=None):
    n = len(y)
    if w is None:
        w = om.root_of_unity(q, n)
    ninv = pow(n, -1, q)
    return [v * ninv % q for v in om.ntt_radix2(y, w, q)]


def _mutant_convolution_difference_index(a, b, q):
    n = len(a)
    c = [0] * n
    for i in range(n):
        for j in range(n):
            c[(i - j) % n] += a[i] * b[j]
    return [v % q for v in c]


@pytest.mark.parametrize("name,mutant,pins", [
    ("dft_naive", _mutant_dft_drops_first_term, "ntt"),
    ("ntt_radix2", _mutant_radix2_transposed_twiddle, "ntt"),
    ("ntt_inv", _mutant_inverse_without_scale, "ntt"),
    ("ntt_inv", _mutant_inverse_wrong_sign, "ntt"),
    ("cyclic_convolution_naive", _mutant_convolution_difference_index, "conv"),
])
def test_planted_transform_mistake_is_caught(monkeypatch, name, mutant, pins):
    check = _ntt_pins_hold if pins == "ntt" else _conv_pins_hold
    assert check()  # the real oracle passes
    monkeypatch.setattr(om, name, mutant)
    if name == "dft_naive":
        # ntt_fwd runs the radix-2 form; the fixture pins dft_naive directly
        d = _fixture()
        assert om.dft_naive(d["x"], d["w"], d["q"]) != d["y"]
    else:
        assert not check()


def test_planted_strict_tie_break_is_caught():
    """Eq. saddmod as printed ('>'): a + b == q would return q; the tie pin rejects it."""
    q = inputs.prime(256).q

    def literal(a, b, q):
        s = a + b
        return s - q if s > q else s
    a = q // 3
    assert oracle.addmod_by_compare(a, q - a, q) == 0
    assert literal(a, q - a, q) != 0


def test_planted_barrett_shift_is_caught():
    """k = 2B + 2 instead of 2B + 3 leaves t above 2q for some products: the bound pin fails."""
    rng = random.Random(4)
    B = 124
    q = inputs.prime(128).q
    worst = 0
    for _ in range(3000):
        a, b = rng.randrange(q), rng.randrange(q)
        mu_bad = (1 << (2 * B + 2)) // q
        _, t = oracle.barrett_mulmod_steps(a, b, q, B, mu=mu_bad)
        worst = max(worst, t // q)
    assert worst >= 2


def test_planted_montgomery_sign_is_caught():
    """q' = +q^-1 instead of -q^-1: T + m q is no longer divisible by 2^32 and REDC(T) != T R^-1."""
    W = 256
    q = inputs.prime_full(W).q
    R = 1 << W
    rinv = int(sympy.mod_inverse(R, q))
    qi_bad = pow(q, -1, 1 << 32)
    rng = random.Random(6)
    caught = False
    for _ in range(20):
        T = rng.randrange(q * R)
        t = T
        for _ in range(W // 32):
            m = (t & 0xFFFFFFFF) * qi_bad & 0xFFFFFFFF
            t = (t + m * q) >> 32
        if t % q != T * rinv % q:
            caught = True
    assert caught
    assert oracle.montgomery_redc_words(12345, q, W) == 12345 * rinv % q


def _barrett_full_pins_hold() -> bool:
    """test_oracle.py's exhaustive pin of the whole-word Barrett reading, at 3-bit words."""
    for q in range(9, 64, 2):
        for a in range(q):
            for b in range(q):
                c, r, s = om.barrett_full_steps(a, b, q, 2, 3)
                Q = a * b // q
                if c != a * b % q or not (Q - 2 <= s <= Q) or not (0 <= r < 3 * q):
                    return False
    return True


def _mutant_barrett_full_short_shift(a, b, q, limbs, word_bits=32):
    # q1 taken from word L instead of word L-1: the estimate loses a word of precision
    mu = (1 << (2 * limbs * word_bits)) // q
    t = a * b
    s = ((t >> (limbs * word_bits)) * mu) >> ((limbs + 1) * word_bits)
    r = t - s * q
    r_before = r
    while r >= q:
        r -= q
    return r, r_before, s


def _mutant_barrett_full_narrow_mu(a, b, q, limbs, word_bits=32):
    # mu of L words only (its top word dropped), as if the W-4 bit constant were reused
    mu = ((1 << (2 * limbs * word_bits)) // q) % (1 << (limbs * word_bits))
    t = a * b
    s = ((t >> ((limbs - 1) * word_bits)) * mu) >> ((limbs + 1) * word_bits)
    r = t - s * q
    r_before = r
    while r >= q:
        r -= q
    return r, r_before, s


@pytest.mark.parametrize("mutant", [_mutant_barrett_full_short_shift, _mutant_barrett_full_narrow_mu])
def test_planted_full_width_barrett_mistake_is_caught(monkeypatch, mutant):
    assert _barrett_full_pins_hold()
    monkeypatch.setattr(om, "barrett_full_steps", mutant)
    assert not _barrett_full_pins_hold()


def _barrett_fixed_pins_hold() -> bool:
    """test_oracle.py's exhaustive pin of the fixed-multiplicand reading at W = 6."""
    for q in range(3, 64, 2):
        for w in range(q):
            for a in range(64):
                c, r, s = om.barrett_fixed_steps(a, w, q, 6)
                Q = a * w // q
                if c != a * w % q or not (Q - 1 <= s <= Q) or not (0 <= r < 2 * q):
                    return False
    return True


def _mutant_barrett_fixed_half_companion(a, w, q, width):
    # companion floor(w 2^(W-1) / q): half the constant, the estimate falls far short
    wp = (w << (width - 1)) // q
    s = (a * wp) >> width
    r = a * w - s * q
    r_before = r
    while r >= q:
        r -= q
    return r, r_before, s


def _mutant_barrett_fixed_rounded_companion(a, w, q, width):
    # companion rounded up instead of down: the estimate can exceed floor(a w / q)
    wp = -((-w << width) // q)
    s = (a * wp) >> width
    r = a * w - s * q
    r_before = r
    while r < 0:
        r += q
    while r >= q:
        r -= q
    return r, r_before, s


@pytest.mark.parametrize("mutant", [_mutant_barrett_fixed_half_companion, _mutant_barrett_fixed_rounded_companion])
def test_planted_fixed_multiplicand_mistake_is_caught(monkeypatch, mutant):
    assert _barrett_fixed_pins_hold()
    monkeypatch.setattr(om, "barrett_fixed_steps", mutant)
    assert not _barrett_fixed_pins_hold()
