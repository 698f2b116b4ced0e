"""CPU oracle for multi-word modular arithmetic, the NTT and modular BLAS.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with the
CUDA path (no kernels, headers, tables or constant generators) and never imports it.

Everything here is Python ``int`` arithmetic: exact, plain and slow, written so that a
reader can check each function against the paper.  Where the paper defines a result
exactly (modular add/sub/mul, the NTT sum), the oracle is that definition written out,
not the word-level algorithm that the GPU runs.

Citations are to the paper "Code Generation for Cryptographic Kernels using
Multi-word Modular Arithmetic on GPU" (Zhang & Franchetti, CGO'25).

Readings where the paper is silent or inconsistent:
  * addmod subtracts q when a + b >= q (Eq. saddmod prints '>', which would return q
    for a + b == q and leave Z_q); results are always canonical in [0, q).
  * The Barrett shift amount k of Eq. mu is taken as 2*MBITS + 3, matching the
    shifts MBITS-2 and MBITS+5 of Listing 1; MBITS = B, the bit length of q, which is
    W - 4 for a W-bit container (Sec. 5.2).
  * The NTT of Eq. ntt is cyclic; its inverse is x(j) = n^-1 sum_k y(k) w^-jk.
  * The primitive n-th root w_n is derived from q: g = the smallest integer >= 2 that
    is a quadratic non-residue mod q, w_max = g^((q-1)/2^s) (s = 2-adicity of q-1),
    w_n = w_max^(2^s / n).
  * Moduli: q = c * 2^32 + 1 with exactly B bits, c drawn from a seeded generator,
    accepted by Miller-Rabin.
  * Full-width moduli (B = W, Sec. 5.2 names Montgomery reduction for them without detail):
    R = 2^W, REDC taken one 32-bit word at a time with q' = -q^-1 mod 2^32, one final
    conditional subtraction; a product of canonical values is REDC(REDC(a b) (R^2 mod q)).
    The same product is also reached by Eq. barrett with whole-word shifts and the constant
    floor(2^(2W) / q) of one word more than q (barrett_full_steps).
"""
from __future__ import annotations

import random

import numpy as np

# --------------------------------------------------------------------- Sec. 2.1, Eq. (1)

def addmod(a: int, b: int, q: int) -> int:
    """c = a + b mod q (Sec. 2.1, first line of the ring operations)."""
    return (a + b) % q


def submod(a: int, b: int, q: int) -> int:
    """c = a - b mod q (Sec. 2.1)."""
    return (a - b) % q


def mulmod(a: int, b: int, q: int) -> int:
    """c = a * b mod q (Sec. 2.1; Eq. barrett states the same exact result)."""
    return (a * b) % q


def axpy(alpha: int, x: int, y: int, q: int) -> int:
    """y' = alpha * x + y mod q (Sec. 2.3, BLAS-1 axpy over Z_q)."""
    return (alpha * x + y) % q


def vec_addmod(a, b, q):
    return [(x + y) % q for x, y in zip(a, b)]


def vec_submod(a, b, q):
    return [(x - y) % q for x, y in zip(a, b)]


def vec_mulmod(a, b, q):
    return [(x * y) % q for x, y in zip(a, b)]


def vec_axpy(alpha, x, y, q):
    return [(alpha * u + v) % q for u, v in zip(x, y)]


# ---------------------------------------------------- Sec. 2.1 Eq. saddmod / ssubmod

def addmod_by_compare(a: int, b: int, q: int) -> int:
    """Eq. saddmod as a conditional subtraction (with the >= reading)."""
    t = a + b
    return t - q if t >= q else t


def submod_by_compare(a: int, b: int, q: int) -> int:
    """Eq. ssubmod: a - b, plus q when a < b."""
    return a - b + q if a < b else a - b


# ------------------------------------------------- Sec. 3.1, Eq. barrett / Eq. mu, Listing 1

def barrett_mu(q: int, mbits: int) -> int:
    """mu = floor(2^k / q) with k = 2*MBITS + 3 (Eq. mu; k read from Listing 1's shifts)."""
    return (1 << (2 * mbits + 3)) // q


def barrett_mulmod_steps(a: int, b: int, q: int, mbits: int, mu: int | None = None):
    """The Barrett sequence of Sec. 3.1 on unbounded integers.

    t = a*b; r = ((t >> (MBITS-2)) * mu) >> (MBITS+5); t -= r*q; one conditional
    subtraction corrects the under-estimate of floor(ab/q).  Returns (c, t_before) so
    tests can check the invariant 0 <= t_before < 2q that makes one correction enough.
    """
    if mu is None:
        mu = barrett_mu(q, mbits)
    t = a * b
    r = t >> (mbits - 2)
    r *= mu
    r >>= mbits + 5
    t -= r * q
    t_before = t
    c = t - q if t >= q else t
    return c, t_before


def barrett_fixed_steps(a: int, w: int, q: int, width: int):
    """Eq. barrett for a fixed multiplicand w < q, with the quotient constant precomputed for w.

    wp = floor(w 2^W / q) (the companion of w); s = floor(a wp / 2^W) estimates floor(a w / q)
    to within one below it for any a < 2^W, so r = a w - s q lies in [0, 2q).  Returns
    (c, r_before, s) with c = a w mod q.
    """
    wp = (w << width) // q
    s = (a * wp) >> width
    r = a * w - s * q
    r_before = r
    while r >= q:
        r -= q
    return r, r_before, s


# ------------------------------------------------------------------ primes and roots

_SMALL_PRIMES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61,
                 67, 71, 73, 79, 83, 89)


def is_probable_prime(n: int, rng: random.Random | None = None, extra_rounds: int = 16) -> bool:
    """Miller-Rabin with the first 24 primes as bases plus `extra_rounds` random bases."""
    if n < 2:
        return False
    for p in _SMALL_PRIMES:
        if n == p:
            return True
        if n % p == 0:
            return False
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    bases = list(_SMALL_PRIMES)
    if rng is not None:
        bases += [rng.randrange(2, n - 1) for _ in range(extra_rounds)]
    for a in bases:
        x = pow(a, d, n)
        if x == 1 or x == n - 1:
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def gen_prime(width: int, seed: int) -> int:
    """NTT-friendly prime q = c*2^32 + 1 of exactly B = W - 4 bits (Sec. 5.2 bit-width rule).

    c is drawn from random.Random("moma:<W>:<seed>") uniformly in [2^(B-33), 2^(B-32)),
    which puts q in [2^(B-1), 2^B); the first candidate passing Miller-Rabin is taken.
    """
    B = width - 4
    rng = random.Random(f"moma:{width}:{seed}")
    while True:
        c = rng.randrange(1 << (B - 33), 1 << (B - 32))
        q = (c << 32) + 1
        if is_probable_prime(q, rng):
            return q


def two_adicity(q: int) -> int:
    s, d = 0, q - 1
    while d % 2 == 0:
        d //= 2
        s += 1
    return s


def smallest_nonresidue(q: int) -> int:
    """Smallest g >= 2 with g^((q-1)/2) = -1 mod q (Euler's criterion)."""
    g = 2
    while pow(g, (q - 1) // 2, q) != q - 1:
        g += 1
    return g


def root_of_unity(q: int, n: int) -> int:
    """Primitive n-th root of unity w_n for n a power of two dividing q-1 (reading above)."""
    s = two_adicity(q)
    if n < 1 or n & (n - 1) or (1 << s) % n:
        raise ValueError("n must be a power of two dividing q-1")
    g = smallest_nonresidue(q)
    w_max = pow(g, (q - 1) >> s, q)
    return pow(w_max, (1 << s) // n, q)


def inverse(a: int, q: int) -> int:
    return pow(a, -1, q)


# --------------------------------------------------------------------- Sec. 2.3, Eq. ntt

def dft_naive(x, w: int, q: int):
    """y(k) = sum_j x(j) w^(jk) mod q, O(n^2), straight from Eq. ntt."""
    n = len(x)
    y = []
    for k in range(n):
        s = 0
        wk = pow(w, k, q)
        p = 1
        for j in range(n):
            s += x[j] * p
            p = p * wk % q
        y.append(s % q)
    return y


def _bit_reverse_permutation(n: int) -> np.ndarray:
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def ntt_radix2(x, w: int, q: int):
    """Same sum as dft_naive, by the iterative radix-2 Cooley-Tukey algorithm.

    Bit-reversed input order, then log2(n) stages of butterflies (u, v) ->
    (u + w^e v, u - w^e v).  Big-integer work is done on numpy object arrays (the
    library only loops; every value is a Python int).
    """
    n = len(x)
    if n & (n - 1):
        raise ValueError("n must be a power of two")
    a = np.array([int(v) % q for v in x], dtype=object)
    if n == 1:
        return [int(a[0])]
    a = a[_bit_reverse_permutation(n)]
    h = 1
    while h < n:
        # twiddles for blocks of size 2h: w_{2h}^j = w^(j * n / (2h)), j < h
        step = pow(w, n // (2 * h), q)
        tw = np.empty(h, dtype=object)
        t = 1
        for j in range(h):
            tw[j] = t
            t = t * step % q
        a = a.reshape(n // (2 * h), 2, h)
        u = a[:, 0, :]
        v = (a[:, 1, :] * tw[None, :]) % q
        a = np.stack([(u + v) % q, (u - v) % q], axis=1).reshape(n)
        h *= 2
    return [int(v) for v in a]


def ntt_fwd(x, q: int, w: int | None = None):
    """Forward cyclic NTT of Eq. ntt with w = root_of_unity(q, n) unless given."""
    n = len(x)
    if w is None:
        w = root_of_unity(q, n)
    return ntt_radix2(x, w, q)


def ntt_inv(y, q: int, w: int | None = None):
    """Inverse: x(j) = n^-1 sum_k y(k) w^(-jk) mod q."""
    n = len(y)
    if w is None:
        w = root_of_unity(q, n)
    z = ntt_radix2(y, inverse(w, q), q)
    ninv = inverse(n, q)
    return [v * ninv % q for v in z]


def ntt_eval_at(x, q: int, k: int, w: int) -> int:
    """One output y(k) of Eq. ntt by Horner's rule in w^k (O(n); for sampled checks)."""
    wk = pow(w, k, q)
    acc = 0
    for c in reversed(x):
        acc = (acc * wk + c) % q
    return acc


def cyclic_convolution_naive(a, b, q: int):
    """c(m) = sum_{i + j = m mod n} a(i) b(j) mod q: the product of Sec. 2.3 reduced mod x^n - 1."""
    n = len(a)
    c = [0] * n
    for i in range(n):
        ai = a[i]
        if ai == 0:
            continue
        for j in range(n):
            c[(i + j) % n] += ai * b[j]
    return [v % q for v in c]


def polymul_cyclic(a, b, q: int):
    """Cyclic product through the transform: inv(fwd(a) * fwd(b)) (Sec. 2.3)."""
    fa = ntt_fwd(a, q)
    fb = ntt_fwd(b, q)
    return ntt_inv([u * v % q for u, v in zip(fa, fb)], q)


# ------------------------------------------------------------ negacyclic variant
# The ring Z_q[x]/(x^n + 1) of lattice schemes: with psi a primitive 2n-th root of unity
# (psi^2 = w_n), the negacyclic transform evaluates f at the odd powers psi^(2k+1).

def psi_root(q: int, n: int) -> int:
    """Primitive 2n-th root, psi = g^((q-1)/(2n)) (the root_of_unity reading at 2n), psi^2 = w_n."""
    return root_of_unity(q, 2 * n)


def ntt_fwd_negacyclic(x, q: int):
    """y(k) = sum_j x(j) psi^(j(2k+1)) = NTT(x(j) psi^j) with w = psi^2."""
    n = len(x)
    psi = psi_root(q, n)
    pre = [x[j] * pow(psi, j, q) % q for j in range(n)]
    return ntt_radix2(pre, psi * psi % q, q)


def ntt_inv_negacyclic(y, q: int):
    """x(j) = n^-1 psi^-j sum_k y(k) w^(-jk)."""
    n = len(y)
    psi = psi_root(q, n)
    z = ntt_inv(y, q, psi * psi % q)
    psi_inv = inverse(psi, q)
    return [z[j] * pow(psi_inv, j, q) % q for j in range(n)]


def negacyclic_convolution_naive(a, b, q: int):
    """c(m) = sum_{i+j=m} a(i) b(j) - sum_{i+j=m+n} a(i) b(j) mod q: the product mod x^n + 1."""
    n = len(a)
    c = [0] * n
    for i in range(n):
        for j in range(n):
            if i + j < n:
                c[i + j] += a[i] * b[j]
            else:
                c[i + j - n] -= a[i] * b[j]
    return [v % q for v in c]


def polymul_negacyclic(a, b, q: int):
    fa, fb = ntt_fwd_negacyclic(a, q), ntt_fwd_negacyclic(b, q)
    return ntt_inv_negacyclic([u * v % q for u, v in zip(fa, fb)], q)


def polymul_naive(a, b):
    """f(x) g(x) = sum_j sum_i a_i b_(j-i) x^j over the integers (Sec. 2.3)."""
    out = [0] * (len(a) + len(b) - 1)
    for i, ai in enumerate(a):
        for j, bj in enumerate(b):
            out[i + j] += ai * bj
    return out


# ------------------------------------------------------------ full-width moduli, Montgomery
# Sec. 5.2 names Montgomery reduction for moduli that fill their container (B = W bits), where
# the Barrett constants of Sec. 3.1 no longer fit.  R = 2^W.  Montgomery's REDC (T -> T R^-1 mod q
# for T < q R) is taken word by word, 32 bits at a time, in the order of the usual
# operand-scanning form: for each of the L words, m = (T mod 2^32) * q' mod 2^32 with
# q' = -q^-1 mod 2^32, T = (T + m q) / 2^32; one final conditional subtraction.

def gen_prime_full(width: int, seed: int) -> int:
    """NTT-friendly prime q = c*2^32 + 1 of exactly W bits (a full-width modulus).

    c is drawn from random.Random("moma-full:<W>:<seed>") uniformly in [2^(W-33), 2^(W-32)).
    """
    rng = random.Random(f"moma-full:{width}:{seed}")
    while True:
        c = rng.randrange(1 << (width - 33), 1 << (width - 32))
        q = (c << 32) + 1
        if is_probable_prime(q, rng):
            return q


def montgomery_qinv_word(q: int) -> int:
    """q' = -q^-1 mod 2^32 (q odd)."""
    return (-pow(q, -1, 1 << 32)) % (1 << 32)


def montgomery_redc_words(T: int, q: int, width: int, final: bool = True) -> int:
    """T R^-1 mod q for 0 <= T < q R, R = 2^W, one 32-bit word of T per step.

    Without the final subtraction the result lies in [0, 2q)."""
    qi = montgomery_qinv_word(q)
    for _ in range(width // 32):
        m = (T & 0xFFFFFFFF) * qi & 0xFFFFFFFF
        T = (T + m * q) >> 32
    if final and T >= q:
        T -= q
    return T


def montgomery_mul(a: int, b: int, q: int, width: int) -> int:
    """a b R^-1 mod q for canonical a, b (REDC of the full product)."""
    return montgomery_redc_words(a * b, q, width)


def mulmod_via_montgomery(a: int, b: int, q: int, width: int) -> int:
    """a b mod q as two Montgomery products: REDC(REDC(a b) (R^2 mod q))."""
    r2 = (1 << (2 * width)) % q
    return montgomery_mul(montgomery_mul(a, b, q, width), r2, q, width)


# Eq. barrett for a full-width modulus, with the shifts taken as whole words: base 2^w, q of L
# words whose top word is nonzero, mu = floor(2^(2Lw) / q) (one word longer than q).

def barrett_full_steps(a: int, b: int, q: int, limbs: int, word_bits: int = 32):
    """a b mod q by the whole-word Barrett sequence; returns (c, r_before, s).

    t = a b; q1 = t >> (L-1) words; s = (q1 * mu) >> (L+1) words; r = t - s q; q is subtracted
    while r >= q.  s is floor(t / q) or up to two less, so r_before lies in [0, 3q).
    """
    mu = (1 << (2 * limbs * word_bits)) // q
    t = a * b
    q1 = t >> ((limbs - 1) * word_bits)
    s = (q1 * mu) >> ((limbs + 1) * word_bits)
    r = t - s * q
    r_before = r
    while r >= q:
        r -= q
    return r, r_before, s
