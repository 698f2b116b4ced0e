// moma_limbs.cuh -- multi-word modular arithmetic on 32-bit machine words (device code).
//
// A residue of a W-bit container is L = W/32 words x[0..L), x[0] least significant
// (Sec. 3, Eq. def_moma writes the same words most significant first).  The modulus q
// has exactly B = W - 4 bits (Sec. 5.2), which leaves 4 bits of headroom in the top word:
// a sum of two residues never carries out of the container, so the carry word of rule
// (moddq_add) is always zero here and is not materialised.
//
// Word-level building blocks follow the rewrite rules of Table 1:
//   (addqdd)+(adc)  multi-word addition        -> add_words  (one add.cc/addc.cc chain)
//   (subddd)        multi-word subtraction     -> sub_words  (one sub.cc/subc.cc chain)
//   (ltd)+(eqd)     multi-word comparison      -> the borrow out of sub_words
//   (moddq_add)     reduction after an add     -> cond_sub
//   (mulqdd)+(addqqq) schoolbook multiplication -> mul_full / mul_lo_acc / mul_hi_trunc
// add_words/sub_words are written as the recursion the paper formalises (Sec. 3.2 "MoMA
// via recursion"): split the operand into a low and a high part, process the low part,
// feed its carry into the high part, and recurse until one machine word remains.  For a
// width that is not a power of two (384, 768 bits) the split takes the largest power of
// two below L for the low part, which is the zero-word pruning of Sec. 4
// ("Non-power-of-two input bit-widths") done at compile time.
//
// Products use operand scanning: row i adds x_i * y into the accumulator with one
// mad.lo.cc chain (low halves of the word products) and one mad.hi.cc chain (high
// halves).  The leaves of rule (mulqdd)'s recursion are exactly these L^2 word products;
// the GPU's multiply-add-with-carry performs the additions of rules (addqdd)/(addqqq) in
// the same instruction, so no separate addition chains are emitted.
//
// Every statement that reads or writes the PTX carry flag is `asm volatile`, which keeps
// the chains in program order in the front end; ptxas tracks the carry dependency.

#pragma once
#include <stdint.h>

#ifndef MOMA_DEV
#define MOMA_DEV __device__ __forceinline__
#endif

namespace moma {

// ------------------------------------------------------------------ PTX carry primitives
#ifndef MOMA_HOST_PRIMITIVES
MOMA_DEV uint32_t add_cc(uint32_t a, uint32_t b) {
  uint32_t r; asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
MOMA_DEV uint32_t addc_cc(uint32_t a, uint32_t b) {
  uint32_t r; asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
MOMA_DEV uint32_t addc(uint32_t a, uint32_t b) {
  uint32_t r; asm volatile("addc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
MOMA_DEV uint32_t sub_cc(uint32_t a, uint32_t b) {
  uint32_t r; asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
MOMA_DEV uint32_t subc_cc(uint32_t a, uint32_t b) {
  uint32_t r; asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
MOMA_DEV uint32_t subc(uint32_t a, uint32_t b) {
  uint32_t r; asm volatile("subc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r;
}
// r = lo(a*b) + c, carry out
MOMA_DEV uint32_t mad_lo_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r; asm volatile("mad.lo.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r;
}
MOMA_DEV uint32_t madc_lo_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r; asm volatile("madc.lo.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r;
}
MOMA_DEV uint32_t madc_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r; asm volatile("madc.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r;
}
MOMA_DEV uint32_t mad_hi_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r; asm volatile("mad.hi.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r;
}
MOMA_DEV uint32_t madc_hi_cc(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r; asm volatile("madc.hi.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r;
}
MOMA_DEV uint32_t madc_hi(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r; asm volatile("madc.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r;
}
MOMA_DEV uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) { return a * b + c; }
MOMA_DEV uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c) { return __umulhi(a, b) + c; }
// (hi:lo) >> s for 0 <= s < 32
MOMA_DEV uint32_t shr_pair(uint32_t lo, uint32_t hi, uint32_t s) { return __funnelshift_r(lo, hi, s); }
// whole word product plus a 64-bit addend: a*b + c < 2^64 whenever c < 2^33
MOMA_DEV uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c) {
  uint64_t r; asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(b), "l"(c)); return r;
}
#endif

// Carry (0/1) left in the flag by the last chain.
MOMA_DEV uint32_t carry_out() { return addc(0u, 0u); }
// Borrow mask left by the last subtraction chain: 0xffffffff if it borrowed, else 0.
MOMA_DEV uint32_t borrow_mask() { return subc(0u, 0u); }

// Compile-time loop: f(IntC<i>{}) for i = I..E-1, so that the index can be a template argument.
template <int V>
struct IntC {
  static constexpr int value = V;
};
template <int I, int E, typename F>
MOMA_DEV void static_for(F&& f) {
  if constexpr (I < E) {
    f(IntC<I>{});
    static_for<I + 1, E>(static_cast<F&&>(f));
  }
}

// Largest power of two strictly below N (N >= 2): the low part of one recursion step.
template <int N, int P = 1, bool MORE = (P * 2 < N)>
struct LowSplit {
  static constexpr int value = P;
};
template <int N, int P>
struct LowSplit<N, P, true> {
  static constexpr int value = LowSplit<N, P * 2>::value;
};

// ------------------------------------------------------------------ rules (addqdd)/(adc)
// c = a + b over N words; CIN: a carry is pending in the flag from a lower part.
template <int N, bool CIN>
MOMA_DEV void add_words(uint32_t* c, const uint32_t* a, const uint32_t* b) {
  if constexpr (N == 1) {
    c[0] = CIN ? addc_cc(a[0], b[0]) : add_cc(a[0], b[0]);
  } else {
    constexpr int H = LowSplit<N>::value;
    add_words<H, CIN>(c, a, b);
    add_words<N - H, true>(c + H, a + H, b + H);
  }
}

// ------------------------------------------------------------------ rule (subddd)
template <int N, bool BIN>
MOMA_DEV void sub_words(uint32_t* c, const uint32_t* a, const uint32_t* b) {
  if constexpr (N == 1) {
    c[0] = BIN ? subc_cc(a[0], b[0]) : sub_cc(a[0], b[0]);
  } else {
    constexpr int H = LowSplit<N>::value;
    sub_words<H, BIN>(c, a, b);
    sub_words<N - H, true>(c + H, a + H, b + H);
  }
}

// ------------------------------------------------------------------ rule (moddq_add)
// x <- x - m when x >= m; valid for x < 2m.  The comparison of rules (ltd)/(eqd) is the
// borrow of the trial subtraction; the select is per word.
template <int L>
MOMA_DEV void cond_sub(uint32_t (&x)[L], const uint32_t* m) {
  uint32_t d[L];
  sub_words<L, false>(d, x, m);
  const uint32_t keep = borrow_mask();
#pragma unroll
  for (int i = 0; i < L; ++i) x[i] = (x[i] & keep) | (d[i] & ~keep);
}

// c = a + b mod q for canonical a, b (Eq. saddmod with the >= reading).
template <int L>
MOMA_DEV void addmod(uint32_t (&c)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                     const uint32_t* q) {
  add_words<L, false>(c, a, b);
  cond_sub<L>(c, q);
}

// c = a - b mod q for canonical a, b (Eq. ssubmod): add q back when the subtraction borrowed.
template <int L>
MOMA_DEV void submod(uint32_t (&c)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                     const uint32_t* q) {
  sub_words<L, false>(c, a, b);
  const uint32_t m = borrow_mask();
  uint32_t t[L];
#pragma unroll
  for (int i = 0; i < L; ++i) t[i] = q[i] & m;
  add_words<L, false>(c, c, t);
}

// ------------------------------------------------------------------ product rows
// r[k] += lo(x * y[k]), k < N, as one chain.  KEEP: leave the top carry in the flag.
template <int N, bool KEEP>
MOMA_DEV void row_lo(uint32_t* r, uint32_t x, const uint32_t* y) {
  if constexpr (N == 1 && !KEEP) {
    r[0] = mad_lo(x, y[0], r[0]);
  } else {
    r[0] = mad_lo_cc(x, y[0], r[0]);
#pragma unroll
    for (int k = 1; k < N - 1; ++k) r[k] = madc_lo_cc(x, y[k], r[k]);
    if constexpr (N > 1) r[N - 1] = KEEP ? madc_lo_cc(x, y[N - 1], r[N - 1]) : madc_lo(x, y[N - 1], r[N - 1]);
  }
}

// r[k] += hi(x * y[k]), k < N, as one chain.
template <int N, bool KEEP>
MOMA_DEV void row_hi(uint32_t* r, uint32_t x, const uint32_t* y) {
  if constexpr (N == 1 && !KEEP) {
    r[0] = mad_hi(x, y[0], r[0]);
  } else {
    r[0] = mad_hi_cc(x, y[0], r[0]);
#pragma unroll
    for (int k = 1; k < N - 1; ++k) r[k] = madc_hi_cc(x, y[k], r[k]);
    if constexpr (N > 1) r[N - 1] = KEEP ? madc_hi_cc(x, y[N - 1], r[N - 1]) : madc_hi(x, y[N - 1], r[N - 1]);
  }
}

// ------------------------------------------------------------------ Eq. muls, full product
// t[0..2L) = x * y (schoolbook, L^2 word products).
// Invariant before row i: t[0..i+L) holds the partial sum, t[i+L] is free.
template <int L>
MOMA_DEV void mul_full(uint32_t (&t)[2 * L], const uint32_t (&x)[L], const uint32_t (&y)[L]) {
#pragma unroll
  for (int k = 0; k < L; ++k) t[k] = x[0] * y[k];
#pragma unroll
  for (int k = L; k < 2 * L; ++k) t[k] = 0u;
  row_hi<L, false>(t + 1, x[0], y);  // t[L] = hi(x0*y[L-1]) + carry: no carry out
#pragma unroll
  for (int i = 1; i < L; ++i) {
    row_lo<L, true>(t + i, x[i], y);
    t[i + L] = carry_out();
    row_hi<L, false>(t + i + 1, x[i], y);  // ends in t[i+L]; the partial sum fits i+L+1 words
  }
}

// r = r + x * y mod 2^(32L): only the word products below the container's top.
template <int L>
MOMA_DEV void mul_lo_acc(uint32_t (&r)[L], const uint32_t (&x)[L], const uint32_t (&y)[L]) {
  static_for<0, L>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    row_lo<L - i, false>(r + i, x[i], y);
    if constexpr (i < L - 1) row_hi<L - 1 - i, false>(r + i + 1, x[i], y);
  });
}

// H ~= floor(x * y / 2^(32L)) from the columns >= L-1 of the product plus the high halves
// of column L-2.  The dropped part is below 2L * 2^(32(L-1)) < 2^(32L), so H is the exact
// floor or one less.  A[p] holds product word L-1+p, p = 0..L.
template <int L>
MOMA_DEV void mul_hi_trunc(uint32_t (&H)[L], const uint32_t (&x)[L], const uint32_t (&y)[L]) {
  uint32_t A[L + 1];
#pragma unroll
  for (int p = 0; p <= L; ++p) A[p] = 0u;
  // row 0: lo(x0*y[L-1]) at p=0; hi(x0*y[L-2]) at p=0, hi(x0*y[L-1]) at p=1
  A[0] = x[0] * y[L - 1];
  row_hi<2, false>(A, x[0], y + (L - 2));
  static_for<1, L>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    if constexpr (i < L - 1) {
      // lo terms j = L-1-i .. L-1 -> p = 0..i ; hi terms j = L-2-i .. L-1 -> p = 0..i+1
      row_lo<i + 1, true>(A, x[i], y + (L - 1 - i));
      A[i + 1] = carry_out();
      row_hi<i + 2, false>(A, x[i], y + (L - 2 - i));
    } else {
      // last row: lo terms j = 0..L-1 -> p = 0..L-1 ; hi terms -> p = 1..L
      row_lo<L, true>(A, x[i], y);
      A[L] = carry_out();
      row_hi<L, false>(A + 1, x[i], y);
    }
  });
#pragma unroll
  for (int k = 0; k < L; ++k) H[k] = A[k + 1];
}

// ------------------------------------------------------------------ wide-product rows
// The same schoolbook sums as above, with each word product formed whole by mad.wide
// (one 32x32->64 multiply) and the running carry of the row passed through the 64-bit
// addend: t = x*y[j] + acc[j] + c, acc[j] = lo(t), c = hi(t).  On GB300 a whole product
// costs 4 multiply-pipe cycles per warp this way, against ~6 for a mad.lo.cc/madc.hi.cc pair.

// acc[0..N) += x*y[0..N) + cin; returns the carry out of acc[N-1].
template <int N>
MOMA_DEV uint32_t roww(uint32_t* acc, uint32_t x, const uint32_t* y, uint32_t cin) {
  uint32_t c = cin;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const uint64_t t = mad_wide(x, y[j], (uint64_t)acc[j] + c);
    acc[j] = (uint32_t)t;
    c = (uint32_t)(t >> 32);
  }
  return c;
}

// t[0..2L) = x * y.
template <int L>
MOMA_DEV void mul_full_w(uint32_t (&t)[2 * L], const uint32_t (&x)[L], const uint32_t (&y)[L]) {
  uint32_t c = 0;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const uint64_t w = mad_wide(x[0], y[j], (uint64_t)c);
    t[j] = (uint32_t)w;
    c = (uint32_t)(w >> 32);
  }
  t[L] = c;
#pragma unroll
  for (int i = 1; i < L; ++i) t[i + L] = roww<L>(t + i, x[i], y, 0u);
}

// r = r + x * y mod 2^(32L).  Row i: whole products below the top word, then one low
// multiply-add for the top word (its carry is not needed).
template <int L>
MOMA_DEV void mul_lo_acc_w(uint32_t (&r)[L], const uint32_t (&x)[L], const uint32_t (&y)[L]) {
  static_for<0, L>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    uint32_t c = 0;
    if constexpr (L - 1 - i > 0) c = roww<L - 1 - i>(r + i, x[i], y, 0u);
    r[L - 1] = x[i] * y[L - 1 - i] + r[L - 1] + c;
  });
}

// Same quotient estimate as mul_hi_trunc (columns >= L-1 plus the high halves of column L-2).
// Row i starts at j0 = L-2-i: that product only contributes its high word, as carry into
// word L-1; A[p] holds word L-1+p.
template <int L>
MOMA_DEV void mul_hi_trunc_w(uint32_t (&H)[L], const uint32_t (&x)[L], const uint32_t (&y)[L]) {
  uint32_t A[L + 1];
#pragma unroll
  for (int p = 0; p <= L; ++p) A[p] = 0u;
  static_for<0, L>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    if constexpr (i < L - 1) {
      // j0 = L-2-i: high word only; then j = L-1-i .. L-1 land on p = 0 .. i
      const uint64_t t0 = mad_wide(x[i], y[L - 2 - i], 0ull);
      A[i + 1] = roww<i + 1>(A, x[i], y + (L - 1 - i), (uint32_t)(t0 >> 32));
    } else {
      A[L] = roww<L>(A, x[i], y, 0u);
    }
  });
#pragma unroll
  for (int k = 0; k < L; ++k) H[k] = A[k + 1];
}

// ------------------------------------------------------------------ Eq. mulk (Karatsuba)
// t = x * y with three half-size products per level (Sec. 2.2, Eq. mulk):
//   x = x1 z + x0, y = y1 z + y0, z = 2^(32 L/2)
//   p0 = x0 y0, p2 = x1 y1, p1 = (x0 + x1)(y0 + y1), t = p0 + (p1 - p0 - p2) z + p2 z^2.
// The half sums carry one extra bit each (cx, cy): p1 = sx sy + (cx sy + cy sx) z + cx cy z^2.
// Recursion stops at KBASE limbs (schoolbook carry chains) or at an odd limb count.
constexpr int kKaratsubaBase = 4;

template <int L>
MOMA_DEV void mul_full_k(uint32_t (&t)[2 * L], const uint32_t (&x)[L], const uint32_t (&y)[L]) {
  if constexpr (L <= kKaratsubaBase || (L % 2) != 0) {
    mul_full<L>(t, x, y);
  } else {
    constexpr int H = L / 2;
    uint32_t x0[H], x1[H], y0[H], y1[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      x0[i] = x[i];
      x1[i] = x[H + i];
      y0[i] = y[i];
      y1[i] = y[H + i];
    }
    uint32_t p0[2 * H], p2[2 * H];
    mul_full_k<H>(p0, x0, y0);
    mul_full_k<H>(p2, x1, y1);
    uint32_t sx[H], sy[H];
    add_words<H, false>(sx, x0, x1);
    const uint32_t cx = carry_out();
    add_words<H, false>(sy, y0, y1);
    const uint32_t cy = carry_out();
    uint32_t p1[2 * H + 1];
    {
      uint32_t pl[2 * H];
      mul_full_k<H>(pl, sx, sy);
#pragma unroll
      for (int i = 0; i < 2 * H; ++i) p1[i] = pl[i];
    }
    p1[2 * H] = cx & cy;
    // p1 += (cx ? sy : 0) z + (cy ? sx : 0) z
    uint32_t m[H];
#pragma unroll
    for (int i = 0; i < H; ++i) m[i] = sy[i] & (0u - cx);
    add_words<H, false>(p1 + H, p1 + H, m);
    p1[2 * H] = addc(p1[2 * H], 0u);
#pragma unroll
    for (int i = 0; i < H; ++i) m[i] = sx[i] & (0u - cy);
    add_words<H, false>(p1 + H, p1 + H, m);
    p1[2 * H] = addc(p1[2 * H], 0u);
    // mid = p1 - p0 - p2 (non-negative, 2H+1 words)
    sub_words<2 * H, false>(p1, p1, p0);
    p1[2 * H] = subc(p1[2 * H], 0u);
    sub_words<2 * H, false>(p1, p1, p2);
    p1[2 * H] = subc(p1[2 * H], 0u);
    // t = p0 + mid z + p2 z^2
#pragma unroll
    for (int i = 0; i < 2 * H; ++i) {
      t[i] = p0[i];
      t[2 * H + i] = p2[i];
    }
    add_words<2 * H + 1, false>(t + H, t + H, p1);
    if constexpr (H > 1) {
#pragma unroll
      for (int i = 3 * H + 1; i < 4 * H - 1; ++i) t[i] = addc_cc(t[i], 0u);
      t[4 * H - 1] = addc(t[4 * H - 1], 0u);
    }
  }
}

// ------------------------------------------------------------------ per-modulus constants
// Kernel-parameter copy of the constants of one modulus (lives in the constant bank).
template <int L>
struct ModK {
  uint32_t q[L];    // modulus, B = 32L - 4 bits (full-width contexts: up to 32L bits)
  uint32_t nq[L];   // 2^(32L) - q, so that  t - s*q = t + s*nq  mod 2^(32L)
  uint32_t mu[L];   // Barrett constant floor(2^(2B+3) / q)  (Eq. mu, k = 2B+3); full-width
                    // contexts: the low L words of floor(2^(64L) / q)
  uint32_t q2[L];   // 2q (full-width contexts: its low L words)
  uint32_t q4[L];   // 4q: bound of the lazy (not fully reduced) values inside a transform
  uint32_t r2[L];   // full-width contexts: R^2 mod q, R = 2^(32L)
  uint32_t qinv;    // full-width contexts: -q^-1 mod 2^32
  uint32_t mu_hi;   // full-width contexts: word L of floor(2^(64L) / q)  (>= 1)
  uint32_t q2_hi;   // full-width contexts: word L of 2q  (0 or 1)
};

// ------------------------------------------------------------------ Sec. 3.1, Eq. barrett
// Barrett reduction of a double-width product t < q^2 with the shifts of Listing 1
// generalised to L words (Listing dmulmod does the same at two words):
//   t1 = t >> (B-2);  s = (t1 * mu) >> (B+5);  c = t - s*q;  if c >= q: c -= q.
// B-2 = 32(L-1) + 26 and B+5 = 32L + 1, so t1 is words L-1..2L-1 shifted by 26 bits and
// s is the high half of t1*mu shifted by one bit.  Only the low L words of t - s*q are
// formed ("the first half matches", Listing dmulmod), as c < 2q < 2^(32L).
// The high half of t1*mu comes from mul_hi_trunc; its error (< L*2^-32 of one unit after
// the shift) keeps c below 2q, so one correction suffices as in Listing 1.
// Returns the quotient estimate s in `s` (callers that need floor(t/q) add the correction).
// HI_WIDE forms the truncated high half t1*mu by whole mad.wide products (the rest by WIDE).
// (With the Karatsuba product, carry chains throughout measured fastest: 37.1 against 34.9
// Gelem/s at 256 bits.)
template <int L, bool WIDE = false, bool HI_WIDE = WIDE>
MOMA_DEV uint32_t barrett_reduce(uint32_t (&c)[L], uint32_t (&s)[L], const uint32_t (&t)[2 * L],
                                 const ModK<L>& k) {
  uint32_t t1[L];
#pragma unroll
  for (int i = 0; i < L; ++i) t1[i] = shr_pair(t[L - 1 + i], t[L + i], 26u);
  uint32_t h[L];
  if constexpr (HI_WIDE) mul_hi_trunc_w<L>(h, t1, k.mu);
  else mul_hi_trunc<L>(h, t1, k.mu);
#pragma unroll
  for (int i = 0; i < L - 1; ++i) s[i] = shr_pair(h[i], h[i + 1], 1u);
  s[L - 1] = h[L - 1] >> 1;
#pragma unroll
  for (int i = 0; i < L; ++i) c[i] = t[i];
  if constexpr (WIDE) mul_lo_acc_w<L>(c, s, k.nq);
  else mul_lo_acc<L>(c, s, k.nq);
  // final correction (the conditional subtraction of Listing 1); report whether it fired
  uint32_t d[L];
  sub_words<L, false>(d, c, k.q);
  const uint32_t keep = borrow_mask();
#pragma unroll
  for (int i = 0; i < L; ++i) c[i] = (c[i] & keep) | (d[i] & ~keep);
  return ~keep & 1u;
}

// c = a * b mod q (Eq. barrett).  WIDE selects the whole-product rows; KARA forms the double
// width product a*b by Karatsuba (Eq. mulk) instead of schoolbook (Eq. muls).
template <int L, bool WIDE = false, bool KARA = false>
MOMA_DEV void mulmod_barrett(uint32_t (&c)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                             const ModK<L>& k) {
  uint32_t t[2 * L];
  if constexpr (KARA) mul_full_k<L>(t, a, b);
  else if constexpr (WIDE) mul_full_w<L>(t, a, b);
  else mul_full<L>(t, a, b);
  uint32_t s[L];
  barrett_reduce<L, WIDE>(c, s, t, k);
}

// ------------------------------------------------------------------ fixed multiplicand
// Barrett with the quotient of the constant precomputed: for a fixed canonical w and its
// companion wp = floor(w * 2^(32L) / q), the quotient of a*w by q is estimated by the high
// half of a*wp, so the reduction needs no double-width product of a*w:
//   s = floor(a*wp / 2^(32L)) (truncated, exact or one less);  r = a*w - s*q mod 2^(32L).
// For any a < 2^(32L): a*w/q - s < 3, so r lies in [0, 3q), which fits the container.
// Used for twiddle factors (tables carry the companion) and for the axpy scalar.
// FE picks the word-product form, splitting the work between the multiply pipe (a whole product
// by mad.wide: 4 cycles; a lo/hi carry-chain pair: 6) and the integer ALU pipe (the carry
// handling of a whole product costs more ALU instructions than that of a carry chain):
//   1: carry chains throughout;
//   2: whole products for the truncated high half a*wp, carry chains for the low halves a*w and
//      s*nq (on GB300 2-3% faster than either uniform form at 256 and 384 bits; the reverse split,
//      carry chains for the high half and whole products for the low halves, measured 4-21% slower).
template <int L, int FE = 1>
MOMA_DEV void mulmod_fixed_lazy(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&w)[L],
                                const uint32_t (&wp)[L], const ModK<L>& k) {
  uint32_t s[L];
#pragma unroll
  for (int i = 0; i < L; ++i) r[i] = 0u;
  if constexpr (FE == 2) mul_hi_trunc_w<L>(s, a, wp);
  else mul_hi_trunc<L>(s, a, wp);
  mul_lo_acc<L>(r, a, w);
  mul_lo_acc<L>(r, s, k.nq);
}

// Canonical form: r in [0, 3q) -> [0, q).
template <int L, int FE = 1>
MOMA_DEV void mulmod_fixed(uint32_t (&r)[L], const uint32_t (&a)[L], const uint32_t (&w)[L],
                           const uint32_t (&wp)[L], const ModK<L>& k) {
  mulmod_fixed_lazy<L, FE>(r, a, w, wp, k);
  cond_sub<L>(r, k.q2);  // [0,3q) -> [0,2q)
  cond_sub<L>(r, k.q);   // -> [0,q)
}

// ------------------------------------------------------------------ full-width moduli
// A modulus that fills its container (up to B = W bits) leaves no headroom: a + b can carry out
// of the W bits, and the Barrett constants above no longer fit.  Sec. 5.2 names Montgomery
// reduction for this case: twiddles and scalars use it (one Montgomery product by a constant kept
// in Montgomery form).  The product of two canonical vectors takes a word-based Barrett reduction
// with an (L+1)-word constant instead (barrett_reduce_full), which needs about half the word
// products of the two Montgomery products it replaces.  Values stay canonical; R = 2^W.

// c = a + b mod q for canonical a, b < q < 2^W: the carry word of rule (moddq_add) is formed
// (the sum may need W+1 bits); subtract q when the sum carried out or is >= q.
template <int L>
MOMA_DEV void addmod_full(uint32_t (&c)[L], const uint32_t (&a)[L], const uint32_t (&b)[L], const uint32_t* q) {
  add_words<L, false>(c, a, b);
  const uint32_t carry = carry_out();
  uint32_t d[L];
  sub_words<L, false>(d, c, q);
  const uint32_t keep = borrow_mask() & (carry - 1u);  // keep the sum: it borrowed and did not carry
#pragma unroll
  for (int i = 0; i < L; ++i) c[i] = (c[i] & keep) | (d[i] & ~keep);
}

// Montgomery product c = a b R^-1 mod q for a, b < q (operand scanning, 32-bit words): for each
// word a_i, t += a_i b, then m = t_0 q' mod 2^32 and t += m q, which clears t_0, and t is shifted
// down one word.  t stays below 2q (L+1 words; one more word holds the carries in between), so
// one conditional subtraction ends it.  2L^2 + L word products.
template <int L>
MOMA_DEV void montmul(uint32_t (&c)[L], const uint32_t (&a)[L], const uint32_t (&b)[L], const ModK<L>& k) {
  uint32_t t[L + 2];
#pragma unroll
  for (int i = 0; i < L + 2; ++i) t[i] = 0u;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    row_lo<L, true>(t, a[i], b);
    t[L] = addc_cc(t[L], 0u);
    t[L + 1] = addc(t[L + 1], 0u);
    row_hi<L, true>(t + 1, a[i], b);
    t[L + 1] = addc(t[L + 1], 0u);
    const uint32_t m = t[0] * k.qinv;
    row_lo<L, true>(t, m, k.q);
    t[L] = addc_cc(t[L], 0u);
    t[L + 1] = addc(t[L + 1], 0u);
    row_hi<L, true>(t + 1, m, k.q);
    t[L + 1] = addc(t[L + 1], 0u);
#pragma unroll
    for (int j = 0; j <= L; ++j) t[j] = t[j + 1];
    t[L + 1] = 0u;
  }
  uint32_t d[L];
  sub_words<L, false>(d, t, k.q);
  const uint32_t borrow = borrow_mask();
  const uint32_t keep = borrow & (0u - (uint32_t)(t[L] == 0u));  // t < q: no carry word, and it borrowed
#pragma unroll
  for (int i = 0; i < L; ++i) c[i] = (t[i] & keep) | (d[i] & ~keep);
}

// c = a b mod q for canonical a, b: REDC(REDC(a b) (R^2 mod q)).
template <int L>
MOMA_DEV void mulmod_mont(uint32_t (&c)[L], const uint32_t (&a)[L], const uint32_t (&b)[L], const ModK<L>& k) {
  uint32_t t[L];
  montmul<L>(t, a, b, k);
  montmul<L>(c, t, k.r2, k);
}

// Word-based Barrett reduction for a modulus that fills its container.  Base b = 2^32; q has L
// words with a nonzero top word, so b^(L-1) < q < b^L (q odd); mu = floor(b^(2L) / q) then has
// L+1 words, b^L < mu < b^(L+1).  For t < q^2:
//   q1 = floor(t / b^(L-1))        words L-1 .. 2L-1 of t (no shift);
//   s ~= floor(q1 mu / b^(L+1))    the truncated high half of q1 mu (exact floor or one less);
//   r = t - s q                    formed mod b^(L+1) as t + s (b^(L+1) - q).
// With Q = floor(t / q): q1 > t/b^(L-1) - 1 and mu > b^(2L)/q - 1 give q1 mu / b^(L+1) in
// (t/q - t/b^(2L) - b^(L-1)/q, t/q], an interval of length below 2, so its floor is Q, Q-1 or Q-2;
// the truncation takes at most one more, hence s in [Q-3, Q] (s < q < b^L: one word fewer than
// q1 mu's high half) and r in [0, 4q), exact in L+1 words.  Two conditional subtractions (2q,
// then q) end it.  Besides the product t: about (L+1)^2 / 2 word products for s and as many for
// the low half of s q, against 2L^2 + L for one Montgomery product (a canonical product needs two).
// r_raw returns r before the subtractions.
template <int L>
MOMA_DEV void barrett_reduce_full(uint32_t (&c)[L], uint32_t (&r_raw)[L + 1], const uint32_t (&t)[2 * L],
                                  const ModK<L>& k) {
  uint32_t q1[L + 1], mu[L + 1], h[L + 1];
#pragma unroll
  for (int i = 0; i <= L; ++i) q1[i] = t[L - 1 + i];
#pragma unroll
  for (int i = 0; i < L; ++i) mu[i] = k.mu[i];
  mu[L] = k.mu_hi;
  mul_hi_trunc<L + 1>(h, q1, mu);  // words L+1 .. 2L+1 of q1 mu; h[L] = 0 since s < b^L
  uint32_t s[L + 1], nq1[L + 1], r[L + 1];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    s[i] = h[i];
    nq1[i] = k.nq[i];
  }
  s[L] = 0u;
  nq1[L] = 0xffffffffu;  // b^(L+1) - q = (b - 1) b^L + (b^L - q)
#pragma unroll
  for (int i = 0; i <= L; ++i) r[i] = t[i];
  mul_lo_acc<L + 1>(r, s, nq1);
#pragma unroll
  for (int i = 0; i <= L; ++i) r_raw[i] = r[i];
  uint32_t m[L + 1];
#pragma unroll
  for (int i = 0; i < L; ++i) m[i] = k.q2[i];
  m[L] = k.q2_hi;
  cond_sub<L + 1>(r, m);  // [0, 4q) -> [0, 2q)
#pragma unroll
  for (int i = 0; i < L; ++i) m[i] = k.q[i];
  m[L] = 0u;
  cond_sub<L + 1>(r, m);  // -> [0, q)
#pragma unroll
  for (int i = 0; i < L; ++i) c[i] = r[i];
}

// c = a b mod q for canonical a, b under a full-width modulus: the double-width product by
// engine ENG (1 carry chains, 2 whole products, 3 Karatsuba), then barrett_reduce_full.
template <int L, int ENG>
MOMA_DEV void mulmod_barrett_full(uint32_t (&c)[L], const uint32_t (&a)[L], const uint32_t (&b)[L],
                                  const ModK<L>& k) {
  uint32_t t[2 * L];
  if constexpr (ENG == 3) mul_full_k<L>(t, a, b);
  else if constexpr (ENG == 2) mul_full_w<L>(t, a, b);
  else mul_full<L>(t, a, b);
  uint32_t r[L + 1];
  barrett_reduce_full<L>(c, r, t, k);
}

}  // namespace moma
