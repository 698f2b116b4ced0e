// moma_bigint.hpp -- small host-side unsigned big integers for per-modulus set-up.
//
// Only used once per modulus or per transform plan (Barrett constant, roots of unity,
// inverses, primality), never on the data path.  Little-endian 32-bit words,
// normalised (no leading zero words).  Straightforward schoolbook algorithms; general
// division is bit-serial shift-and-subtract (used to set up a Reducer), repeated
// reductions by one modulus go through Reducer (quotient from a precomputed reciprocal).
#pragma once
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace moma {

struct BigU {
  std::vector<uint32_t> w;  // little-endian words, no leading zeros

  BigU() = default;
  explicit BigU(uint64_t v) {
    while (v) {
      w.push_back((uint32_t)v);
      v >>= 32;
    }
  }
  static BigU from_words(const uint32_t* p, int n) {
    BigU r;
    r.w.assign(p, p + n);
    r.trim();
    return r;
  }
  void trim() {
    while (!w.empty() && w.back() == 0) w.pop_back();
  }
  bool is_zero() const { return w.empty(); }
  int bits() const {
    if (w.empty()) return 0;
    uint32_t top = w.back();
    int b = 0;
    while (top) {
      ++b;
      top >>= 1;
    }
    return (int)(w.size() - 1) * 32 + b;
  }
  bool bit(int i) const {
    size_t k = (size_t)i / 32;
    return k < w.size() && ((w[k] >> (i % 32)) & 1u);
  }
  uint32_t word(size_t i) const { return i < w.size() ? w[i] : 0u; }
  void to_words(uint32_t* out, int n) const {
    for (int i = 0; i < n; ++i) out[i] = word((size_t)i);
  }
  bool is_odd() const { return !w.empty() && (w[0] & 1u); }
};

inline int cmp(const BigU& a, const BigU& b) {
  if (a.w.size() != b.w.size()) return a.w.size() < b.w.size() ? -1 : 1;
  for (size_t i = a.w.size(); i-- > 0;) {
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  }
  return 0;
}

inline BigU add(const BigU& a, const BigU& b) {
  BigU r;
  size_t n = std::max(a.w.size(), b.w.size());
  r.w.resize(n + 1);
  uint64_t c = 0;
  for (size_t i = 0; i < n; ++i) {
    c += (uint64_t)a.word(i) + b.word(i);
    r.w[i] = (uint32_t)c;
    c >>= 32;
  }
  r.w[n] = (uint32_t)c;
  r.trim();
  return r;
}

// a - b, requires a >= b
inline BigU sub(const BigU& a, const BigU& b) {
  BigU r;
  r.w.resize(a.w.size());
  int64_t br = 0;
  for (size_t i = 0; i < a.w.size(); ++i) {
    int64_t d = (int64_t)a.w[i] - (int64_t)b.word(i) - br;
    br = d < 0;
    r.w[i] = (uint32_t)(d + (br ? (int64_t)1 << 32 : 0));
  }
  r.trim();
  return r;
}

inline BigU mul(const BigU& a, const BigU& b) {
  BigU r;
  if (a.is_zero() || b.is_zero()) return r;
  r.w.assign(a.w.size() + b.w.size(), 0u);
  for (size_t i = 0; i < a.w.size(); ++i) {
    uint64_t c = 0;
    for (size_t j = 0; j < b.w.size(); ++j) {
      c += (uint64_t)a.w[i] * b.w[j] + r.w[i + j];
      r.w[i + j] = (uint32_t)c;
      c >>= 32;
    }
    r.w[i + b.w.size()] = (uint32_t)c;
  }
  r.trim();
  return r;
}

inline BigU shl(const BigU& a, int s) {
  if (a.is_zero()) return a;
  BigU r;
  int ws = s / 32, bs = s % 32;
  r.w.assign(a.w.size() + ws + 1, 0u);
  for (size_t i = 0; i < a.w.size(); ++i) {
    uint64_t v = (uint64_t)a.w[i] << bs;
    r.w[i + ws] |= (uint32_t)v;
    r.w[i + ws + 1] |= (uint32_t)(v >> 32);
  }
  r.trim();
  return r;
}

inline BigU shr(const BigU& a, int s) {
  int ws = s / 32, bs = s % 32;
  BigU r;
  if ((size_t)ws >= a.w.size()) return r;
  r.w.assign(a.w.size() - ws, 0u);
  for (size_t i = 0; i < r.w.size(); ++i) {
    uint64_t v = a.word(i + ws) | ((uint64_t)a.word(i + ws + 1) << 32);
    r.w[i] = (uint32_t)(v >> bs);
  }
  r.trim();
  return r;
}

// q = a / b, r = a % b (b != 0), bit-serial restoring division.
inline void divmod(const BigU& a, const BigU& b, BigU* q, BigU* r) {
  BigU quo, rem;
  int nb = a.bits();
  quo.w.assign((size_t)(nb + 31) / 32 + 1, 0u);
  for (int i = nb - 1; i >= 0; --i) {
    rem = shl(rem, 1);
    if (a.bit(i)) {
      if (rem.w.empty()) rem.w.push_back(0u);
      rem.w[0] |= 1u;
    }
    if (cmp(rem, b) >= 0) {
      rem = sub(rem, b);
      quo.w[(size_t)i / 32] |= 1u << (i % 32);
    }
  }
  quo.trim();
  if (q) *q = quo;
  if (r) *r = rem;
}

inline BigU mod(const BigU& a, const BigU& m) {
  BigU r;
  divmod(a, m, nullptr, &r);
  return r;
}

// Fixed-modulus reduction for repeated use (powers, primality): quotient estimated with
// mu = floor(2^k / m), k = 2*bits(m) + 8, exact after at most two corrections for x < 2^k.
struct Reducer {
  BigU m, mu;
  int k = 0;
  explicit Reducer(const BigU& mod_) : m(mod_) {
    k = 2 * m.bits() + 8;
    divmod(pow2(k), m, &mu, nullptr);
  }
  static BigU pow2(int e) { return shl(BigU(1), e); }
  // q = x / m, r = x % m for x < 2^k
  void divmod_(const BigU& x, BigU* q, BigU* r) const {
    BigU qh = shr(mul(x, mu), k);
    BigU rr = sub(x, mul(qh, m));
    while (cmp(rr, m) >= 0) {
      rr = sub(rr, m);
      qh = add(qh, BigU(1));
    }
    if (q) *q = qh;
    if (r) *r = rr;
  }
  BigU mod(const BigU& x) const {
    BigU r;
    divmod_(x, nullptr, &r);
    return r;
  }
  BigU mulmod(const BigU& a, const BigU& b) const { return mod(mul(a, b)); }
  BigU powmod(const BigU& base, const BigU& e) const {
    BigU r(1), b = mod(base);
    for (int i = e.bits() - 1; i >= 0; --i) {
      r = mulmod(r, r);
      if (e.bit(i)) r = mulmod(r, b);
    }
    return r;
  }
};

inline BigU pow2(int k) { return shl(BigU(1), k); }

// Miller-Rabin with the first 24 primes as bases.
inline bool probably_prime(const BigU& n) {
  static const uint32_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37,
                                   41, 43, 47, 53, 59, 61, 67, 71, 73, 79, 83, 89};
  if (n.bits() <= 32) {
    uint32_t v = n.word(0);
    if (v < 2) return false;
    for (uint32_t p : bases) {
      if (v == p) return true;
      if (v % p == 0) return false;
    }
  }
  if (!n.is_odd()) return false;
  Reducer red(n);
  BigU one(1), nm1 = sub(n, one), d = nm1;
  int s = 0;
  while (!d.is_odd()) {
    d = shr(d, 1);
    ++s;
  }
  for (uint32_t a : bases) {
    BigU x = red.powmod(BigU(a), d);
    if (cmp(x, one) == 0 || cmp(x, nm1) == 0) continue;
    bool composite = true;
    for (int i = 1; i < s; ++i) {
      x = red.mulmod(x, x);
      if (cmp(x, nm1) == 0) {
        composite = false;
        break;
      }
    }
    if (composite) return false;
  }
  return true;
}

}  // namespace moma
