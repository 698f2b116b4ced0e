// Test harness for the library's host-side big integers (moma_bigint.hpp), which set up every
// per-modulus constant (Barrett mu, companions, roots, R^2, primality).  Reads one operation per
// line from stdin -- "<op> <hex> <hex> [<hex>]" -- and writes the result(s) in hex, one line each.
#include <cstdio>
#include <iostream>
#include <sstream>
#include <string>

#include "moma_bigint.hpp"

using moma::BigU;

static BigU from_hex(const std::string& s) {
  BigU r;
  for (char ch : s) {
    uint32_t d = (ch >= '0' && ch <= '9') ? ch - '0' : (ch >= 'a' && ch <= 'f') ? ch - 'a' + 10 : ch - 'A' + 10;
    r = moma::add(moma::shl(r, 4), BigU(d));
  }
  return r;
}

static std::string to_hex(const BigU& a) {
  if (a.is_zero()) return "0";
  std::string s;
  char buf[9];
  for (size_t i = a.w.size(); i-- > 0;) {
    std::snprintf(buf, sizeof buf, i + 1 == a.w.size() ? "%x" : "%08x", a.w[i]);
    s += buf;
  }
  return s;
}

int main() {
  std::string line;
  while (std::getline(std::cin, line)) {
    std::istringstream in(line);
    std::string op, x, y, z;
    in >> op >> x >> y >> z;
    const BigU a = from_hex(x), b = y.empty() ? BigU() : from_hex(y), m = z.empty() ? BigU() : from_hex(z);
    if (op == "add") {
      std::cout << to_hex(moma::add(a, b)) << "\n";
    } else if (op == "sub") {
      std::cout << to_hex(moma::sub(a, b)) << "\n";
    } else if (op == "mul") {
      std::cout << to_hex(moma::mul(a, b)) << "\n";
    } else if (op == "shl") {
      std::cout << to_hex(moma::shl(a, (int)b.word(0))) << "\n";
    } else if (op == "shr") {
      std::cout << to_hex(moma::shr(a, (int)b.word(0))) << "\n";
    } else if (op == "cmp") {
      std::cout << moma::cmp(a, b) << "\n";
    } else if (op == "divmod") {
      BigU q, r;
      moma::divmod(a, b, &q, &r);
      std::cout << to_hex(q) << " " << to_hex(r) << "\n";
    } else if (op == "red_divmod") {  // a < 2^k of the Reducer for modulus b
      moma::Reducer red(b);
      BigU q, r;
      red.divmod_(a, &q, &r);
      std::cout << to_hex(q) << " " << to_hex(r) << "\n";
    } else if (op == "mulmod") {
      std::cout << to_hex(moma::Reducer(m).mulmod(a, b)) << "\n";
    } else if (op == "powmod") {
      std::cout << to_hex(moma::Reducer(m).powmod(a, b)) << "\n";
    } else if (op == "prime") {
      std::cout << (moma::probably_prime(a) ? 1 : 0) << "\n";
    } else if (op == "words") {  // to_words / from_words round trip at b words
      uint32_t w[80] = {};
      a.to_words(w, (int)b.word(0));
      std::cout << to_hex(BigU::from_words(w, (int)b.word(0))) << "\n";
    } else {
      std::cout << "?\n";
    }
  }
  return 0;
}
