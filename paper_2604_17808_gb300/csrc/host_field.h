// host_field.h -- host-side 256-bit modular arithmetic for plan constants.
//
// Only a few hundred operations per plan (roots of unity, N^-1, coset
// powers, Montgomery conversions), so this favours obviously-correct code:
// multiplication is MSB-first double-and-add with a modular reduction after
// every addition, and Montgomery conversion x -> x * 2^256 mod p is 256
// modular doublings.  Both moduli are below 2^255, so a + b < 2^256 never
// overflows four limbs.
#pragma once

#include <cstdint>
#include <cstring>

namespace gb300ntt {

struct U256 {
  uint64_t w[4];
};

inline U256 u256(uint64_t v) { return U256{{v, 0, 0, 0}}; }

inline bool u256_geq(const U256 &a, const U256 &b) {
  for (int i = 3; i >= 0; --i)
    if (a.w[i] != b.w[i]) return a.w[i] > b.w[i];
  return true;
}

inline bool u256_is_zero(const U256 &a) { return (a.w[0] | a.w[1] | a.w[2] | a.w[3]) == 0; }

inline U256 u256_add_raw(const U256 &a, const U256 &b) {
  U256 r;
  uint64_t c = 0;
  for (int i = 0; i < 4; ++i) {
    const uint64_t s = a.w[i] + c;
    const uint64_t c1 = s < c;
    r.w[i] = s + b.w[i];
    c = c1 + (r.w[i] < s);
  }
  return r;
}

inline U256 u256_sub_raw(const U256 &a, const U256 &b) {
  U256 r;
  uint64_t bw = 0;
  for (int i = 0; i < 4; ++i) {
    const uint64_t d = a.w[i] - b.w[i];
    const uint64_t b1 = a.w[i] < b.w[i];
    r.w[i] = d - bw;
    bw = b1 | (d < bw);
  }
  return r;
}

inline U256 u256_shr(const U256 &a, unsigned s) {
  U256 r = a;
  for (unsigned k = 0; k < s; ++k)
    for (int i = 0; i < 4; ++i) r.w[i] = (r.w[i] >> 1) | (i < 3 ? (r.w[i + 1] << 63) : 0);
  return r;
}

class HostField {
 public:
  U256 p;
  uint64_t generator;
  unsigned two_adicity;

  HostField(const U256 &modulus, uint64_t g, unsigned adicity) : p(modulus), generator(g), two_adicity(adicity) {}

  U256 add(const U256 &a, const U256 &b) const {
    U256 s = u256_add_raw(a, b);
    return u256_geq(s, p) ? u256_sub_raw(s, p) : s;
  }
  U256 sub(const U256 &a, const U256 &b) const {
    return u256_geq(a, b) ? u256_sub_raw(a, b) : u256_add_raw(u256_sub_raw(p, b), a);
  }
  U256 reduce_small(uint64_t v) const {
    U256 r = u256(v);
    while (u256_geq(r, p)) r = u256_sub_raw(r, p);
    return r;
  }
  U256 mul(const U256 &a, const U256 &b) const {
    U256 acc = u256(0);
    for (int i = 255; i >= 0; --i) {
      acc = add(acc, acc);
      if ((b.w[i / 64] >> (i % 64)) & 1) acc = add(acc, a);
    }
    return acc;
  }
  U256 pow(const U256 &a, const U256 &e) const {
    U256 acc = u256(1), base = a;
    for (int i = 0; i < 256; ++i) {
      if ((e.w[i / 64] >> (i % 64)) & 1) acc = mul(acc, base);
      base = mul(base, base);
    }
    return acc;
  }
  U256 pow(const U256 &a, uint64_t e) const { return pow(a, u256(e)); }
  U256 inv(const U256 &a) const { return pow(a, u256_sub_raw(p, u256(2))); }
  // x * 2^256 mod p
  U256 to_mont(const U256 &a) const {
    U256 r = a;
    for (int i = 0; i < 256; ++i) r = add(r, r);
    return r;
  }
  // x * 2^-256 mod p
  U256 from_mont(const U256 &a) const { return mul(a, r_inv()); }
  U256 r_inv() const { return inv(to_mont(u256(1))); }
  // omega_N = g^((p-1)/N), N = 2^log_n <= 2^two_adicity
  U256 root_of_unity(unsigned log_n) const {
    return pow(reduce_small(generator), u256_shr(u256_sub_raw(p, u256(1)), log_n));
  }
};

inline HostField host_field(int field) {
  if (field == 0)
    return HostField(U256{{0xffffffff00000001ULL, 0x53bda402fffe5bfeULL, 0x3339d80809a1d805ULL,
                           0x73eda753299d7d48ULL}},
                     7, 32);
  return HostField(U256{{0x43e1f593f0000001ULL, 0x2833e84879b97091ULL, 0xb85045b68181585dULL,
                         0x30644e72e131a029ULL}},
                   5, 28);
}

}  // namespace gb300ntt
