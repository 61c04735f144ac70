// ntt_rns.cu -- host side of the RNS lazy multiplication (ntt_rns.cuh):
// the two residue bases, the constant tables and byte matrices, and the
// C ABI.  MORPH, Sec. 3.2.3-3.2.4 and Alg. 1.
//
// Bases (both fields): Q = the I largest primes below 2^31, I the fewest
// with Q > 4 L^2, L = (sum q + I) M; P = the next primes below them, the
// fewest with P > 2^20 L.  The tables are built here from their
// definitions with a small host bignum and the host field arithmetic, and
// uploaded once per (device, field).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "host_field.h"
#include "ntt_plan.h"
#include "ntt_rns.cuh"

using namespace gb300ntt;

namespace gb300ntt {
namespace {

#define NTT_TRY_RNS(expr)              \
  do {                                 \
    const ntt_status _s = (expr);      \
    if (_s != NTT_OK) return _s;       \
  } while (0)

// ------------------------------------------------------------ host bignum

using Big = std::vector<uint64_t>;   // little-endian 64-bit limbs

void big_trim(Big &a) {
  while (!a.empty() && a.back() == 0) a.pop_back();
}

Big big_mul_small(const Big &a, uint64_t m) {
  Big r(a.size() + 1, 0);
  unsigned __int128 carry = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    const unsigned __int128 t = (unsigned __int128)a[i] * m + carry;
    r[i] = (uint64_t)t;
    carry = t >> 64;
  }
  r[a.size()] = (uint64_t)carry;
  big_trim(r);
  return r;
}

Big big_mul(const Big &a, const Big &b) {
  Big r(a.size() + b.size() + 1, 0);
  for (size_t i = 0; i < a.size(); ++i) {
    unsigned __int128 carry = 0;
    for (size_t j = 0; j < b.size(); ++j) {
      const unsigned __int128 t = (unsigned __int128)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint64_t)t;
      carry = t >> 64;
    }
    size_t k = i + b.size();
    while (carry) {
      const unsigned __int128 t = (unsigned __int128)r[k] + carry;
      r[k++] = (uint64_t)t;
      carry = t >> 64;
    }
  }
  big_trim(r);
  return r;
}

Big big_shl(const Big &a, unsigned s) {
  Big r(a.size() + s / 64 + 1, 0);
  for (size_t i = 0; i < a.size(); ++i) {
    const unsigned w = s / 64, b = s % 64;
    r[i + w] |= a[i] << b;
    if (b) r[i + w + 1] |= a[i] >> (64 - b);
  }
  big_trim(r);
  return r;
}

int big_cmp(const Big &a, const Big &b) {
  if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
  for (size_t i = a.size(); i-- > 0;)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}

Big big_of(const U256 &a) {
  Big r(a.w, a.w + 4);
  big_trim(r);
  return r;
}

// ------------------------------------------------------- small-number math

uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }

uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = mulmod64(r, a, m);
    a = mulmod64(a, a, m);
    e >>= 1;
  }
  return r;
}

// Miller-Rabin with bases 2, 7, 61: deterministic below 2^32.
bool is_prime_u32(uint32_t n) {
  if (n < 2) return false;
  for (uint32_t p : {2u, 3u, 5u, 7u, 11u, 13u, 17u, 19u, 23u, 29u, 31u, 37u, 41u, 43u, 47u, 53u, 59u, 61u})
    if (n % p == 0) return n == p;
  uint32_t d = n - 1, s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  for (uint32_t a : {2u, 7u, 61u}) {
    uint64_t x = powmod64(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool composite = true;
    for (uint32_t r = 1; r < s; ++r) {
      x = mulmod64(x, x, n);
      if (x == n - 1) {
        composite = false;
        break;
      }
    }
    if (composite) return false;
  }
  return true;
}

uint64_t u256_mod_small(const U256 &a, uint64_t m) {
  unsigned __int128 r = 0;
  for (int i = 3; i >= 0; --i) r = ((r << 64) | a.w[i]) % m;
  return (uint64_t)r;
}

uint32_t bf16_bits_of_byte(uint32_t v) {
  const float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u >> 16;
}

// --------------------------------------------------------------- tables

struct RnsField {
  bool ready = false;
  int num_p = 0;
  RnsConst c{};
  std::vector<uint32_t> q, p;
  uint4 *d_e1 = nullptr, *d_e2 = nullptr;
  uint32_t *d_err = nullptr;
};

std::mutex g_rns_mu;
RnsField g_rns[8][2];   // [device][field]

void build_basis(int field, std::vector<uint32_t> &q, std::vector<uint32_t> &p) {
  const HostField F = host_field(field);
  const Big M = big_of(F.p);
  uint32_t cand = 0x7FFFFFFFu;   // largest primes below 2^31, descending
  auto next_prime = [&]() {
    while (!is_prime_u32(cand)) --cand;
    return cand--;
  };
  q.clear();
  p.clear();
  Big Q{1}, L;
  uint64_t sum = 0;
  for (;;) {
    const uint32_t qi = next_prime();
    q.push_back(qi);
    Q = big_mul_small(Q, qi);
    sum += qi;
    L = big_mul_small(M, sum + q.size());
    if (big_cmp(Q, big_mul_small(big_mul(L, L), 4)) > 0) break;
  }
  Big P{1};
  const Big bound = big_shl(L, 20);
  while (big_cmp(P, bound) <= 0) {
    const uint32_t pj = next_prime();
    p.push_back(pj);
    P = big_mul_small(P, pj);
  }
}

ntt_status build_field(int device, int field, RnsField &R) {
  const HostField F = host_field(field);
  std::vector<uint32_t> &q = R.q, &p = R.p;
  build_basis(field, q, p);
  const int I = (int)q.size(), J = (int)p.size();
  if (I != kRnsI || J > kRnsMaxJ || (J != 10 && J != 11)) return NTT_ERR_UNSUPPORTED;
  R.num_p = J;
  RnsConst &C = R.c;
  std::memset(&C, 0, sizeof C);
  // base Q constants
  for (int i = 0; i < I; ++i) {
    const uint64_t qi = q[i];
    C.q[i] = q[i];
    uint32_t inv = 1;   // q^-1 mod 2^32 by Newton's iteration
    for (int t = 0; t < 5; ++t) inv *= 2u - q[i] * inv;
    C.q_ninv[i] = 0u - inv;
    uint64_t qhat = 1;
    for (int t = 0; t < I; ++t)
      if (t != i) qhat = mulmod64(qhat, q[t], qi);
    const uint64_t qhat_inv = powmod64(qhat, qi - 2, qi);
    const uint64_t two64 = mulmod64((uint64_t)1 << 32, (uint64_t)1 << 32, qi);
    C.q_hat_inv_m[i] = (uint32_t)mulmod64(qhat_inv, two64, qi);
    C.f[i] = (uint32_t)((((uint64_t)1 << kRnsShift) + qi - 1) / qi);
    C.q_mu[i] = UINT64_MAX / qi;
    uint64_t pm = 1;
    for (int j = 0; j < J; ++j) pm = mulmod64(pm, p[j], qi);
    C.g2[i] = (uint32_t)((qi - pm) % qi);
  }
  // base P constants
  std::vector<uint64_t> p_hat_inv(J);
  for (int j = 0; j < J; ++j) {
    const uint64_t pj = p[j];
    C.p[j] = p[j];
    C.f2[j] = (uint32_t)((((uint64_t)1 << kRnsShift) + pj - 1) / pj);
    C.p_mu[j] = UINT64_MAX / pj;
    uint64_t phat = 1;
    for (int t = 0; t < J; ++t)
      if (t != j) phat = mulmod64(phat, p[t], pj);
    p_hat_inv[j] = powmod64(phat, pj - 2, pj);
  }
  // (Q/q_i) mod M and Q mod M with the field arithmetic
  std::vector<U256> w(I);
  U256 q_mod_m = u256(1);
  for (int i = 0; i < I; ++i) q_mod_m = F.mul(q_mod_m, u256(q[i]));
  for (int i = 0; i < I; ++i) {
    U256 acc = u256(1);
    for (int t = 0; t < I; ++t)
      if (t != i) acc = F.mul(acc, u256(q[t]));
    w[i] = acc;
  }
  const U256 m_minus = u256_sub_raw(F.p, q_mod_m);   // M - (Q mod M), in (0, M]
  for (int j = 0; j < J; ++j)
    C.g[j] = (uint32_t)mulmod64(u256_mod_small(m_minus, p[j]), p_hat_inv[j], p[j]);
  // E1: rows n = 4j + h, columns k = 4i + b; E2: rows n = 4i + h, columns k = 4j + b
  std::vector<uint16_t> e1((size_t)kRnsN1 * kRnsK1, 0), e2((size_t)kRnsN2 * kRnsK2, 0);
  for (int i = 0; i < I; ++i)
    for (int b = 0; b < 4; ++b)
      for (int j = 0; j < J; ++j) {
        const uint64_t pj = p[j];
        const uint64_t val =
            mulmod64(mulmod64(u256_mod_small(w[i], pj), ((uint64_t)1 << (8 * b)) % pj, pj), p_hat_inv[j], pj);
        for (int h = 0; h < 4; ++h) {
          const uint32_t off = core_offset(4 * j + h, 4 * i + b, kRnsK1) / 2;
          e1[off] = (uint16_t)bf16_bits_of_byte((uint32_t)(val >> (8 * h)) & 0xFFu);
        }
      }
  for (int j = 0; j < J; ++j)
    for (int b = 0; b < 4; ++b)
      for (int i = 0; i < I; ++i) {
        const uint64_t qi = q[i];
        uint64_t phat = 1;
        for (int t = 0; t < J; ++t)
          if (t != j) phat = mulmod64(phat, p[t], qi);
        const uint64_t val = mulmod64(phat, ((uint64_t)1 << (8 * b)) % qi, qi);
        for (int h = 0; h < 4; ++h) {
          const uint32_t off = core_offset(4 * i + h, 4 * j + b, kRnsK2) / 2;
          e2[off] = (uint16_t)bf16_bits_of_byte((uint32_t)(val >> (8 * h)) & 0xFFu);
        }
      }
  ntt_status s = cuda_status(cudaMalloc(&R.d_e1, e1.size() * 2));
  if (s == NTT_OK) s = cuda_status(cudaMalloc(&R.d_e2, e2.size() * 2));
  if (s == NTT_OK) s = cuda_status(cudaMalloc(&R.d_err, sizeof(uint32_t)));
  if (s == NTT_OK) s = cuda_status(cudaMemcpy(R.d_e1, e1.data(), e1.size() * 2, cudaMemcpyHostToDevice));
  if (s == NTT_OK) s = cuda_status(cudaMemcpy(R.d_e2, e2.data(), e2.size() * 2, cudaMemcpyHostToDevice));
  if (s == NTT_OK) s = cuda_status(cudaMemset(R.d_err, 0, sizeof(uint32_t)));
  if (s == NTT_OK && J == 11)
    s = cuda_status(cudaFuncSetAttribute(rns_mul_kernel<11>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         rns_smem_bytes()));
  if (s == NTT_OK && J == 10)
    s = cuda_status(cudaFuncSetAttribute(rns_mul_kernel<10>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         rns_smem_bytes()));
  (void)device;
  return s;
}

ntt_status rns_field(int field, RnsField **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NTT_ERR_NO_DEVICE;
  if (dev < 0 || dev >= 8) return NTT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_rns_mu);
  RnsField &R = g_rns[dev][field];
  if (!R.ready) {
    NTT_TRY_RNS(build_field(dev, field, R));
    R.ready = true;
  }
  *out = &R;
  return NTT_OK;
}

}  // namespace
}  // namespace gb300ntt

extern "C" {

ntt_status ntt_rns_basis_get(ntt_field field, ntt_rns_basis *out) {
  if (!out || (field != NTT_FIELD_BLS12_381_FR && field != NTT_FIELD_BN254_FR)) return NTT_ERR_INVALID_ARG;
  std::vector<uint32_t> q, p;
  build_basis((int)field, q, p);
  std::memset(out, 0, sizeof *out);
  out->num_q = (uint32_t)q.size();
  out->num_p = (uint32_t)p.size();
  out->words_per_element = kRnsWords;
  out->shift = kRnsShift;
  for (size_t i = 0; i < q.size() && i < 24; ++i) out->q[i] = q[i];
  for (size_t j = 0; j < p.size() && j < 16; ++j) out->p[j] = p[j];
  return NTT_OK;
}

ntt_status ntt_rns_mul(ntt_field field, const void *d_x, const void *d_y, void *d_out, uint64_t count, uint32_t reps,
                       ntt_stream stream) {
  if (field != NTT_FIELD_BLS12_381_FR && field != NTT_FIELD_BN254_FR) return NTT_ERR_INVALID_ARG;
  if (reps == 0) return NTT_ERR_INVALID_ARG;
  if (!d_x || !d_y || !d_out || ((uintptr_t)d_x | (uintptr_t)d_y | (uintptr_t)d_out) % 16) return NTT_ERR_INVALID_ARG;
  if (count == 0) return NTT_OK;
  RnsField *R = nullptr;
  const ntt_status s = rns_field((int)field, &R);
  if (s != NTT_OK) return s;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NTT_ERR_CUDA;
  RnsArgs a{};
  a.x = (const uint4 *)d_x;
  a.y = (const uint4 *)d_y;
  a.out = (uint4 *)d_out;
  a.count = count;
  a.reps = reps;
  a.e1 = R->d_e1;
  a.e2 = R->d_e2;
  a.err = R->d_err;
  a.wait_ns = 1000000000ull;
  const uint64_t tiles = (count + kRnsThreads - 1) / kRnsThreads;
  const uint64_t slots = (uint64_t)sms * 4;
  const unsigned grid = (unsigned)(tiles < slots ? tiles : slots);
  if (R->num_p == 11)
    rns_mul_kernel<11><<<grid, kRnsThreads, rns_smem_bytes(), (cudaStream_t)stream>>>(a, R->c);
  else
    rns_mul_kernel<10><<<grid, kRnsThreads, rns_smem_bytes(), (cudaStream_t)stream>>>(a, R->c);
  return cuda_status(cudaGetLastError());
}

ntt_status ntt_rns_poll_error(ntt_field field, uint32_t *code) {
  if (!code || (field != NTT_FIELD_BLS12_381_FR && field != NTT_FIELD_BN254_FR)) return NTT_ERR_INVALID_ARG;
  *code = 0;
  RnsField *R = nullptr;
  const ntt_status s = rns_field((int)field, &R);
  if (s != NTT_OK) return s;
  ntt_status st = cuda_status(cudaMemcpy(code, R->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (st == NTT_OK) st = cuda_status(cudaMemset(R->d_err, 0, sizeof(uint32_t)));
  return st;
}

}  // extern "C"
