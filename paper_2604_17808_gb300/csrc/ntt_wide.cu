// ntt_wide.cu -- host side of the 377- and 753-bit transforms (ntt_wide.cuh):
// field constants, per-(device, field, size) tables, pass launches, C ABI.
//
// The moduli (the smallest primes c 2^32 + 1, c odd, above floor(pi
// 2^(b-2)) for b = 377 and 753; generators 7 and 11, the smallest quadratic
// non-residues) are public constants of this library, written out below.
// The host derives R mod p, R^2 mod p and (p - 1) / 2^32 from them with a
// small fixed-width arithmetic; every root of unity, inverse and table is
// computed on the device (wide_constants_kernel, wide_table_kernel).
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <new>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "ntt_plan.h"
#include "ntt_wide.cuh"

namespace gb300ntt {
namespace {

const uint32_t kP377[12] = {0x00000001u, 0xBBDF2BD5u, 0xF31C6809u, 0x44A29410u, 0x4C762736u, 0xE804177Du,
                            0x1114CF98u, 0xA252049Cu, 0x1701B839u, 0x69898CC5u, 0x4442D184u, 0x01921FB5u};
const uint32_t kP753[24] = {0x00000001u, 0x6FDBDCD3u, 0xB96DE80Du, 0xDAD617FEu, 0x85D34C6Fu, 0xFD8DE898u,
                            0x6AECC4BCu, 0x848BC90Bu, 0x6ADADAA3u, 0x286E9FC2u, 0x14DBE4BEu, 0x86366056u,
                            0x33679A74u, 0x09BBDF2Au, 0x10F31C68u, 0x3644A294u, 0x7D4C7627u, 0x98E80417u,
                            0x9C1114CFu, 0x39A25204u, 0xC51701B8u, 0x8469898Cu, 0xB54442D1u, 0x0001921Fu};

#define NTT_TRY_W(expr)                \
  do {                                 \
    const ntt_status _s = (expr);      \
    if (_s != NTT_OK) return _s;       \
  } while (0)

// x = 2 x mod p on NL-limb numbers (x < p).
template <int NL>
void host_double_mod(uint32_t x[NL], const uint32_t p[NL]) {
  uint32_t carry = 0;
  for (int j = 0; j < NL; ++j) {
    const uint32_t nc = x[j] >> 31;
    x[j] = (x[j] << 1) | carry;
    carry = nc;
  }
  bool ge = carry != 0;
  if (!ge) {
    ge = true;
    for (int j = NL - 1; j >= 0; --j)
      if (x[j] != p[j]) {
        ge = x[j] > p[j];
        break;
      }
  }
  if (ge) {
    int64_t br = 0;
    for (int j = 0; j < NL; ++j) {
      const int64_t v = (int64_t)x[j] - p[j] + br;
      x[j] = (uint32_t)v;
      br = v >> 32;
    }
  }
}

template <int NL32>
WideConst<NL32> make_const(const uint32_t p[NL32], uint32_t gen) {
  constexpr int L = WideShape<NL32>::L;
  WideConst<NL32> c{};
  std::memcpy(c.p32, p, sizeof c.p32);
  auto to29 = [&](uint32_t out[L], const uint32_t x[NL32]) {
    for (int j = 0; j < L; ++j) {
      const int bit = 29 * j, w = bit >> 5, sh = bit & 31;
      const uint64_t lo = w < NL32 ? x[w] : 0u, hi = w + 1 < NL32 ? x[w + 1] : 0u;
      out[j] = (uint32_t)(((hi << 32) | lo) >> sh) & kM29;
    }
  };
  to29(c.p, p);
  uint32_t inv = 1;   // p^-1 mod 2^32 by Newton's iteration
  for (int t = 0; t < 5; ++t) inv *= 2u - p[0] * inv;
  c.ninv = (0u - inv) & kM29;
  uint32_t x[NL32] = {1};
  for (int b = 0; b < 29 * L; ++b) host_double_mod<NL32>(x, p);   // R mod p, R = 2^(29 L)
  to29(c.one, x);
  for (int b = 0; b < 29 * L; ++b) host_double_mod<NL32>(x, p);   // R^2 mod p
  to29(c.r2, x);
  for (int j = 0; j < NL32; ++j) c.exp_c[j] = j + 1 < NL32 ? p[j + 1] : 0u;   // (p - 1) >> 32 (p0 = 1)
  c.gen = gen;
  return c;
}

int limbs_of(int field) { return field == NTT_FIELD_W377 ? 12 : 24; }
int tile_log(int field) { return field == NTT_FIELD_W377 ? WideShape<12>::kLog : WideShape<24>::kLog; }

struct WidePlan {
  uint32_t log_n = 0, num_passes = 0;
  uint32_t pass_log[kMaxPasses] = {};
  uint4 *dft_tw[2][12] = {};
  uint4 *tw[2][kMaxPasses] = {};
  uint4 *pre_inv = nullptr;
  uint4 *scratch = nullptr;
  uint4 *coset_pre = nullptr;    // s^i, i < N: first-pass input factors of the coset forward kind
  uint4 *coset_post = nullptr;   // s^-i, i < N: last-pass output factors of the coset inverse kind
  uint32_t coset_shift[24] = {}; // the s of those tables (32-bit words, standard form)
  bool coset_ready = false;      // the two tables hold the powers of coset_shift
  uint32_t *kbuf = nullptr;      // constants scratch of the table builders
  std::vector<void *> allocs;
};

std::mutex g_wide_mu;
bool g_wide_ready[8] = {};
std::map<std::tuple<int, int, uint32_t>, WidePlan *> g_wide_plans;   // (device, field, log_n)

ntt_status cuda_w(cudaError_t e) { return cuda_status(e); }

template <int NL32>
ntt_status gen_table(uint4 *out, uint32_t log_m, int dir, bool use_m_inv, uint32_t log_mp, uint64_t count, int two_d,
                     bool constant, uint32_t *kbuf, cudaStream_t st) {
  constexpr int L = WideShape<NL32>::L;
  wide_constants_kernel<NL32><<<1, 1, 0, st>>>(kbuf, log_m);
  const uint32_t *ladder = constant ? nullptr : kbuf + (dir ? 32 : 0) * L;
  const uint32_t *init = kbuf + (use_m_inv ? 64 : 65) * L;
  uint64_t blocks = (count + 255) / 256;
  if (blocks > 152ull * 32) blocks = 152ull * 32;
  wide_table_kernel<NL32><<<(unsigned)(blocks ? blocks : 1), 256, 0, st>>>(out, log_mp, ladder, init, count, two_d);
  return cuda_w(cudaGetLastError());
}

ntt_status alloc_w(WidePlan *w, uint4 **out, uint64_t bytes) {
  void *p = nullptr;
  const cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_w(e);
  }
  w->allocs.push_back(p);
  *out = (uint4 *)p;
  return NTT_OK;
}

template <int NL32>
ntt_status build_wide(int field, uint32_t log_n, WidePlan *w) {
  constexpr int L = WideShape<NL32>::L, LP = WideShape<NL32>::LP;
  const uint32_t TL = (uint32_t)tile_log(field);
  const uint32_t P = (log_n + TL - 1) / TL;
  if (P > (uint32_t)kMaxPasses) return NTT_ERR_UNSUPPORTED;
  w->log_n = log_n;
  w->num_passes = P;
  for (uint32_t j = 0; j < P; ++j) w->pass_log[j] = log_n / P + (j < log_n % P ? 1 : 0);
  const uint64_t eb = 4ull * LP;   // table entry: LP words of 29-bit limbs
  uint32_t *kbuf = nullptr;
  if (cudaMalloc(&kbuf, 66 * 4 * L) != cudaSuccess) return NTT_ERR_OOM;
  w->allocs.push_back(kbuf);
  w->kbuf = kbuf;
  cudaStream_t st = nullptr;
  for (uint32_t j = 0; j < P; ++j) {
    const uint32_t logs = w->pass_log[j];
    for (int dir = 0; dir < 2; ++dir) {
      if (w->dft_tw[dir][logs]) continue;
      const uint64_t cnt = logs ? (1ull << (logs - 1)) : 1;
      NTT_TRY_W(alloc_w(w, &w->dft_tw[dir][logs], cnt * eb));
      NTT_TRY_W(gen_table<NL32>(w->dft_tw[dir][logs], logs, dir, false, 0, cnt, 0, false, kbuf, st));
    }
  }
  uint32_t log_m = w->pass_log[0];
  for (uint32_t j = 1; j < P; ++j) {
    const uint32_t logs = w->pass_log[j], log_mp = log_m;
    log_m += logs;
    for (int dir = 0; dir < 2; ++dir) {
      NTT_TRY_W(alloc_w(w, &w->tw[dir][j], (1ull << log_m) * eb));
      NTT_TRY_W(gen_table<NL32>(w->tw[dir][j], log_m, dir, dir == 1 && j == P - 1, log_mp, 1ull << log_m, 1, false,
                                kbuf, st));
    }
  }
  if (P == 1) {   // single-pass inverse: N^-1 as the pass-0 multiplier
    NTT_TRY_W(alloc_w(w, &w->pre_inv, (1ull << log_n) * eb));
    NTT_TRY_W(gen_table<NL32>(w->pre_inv, log_n, 0, true, 0, 1ull << log_n, 0, true, kbuf, st));
  }
  if (P > 1) NTT_TRY_W(alloc_w(w, &w->scratch, (1ull << log_n) * 4ull * NL32));   // memory-layout elements
  return cuda_w(cudaDeviceSynchronize());
}

// The coset tables of shift s (NL32 words, 0 < s < p), s^i and s^-i for
// i < N: allocated on the first coset call for this (device, field, size),
// rewritten in place when a call brings another shift (after the device is
// idle: transforms enqueued earlier may still read the old tables).
template <int NL32>
ntt_status build_wide_coset(WidePlan *w, const uint32_t *shift) {
  constexpr int L = WideShape<NL32>::L, LP = WideShape<NL32>::LP;
  const uint64_t n = 1ull << w->log_n, eb = 4ull * LP;
  if (!w->coset_post) {
    const size_t kept = w->allocs.size();
    uint4 *pre = nullptr, *post = nullptr;
    ntt_status s = alloc_w(w, &pre, n * eb);
    if (s == NTT_OK) s = alloc_w(w, &post, n * eb);
    if (s != NTT_OK) {   // forward and inverse stay usable
      for (size_t i = kept; i < w->allocs.size(); ++i) cudaFree(w->allocs[i]);
      w->allocs.resize(kept);
      return s;
    }
    w->coset_pre = pre;
    w->coset_post = post;
  } else {
    NTT_TRY_W(cuda_w(cudaDeviceSynchronize()));
  }
  w->coset_ready = false;   // until the tables below are written
  uint4 *pre = w->coset_pre, *post = w->coset_post;
  cudaStream_t st = nullptr;
  NTT_TRY_W(cuda_w(cudaMemcpy(w->kbuf + 64 * L, shift, 4 * NL32, cudaMemcpyHostToDevice)));
  wide_coset_constants_kernel<NL32><<<1, 1, 0, st>>>(w->kbuf);
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 152ull * 32) blocks = 152ull * 32;
  wide_table_kernel<NL32><<<(unsigned)blocks, 256, 0, st>>>(pre, 0, w->kbuf, w->kbuf + 65 * L, n, 0);
  wide_table_kernel<NL32><<<(unsigned)blocks, 256, 0, st>>>(post, 0, w->kbuf + 32 * L, w->kbuf + 65 * L, n, 0);
  NTT_TRY_W(cuda_w(cudaGetLastError()));
  NTT_TRY_W(cuda_w(cudaDeviceSynchronize()));
  std::memcpy(w->coset_shift, shift, 4 * NL32);
  w->coset_ready = true;
  return NTT_OK;
}

template <int NL, int LOGS>
cudaError_t wide_launch(int mode, const PassArgs &a, uint64_t tiles, cudaStream_t st) {
  const int smem = WideShape<NL>::kBytes;
  switch (mode) {
    case kModeInner: wide_pass_kernel<NL, LOGS, kModeInner><<<(unsigned)tiles, 256, smem, st>>>(a); break;
    case kModeFirst: wide_pass_kernel<NL, LOGS, kModeFirst><<<(unsigned)tiles, 256, smem, st>>>(a); break;
    default: wide_pass_kernel<NL, LOGS, kModeFirstPre><<<(unsigned)tiles, 256, smem, st>>>(a); break;
  }
  return cudaGetLastError();
}

template <int NL, int LOGS>
cudaError_t wide_attr() {
  const int smem = WideShape<NL>::kBytes;
  cudaError_t e = cudaFuncSetAttribute(wide_pass_kernel<NL, LOGS, kModeInner>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wide_pass_kernel<NL, LOGS, kModeFirst>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(wide_pass_kernel<NL, LOGS, kModeFirstPre>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
  return e;
}

template <int NL>
cudaError_t wide_set_attrs() {
  cudaError_t e = wide_attr<NL, 1>();
  if (e == cudaSuccess) e = wide_attr<NL, 2>();
  if (e == cudaSuccess) e = wide_attr<NL, 3>();
  if (e == cudaSuccess) e = wide_attr<NL, 4>();
  if (e == cudaSuccess) e = wide_attr<NL, 5>();
  if (e == cudaSuccess) e = wide_attr<NL, 6>();
  if (e == cudaSuccess) e = wide_attr<NL, 7>();
  if (e == cudaSuccess) e = wide_attr<NL, 8>();
  if (e == cudaSuccess) e = wide_attr<NL, 9>();
  if constexpr (WideShape<NL>::kLog >= 10) {
    if (e == cudaSuccess) e = wide_attr<NL, 10>();
  }
  return e;
}

template <int NL>
cudaError_t wide_dispatch(int logs, int mode, const PassArgs &a, uint64_t tiles, cudaStream_t st) {
  switch (logs) {
    case 1: return wide_launch<NL, 1>(mode, a, tiles, st);
    case 2: return wide_launch<NL, 2>(mode, a, tiles, st);
    case 3: return wide_launch<NL, 3>(mode, a, tiles, st);
    case 4: return wide_launch<NL, 4>(mode, a, tiles, st);
    case 5: return wide_launch<NL, 5>(mode, a, tiles, st);
    case 6: return wide_launch<NL, 6>(mode, a, tiles, st);
    case 7: return wide_launch<NL, 7>(mode, a, tiles, st);
    case 8: return wide_launch<NL, 8>(mode, a, tiles, st);
    case 9: return wide_launch<NL, 9>(mode, a, tiles, st);
    case 10:
      if constexpr (WideShape<NL>::kLog >= 10) return wide_launch<NL, 10>(mode, a, tiles, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

// The (device, field, size) tables, built on first use; with a shift
// (NL32 words), also the coset tables of that shift.  The caller holds
// g_wide_mu until its transform is enqueued, so no other call can rewrite
// the coset tables in between.
ntt_status wide_plan(int field, uint32_t log_n, const uint32_t *shift, WidePlan **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NTT_ERR_NO_DEVICE;
  if (dev < 0 || dev >= 8) return NTT_ERR_UNSUPPORTED;
  if (!g_wide_ready[dev]) {
    const WideConst<12> c12 = make_const<12>(kP377, 7);
    const WideConst<24> c24 = make_const<24>(kP753, 11);
    NTT_TRY_W(cuda_w(cudaMemcpyToSymbol(c_wide12, &c12, sizeof c12)));
    NTT_TRY_W(cuda_w(cudaMemcpyToSymbol(c_wide24, &c24, sizeof c24)));
    NTT_TRY_W(cuda_w(wide_set_attrs<12>()));
    NTT_TRY_W(cuda_w(wide_set_attrs<24>()));
    g_wide_ready[dev] = true;
  }
  auto key = std::make_tuple(dev, field, log_n);
  auto it = g_wide_plans.find(key);
  WidePlan *w = nullptr;
  if (it != g_wide_plans.end()) {
    w = it->second;
  } else {
    w = new (std::nothrow) WidePlan();
    if (!w) return NTT_ERR_OOM;
    const ntt_status s = limbs_of(field) == 12 ? build_wide<12>(field, log_n, w) : build_wide<24>(field, log_n, w);
    if (s != NTT_OK) {
      for (void *p : w->allocs) cudaFree(p);
      delete w;
      return s;
    }
    g_wide_plans[key] = w;
  }
  if (shift && (!w->coset_ready || std::memcmp(w->coset_shift, shift, 4 * limbs_of(field)) != 0)) {
    // a failure leaves forward and inverse usable and the coset tables
    // marked unwritten (the next coset call writes them again)
    NTT_TRY_W(limbs_of(field) == 12 ? build_wide_coset<12>(w, shift) : build_wide_coset<24>(w, shift));
  }
  *out = w;
  return NTT_OK;
}

// 0 < s < p for a shift of NL32 little-endian words.
bool shift_in_range(ntt_field field, const uint32_t *sw) {
  const int nl = limbs_of((int)field);
  const uint32_t *p = field == NTT_FIELD_W377 ? kP377 : kP753;
  bool zero = true;
  for (int j = 0; j < nl; ++j) zero = zero && sw[j] == 0;
  if (zero) return false;
  for (int j = nl - 1; j >= 0; --j)
    if (sw[j] != p[j]) return sw[j] < p[j];
  return false;   // s == p
}

// One transform; `shift` (NL32 words, checked by the caller) is used by the
// coset kinds only.  The table lock is held until every pass is enqueued.
ntt_status wide_transform(ntt_field field, ntt_kind kind, uint32_t log_n, const uint32_t *shift, const void *d_in,
                          void *d_out, ntt_stream stream) {
  std::lock_guard<std::mutex> lk(g_wide_mu);
  WidePlan *w = nullptr;
  const bool coset = kind == NTT_KIND_COSET || kind == NTT_KIND_COSET_INVERSE;
  const ntt_status s = wide_plan((int)field, log_n, coset ? shift : nullptr, &w);
  if (s != NTT_OK) return s;
  const int NL = limbs_of((int)field);
  const uint32_t TL = (uint32_t)tile_log((int)field);
  const int dir = (kind == NTT_KIND_INVERSE || kind == NTT_KIND_COSET_INVERSE) ? 1 : 0;
  const uint32_t P = w->num_passes;
  uint4 *work = (P > 1 && d_in == d_out) ? w->scratch : (uint4 *)d_out;
  for (uint32_t j = 0; j < P; ++j) {
    const uint32_t logs = w->pass_log[j];
    PassArgs a{};
    a.dft_tw = w->dft_tw[dir][logs];
    a.num_sub = 1ull << (log_n - logs);
    int mode;
    if (j == 0) {
      a.src = (const uint4 *)d_in;
      a.dst = P == 1 ? (uint4 *)d_out : work;
      a.log_mp = log_n - logs;
      a.num_digits = P - 1;
      uint32_t dshift = 0;
      for (uint32_t d = 1; d < P; ++d) {
        a.digit_log[d - 1] = (uint8_t)w->pass_log[d];
        a.digit_shift[d - 1] = (uint8_t)dshift;
        dshift += w->pass_log[d];
      }
      a.mul = kind == NTT_KIND_COSET ? w->coset_pre : (P == 1 && dir == 1) ? w->pre_inv : nullptr;
      mode = a.mul ? kModeFirstPre : kModeFirst;
    } else {
      uint32_t log_mp = 0;
      for (uint32_t i = 0; i < j; ++i) log_mp += w->pass_log[i];
      a.src = work;
      a.dst = j == P - 1 ? (uint4 *)d_out : work;
      a.log_mp = log_mp;
      a.mul = w->tw[dir][j];
      mode = kModeInner;
    }
    if (j == P - 1 && kind == NTT_KIND_COSET_INVERSE) a.post = w->coset_post;
    const uint64_t g = 1ull << (TL - logs);
    const uint64_t tiles = (a.num_sub + g - 1) / g;
    const cudaError_t e = NL == 12 ? wide_dispatch<12>((int)logs, mode, a, tiles, (cudaStream_t)stream)
                                   : wide_dispatch<24>((int)logs, mode, a, tiles, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return NTT_OK;
}

}  // namespace
}  // namespace gb300ntt

using namespace gb300ntt;

extern "C" {

ntt_status ntt_field_element_bytes(ntt_field field, uint32_t *bytes) {
  if (!bytes) return NTT_ERR_INVALID_ARG;
  switch (field) {
    case NTT_FIELD_BLS12_381_FR:
    case NTT_FIELD_BN254_FR: *bytes = 32; return NTT_OK;
    case NTT_FIELD_W377: *bytes = 48; return NTT_OK;
    case NTT_FIELD_W753: *bytes = 96; return NTT_OK;
    default: return NTT_ERR_INVALID_ARG;
  }
}

ntt_status ntt_wide_transform(ntt_field field, ntt_kind kind, uint32_t log_n, const void *d_in, void *d_out,
                              ntt_stream stream) {
  if (field != NTT_FIELD_W377 && field != NTT_FIELD_W753) return NTT_ERR_INVALID_ARG;
  if (kind != NTT_KIND_FORWARD && kind != NTT_KIND_INVERSE && kind != NTT_KIND_COSET && kind != NTT_KIND_COSET_INVERSE)
    return NTT_ERR_INVALID_ARG;
  if (log_n < 1 || log_n > 24) return NTT_ERR_UNSUPPORTED;
  if (!d_in || !d_out || ((uintptr_t)d_in | (uintptr_t)d_out) % 16) return NTT_ERR_INVALID_ARG;
  uint32_t gen[24] = {field == NTT_FIELD_W377 ? 7u : 11u};   // the default shift: the generator
  return wide_transform(field, kind, log_n, gen, d_in, d_out, stream);
}

ntt_status ntt_wide_transform_shift(ntt_field field, ntt_kind kind, uint32_t log_n, const uint32_t *h_shift,
                                    const void *d_in, void *d_out, ntt_stream stream) {
  if (field != NTT_FIELD_W377 && field != NTT_FIELD_W753) return NTT_ERR_INVALID_ARG;
  if (kind != NTT_KIND_COSET && kind != NTT_KIND_COSET_INVERSE) return NTT_ERR_INVALID_ARG;
  if (log_n < 1 || log_n > 24) return NTT_ERR_UNSUPPORTED;
  if (!d_in || !d_out || ((uintptr_t)d_in | (uintptr_t)d_out) % 16) return NTT_ERR_INVALID_ARG;
  if (!h_shift || !shift_in_range(field, h_shift)) return NTT_ERR_INVALID_ARG;
  return wide_transform(field, kind, log_n, h_shift, d_in, d_out, stream);
}

}  // extern "C"
