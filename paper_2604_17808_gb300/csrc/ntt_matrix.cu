// ntt_matrix.cu -- plan resources and launches of the matrix-form path.
//
// The matrix path runs every pass as a tensor-core product with a byte
// matrix E (ntt_matrix.cuh).  Its passes are at most 2^3 points (K = N =
// 32 S <= 256 keeps every fp32 partial sum within 2^22), so a plan on this
// path owns a nested plan with that split whose inter-pass, coset and
// inverse tables are used as on the butterfly path -- except that each
// pass's epilogue applies the NEXT pass's input factors, and the pass-0
// factors (coset powers; N^-1 of a single-pass inverse) are folded into the
// pass-0 matrix E.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "host_field.h"
#include "ntt_launch.h"
#include "ntt_matrix.cuh"
#include "ntt_plan.h"

namespace gb300ntt {

constexpr uint32_t kMatrixMaxPassLog = 3;

namespace {

// Balanced base-256 digits of a canonical value (< 2^255): digit h in
// [-128, 127], sum_h digit_h 2^(8h) = v.  The top digit stays below 128
// because v < 2^255.
void balanced_digits(const U256 &v, int out[32]) {
  int carry = 0;
  for (int h = 0; h < 32; ++h) {
    int d = (int)((v.w[h / 8] >> (8 * (h % 8))) & 0xFF) + carry;
    carry = d >= 128 ? 1 : 0;
    out[h] = d - (carry << 8);
  }
}

// IEEE fp16 bit pattern of an integer in [-128, 128] (exact).
uint16_t f16_bits(int v) {
  if (v == 0) return 0;
  const uint16_t sign = v < 0 ? 0x8000 : 0;
  unsigned a = (unsigned)(v < 0 ? -v : v);
  int e = 0;
  while ((a >> (e + 1)) != 0) ++e;                      // a in [2^e, 2^(e+1))
  const unsigned mant = (a << (10 - e)) & 0x3FF;        // 10 fraction bits
  return (uint16_t)(sign | ((unsigned)(e + 15) << 10) | mant);
}

// Effective pass matrix V[n][k] = pre_n omega^(nk) (row-major n * S + k).
std::vector<U256> pass_matrix(const HostField &F, uint32_t logs, bool inverse, const std::vector<U256> &pre) {
  const uint32_t S = 1u << logs;
  U256 w = F.root_of_unity(logs);
  if (inverse) w = F.inv(w);
  std::vector<U256> V((size_t)S * S);
  for (uint32_t n = 0; n < S; ++n)
    for (uint32_t k = 0; k < S; ++k) {
      const U256 t = F.pow(w, (uint64_t)((n * k) % S));
      V[(size_t)n * S + k] = pre.empty() ? t : F.mul(pre[n], t);
    }
  return V;
}

U256 times_pow2(const HostField &F, U256 v, unsigned e) {
  for (unsigned i = 0; i < e; ++i) v = F.add(v, v);
  return v;
}

// E[(k,h),(n,b)] = digit h of V[n][k] 2^(8b) g mod p, fp16, in the K-major
// B-operand layout (N = K = 32 S), and the merge offsets
// O_k = g C sum_n V[n][k] - B sum_h 2^(8h) mod p, C = 128 sum_b 2^(8b),
// B = 0x4B400000 (the fp32 pattern of 1.5 2^23 in every accumulator), with
// g = 2^32 for passes whose epilogue is the 9-row Montgomery product (its
// 2^-288 leaves 2^-32 after the table's 2^256) and g = 1 for a last pass
// reduced by Barrett.
void build_e16(const HostField &F, uint32_t logs, const std::vector<U256> &V, bool scaled, std::vector<uint8_t> *e,
               uint32_t off[8][8]) {
  const uint32_t S = 1u << logs, K = 32 * S;
  const unsigned gexp = scaled ? 32 : 0;
  e->assign((size_t)K * K * 2, 0);
  for (uint32_t n = 0; n < S; ++n) {
    for (uint32_t k = 0; k < S; ++k) {
      U256 wv = times_pow2(F, V[(size_t)n * S + k], gexp);
      for (uint32_t b = 0; b < 32; ++b) {
        int dg[32];
        balanced_digits(wv, dg);
        for (uint32_t h = 0; h < 32; ++h) {
          const uint16_t bits = f16_bits(dg[h]);
          std::memcpy(&(*e)[core_offset(32 * k + h, 32 * n + b, K)], &bits, 2);
        }
        wv = times_pow2(F, wv, 8);
      }
    }
  }
  U256 sigma = u256(0), pw = u256(1);   // sum_{i<32} 2^(8i) mod p
  for (int i = 0; i < 32; ++i) {
    sigma = F.add(sigma, pw);
    pw = times_pow2(F, pw, 8);
  }
  const U256 c = F.mul(F.reduce_small(128), sigma);
  const U256 bsig = F.mul(F.reduce_small(0x4B400000u), sigma);
  std::memset(off, 0, sizeof(uint32_t) * 64);
  for (uint32_t k = 0; k < S; ++k) {
    U256 colsum = u256(0);
    for (uint32_t n = 0; n < S; ++n) colsum = F.add(colsum, V[(size_t)n * S + k]);
    const U256 corr = times_pow2(F, F.mul(c, colsum), gexp);
    const U256 o = F.sub(corr, bsig);
    for (int i = 0; i < 4; ++i) {
      off[k][2 * i] = (uint32_t)o.w[i];
      off[k][2 * i + 1] = (uint32_t)(o.w[i] >> 32);
    }
  }
}

ntt_status upload(ntt_plan p, const std::vector<uint8_t> &buf, uint4 **out) {
  if (*out) {
    cudaFree(*out);
    *out = nullptr;
  }
  ntt_status s = cuda_status(cudaMalloc(out, buf.size()));
  if (s == NTT_OK) s = cuda_status(cudaMemcpy(*out, buf.data(), buf.size(), cudaMemcpyHostToDevice));
  return s;
}

// floor(2^288 / p) by binary long division (the quotient has 34 bits).
uint64_t barrett_mu(const HostField &F) {
  U256 r = u256(0);
  uint64_t q = 0;
  for (int i = 288; i >= 0; --i) {
    r = u256_add_raw(r, r);   // r < p < 2^255: no overflow
    if (i == 288) r = u256_add_raw(r, u256(1));
    if (u256_geq(r, F.p)) {
      r = u256_sub_raw(r, F.p);
      if (i < 64) q |= 1ull << i;
    }
  }
  return q;
}

// Pass-0 factors pre_n of table kind tk for the nested plan q (empty: all 1).
std::vector<U256> pass0_factors(const HostField &F, ntt_plan q, int tk) {
  const uint32_t logs0 = q->pass_log[0], S0 = 1u << logs0;
  std::vector<U256> pre;
  if (tk == kInverse && q->num_passes == 1) {
    const U256 ninv = F.inv(F.reduce_small(1ull << q->log_n));
    pre.assign(S0, ninv);
  } else if (tk == kCoset) {
    // s^(n N / S_0)
    const U256 step = F.pow(q->coset_shift, 1ull << (q->log_n - logs0));
    pre.resize(S0);
    U256 acc = u256(1);
    for (uint32_t n = 0; n < S0; ++n) {
      pre[n] = acc;
      acc = F.mul(acc, step);
    }
  }
  return pre;
}

}  // namespace

bool matrix_path_available(ntt_plan) { return true; }

void release_matrix_resources(ntt_plan p) {
  MatrixResources *m = p->matrix;
  if (!m) return;
  if (m->nested) ntt_plan_destroy(m->nested);
  for (auto &dir : m->e_inner)
    for (auto &lg : dir)
      for (uint4 *q : lg)
        if (q) cudaFree(q);
  for (auto &tk : m->e_first)
    for (uint4 *q : tk)
      if (q) cudaFree(q);
  if (m->err) cudaFree(m->err);
  delete m;
  p->matrix = nullptr;
}

// (Re)build the pass-0 matrix of the coset kind (after a coset-shift change).
ntt_status matrix_build_coset(ntt_plan p) {
  MatrixResources *m = p->matrix;
  if (!m || !m->nested || !p->has_coset) return NTT_OK;
  const HostField F = host_field(p->field);
  ntt_plan q = m->nested;
  std::vector<uint8_t> buf;
  const std::vector<U256> V = pass_matrix(F, q->pass_log[0], false, pass0_factors(F, q, kCoset));
  const int sc = q->num_passes > 1 ? 1 : 0;   // a single pass of a coset forward ends in Barrett
  build_e16(F, q->pass_log[0], V, sc == 1, &buf, m->off_first[kCoset][sc]);
  return upload(p, buf, &m->e_first[kCoset][sc]);
}

static ntt_status ensure_matrix(ntt_plan p) {
  if (p->matrix) return NTT_OK;
  MatrixResources *m = new (std::nothrow) MatrixResources();
  if (!m) return NTT_ERR_OOM;
  p->matrix = m;
  ntt_plan q = new (std::nothrow) ntt_plan_s();
  if (!q) return NTT_ERR_OOM;
  m->nested = q;
  q->device = p->device;
  q->field = p->field;
  q->log_n = p->log_n;
  q->has_coset = p->has_coset;
  q->sm_count = p->sm_count;
  cudaStream_t st = nullptr;
  ntt_status s = cuda_status(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  const std::vector<uint32_t> split = split_passes_max(p->log_n, kMatrixMaxPassLog);
  if (s == NTT_OK) s = build_plan(q, st, &split);
  if (s == NTT_OK && p->has_coset && !u256_is_zero(p->coset_shift) &&
      !(p->coset_shift.w[0] == host_field(p->field).generator && p->coset_shift.w[1] == 0 &&
        p->coset_shift.w[2] == 0 && p->coset_shift.w[3] == 0))
    s = build_coset_tables(q, p->coset_shift, st);
  if (st) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (s == NTT_OK) s = cuda_status(e);
    cudaStreamDestroy(st);
  }
  if (s != NTT_OK) return s;
  const HostField F = host_field(p->field);
  std::vector<uint8_t> buf;
  const uint32_t P = q->num_passes;
  // Matrices needed: [scaled] = the pass ends in the 9-row Montgomery product
  // (every pass but the last, and the last pass of a coset inverse, whose
  // factor is s^-n); unscaled = a last pass reduced by Barrett.
  auto need = [&](ntt_status *st, uint4 **slot, uint32_t logs, bool inverse, const std::vector<U256> &pre,
                  bool scaled, uint32_t off[8][8]) {
    if (*st != NTT_OK || *slot) return;
    build_e16(F, logs, pass_matrix(F, logs, inverse, pre), scaled, &buf, off);
    *st = upload(p, buf, slot);
    if (*st == NTT_OK) p->device_bytes += buf.size();
  };
  for (uint32_t j = 1; j < P; ++j) {
    const uint32_t logs = q->pass_log[j];
    for (int dir = 0; dir < 2; ++dir) {
      const bool last = j == P - 1;
      if (!last || (dir == 1 && p->has_coset))
        need(&s, &m->e_inner[dir][logs][1], logs, dir == 1, {}, true, m->off_inner[dir][logs][1]);
      if (last) need(&s, &m->e_inner[dir][logs][0], logs, dir == 1, {}, false, m->off_inner[dir][logs][0]);
    }
  }
  for (int tk = kForward; tk <= kCoset; ++tk) {
    if (tk == kCoset && !p->has_coset) continue;
    const std::vector<U256> pre = pass0_factors(F, q, tk);
    const uint32_t logs = q->pass_log[0];
    if (P > 1 || (tk == kInverse && p->has_coset))
      need(&s, &m->e_first[tk][1], logs, tk == kInverse, pre, true, m->off_first[tk][1]);
    if (P == 1) need(&s, &m->e_first[tk][0], logs, tk == kInverse, pre, false, m->off_first[tk][0]);
  }
  if (s != NTT_OK) return s;
  m->mu = barrett_mu(F);
  const U256 one = F.to_mont(u256(1));
  for (int i = 0; i < 4; ++i) {
    m->one[2 * i] = (uint32_t)one.w[i];
    m->one[2 * i + 1] = (uint32_t)(one.w[i] >> 32);
  }
  s = cuda_status(cudaMalloc(&m->err, sizeof(uint32_t)));
  if (s == NTT_OK) s = cuda_status(cudaMemset(m->err, 0, sizeof(uint32_t)));
  p->device_bytes += q->device_bytes;
  return s;
}

ntt_status prepare_matrix_path(ntt_plan p) {
  const ntt_status s = ensure_matrix(p);
  if (s != NTT_OK) release_matrix_resources(p);
  return s;
}

uint32_t matrix_launches(ntt_plan p) { return p->matrix && p->matrix->nested ? p->matrix->nested->num_passes : 0; }

ntt_status matrix_poll_error(ntt_plan p, uint32_t *code) {
  *code = 0;
  if (!p->matrix || !p->matrix->err) return NTT_OK;
  ntt_status s = cuda_status(cudaMemcpy(code, p->matrix->err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (s == NTT_OK) s = cuda_status(cudaMemset(p->matrix->err, 0, sizeof(uint32_t)));
  return s;
}

ntt_status enqueue_matrix_transform(ntt_plan p, int kind, const void *in, void *out, cudaStream_t st) {
  MatrixResources *m = p->matrix;
  if (!m || !m->nested) return NTT_ERR_UNSUPPORTED;
  ntt_plan q = m->nested;
  const FieldLaunchers &L = launchers(p->field);
  const int tk = table_kind(kind);
  const int dir = tk == kInverse ? 1 : 0;
  uint32_t log_m = 0;
  const uint32_t P = q->num_passes;
  for (uint32_t j = 0; j < P; ++j) {
    MatrixPassArgs ma{};
    int mode = 0;
    build_pass_args(q, kind, in, out, j, &ma.a, &mode);
    const uint32_t logs = q->pass_log[j];
    log_m += logs;
    // the last pass without output factors ends in a Barrett reduction
    const bool barrett = j == P - 1 && !ma.a.post;
    const int sc = barrett ? 0 : 1;
    if (j == 0) {
      ma.e = m->e_first[tk][sc];
      std::memcpy(ma.off, m->off_first[tk][sc], sizeof ma.off);
      mode = kModeFirst;   // the pass-0 factors are in E
    } else {
      ma.e = m->e_inner[dir][logs][sc];
      std::memcpy(ma.off, m->off_inner[dir][logs][sc], sizeof ma.off);
    }
    ma.barrett = barrett ? 1u : 0u;
    ma.mu = m->mu;
    if (!ma.e) return NTT_ERR_UNSUPPORTED;
    if (j + 1 < P) {
      ma.next = q->tw[tk][j + 1];
      ma.next_log = log_m + q->pass_log[j + 1];
    }
    ma.post = ma.a.post;   // last pass of a coset inverse: s^-n
    std::memcpy(ma.one, m->one, sizeof ma.one);
    ma.err = m->err;
    ma.wait_ns = 1000000000ull;
    const uint64_t tiles = (ma.a.num_sub + kMatRows - 1) / kMatRows;
    const uint32_t grid = (uint32_t)(tiles < (uint64_t)p->sm_count ? tiles : (uint64_t)p->sm_count);
    cudaError_t e = timing_begin(p, (int)j, st);
    if (e == cudaSuccess) e = L.matrix_pass((int)logs, mode, ma, grid, st);
    if (e == cudaSuccess) e = timing_end(p, st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return NTT_OK;
}

}  // namespace gb300ntt
