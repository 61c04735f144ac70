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
//
// Early passes (few distinct q, many rows each) are folded: their input
// factors c(q, n) go into one matrix E_q per q, so the pass before them
// needs no factor and ends in a Barrett reduction instead of the 9-row
// Montgomery product -- the bulk of the epilogue's integer work.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "host_field.h"
#include "ntt_launch.h"
#include "ntt_matrix.cuh"
#include "ntt_plan.h"

namespace gb300ntt {

constexpr uint32_t kMatrixMaxPassLog = 3;
// A pass is folded when every q has at least 2^11 rows (16 tiles of 128):
// E_q is then loaded once per 16 tiles or fewer.
constexpr uint32_t kMatFoldMinLog = 11;
constexpr uint32_t kMatFoldGroup = 4;   // four neighbouring q: one 128-byte line

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

// DFT matrix omega_S^(nk) (row-major n * S + k).
std::vector<U256> dft_matrix(const HostField &F, uint32_t logs, bool inverse) {
  const uint32_t S = 1u << logs;
  U256 w = F.root_of_unity(logs);
  if (inverse) w = F.inv(w);
  std::vector<U256> pw(S);
  pw[0] = u256(1);
  for (uint32_t i = 1; i < S; ++i) pw[i] = F.mul(pw[i - 1], w);
  std::vector<U256> D((size_t)S * S);
  for (uint32_t n = 0; n < S; ++n)
    for (uint32_t k = 0; k < S; ++k) D[(size_t)n * S + k] = pw[(n * k) % S];
  return D;
}

// Effective pass matrix V[n][k] = pre_n D[n][k] (pre empty: all 1).
std::vector<U256> with_factors(const HostField &F, uint32_t logs, const std::vector<U256> &D,
                               const std::vector<U256> &pre) {
  const uint32_t S = 1u << logs;
  std::vector<U256> V = D;
  if (!pre.empty())
    for (uint32_t n = 0; n < S; ++n)
      for (uint32_t k = 0; k < S; ++k) V[(size_t)n * S + k] = F.mul(pre[n], D[(size_t)n * S + k]);
  return V;
}

std::vector<U256> pass_matrix(const HostField &F, uint32_t logs, bool inverse, const std::vector<U256> &pre) {
  return with_factors(F, logs, dft_matrix(F, logs, inverse), pre);
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

template <class T>
ntt_status upload(ntt_plan, const std::vector<uint8_t> &buf, T **out) {
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

// cuTensorMapEncodeTiled, fetched once through the runtime (no link to the
// driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// The pass input as a 4-D tensor of 64-bit words {4, Mp, S, N / (Mp S)}
// (element q + n Mp + o Mp S of the vector at coordinates (., q, n, o)), and
// the box one chunk copies: the tile's rows d = q + o Mp of one input n --
// 128 consecutive d ({4, min(Mp, rows), 1, rows / min(Mp, rows)}), or for a
// folded pass 128 consecutive o of one q ({4, 1, 1, 128}).
ntt_status encode_input_map(CUtensorMap *map, const PassArgs &a, uint32_t log_n, uint32_t logs, bool fold) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return NTT_ERR_CUDA;
  const uint64_t mp = 1ull << a.log_mp, S = 1ull << logs;
  const cuuint64_t dims[4] = {4, mp, S, (1ull << log_n) >> (a.log_mp + logs)};
  const cuuint64_t strides[3] = {32, 32 * mp, 32 * mp * S};
  const uint64_t rows = a.num_sub < (uint64_t)kMatRows ? a.num_sub : (uint64_t)kMatRows;
  const uint64_t bm = fold ? 1 : std::min(mp, rows);
  const cuuint32_t box[4] = {4, (cuuint32_t)bm, 1, (cuuint32_t)(fold ? kMatRows : rows / bm)};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<uint4 *>(a.src), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        fold ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? NTT_OK : NTT_ERR_CUDA;
}

// Passes 1..f of nested plan q that are folded: each q needs at least
// 2^kMatFoldMinLog rows, and the last pass is never folded.
uint32_t fold_passes(ntt_plan q) {
  uint32_t f = 0, L = q->pass_log[0];
  for (uint32_t j = 1; j + 1 < q->num_passes; ++j) {
    L += q->pass_log[j];
    if (q->log_n < L + kMatFoldMinLog) break;
    f = j;
  }
  return f;
}

uint32_t pass_log_mp(ntt_plan q, uint32_t j) {
  uint32_t l = 0;
  for (uint32_t i = 0; i < j; ++i) l += q->pass_log[i];
  return l;
}

// Run body(i) for i < count on the host's cores.
template <class Body>
void parallel_for(uint64_t count, const Body &body) {
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  const uint64_t nt = std::min<uint64_t>(hw, count);
  if (nt <= 1) {
    for (uint64_t i = 0; i < count; ++i) body(i);
    return;
  }
  std::vector<std::thread> pool;
  for (uint64_t t = 0; t < nt; ++t)
    pool.emplace_back([&, t] {
      for (uint64_t i = t; i < count; i += nt) body(i);
    });
  for (auto &th : pool) th.join();
}

void free_fold(MatrixResources *m, int tk) {
  for (uint32_t j = 0; j < (uint32_t)kMaxPasses; ++j) {
    if (m->e_fold[tk][j]) cudaFree(m->e_fold[tk][j]);
    if (m->off_fold[tk][j]) cudaFree(m->off_fold[tk][j]);
    m->e_fold[tk][j] = nullptr;
    m->off_fold[tk][j] = nullptr;
  }
}

// E_q and the merge offsets of every folded pass of table kind tk: V[n][k]
// = c(q, n) omega_S^(+-nk), c(q, n) = entry q + n Mp of the pass's input
// factor table (read back from the device, Montgomery form).  The last
// folded pass ends in the Montgomery product with the next pass's factors
// (E scaled by 2^32); the others feed a folded pass and end in Barrett.
ntt_status build_fold_tables(ntt_plan p, int tk) {
  MatrixResources *m = p->matrix;
  ntt_plan q = m->nested;
  free_fold(m, tk);
  if (m->fold == 0) return NTT_OK;
  const HostField F = host_field(p->field);
  const U256 rinv = F.r_inv();
  for (uint32_t j = 1; j <= m->fold; ++j) {
    const uint32_t logs = q->pass_log[j], S = 1u << logs, K = 32 * S;
    const uint64_t mp = 1ull << pass_log_mp(q, j);
    const size_t eb = (size_t)K * K * 2;
    std::vector<uint32_t> raw((size_t)mp * S * 8);
    ntt_status s =
        cuda_status(cudaMemcpy(raw.data(), q->tw[tk][j], raw.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (s != NTT_OK) return s;
    const std::vector<U256> D = dft_matrix(F, logs, tk == kInverse);
    std::vector<uint8_t> all(mp * eb);
    std::vector<uint32_t> offs((size_t)mp * S * 8);
    const bool scaled = j == m->fold;
    parallel_for(mp, [&](uint64_t qi) {
      std::vector<U256> pre(S);
      for (uint32_t n = 0; n < S; ++n) {
        const uint32_t *w = &raw[(qi + (uint64_t)n * mp) * 8];
        U256 v;
        for (int i = 0; i < 4; ++i) v.w[i] = (uint64_t)w[2 * i] | ((uint64_t)w[2 * i + 1] << 32);
        pre[n] = F.mul(v, rinv);
      }
      std::vector<uint8_t> buf;
      uint32_t off[8][8];
      build_e16(F, logs, with_factors(F, logs, D, pre), scaled, &buf, off);
      std::memcpy(&all[qi * eb], buf.data(), eb);
      for (uint32_t k = 0; k < S; ++k) std::memcpy(&offs[(qi * S + k) * 8], off[k], 32);
    });
    s = upload(p, all, &m->e_fold[tk][j]);
    std::vector<uint8_t> ob(offs.size() * sizeof(uint32_t));
    std::memcpy(ob.data(), offs.data(), ob.size());
    if (s == NTT_OK) s = upload(p, ob, &m->off_fold[tk][j]);
    if (s != NTT_OK) return s;
  }
  return NTT_OK;
}

uint64_t fold_bytes(const MatrixResources *m, ntt_plan q) {
  uint64_t b = 0;
  for (uint32_t j = 1; j <= m->fold; ++j) {
    const uint64_t S = 1ull << q->pass_log[j], K = 32 * S;
    b += (1ull << pass_log_mp(q, j)) * (K * K * 2 + S * 32);
  }
  return b;
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
  for (int tk = 0; tk < 3; ++tk) free_fold(m, tk);
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
  // pass 0 of a coset forward ends in Barrett when it is the only pass or
  // feeds a folded pass
  const int sc = q->num_passes > 1 && m->fold == 0 ? 1 : 0;
  build_e16(F, q->pass_log[0], V, sc == 1, &buf, m->off_first[kCoset][sc]);
  ntt_status s = upload(p, buf, &m->e_first[kCoset][sc]);
  if (s == NTT_OK) s = build_fold_tables(p, kCoset);
  return s;
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
  m->fold = fold_passes(q);
  for (uint32_t j = m->fold + 1; j < P; ++j) {
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
    // pass 0 ends in Barrett when it is the only pass (no coset inverse) or
    // feeds a folded pass
    if ((P > 1 && m->fold == 0) || (P == 1 && tk == kInverse && p->has_coset))
      need(&s, &m->e_first[tk][1], logs, tk == kInverse, pre, true, m->off_first[tk][1]);
    if (P == 1 || m->fold > 0) need(&s, &m->e_first[tk][0], logs, tk == kInverse, pre, false, m->off_first[tk][0]);
    if (s == NTT_OK) s = build_fold_tables(p, tk);
    if (s == NTT_OK) p->device_bytes += fold_bytes(m, q);
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
    const bool folded = j >= 1 && j <= m->fold;
    // no factor (Barrett) for the last pass without output factors and for
    // a pass that feeds a folded pass
    const bool barrett = (j == P - 1 && !ma.a.post) || j < m->fold;
    const int sc = barrett ? 0 : 1;
    if (j == 0) {
      ma.e = m->e_first[tk][sc];
      std::memcpy(ma.off, m->off_first[tk][sc], sizeof ma.off);
      mode = kModeFirst;   // the pass-0 factors are in E
    } else if (folded) {
      ma.e = m->e_fold[tk][j];
      ma.off_fold = m->off_fold[tk][j];
      ma.fold = 1;
      ma.fold_group = kMatFoldGroup;
      // 2^(log_n - L_j) rows per q, at least 2^kMatFoldMinLog
      const uint32_t rows_log = q->log_n - log_m;
      ma.tiles_per_q_log = rows_log - 7;
      if (!ma.off_fold || rows_log < kMatFoldMinLog || (1ull << ma.a.log_mp) < kMatFoldGroup)
        return NTT_ERR_UNSUPPORTED;
    } else {
      ma.e = m->e_inner[dir][logs][sc];
      std::memcpy(ma.off, m->off_inner[dir][logs][sc], sizeof ma.off);
    }
    ma.barrett = barrett ? 1u : 0u;
    ma.lazy = j + 1 < P ? 1u : 0u;   // the last pass's outputs are canonical
    ma.mu = m->mu;
    if (!ma.e) return NTT_ERR_UNSUPPORTED;
    if (j + 1 < P && !barrett) {
      ma.next = q->tw[tk][j + 1];
      ma.next_log = log_m + q->pass_log[j + 1];
    }
    ma.post = ma.a.post;   // last pass of a coset inverse: s^-n
    std::memcpy(ma.one, m->one, sizeof ma.one);
    ma.err = m->err;
    ma.wait_ns = 1000000000ull;
    CUtensorMap map;
    const ntt_status ms = encode_input_map(&map, ma.a, q->log_n, logs, folded);
    if (ms != NTT_OK) return ms;
    const uint64_t units = folded ? ((1ull << ma.a.log_mp) / kMatFoldGroup) << ma.tiles_per_q_log
                                  : (ma.a.num_sub + kMatRows - 1) / kMatRows;
    const uint64_t sms = (uint64_t)p->sm_count;
    // folded: whole groups of CTAs
    const uint32_t grid = folded ? (uint32_t)(std::min(units, sms / kMatFoldGroup) * kMatFoldGroup)
                                 : (uint32_t)std::min(units, sms);
    cudaError_t e = timing_begin(p, (int)j, st);
    if (e == cudaSuccess) e = L.matrix_pass((int)logs, mode, ma, map, grid, st);
    if (e == cudaSuccess) e = timing_end(p, st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return NTT_OK;
}

}  // namespace gb300ntt
