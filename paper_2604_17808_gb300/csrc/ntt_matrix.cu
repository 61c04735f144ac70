// ntt_matrix.cu -- plan resources and launches of the matrix-form path.
//
// The matrix path runs every pass as a tensor-core product with a byte
// matrix E (ntt_matrix.cuh).  Its passes are at most 2^3 points (K = N =
// 32 S <= 256 keeps every fp32 partial sum exact), so a plan on this path
// owns a nested plan with that split: the nested plan's inter-pass tables,
// coset and inverse factors are used exactly as on the butterfly path; its
// DFT twiddle tables are replaced by E.
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

int signed_digit(const U256 &v, int b, int *carry) {
  int d = (int)((v.w[b / 8] >> (8 * (b % 8))) & 0xFF) + *carry;
  *carry = d >= 128 ? 1 : 0;
  return d - (*carry << 8);
}

uint16_t bf16_bits(int v) {
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);  // exact for |v| <= 256
}

// E[(k,h), (n,b)] = signed digit h of omega_S^(dir * n k) * 2^(8b) * 2^256 mod p,
// stored as the K-major B operand (N = K = 32 S rows/columns).
std::vector<uint8_t> build_e(const HostField &F, uint32_t logs, bool inverse) {
  const uint32_t S = 1u << logs, K = 32 * S;
  std::vector<uint8_t> buf((size_t)K * K * 2, 0);
  U256 w = F.root_of_unity(logs);
  if (inverse) w = F.inv(w);
  for (uint32_t n = 0; n < S; ++n) {
    for (uint32_t k = 0; k < S; ++k) {
      U256 v = F.to_mont(F.pow(w, (uint64_t)((n * k) % S)));
      for (uint32_t b = 0; b < 32; ++b) {
        int carry = 0;
        for (uint32_t h = 0; h < 32; ++h) {
          const int dg = signed_digit(v, (int)h, &carry);
          const uint16_t bits = bf16_bits(dg);
          const uint32_t off = core_offset(32 * k + h, 32 * n + b, K);
          std::memcpy(&buf[off], &bits, 2);
        }
        for (int i = 0; i < 8; ++i) v = F.add(v, v);  // * 2^8
      }
    }
  }
  return buf;
}

}  // namespace

bool matrix_path_available(ntt_plan) { return true; }

void release_matrix_resources(ntt_plan p) {
  MatrixResources *m = p->matrix;
  if (!m) return;
  if (m->nested) ntt_plan_destroy(m->nested);
  for (auto &row : m->e)
    for (uint4 *q : row)
      if (q) cudaFree(q);
  if (m->err) cudaFree(m->err);
  delete m;
  p->matrix = nullptr;
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
  for (uint32_t j = 0; j < q->num_passes; ++j) {
    const uint32_t logs = q->pass_log[j];
    for (int dir = 0; dir < 2; ++dir) {
      if (m->e[dir][logs]) continue;
      const std::vector<uint8_t> buf = build_e(F, logs, dir == 1);
      s = cuda_status(cudaMalloc(&m->e[dir][logs], buf.size()));
      if (s == NTT_OK) s = cuda_status(cudaMemcpy(m->e[dir][logs], buf.data(), buf.size(), cudaMemcpyHostToDevice));
      if (s != NTT_OK) return s;
      p->device_bytes += buf.size();
    }
  }
  U256 off = F.p;  // 2^18 * p (< 2^274), nine limbs
  uint32_t limbs[9] = {};
  for (int i = 0; i < 4; ++i) {
    limbs[2 * i] = (uint32_t)off.w[i];
    limbs[2 * i + 1] = (uint32_t)(off.w[i] >> 32);
  }
  for (int sh = 0; sh < 18; ++sh) {
    uint32_t c = 0;
    for (int i = 0; i < 9; ++i) {
      const uint32_t nc = limbs[i] >> 31;
      limbs[i] = (limbs[i] << 1) | c;
      c = nc;
    }
  }
  std::memcpy(m->offset, limbs, sizeof limbs);
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
  const int dir = table_kind(kind) == kInverse ? 1 : 0;
  for (uint32_t j = 0; j < q->num_passes; ++j) {
    MatrixPassArgs ma{};
    int mode = 0;
    build_pass_args(q, kind, in, out, j, &ma.a, &mode);
    const uint32_t logs = q->pass_log[j];
    ma.e = m->e[dir][logs];
    std::memcpy(ma.offset, m->offset, sizeof ma.offset);
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
