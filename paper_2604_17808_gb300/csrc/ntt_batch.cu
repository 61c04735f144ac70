// ntt_batch.cu -- batched submission of many transforms.
#include "ntt_plan.h"

using namespace gb300ntt;

extern "C" ntt_status ntt_batch_submit(const ntt_job *jobs, size_t n, ntt_stream stream) {
  if (!jobs && n) return NTT_ERR_INVALID_ARG;
  for (size_t i = 0; i < n; ++i) {
    const ntt_job &j = jobs[i];
    if (!j.plan || j.in == j.out) return NTT_ERR_INVALID_ARG;
    if (j.kind < 0 || j.kind > 2 || (j.kind == kCoset && !j.plan->has_coset)) return NTT_ERR_INVALID_ARG;
    ntt_status s = check_buffer(j.in);
    if (s == NTT_OK) s = check_buffer(j.out);
    if (s != NTT_OK) return s;
  }
  for (size_t i = 0; i < n; ++i) {
    const ntt_status s = enqueue_transform(jobs[i].plan, jobs[i].kind, jobs[i].in, jobs[i].out, (cudaStream_t)stream);
    if (s != NTT_OK) return s;
  }
  return NTT_OK;
}
