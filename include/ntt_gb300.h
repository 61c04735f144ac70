/*
 * ntt_gb300.h -- C ABI of the GB300 (sm_103a) 255-bit number-theoretic
 * transform library.
 *
 * The operation (MORPH, Sec. 2.3.1, the NTT definition): for a
 * vector x of N = 2^log_n elements of the prime field F_M,
 *
 *     forward:  X_k = sum_{n<N} x_n * omega_N^{k n}            mod M
 *     inverse:  x_n = N^{-1} * sum_{k<N} X_k * omega_N^{-k n}   mod M
 *     coset:    X_k = sum_{n<N} x_n * (s * omega_N^k)^n          mod M
 *
 * with omega_N = g^((M-1)/N), g the field's multiplicative generator (7 for
 * BLS12-381 Fr, 5 for BN254 Fr) and s the coset shift (default g).  The
 * paper states the forward transform; inverse and coset are the standard
 * companions of a prover's evaluation / interpolation step.  The results are
 * exact: no rounding, outputs canonical in [0, M).
 *
 * Data layout (every buffer, host or device): N elements, element i at byte
 * offset 32*i, each element four little-endian uint64 limbs (limb 0 least
 * significant), standard (not Montgomery) representation, canonical in
 * [0, M), natural order in and out.  Device buffers must be 32-byte aligned
 * (one element; the kernels move each element with one 256-bit access).
 *
 * Ownership: the caller owns every input and output buffer.  A plan owns its
 * device-resident twiddle tables and one scratch vector of N elements, all
 * allocated by ntt_plan_create on the current CUDA device and freed by
 * ntt_plan_destroy.
 *
 * Streams and asynchrony: ntt_forward / ntt_inverse / ntt_coset_forward /
 * ntt_batch_submit only enqueue work on `stream` (a cudaStream_t; NULL is the
 * legacy default stream) and return without synchronising.  Their status
 * covers argument and launch errors only.  Errors detected on the device
 * (a bounded wait that ran out, see ntt_batch_submit) are read afterwards
 * with ntt_batch_poll_error.
 *
 * Concurrency: a plan is immutable after creation (except the two setters
 * below, which must not race with transforms).  Out-of-place transforms
 * (in != out) on one plan may run concurrently on several streams.  In-place
 * transforms (in == out) with more than one pass use the plan's scratch
 * vector, so concurrent in-place transforms on one plan race: order them on
 * one stream or use one plan per stream.
 *
 * Errors: every call returns an ntt_status; NTT_ERR_INVALID_ARG for a NULL
 * plan or buffer, a misaligned buffer or an unknown enum value;
 * NTT_ERR_UNSUPPORTED for log_n outside [1, min(2-adicity, 28)];
 * NTT_ERR_OOM when a device allocation fails; NTT_ERR_CUDA for any other CUDA
 * runtime error (the CUDA error is kept by the runtime as usual).  Inputs
 * must be canonical (< M): non-canonical inputs are a precondition violation
 * and give unspecified (but memory-safe) outputs.
 */
#ifndef NTT_GB300_H
#define NTT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
/* Same type as cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st *ntt_stream;

typedef enum ntt_status {
    NTT_OK = 0,
    NTT_ERR_INVALID_ARG = 1,
    NTT_ERR_UNSUPPORTED = 2,
    NTT_ERR_OOM = 3,
    NTT_ERR_CUDA = 4,
    NTT_ERR_TIMEOUT = 5,   /* a device-side bounded wait ran out */
    NTT_ERR_BUDGET = 6,    /* a memory budget would be exceeded */
    NTT_ERR_NO_DEVICE = 7, /* no usable CUDA device of compute capability 10.3 */
    NTT_ERR_BOUNDS = 8     /* debug builds (NTT_DEBUG): a kernel index fell outside its buffer */
} ntt_status;

typedef enum ntt_field {
    NTT_FIELD_BLS12_381_FR = 0, /* r = 0x73eda753...ffffffff00000001, 255 bits, 2-adicity 32, g = 7 */
    NTT_FIELD_BN254_FR = 1,     /* r = 0x30644e72...43e1f593f0000001, 254 bits, 2-adicity 28, g = 5 */
    /* Wider fields for the paper's 377- and 753-bit rows (Sec. 4.3.1, Tab. 3),
     * used through ntt_wide_transform only: the smallest primes c 2^32 + 1
     * (c odd) above floor(pi 2^(b-2)), 2-adicity 32, generators 7 and 11. */
    NTT_FIELD_W377 = 2,         /* 0x1921fb54...bdf2bd500000001, 377 bits; 48-byte elements */
    NTT_FIELD_W753 = 3          /* 0x1921fb54...dcd300000001, 753 bits; 96-byte elements */
} ntt_field;

typedef enum ntt_kind {
    NTT_KIND_FORWARD = 0,
    NTT_KIND_INVERSE = 1,
    NTT_KIND_COSET = 2,     /* coset forward: X_k = sum_n x_n (s omega^k)^n */
    NTT_KIND_COSET_INVERSE = 3 /* coset inverse: x_n = s^-n N^-1 sum_k X_k omega^-nk
                                  (interpolation from the coset s<omega>; undoes
                                  NTT_KIND_COSET).  Not in the paper, which states
                                  the forward transform only (Sec. 2.3.1); it is the
                                  prover step after pointwise work on coset
                                  evaluations. */
} ntt_kind;

typedef enum ntt_path {
    NTT_PATH_AUTO = 0,      /* the library's choice (butterfly passes) */
    NTT_PATH_BUTTERFLY = 1, /* radix-2^k shared-memory butterfly passes on 32-bit IMAD (Fig. 5a) */
    NTT_PATH_MATRIX = 2     /* matrix-form column DFT on tensor cores (Sec. 3.3.2; Alg. 1 ByteDecompose/Einsum/ByteMerge) */
} ntt_path;

typedef struct ntt_plan_s *ntt_plan;

/*
 * Create a plan for N = 2^log_n elements of `field` on the current CUDA
 * device.  Builds (on the device) the twiddle tables of the forward and the
 * inverse transform, and of the coset transform when `coset` is nonzero
 * (shift = the field's generator) and its inverse, and allocates the scratch
 * vector.  Cost: a few milliseconds plus about (3 + 2 * coset) * 32 * N bytes
 * of device memory.  On success *out holds the plan; on failure *out is NULL.
 */
ntt_status ntt_plan_create(ntt_plan *out, ntt_field field, uint32_t log_n, int coset);

/*
 * Choose the path used by later transforms on this plan.  The first switch
 * to NTT_PATH_MATRIX builds that path's resources: a nested plan of passes of
 * at most 2^3 points with its own tables, the byte matrices E of its passes
 * and, from 2^17 points on, the per-q matrices of its folded passes (built on
 * the host's cores; at 2^24 about 73 MB per table kind and well under a
 * second; more than 1 GB from 2^26 on).  They stay with the plan until it is
 * destroyed; switching back and forth costs nothing more.  Outputs are
 * byte-identical on both paths.
 */
ntt_status ntt_plan_set_path(ntt_plan plan, ntt_path path);

/*
 * Replace the coset shift s (four little-endian limbs, canonical, nonzero)
 * and rebuild the coset tables.  Synchronous.  Requires a plan created with
 * coset != 0.
 */
ntt_status ntt_plan_set_coset_shift(ntt_plan plan, const uint64_t shift[4]);

/* Free the plan's device memory.  Waits for the device first.  NULL is OK. */
ntt_status ntt_plan_destroy(ntt_plan plan);

/*
 * The transforms, device buffers, stream-ordered.  d_in and d_out hold N
 * elements each (layout above); d_in == d_out (in place) is allowed.  The
 * two coset kinds need a plan created with coset != 0 (else
 * NTT_ERR_INVALID_ARG).
 */
ntt_status ntt_forward(ntt_plan plan, const void *d_in, void *d_out, ntt_stream stream);
ntt_status ntt_inverse(ntt_plan plan, const void *d_in, void *d_out, ntt_stream stream);
ntt_status ntt_coset_forward(ntt_plan plan, const void *d_in, void *d_out, ntt_stream stream);
ntt_status ntt_coset_inverse(ntt_plan plan, const void *d_in, void *d_out, ntt_stream stream);

/* Same as the calls above, with the kind as an argument. */
ntt_status ntt_execute(ntt_plan plan, ntt_kind kind, const void *d_in, void *d_out, ntt_stream stream);

/*
 * End-to-end transform of HOST buffers: copies h_in (N elements) to the
 * device buffer d_work (N elements, caller-owned), transforms it in place and
 * copies the result to h_out, all on `stream`, then synchronises the stream.
 * Host buffers should be page-locked for the copies to be asynchronous.
 */
ntt_status ntt_transform_host(ntt_plan plan, ntt_kind kind, const void *h_in, void *h_out,
                              void *d_work, ntt_stream stream);

/*
 * Asynchronous form of ntt_transform_host: enqueues the host-to-device copy,
 * the in-place transform of d_work and the device-to-host copy on `stream`
 * and returns without synchronising.  h_in, h_out and d_work must stay
 * valid (and h_in unmodified) until the stream has passed this work; with
 * page-locked host buffers, transforms on different streams overlap their
 * copies with each other's kernels.
 */
ntt_status ntt_transform_host_async(ntt_plan plan, ntt_kind kind, const void *h_in, void *h_out, void *d_work,
                                    ntt_stream stream);

/*
 * Read back the plan's structure: number of passes and the log2 size of each
 * pass's sub-transforms (of the path selected: on the matrix path its own
 * split into passes of at most 2^3 points), the number of kernel launches one
 * transform makes and, on the matrix path, how many of its passes
 * (passes 1 .. matrix_folded_passes) take their input factors folded into
 * per-q byte matrices (so that the pass before them ends in a Barrett
 * reduction instead of a Montgomery product).
 */
/* Most passes a transform is split into (the matrix path splits 2^28 into
 * ten passes of at most 2^3 points). */
#define NTT_MAX_PASSES 12

typedef struct ntt_plan_desc {
    uint32_t field;
    uint32_t log_n;
    uint32_t num_passes;
    uint32_t pass_log[NTT_MAX_PASSES];
    uint32_t launches_per_transform;
    uint32_t path;
    uint64_t device_bytes;
    uint32_t matrix_folded_passes;
    uint32_t reserved;
} ntt_plan_desc;
ntt_status ntt_plan_describe(ntt_plan plan, ntt_plan_desc *out);

/*
 * Copy `count` entries (from entry `first`) of one device twiddle table to
 * host memory, converted to standard form, so that tests can check the
 * tables against an independent computation.  table: 0 = the DFT twiddles
 * omega_S^i (i < S/2) of pass `pass`'s sub-transform size S; 1 = the input
 * multipliers of pass `pass` (pass >= 1: omega_M^{n q} [times s^{...} and
 * N^-1 folded in], row-major [n][q]; pass 0: the coset / scale factors);
 * 2 = the output multipliers s^-n (n < N) of the last pass of a coset
 * inverse (kind NTT_KIND_COSET_INVERSE, pass = the last pass).
 * Synchronous.
 */
ntt_status ntt_plan_read_table(ntt_plan plan, ntt_kind kind, uint32_t pass, uint32_t table,
                               uint64_t first, uint64_t count, void *h_out);

/*
 * Autotuner: time candidate configurations of this plan's transform on the
 * device and keep the fastest -- butterfly-path pass splits (balanced splits
 * for every maximum pass size 2^4..2^11, in both orders) x tile shapes (1024-
 * or 2048-element tiles), and the matrix path.  Each candidate runs one
 * untimed and `reps` timed forward transforms (reps = 0: 3) on scratch
 * buffers it allocates.  The plan's tables are rebuilt for the winner;
 * cached batched job lists that use the plan are dropped.  The choice is
 * remembered for (GPU, field, log_n): later ntt_plan_create calls in this
 * process use it, and when the environment variable NTT_TUNE_CACHE names a
 * file the choices are also written there and read by later processes.
 * Synchronous; takes tens to hundreds of milliseconds.  result may be NULL.
 */
typedef struct ntt_tune_result {
    uint32_t path;            /* ntt_path chosen */
    uint32_t num_passes;      /* butterfly passes (the matrix path has its own split) */
    uint32_t pass_log[NTT_MAX_PASSES];
    uint32_t tile_log[NTT_MAX_PASSES];  /* log2 of each pass's tile (10 or 11) */
    uint32_t candidates;
    double best_ms;           /* forward transform, winner */
    double default_ms;        /* forward transform, configuration before tuning */
} ntt_tune_result;
ntt_status ntt_plan_autotune(ntt_plan plan, uint32_t reps, ntt_tune_result *result);

/*
 * Rebuild the plan's butterfly path for an explicit pass split: num_passes
 * (1..NTT_MAX_PASSES) sub-transform sizes 2^pass_log[j] (each 1..11, summing
 * to log_n; pass 0 transforms the digit of largest stride, Sec. 3.3.2's
 * 3-/5-step decomposition with P passes), passes of at most 2^10 points on
 * tiles of 2^tile_log elements (10 or 11; larger passes always use 11).  The
 * plan's tables are rebuilt (coset shift kept) and its path set to
 * NTT_PATH_BUTTERFLY; cached batched job lists that use the plan are
 * dropped.  This is the autotuner's own step, for callers (and tests) that
 * choose a split themselves.  Synchronous; NTT_ERR_INVALID_ARG for a split
 * that does not fit these rules.
 */
ntt_status ntt_plan_set_passes(ntt_plan plan, uint32_t num_passes, const uint32_t *pass_log, uint32_t tile_log);

/*
 * Batched submission (the paper batches NTTs to fill its matrix units,
 * Sec. 4.4 / Fig. 7): many independent transforms of possibly different
 * sizes, kinds and fields, run as one persistent kernel launch per field in
 * which the CTAs pull (job, pass, tile) work items from a device queue.
 * jobs[i].plan fixes field and size; kind is an ntt_kind; in/out are device
 * buffers as above.  Jobs must not overlap in memory, and in != out for every
 * job (in-place jobs are rejected with NTT_ERR_INVALID_ARG: the batched path
 * works in the output buffer).  Jobs whose plan is on the matrix path run as
 * ordinary transforms inside the same graph (see ntt_batch_autotune).
 *
 * The first submission of a given job list (same plans, kinds and pointers)
 * builds its work-item table on the device and captures the launch sequence
 * into a CUDA graph (synchronous, a few hundred microseconds); later
 * submissions of the same list replay the graph (asynchronous).  Up to 16
 * job lists are cached; destroying a plan drops the lists that use it.
 * Submissions of one job list must not overlap in time (they share the
 * list's device counters): order them on one stream.
 *
 * Every device-side wait of a batch is bounded (ntt_batch_set_wait_limit,
 * default 2 s); when one runs out the kernel stops and records
 * NTT_ERR_TIMEOUT, which ntt_batch_poll_error reports.
 */
typedef struct ntt_job {
    ntt_plan plan;
    int32_t kind;
    const void *in;
    void *out;
} ntt_job;
ntt_status ntt_batch_submit(const ntt_job *jobs, size_t n, ntt_stream stream);

/*
 * Autotuner of a job list (the batch-size ablation of Sec. 4.4 / Fig. 7 asks
 * how batching should be organised; here it is measured per job list).
 * Candidates: every job in the persistent kernel; or, for each distinct job
 * size 2^t of the list, the jobs of 2^t points and more taken out of it and
 * run as ordinary transforms (each on its plan's own path and pass split,
 * e.g. as chosen by ntt_plan_autotune) over 1, 2 or 4 parallel branches of
 * the same CUDA graph, concurrently with the persistent kernel for the rest.
 * Each candidate runs the list once untimed and `reps` times timed (reps = 0:
 * 3), so the output buffers end up holding the jobs' results.  The fastest
 * policy is kept for the list's signature (the multiset of field, size,
 * kind and path of its jobs): later ntt_batch_submit calls of any list with
 * that signature follow it, and with NTT_TUNE_CACHE set the policies are
 * also written to "<NTT_TUNE_CACHE>.batch" and read by later processes.
 * Synchronous.  result may be NULL.
 */
typedef struct ntt_batch_tune_result {
    uint32_t split_log;      /* jobs of 2^split_log points and more run alone (0: none) */
    uint32_t branches;       /* parallel graph branches for them (0: none) */
    uint32_t candidates;
    double best_ms;          /* the list under the chosen policy */
    double persistent_ms;    /* every job in the persistent kernel */
    double loop_ms;          /* one ntt_execute per job on one stream */
} ntt_batch_tune_result;
ntt_status ntt_batch_autotune(const ntt_job *jobs, size_t n, uint32_t reps, ntt_batch_tune_result *result);

/*
 * ntt_batch_submit without any allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * while they submit work -- services that reserve all their device memory
 * up front and must not allocate once they are serving, and submitters on
 * a latency path, where cudaMalloc's implicit device synchronisation would
 * stall work already queued on other streams.
 * ntt_batch_submit allocates a work-item table and counters per new job
 * list; this call instead runs the same persistent
 * batched kernel with its table and counters in one fixed-size array that
 * the library holds in device memory (about 55 KB on every GPU that loads
 * the library, until the process exits).  It calls no cudaMalloc, cudaFree
 * or other allocating routine; the caller passes the plans (created
 * beforehand) and the input and output buffers, as for ntt_batch_submit.
 *
 * Limits: at most 64 jobs per call and at most 256 passes of jobs per field
 * (the jobs' pass counts summed; NTT_ERR_UNSUPPORTED beyond, nothing
 * launched); same job rules as ntt_batch_submit (in != out, butterfly-path
 * plans, no overlap).  n == 0 launches nothing.
 * d_status: device pointer to one uint32_t (4-byte aligned), set to 0 at the
 * start of the call and to NTT_ERR_TIMEOUT if a device wait of the kernel
 * ran out.  It may be NULL: the error is then kept in the array's own error
 * word until ntt_batch_poll_error reads and clears it, and until then later
 * calls made without a status pointer stop at once (like ntt_batch_submit
 * after an unpolled error).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, which may load the library's device code on that
 * device, and so may allocate): make that first call before the phase in
 * which the caller must not allocate.  The address is
 * kept until ntt_batch_cache_clear, which must be called after a
 * cudaDeviceReset.  Every call on a device shares the one array, which keeps
 * the last call's contents (the call clears the counters it needs): calls
 * whose work overlaps on the GPU race -- order them on one stream.
 */
ntt_status ntt_batch_submit_static(const ntt_job *jobs, size_t n, uint32_t *d_status, ntt_stream stream);

/* First error recorded by batched kernels on the current device since the
 * last poll (0 = none), then cleared: ntt_batch_submit's word, else the word
 * of ntt_batch_submit_static calls made without a status pointer.
 * Synchronises the device. */
ntt_status ntt_batch_poll_error(uint32_t *code);

/* Bound of every device-side wait of batches built from now on (ns, > 0).
 * Drops the cached job lists. */
ntt_status ntt_batch_set_wait_limit(uint64_t ns);

/* Test hook (fault injection on the host): when enabled, every job list
 * built from now on makes one of its device waits unsatisfiable, so that
 * the bounded-wait path runs out and reports NTT_ERR_TIMEOUT.  No GPU fault
 * is involved.  Drops the cached job lists. */
ntt_status ntt_batch_debug_stall(int enable);

/* Drop every cached job list (synchronises the device), the batch policies
 * of ntt_batch_autotune held in memory (those in "<NTT_TUNE_CACHE>.batch"
 * are read again) and the device addresses looked up by
 * ntt_batch_submit_static. */
ntt_status ntt_batch_cache_clear(void);

/*
 * Per-pass launch timing.  While enabled, every pass launch of this plan's
 * transforms is bracketed by two CUDA events recorded on the launch's own
 * stream.  ntt_plan_read_timing synchronises those events and returns, per
 * pass (up to NTT_MAX_PASSES), the summed device time in milliseconds and
 * the number of launches timed since the last read, then clears the record.  Timing adds
 * two event records per launch; leave it off outside measurements.
 */
ntt_status ntt_plan_enable_timing(ntt_plan plan, int enable);
ntt_status ntt_plan_read_timing(ntt_plan plan, double ms_per_pass[NTT_MAX_PASSES],
                                uint64_t launches_per_pass[NTT_MAX_PASSES]);

/*
 * Device-detected error of the plan's last transforms (0 = none), cleared on
 * read.  Synchronises the device.  In a debug build of the library (compiled
 * with NTT_DEBUG: every vector and table access of the butterfly pass
 * kernels, single and batched, is checked against the extent the plan
 * recorded for it, and an access out of range is skipped instead of made),
 * a failed check reports NTT_ERR_BOUNDS here.  ntt_build_is_debug tells
 * which build is loaded.
 */
ntt_status ntt_plan_poll_error(ntt_plan plan, uint32_t *code);
int ntt_build_is_debug(void);

/*
 * Test hook of debug builds: the next butterfly transform of this plan runs
 * with the recorded vector extent halved, so that the bounds checks of its
 * kernels fire on in-range accesses (which are then skipped: no access is
 * ever made outside a buffer) and NTT_ERR_BOUNDS reaches
 * ntt_plan_poll_error.  Release builds return NTT_ERR_UNSUPPORTED.
 */
ntt_status ntt_debug_shrink_next_extent(ntt_plan plan);

/*
 * Serving runtime (continuous batching).  A server keeps plans with their
 * twiddle tables resident for both fields and every size in
 * [min_log_n, max_log_n] (coset tables included), admits requests against
 * a device-memory budget (resident tables + two N-element device buffers
 * per admitted request), and runs admitted requests as batches (see
 * ntt_batch_submit) on up to max_inflight streams, so that requests that
 * arrive while others are on the GPU are admitted as soon as memory and a
 * stream slot free up, and their work overlaps on the device.  A worker
 * thread owned by the server does admission, dispatch and retirement.
 *
 * Requests use HOST buffers (page-locked for asynchronous copies): h_in is
 * read and h_out written by the server between submit and completion; the
 * caller must keep both alive until ntt_server_wait / ntt_server_query
 * report completion.  Results are bit-identical to a transform run alone.
 * Timestamps (seconds since server creation): arrive = submit, admit =
 * device buffers reserved, finish = the batch's device-to-host copy done
 * and observed by the worker; latency = finish - arrive.
 */
typedef struct ntt_server_s *ntt_server;

typedef struct ntt_server_config {
    uint64_t memory_budget_bytes; /* default 64 GiB (0 = default) */
    uint32_t min_log_n;           /* default 12 */
    uint32_t max_log_n;           /* default 24 */
    uint32_t max_inflight;        /* batches in flight (streams), default 3, at most 16 */
    uint32_t max_batch_jobs;      /* requests per batch, default 64 */
    uint64_t max_batch_elements;  /* elements per batch, default 2^26 (a single larger request still runs) */
} ntt_server_config;

typedef struct ntt_server_stats {
    uint64_t submitted;
    uint64_t completed;
    uint64_t batches;
    uint64_t queued;              /* waiting for admission or dispatch */
    uint64_t resident_bytes;      /* plans and twiddle tables */
    uint64_t peak_device_bytes;   /* resident + request buffers, high-water mark */
    uint64_t budget_bytes;
} ntt_server_stats;

/* cfg may be NULL (all defaults).  NTT_ERR_BUDGET if the resident tables
 * plus one largest request exceed the budget. */
ntt_status ntt_server_create(const ntt_server_config *cfg, ntt_server *out);
/* Enqueue one request; *ticket identifies it.  Non-blocking. */
ntt_status ntt_server_submit(ntt_server server, ntt_field field, ntt_kind kind, uint32_t log_n, const void *h_in,
                             void *h_out, uint64_t *ticket);
/* *done = 1 once h_out holds the result. */
ntt_status ntt_server_query(ntt_server server, uint64_t ticket, int *done);
/* Block until the request is done (NTT_ERR_TIMEOUT after timeout_s > 0). */
ntt_status ntt_server_wait(ntt_server server, uint64_t ticket, double timeout_s);
ntt_status ntt_server_request_times(ntt_server server, uint64_t ticket, double *arrive_s, double *admit_s,
                                    double *finish_s);
/* Forget a completed request (its record and timestamps). */
ntt_status ntt_server_release(ntt_server server, uint64_t ticket);
ntt_status ntt_server_get_stats(ntt_server server, ntt_server_stats *out);
/* Finish every submitted request, then free the server. */
ntt_status ntt_server_destroy(ntt_server server);

/*
 * Pointwise quotient of a prover on coset evaluations, fused into one kernel
 * (one pass over the vectors: 3 reads, 1 write per element):
 *   out[i] = (a[i] * b[i] - c[i]) * z[i mod z_len] mod M,  i < count.
 * a, b, c, out: device vectors of `count` elements (layout above, canonical;
 * out may alias an input).  h_z: z_len elements in HOST memory, standard
 * form, canonical; z_len a power of two, 1..64.  The typical z is the
 * inverse of the vanishing polynomial X^n - 1 of an n-point domain on a
 * coset of 2^k n points, which takes 2^k values (z_len = 2^k).  The paper
 * has no counterpart (its workload is the transform); this is the step
 * between a prover's coset transforms and the coset inverse.
 * Stream-ordered; h_z is read before the call returns (no device memory is
 * allocated).  NTT_ERR_INVALID_ARG for a bad field, z_len, z value or
 * buffer.
 */
ntt_status ntt_pointwise_quotient(ntt_field field, const void *d_a, const void *d_b, const void *d_c,
                                  const uint64_t *h_z, uint32_t z_len, void *d_out, uint64_t count,
                                  ntt_stream stream);

/*
 * NTT of 2^log_n elements (1 <= log_n <= 24) over the 377- or 753-bit
 * field, any of the four kinds (forward, inverse, coset and coset inverse;
 * the coset shift s is the field's generator, 7 resp. 11): element i is 12
 * (resp. 24) little-endian uint32 words at byte offset 48 i (resp. 96 i),
 * standard form, canonical, natural order; device buffers 16-byte aligned;
 * d_in == d_out allowed.  Same pass decomposition as the 256-bit
 * transforms, with a generic-limb Montgomery product; the coset factors
 * s^i ride on the first pass's loads and the coset inverse's s^-i on the
 * last pass's stores.  The first call for a (device, field, log_n) builds
 * the tables on the device, and the first coset call of either coset kind
 * the two coset tables (2 * 4 * LP * 2^log_n bytes, LP = 16 resp. 28);
 * both synchronous, kept until the process exits.  Stream-ordered.  The
 * tables and an in-place call's scratch vector belong to the (device,
 * field, log_n), not to the caller: two in-place calls of the same field
 * and size must not run at the same time on different streams.
 * NTT_ERR_INVALID_ARG for another field or kind, or unaligned or null
 * buffers; NTT_ERR_UNSUPPORTED for other sizes.
 */
ntt_status ntt_wide_transform(ntt_field field, ntt_kind kind, uint32_t log_n, const void *d_in, void *d_out,
                              ntt_stream stream);
/*
 * The coset kinds of ntt_wide_transform with a caller-chosen shift s:
 * h_shift points to 12 (377-bit) or 24 (753-bit) little-endian uint32 words
 * in host memory, standard form, 0 < s < p; kind is NTT_KIND_COSET or
 * NTT_KIND_COSET_INVERSE.  The (device, field, log_n) keeps the coset
 * tables of one shift: a call with another shift than the last one waits
 * for the device to be idle (cudaDeviceSynchronize), rewrites the tables
 * and then enqueues its transform.  NTT_ERR_INVALID_ARG for a null, zero or
 * out-of-range shift, another kind, or the errors of ntt_wide_transform.
 */
ntt_status ntt_wide_transform_shift(ntt_field field, ntt_kind kind, uint32_t log_n, const uint32_t *h_shift,
                                    const void *d_in, void *d_out, ntt_stream stream);
/* Bytes of one element of `field` in memory (32, 32, 48, 96). */
ntt_status ntt_field_element_bytes(ntt_field field, uint32_t *bytes);

/*
 * The paper's RNS lazy modular multiplication (MORPH Sec. 3.2.3-3.2.4,
 * Alg. 1 "MXU RNS Lazy") on the tensor cores, for measuring it against the
 * 32-bit IMAD Montgomery product the transforms use.
 *
 * Representation: an element of F_M is carried as an integer in [0, L),
 * L = (sum_i q_i + num_q) M, congruent to it ("lazy"), by its residues
 * modulo the num_q primes q_i of base Q (the largest primes below 2^31,
 * as many as give Q > 4 L^2).  Memory layout: words_per_element (20)
 * uint32 per element, residue i in word i, the remaining words zero; 16-byte
 * aligned device buffers.  A second base P of num_p primes (the next ones
 * below, as many as give P > 2^20 L) serves the reduction.
 *
 * ntt_rns_mul computes, for every element e < count, out[e] = x[e] *
 * y[e]^reps as a lazy element (congruent mod M, in [0, L)): each product
 * is two 32-bit Montgomery products per residue, a quotient estimate
 * scaled by 2^shift, a byte product (ByteDecompose, Einsum on tcgen05,
 * ByteMerge) into base P, and an exact base extension (a second byte
 * product) back to base Q.  Inputs must be canonical residues of an
 * integer in [0, L).  Stream-ordered.  The first call per (device, field)
 * builds and uploads the constant tables (synchronous, ~30 KB).  A device
 * wait that runs out records NTT_ERR_TIMEOUT, read by ntt_rns_poll_error
 * (which synchronises and clears it).
 */
typedef struct ntt_rns_basis {
    uint32_t num_q, num_p;
    uint32_t words_per_element;
    uint32_t shift;
    uint32_t q[24];
    uint32_t p[16];
} ntt_rns_basis;
ntt_status ntt_rns_basis_get(ntt_field field, ntt_rns_basis *out);
ntt_status ntt_rns_mul(ntt_field field, const void *d_x, const void *d_y, void *d_out, uint64_t count,
                       uint32_t reps, ntt_stream stream);
ntt_status ntt_rns_poll_error(ntt_field field, uint32_t *code);

/*
 * Diagnostic: element-wise Montgomery product of device vectors,
 * out[i] = a[i] * b[i] * 2^-256 mod M, the field multiplication every
 * butterfly uses (the paper's "radix Mont" baseline, Sec. 2.3.2: 8 32-bit
 * digits, O(D^2) product and Montgomery reduction).  count elements each,
 * layout as above, inputs canonical.  Stream-ordered.
 */
ntt_status ntt_field_mont_mul(ntt_field field, const void *d_a, const void *d_b, void *d_out, uint64_t count,
                              ntt_stream stream);

/*
 * Diagnostic / throughput probe of the field multiplication: out[i] =
 * a[i] * (b[i] * 2^-256)^reps mod M, i.e. `reps` dependent Montgomery
 * products per element.  variant 0: one thread per element, carry chains in
 * registers (what every kernel of this library uses); variant 1: eight lanes
 * per element, one 32-bit limb each, carries moved between lanes by warp
 * shuffles (the warp-cooperative form).  Same results; the two exist to
 * measure the difference.  count elements, reps >= 1.  Stream-ordered.
 */
ntt_status ntt_field_mont_mul_rep(ntt_field field, const void *d_a, const void *d_b, void *d_out, uint64_t count,
                                  uint32_t reps, int variant, ntt_stream stream);

/* Human-readable name of a status code (static storage). */
const char *ntt_status_string(ntt_status status);

/* Library version as major*10000 + minor*100 + patch. */
uint32_t ntt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NTT_GB300_H */
