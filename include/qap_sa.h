/*
 * qap_sa.h -- C ABI of libqapsa: Delta-matrix simulated annealing (SA) for the
 * quadratic assignment problem (QAP) on one NVIDIA GB300 GPU (sm_103a).
 *
 * Method: G. Paul, "A GPU implementation of the Simulated Annealing Heuristic
 * for the Quadratic Assignment Problem", arXiv:1208.2675.
 *   - cost of an assignment p:            Eq. (1), section 1
 *   - acceptance of a proposed swap:      Eq. (2), section 2.1
 *   - the Delta-matrix loop (a)-(e):      section 2.2
 *   - window search (a subset of proposals), first accepted one in sequential order:
 *                                         section 3 (ii)
 *   - B' kept permuted for coalescing:    Eq. (3), section 3 (i)
 *
 * Conventions for every entry point:
 *   - Matrices are row-major N x N int32 (element (i,j) at index i*N + j).
 *     A[i][j] is the flow between facilities i and j, B[x][y] the distance
 *     between locations x and y; p[i] is the location of facility i.
 *     Any int32 entries are accepted as long as 8 N max|A| max|B| <= 2^31 - 1
 *     (every swap cost and Gram sum then fits int32).  The symmetric instances
 *     with zero diagonals and entries in [-127, 127] (the family of section 4)
 *     run on the on-chip tiers; asymmetric instances (the general swap cost),
 *     nonzero diagonals, wider entries, random proposal order and N beyond a
 *     cluster's capacity run on tier 3 (qap_sa_info.tier).
 *   - Unless a name ends in _device, pointers are HOST pointers; the library
 *     copies what it needs and never keeps a caller pointer after returning.
 *   - Return value: QAP_OK (0) or a negative QAP_E_* status; on error nothing
 *     the caller owns has been written and *out handles are left NULL.
 *   - A handle is not thread-safe; distinct handles are independent and may be
 *     used from different threads.
 *   - There is no CPU fallback: if no usable CUDA device is present every
 *     create call returns QAP_E_CUDA.
 */
#ifndef QAP_SA_H
#define QAP_SA_H

#include <stdint.h>

#if defined(__GNUC__)
#define QAP_EXPORT __attribute__((visibility("default")))
#else
#define QAP_EXPORT
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define QAP_OK            0
#define QAP_E_INVAL      (-1) /* null pointer; N < 2; p0 not a permutation;
                                 T0 or Tf not finite and > 0; total_iters == 0;
                                 unknown schedule flags */
#define QAP_E_RANGE      (-2) /* the swap-cost bound 8 N max|A| max|B| exceeds
                                 2^31 - 1; or it + iters > total_iters */
#define QAP_E_NOMEM      (-3) /* device or host allocation failed */
#define QAP_E_CUDA       (-4) /* a CUDA call failed (message via strerror) */
#define QAP_E_TIMEOUT    (-5) /* a bounded device-side wait expired */
#define QAP_E_STATE      (-6) /* the device reported an inconsistent state */
#define QAP_E_UNSUPPORTED (-7) /* N larger than the largest supported tier
                                  (qap_sa_max_n, qap_sa_max_n_tier); a tier-3
                                  chain in a batch or a served request */

/* ---- cooling schedule ---------------------------------------------------- */
/* Temperature T of Eq. (2) is lowered after every iteration (section 2.1) by
 * the geometric law T(it) = T0 * alpha^it, alpha = (Tf / T0)^(1 / (I - 1)),
 * it = 0 .. I - 1, evaluated bit-reproducibly as a product of per-byte tables
 * built by repeated squaring of alpha (see qap_sa_temperature).              */
#define QAP_T_RELATIVE 1u /* t0 multiplies mean |Delta_0| over the M pairs,
                             tf multiplies T0; if every Delta_0 is zero t0 and
                             tf are used as absolute temperatures */
#define QAP_ORDER_RANDOM 2u /* proposals drawn at random (section 2.1) instead
                             of the sequential cyclic order: the pair proposed
                             at iteration it is pair number (x * M) >> 32 of
                             the row-major enumeration, x word 0 of
                             Philox4x32-10(counter = (it low, it high,
                             stream_id, 1), key = (seed low, seed high)) */

typedef struct qap_schedule {
  double t0;            /* T0, or its multiplier with QAP_T_RELATIVE        */
  double tf;            /* Tf, or its multiplier with QAP_T_RELATIVE        */
  uint64_t total_iters; /* I: the schedule spans it = 0 .. I - 1 (>= 1)     */
  uint32_t flags;       /* QAP_T_RELATIVE | QAP_ORDER_RANDOM, or 0          */
  uint32_t stream_id;   /* Philox counter word 2: the chain's random stream */
} qap_schedule;

/* ---- one chain ----------------------------------------------------------- */
typedef struct qap_sa qap_sa; /* opaque; created by qap_sa_create*, freed by
                                 qap_sa_destroy */

/* Step (a) of section 2.2: copy A, B, p0 to the device, build B' (Eq. 3),
 * the initial Delta for all M = N(N-1)/2 pairs r < s and the cost C0 of
 * Eq. (1), then fix the schedule.  Random numbers: the r of Eq. (2) at
 * iteration it is u = (x + 0.5) / 2^32 with x word (it mod 4) of
 * Philox4x32-10(counter = (it/4 low, it/4 high, stream_id, 0),
 * key = (seed low, seed high)).  Blocks until the set-up is done.
 *   A, B  : host, N*N int32 each, row-major, symmetric, zero diagonal
 *   N     : 2 .. qap_sa_max_n()
 *   p0    : host, N int32, a permutation of 0 .. N-1
 *   sched : host, read during the call only
 *   out   : receives the new handle                                         */
QAP_EXPORT int qap_sa_create(const int32_t *A, const int32_t *B, int32_t N,
                  const int32_t *p0, const qap_schedule *sched, uint64_t seed,
                  qap_sa **out);

/* As qap_sa_create, but A, B and p0 are DEVICE pointers (same layouts) that
 * must stay valid until this call returns, and all device work of the handle
 * is issued on `cuda_stream` (a cudaStream_t; NULL = a stream the library
 * creates and owns).  The caller's buffers are only read.                   */
QAP_EXPORT int qap_sa_create_device(const int32_t *A, const int32_t *B, int32_t N,
                         const int32_t *p0, const qap_schedule *sched,
                         uint64_t seed, void *cuda_stream, qap_sa **out);

/* Steps (b)-(d) of section 2.2 for exactly `iters` more iterations: proposals
 * are the pairs r < s in row-major cyclic order, pair(it mod M); each is
 * accepted by Eq. (2) (delta <= 0 always; otherwise iff
 * (double)delta < -(T(it) * log(u)) in IEEE binary64); on acceptance p, the
 * cost and Delta are updated.  Windows of consecutive proposals are tested in
 * parallel and the first accepted one in sequential order is taken
 * (section 3 (ii)), so the trajectory equals the sequential one.  While the
 * acceptance rate is high the swap cost of a proposal is evaluated directly
 * from A and B' instead of being read from Delta (the same exact integer) and
 * Delta is rebuilt from its definition before it is read again, so Delta is
 * always current between calls (qap_sa_delta).
 * run(a); run(b) gives the same state as run(a + b).  Blocks until done.
 * Returns QAP_E_RANGE if it + iters > total_iters.                          */
QAP_EXPORT int qap_sa_run(qap_sa *h, uint64_t iters);

/* As qap_sa_run but only enqueues the work on the handle's stream and
 * returns; qap_sa_sync waits for it and reports device-side errors.         */
QAP_EXPORT int qap_sa_run_async(qap_sa *h, uint64_t iters);
QAP_EXPORT int qap_sa_sync(qap_sa *h);

/* Current state after a stream sync: p (N int32, host), the int64 cost of
 * Eq. (1) for p, and the number of accepted swaps.  Any output pointer may
 * be NULL.                                                                  */
QAP_EXPORT int qap_sa_result(qap_sa *h, int32_t *p_out, int64_t *cost,
                  uint64_t *accepts);

/* As qap_sa_result, into DEVICE buffers, enqueued on the handle's stream
 * without a host sync.  Any output pointer may be NULL.                     */
QAP_EXPORT int qap_sa_result_device(qap_sa *h, int32_t *p_out, int64_t *cost,
                         uint64_t *accepts);

/* Diagnostics of the current state (after a stream sync). */
typedef struct qap_sa_info {
  int32_t N;
  int32_t tier;           /* 1 = one CTA (Delta in its registers or its
                             Tensor Memory, A and B' in its shared memory);
                             2 = a thread-block cluster (Delta in the
                             cluster's Tensor Memory, A and B' split over the
                             cluster's shared memory), for N beyond one SM;
                             3 = a persistent grid (Delta in global memory,
                             rows staged by TMA, one grid barrier per
                             accepted swap) for general instances, random
                             order, wide entries and N beyond a cluster    */
  uint64_t iterations;    /* it: iterations done                            */
  uint64_t accepts;
  int64_t cost;
  uint64_t near_ties;     /* evaluations with |delta + T ln u| < 1e-9 T     */
  uint64_t exact_evals;   /* acceptance tests decided in binary64           */
  uint64_t windows;       /* windows scanned                                */
  double T0, Tf, alpha;   /* the schedule actually used                     */
  uint64_t total_iters;
  uint64_t smem_bytes;    /* dynamic shared memory of the SA kernel         */
  uint64_t direct_iters;  /* iterations whose proposal was evaluated directly
                             (high acceptance) instead of read from Delta  */
  uint64_t direct_accepts;/* accepted swaps among them (no Delta update)    */
  uint64_t warp_iters;    /* direct iterations run by one warp alone, with no
                             block barrier (while the acceptance rate is
                             above 1/512, or 1/64 for N above ~180)        */
  int32_t ctas;           /* CTAs (= SMs) the chain holds while it runs     */
  int32_t threads;        /* threads per CTA of the SA kernel               */
  uint64_t hot_iters;     /* iterations run by the hot-phase kernel of the
                             cluster tier (one SM, rows of A and B' in L2)
                             while the acceptance rate was high            */
  uint64_t hot_accepts;   /* accepted swaps among them                      */
} qap_sa_info;
QAP_EXPORT int qap_sa_get_info(qap_sa *h, qap_sa_info *out);

/* Device time of a handle's kernels, by kind, from CUDA events recorded on
 * the handle's stream around every launch of qap_sa_run / qap_sa_run_async
 * while timing is on (off by default; events cost a few microseconds per
 * launch of 2^26 iterations).  Kinds:                                      */
#define QAP_KT_HOT 0   /* the cluster tier's hot-phase kernel (one SM)      */
#define QAP_KT_SA 1    /* the SA kernel of the chain's tier (one SM,
                          cluster or grid)                                  */
#define QAP_KT_AUX 2   /* the B' and Delta rebuilds between them            */
#define QAP_KT_COUNT 3
/* on != 0 starts timing (and clears what was counted), 0 stops it.
 * QAP_E_INVAL for h == NULL.                                               */
QAP_EXPORT int qap_sa_set_timing(qap_sa *h, int on);
/* After a sync of the handle's stream: seconds[k] and launches[k], k <
 * QAP_KT_COUNT (caller-owned arrays), the device time and the number of timed
 * launches of kind k (a rebuild of B' and Delta, two or three small kernels,
 * counts as one) since timing was switched on or last read; the counts start
 * again.
 * QAP_E_INVAL for NULL arguments, QAP_E_CUDA if an event failed.            */
QAP_EXPORT int qap_sa_kernel_times(qap_sa *h, double *seconds, uint64_t *launches);

/* The current Delta (after a stream sync) as M int32 values in pair order
 * (r < s, row-major): delta_out[m] is the cost change of swapping pair(m).  */
QAP_EXPORT int qap_sa_delta(qap_sa *h, int32_t *delta_out);

/* T(it) of the handle's schedule as a binary64 (see qap_schedule).          */
QAP_EXPORT double qap_sa_temperature(const qap_sa *h, uint64_t it);

/* Near-ties of the handle (after a stream sync): the test of Eq. (2) is
 * decided in binary64 with CUDA's log, and a test with
 * |delta + T ln u| < 1e-9 T is a near-tie, where another libm's log could decide
 * it the other way.  Writes the iteration indices of the first
 * min(cap, 8) near-ties to it_out (host, cap uint64) and their total count to
 * *count (may be NULL).  QAP_E_INVAL if h is NULL, cap < 0, or cap > 0 with
 * it_out NULL.                                                              */
QAP_EXPORT int qap_sa_near_tie_log(qap_sa *h, uint64_t *it_out, int32_t cap,
                                   uint64_t *count);

/* Eq. (2) (section 2.1) for given proposals, decided exactly as the SA kernels
 * decide it inside a window (section 3 (ii)), with the handle's schedule and
 * random stream: probe k is the proposal of iteration it[k] with swap cost
 * delta[k] in a window that starts at iteration it0[k].  For a diagnostic of
 * the binary32 pre-test against the binary64 rule; it changes no state.
 *   it, it0, delta : host, n entries each; it0[k] <= it[k] < it0[k] + 2^30
 *   out            : host, n int32: bit 0 the decision (1 = accept); bits 2-3
 *                    the binary32 interval of the prepared per-window tables
 *                    (0 reject, 1 accept, 2 undecided -> binary64); bits 4-5
 *                    the interval of the in-window pre-test; bit 6 set when
 *                    the integer pre-filter of a window of it - it0 + 1
 *                    proposals rejects; bit 7 set when the binary64 test saw
 *                    a near-tie
 * Blocks until done.  QAP_E_INVAL for NULL arguments or n < 0, QAP_E_RANGE for
 * an offset outside [0, 2^30).                                              */
QAP_EXPORT int qap_sa_accept_probe(qap_sa *h, int32_t n, const uint64_t *it,
                                   const uint64_t *it0, const int32_t *delta,
                                   int32_t *out);

/* Failure detection without a fault (the paper has no counterpart): while on
 * != 0, the grid barrier of a tier-3 handle's launches expects one arrival
 * more than its CTAs make, so every CTA's bounded wait (about two seconds)
 * expires; the kernel records the expiry and returns, and qap_sa_run /
 * qap_sa_sync return QAP_E_TIMEOUT.  The handle's state is then invalid:
 * destroy it.  The device and other handles stay usable.  QAP_E_INVAL for
 * h == NULL, QAP_E_UNSUPPORTED for a handle on another tier.               */
QAP_EXPORT int qap_sa_inject_barrier_fault(qap_sa *h, int on);

/* Frees every resource of the handle (NULL is ignored).                     */
QAP_EXPORT void qap_sa_destroy(qap_sa *h);

/* ---- batch of independent chains ------------------------------------------
 * Many independent chains -- repeated runs of the heuristic (section 2.3), here
 * independent problems of uneven N -- advanced together by one persistent
 * launch captured in a CUDA graph: each CTA of a one-CTA-per-SM grid takes
 * the next chain from a longest-first work list and runs it with the same
 * kernel code as a single chain, so every chain's trajectory equals the one
 * qap_sa_run gives it alone.                                                */
typedef struct qap_problem {
  const int32_t *A;     /* host, N*N int32, as for qap_sa_create            */
  const int32_t *B;     /* host, N*N int32                                  */
  const int32_t *p0;    /* host, N int32 permutation                        */
  int32_t N;
  uint32_t reserved;    /* must be 0                                        */
  qap_schedule sched;   /* its own schedule and random stream (stream_id)   */
  uint64_t seed;
} qap_problem;

typedef struct qap_batch qap_batch; /* opaque; freed by qap_batch_destroy */

/* Set-up (step (a)) of every problem; host inputs are read during the call
 * only.  Errors as qap_sa_create, for the first problem that fails.         */
QAP_EXPORT int qap_batch_create(const qap_problem *probs, int32_t count,
                                qap_batch **out);
/* Advances chain i by iters[i] iterations (iters == NULL: every chain to its
 * total_iters) in one graph launch; blocks until done.  QAP_E_RANGE if a
 * chain would pass its total_iters (nothing runs then).                     */
QAP_EXPORT int qap_batch_run(qap_batch *b, const uint64_t *iters);
/* State of chain i, as qap_sa_result / qap_sa_get_info.                      */
QAP_EXPORT int qap_batch_result(qap_batch *b, int32_t i, int32_t *p_out,
                                int64_t *cost, uint64_t *accepts);
QAP_EXPORT int qap_batch_get_info(qap_batch *b, int32_t i, qap_sa_info *out);
QAP_EXPORT void qap_batch_destroy(qap_batch *b);

/* ---- serving: continuous batching of solve requests -----------------------
 * A worker thread of the library admits submitted requests in arrival order as
 * soon as SMs (one per chain, or the chain's cluster size for large N) and
 * device memory (the budget) are free, runs each on its own stream, and keeps
 * every chain's state on the device until it finishes.  Requests that arrive
 * while others run are admitted as slots free up and overlap with them.  The
 * paper has no counterpart; each request's result equals qap_sa_run's for the
 * same problem.                                                               */
typedef struct qap_server_cfg {
  int32_t max_sms;          /* SMs the server may fill with chains (0 = all but
                               four, which stay free for the set-up and
                               rebuild kernels of admissions: an SM holding a
                               chain has no room left for them)             */
  uint32_t reserved;        /* must be 0                                       */
  uint64_t mem_budget_bytes;/* device bytes for chains (0 = 80 % of free)      */
} qap_server_cfg;

typedef struct qap_result {
  int32_t done;       /* 1 once the request has finished                      */
  int32_t status;     /* its status code (valid when done)                    */
  int64_t cost;       /* Eq. (1) of the final assignment                      */
  uint64_t accepts;
  uint64_t iterations;
  double queue_s;     /* seconds from submit to admission                     */
  double latency_s;   /* seconds from submit to completion                    */
} qap_result;

typedef struct qap_server qap_server; /* opaque; freed by qap_server_stop */

/* Starts the worker on the current device; cfg may be NULL.                  */
QAP_EXPORT int qap_server_start(const qap_server_cfg *cfg, qap_server **out);
/* Queues `iters` iterations of problem q (inputs copied during the call;
 * iters <= q->sched.total_iters); *ticket identifies the request.  Only chains
 * of the on-chip tiers are served (symmetric, zero diagonal, entries in
 * [-127, 127], sequential order, N <= qap_sa_max_n_tier(2)); others return
 * QAP_E_UNSUPPORTED.                                                         */
QAP_EXPORT int qap_server_submit(qap_server *s, const qap_problem *q,
                                 uint64_t iters, uint64_t *ticket);
/* Non-blocking: fills *out (out->done = 0 while pending); when done and p_out
 * is not NULL, copies the final assignment (N int32) into it.               */
QAP_EXPORT int qap_server_poll(qap_server *s, uint64_t ticket, qap_result *out,
                               int32_t *p_out);
/* Largest number of requests that were on the device at the same time.     */
QAP_EXPORT int qap_server_max_running(qap_server *s);
/* Finishes every queued and running request, stops the worker, frees all.   */
QAP_EXPORT int qap_server_stop(qap_server *s);

/* ---- set-up without allocation ---------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot call cudaMalloc -- programs whose device memory belongs to another
 * allocator (a framework's caching pool) or to a fixed budget, and loops that
 * must not stall on the device-wide synchronisation cudaMalloc and cudaFree may
 * imply.  It computes what qap_sa_create computes first (step (a): the swap
 * costs Delta for every pair and the cost of Eq. (1)) and allocates nothing:
 * its intermediates live in one static device array of about 400 KB that every
 * GPU loading the library holds until the process exits.
 *   A, B, p   : DEVICE pointers, same layouts and rules as qap_sa_create
 *   N         : 2 .. QAP_NOALLOC_MAX_N; larger N returns QAP_E_RANGE
 *   delta_out : DEVICE, M = N(N-1)/2 int32 in pair order (as qap_sa_delta)
 *   cost_out  : DEVICE, one int64
 *   cuda_stream : the cudaStream_t the work is issued on (NULL = default)
 * Blocks until the work is done.  Returns QAP_E_INVAL / QAP_E_RANGE for the
 * same input defects as qap_sa_create; in that case the outputs hold
 * unspecified values.  The first call on a device looks up the array's device
 * address (with that device current); make that first call before any stream
 * capture.  The address is kept for the life of the process: after a
 * cudaDeviceReset it is stale, and this entry point must not be called again
 * on that device.  All calls share the one array, so calls that overlap on the
 * GPU (from several threads or streams) race: serialise them.                */
#define QAP_NOALLOC_MAX_N 256
QAP_EXPORT int qap_sa_setup_noalloc(const int32_t *A, const int32_t *B, int32_t N,
                                    const int32_t *p, int32_t *delta_out,
                                    int64_t *cost_out, void *cuda_stream);

/* ---- tuning ----------------------------------------------------------------
 * The paper leaves the number of proposals tested in parallel as an
 * adjustable parameter (section 3 (ii)); this library has more such knobs,
 * none of which changes a trajectory: which tier runs a chain, when the swap
 * cost of a proposal is read from Delta or evaluated directly, when one warp
 * runs the direct mode alone, how many CTAs a grid-tier chain uses.  qap_tune
 * measures them on the current GPU; qap_knobs_set makes a choice the default
 * for a range of N.  Environment variables read at create time override them:
 * QAPSA_TIER, QAPSA_T3_GRID, QAPSA_HYBRID_RATE, QAPSA_WARP_RATE,
 * QAPSA_CLUSTER_HYBRID_RATE; and for the cluster tier's hot phase (one SM
 * while the block acceptance rate is at least the hand-over rate)
 * QAPSA_HOT (0: off), QAPSA_HOT_RATE (the hand-over rate, default 0.009) and
 * QAPSA_HOT_WARPS (proposal warps, rounded down to a power of two, default 8). */
typedef struct qap_knobs {
  int32_t tier;               /* 0: the default choice; 3: the grid tier even
                                 where an on-chip tier could take the chain;
                                 1 or 2: the on-chip tier for N's size (never
                                 for instances only tier 3 can run)            */
  int32_t t3_grid;            /* CTAs of a grid-tier chain (0: one per SM)     */
  float hybrid_rate;          /* one SM: Delta maintained below this block
                                 acceptance rate (< 0: the default 5e-4)       */
  float warp_rate;            /* one SM: one warp runs the direct mode alone
                                 from this rate (< 0: the default)             */
  float cluster_hybrid_rate;  /* cluster: direct mode above this rate (< 0:
                                 the default 2e-3; 0: Delta mode throughout)  */
  uint32_t reserved;          /* must be 0                                     */
} qap_knobs;

/* Makes `k` the knobs of every chain created afterwards with n_lo <= N <= n_hi
 * (a later call for an overlapping range takes precedence; k == NULL clears
 * all ranges).  The QAPSA_* environment variables still override a knob.
 * Process-wide and thread-safe.  QAP_E_INVAL for n_lo > n_hi or reserved != 0. */
QAP_EXPORT int qap_knobs_set(int32_t n_lo, int32_t n_hi, const qap_knobs *k);

/* Measures the candidate knobs for problems of size N on the current GPU and
 * returns the fastest in *best (and its time in *seconds, may be NULL): each
 * candidate runs the same seeded uniform symmetric instance (entries in
 * [0, 99], zero diagonal) over a whole geometric schedule of `iters`
 * iterations from T0 = 0.5 mean|Delta_0| to Tf = 1e-3 T0, the schedule form of
 * the library's workloads.  Candidates: the grid tier against the on-chip one
 * (N > 2), the direct/Delta switch rates of the on-chip tier, and for the grid
 * tier one CTA per SM or half as many.  Blocks; takes a few times a run of
 * `iters` iterations.  Errors as qap_sa_create.                               */
QAP_EXPORT int qap_tune(int32_t N, uint64_t iters, qap_knobs *best, double *seconds);

/* ---- library ------------------------------------------------------------- */
/* Largest N any tier supports on the current device (0 if no device).      */
QAP_EXPORT int32_t qap_sa_max_n(void);

/* Largest N of one tier on the current device (0 if no device or an unknown
 * tier): 1 = one SM (about 276), 2 = a cluster of up to 16 SMs (1136),
 * 3 = the grid tier for symmetric instances, 4 = the grid tier for general
 * (asymmetric) instances.                                                    */
QAP_EXPORT int32_t qap_sa_max_n_tier(int32_t tier);

/* Static text for a status code; for QAP_E_CUDA the last CUDA error text of
 * the calling thread is appended.                                            */
QAP_EXPORT const char *qap_sa_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* QAP_SA_H */
