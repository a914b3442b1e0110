// qap_sa.cu -- host runtime of libqapsa: the C ABI declared in
// include/qap_sa.h.  Validates inputs, owns device memory and streams, fixes
// the cooling schedule, and launches the kernels of sa_kernels.cuh.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>

#include "qap_sa.h"
#include "qap_internal.h"
#include "sa_tier2.cuh"
#include "sa_tier3.cuh"
#include "sa_hot.cuh"

#include <chrono>
#include <vector>

using namespace qapsa;

__global__ void classify_kernel(const int *A32, const int *B32, const int *p0, int N,
                                int *count, SetupOut *out);

namespace {

thread_local char g_errbuf[256];

int cuda_fail(cudaError_t e, const char *what) {
  snprintf(g_errbuf, sizeof g_errbuf, "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? QAP_E_NOMEM : QAP_E_CUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Iterations per launch of the SA kernel: bounds the length of one kernel and
// lets the host see device errors between launches.  run(a); run(b) equals
// run(a + b), so the split does not change the trajectory.
unsigned long long chunk_iters() {
  static unsigned long long v = [] {
    const char *e = getenv("QAPSA_CHUNK_ITERS");
    unsigned long long x = e ? strtoull(e, nullptr, 10) : 0ull;
    return x ? x : (1ull << 26);
  }();
  return v;
}

// Set once by preload_kernels (see there).
int g_tmem_min_smem = 0;   // least dynamic shared memory of a TMEM-kernel launch
bool g_tmem_ok = true;     // one TMEM-holding CTA per SM is guaranteed

// Knobs registered with qap_knobs_set (later ranges first), and the knobs of
// qap_tune's trial chains on the calling thread.
struct KnobRange {
  int lo, hi;
  qap_knobs k;
};
std::mutex g_knob_mu;
std::vector<KnobRange> g_knobs;
thread_local const qap_knobs *t_knob_override = nullptr;

qap_knobs default_knobs() {
  qap_knobs k{};
  k.tier = 0;
  k.t3_grid = 0;
  k.hybrid_rate = -1.0f;
  k.warp_rate = -1.0f;
  k.cluster_hybrid_rate = -1.0f;
  k.reserved = 0;
  return k;
}

qap_knobs knobs_for(int N) {
  if (t_knob_override) return *t_knob_override;
  std::lock_guard<std::mutex> lock(g_knob_mu);
  for (auto it = g_knobs.rbegin(); it != g_knobs.rend(); ++it)
    if (it->lo <= N && N <= it->hi) return it->k;
  return default_knobs();
}

int device_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
      cudaSuccess)
    return 0;
  return v;
}

// Row stride of the int8 A and B' rows: 16 bytes times an odd number, so that
// eight threads reading 16-byte chunks of eight consecutive rows hit distinct
// bank groups.
constexpr int row_stride(int N) { return 16 * (((N + 15) / 16) | 1); }

// Height of the register tiles of Delta.
int tile_rows(int) { return kT1R; }

// R x 4 tiles of the upper triangle that hold at least one pair u < v < N,
// row-block major, each encoded as first_row << 16 | first_column.
std::vector<int> make_tiles(int N, int R) {
  std::vector<int> t;
  for (int u0 = 0; u0 < N - 1; u0 += R)
    for (int v0 = 0; v0 < N; v0 += 4) {
      bool any = false;
      for (int i = 0; i < R && !any; ++i)
        for (int c = 0; c < 4 && !any; ++c) {
          const int u = u0 + i, v = v0 + c;
          any = u < v && v < N;
        }
      if (any) t.push_back(u0 << 16 | v0);
    }
  return t;
}

int pow2_floor(int x) {
  int p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

// The cooling schedule, built exactly as the header documents it.
struct Schedule {
  double T0, Tf, alpha;
  unsigned long long I;
  double P[8][256];
};

void build_schedule(Schedule *S, double T0, double Tf, unsigned long long I) {
  S->T0 = T0;
  S->Tf = Tf;
  S->I = I;
  const double ratio = Tf / T0;
  S->alpha = (I >= 2) ? pow(ratio, 1.0 / (double)(I - 1)) : 1.0;
  double sq[64];
  sq[0] = S->alpha;
  for (int i = 1; i < 64; ++i) sq[i] = sq[i - 1] * sq[i - 1];
  for (int b = 0; b < 8; ++b)
    for (int v = 0; v < 256; ++v) {
      double f = 1.0;
      for (int bit = 0; bit < 8; ++bit)
        if (v & (1 << bit)) f = f * sq[8 * b + bit];
      S->P[b][v] = f;
    }
}

double schedule_T(const Schedule &S, unsigned long long it) {
  double T = S.T0;
  for (int b = 7; b >= 0; --b) T = T * S.P[b][(it >> (8 * b)) & 255u];
  return T;
}

}  // namespace

// Largest window offset the probe accepts (windows are at most M < 2^31 long).
constexpr unsigned long long kProbeMaxOffset = 1ull << 30;

// Eq. (2) for given proposals, decided as the SA kernels decide it, for tests of
// the binary32 pre-test against binary64.  Probe k is the proposal of iteration
// it[k] with swap cost delta[k], in a window that starts at it0[k] <= it[k].
// out[k] bit 0: the decision (binary32 interval, binary64 when undecided);
// bits 2-3: the interval of the prepared tables (0 reject, 1 accept,
// 2 undecided); bits 4-5: the interval of the in-window pre-test; bit 6: the
// integer pre-filter of a window of it[k] - it0[k] + 1 proposals rejects;
// bit 7: the binary64 test saw a near-tie.
__global__ void accept_probe_kernel(ChainDev g, int n, const unsigned long long *its,
                                    const unsigned long long *it0s, const int *deltas,
                                    int *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const unsigned long long it = its[k], it0 = it0s[k];
  const int dv = deltas[k];
  const int j = (int)(it - it0);
  // the prepared tables: the Philox block of it, T of the block's first iteration
  const unsigned long long q = it >> 2;
  const int w = (int)(it & 3u);
  const uint4 x = rng_block(g.seed, g.stream, q);
  const float Tq = g.T0f * exp2f(u64_to_f32(q << 2) * g.log2a_f);
  const float2 bt = accept_interval(g.mrel, Tq * exp2f((float)w * g.log2a_f), word_of(x, w));
  const float df = (float)dv;
  const int dt = dv <= 0 ? 1 : (df < bt.x ? 1 : (!(df > bt.y) ? 2 : 0));
  // the in-window pre-test and the integer pre-filter of a window [it0, it]
  const float Tw = g.T0f * exp2f(u64_to_f32(it0) * g.log2a_f);
  const unsigned o = pretest_cells(g.seed, g.stream, g.log2a_f, g.mrel, it0, Tw, j, 0, 0, 0,
                                   dv, 0, 0, 0, 1u);
  const int dw = dv <= 0 ? 1 : ((o & 1u) ? 1 : (((o >> 4) & 1u) ? 2 : 0));
  const float Te = Tw * exp2f((float)(j + 1) * g.log2a_f);
  const float tmax = fmaxf(Tw, Te) * 24.5f;
  const int thr = (tmax < 1.0e9f) ? (int)ceilf(tmax) + 1 : 0x7FFFFFFF;
  const int filt = dv > thr ? 1 : 0;
  unsigned long long nt = 0;
  const int ex = dv <= 0 ? 1 : exact_accept(g.seed, g.stream, g.T0, g.P, dv, it, &nt, nullptr);
  out[k] = ex | (dt << 2) | (dw << 4) | (filt << 6) | ((nt ? 1 : 0) << 7);
}

struct qap_sa {
  int N = 0, S = 0, M = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int8_t *A8 = nullptr, *Bp8 = nullptr;
  int *delta = nullptr, *p = nullptr, *d = nullptr;
  ChainStatus *st = nullptr;
  double *P = nullptr;
  int *tiles = nullptr;
  Schedule sched;
  ChainDev dev{};
  T1Layout layout{};
  int R = 4, nthreads = 0;
  int cluster = 1;      // CTAs per chain (tier 2)
  int smem_bytes = 0;   // dynamic shared memory of the SA kernel
  unsigned long long it_host = 0;  // iterations enqueued so far
  int tier = 1;
  // tier 2: the hot-phase kernel (one CTA of hot_warps warps, rows in L2) runs
  // each piece first while the chain's acceptance is at least hot_lo
  int hot = 0;
  int8_t *B8 = nullptr;  // B as int8 rows of stride S (the hot-phase kernel's)
  int hot_warps = 0;
  int hot_smem = 0;
  float hot_lo = 0.0f;
  // tier 3 (a persistent grid, Delta in global memory)
  int general = 0;                 // the general (asymmetric) swap-cost forms
  int random_order = 0;            // proposals drawn at random
  int *A3 = nullptr, *AT3 = nullptr, *B3 = nullptr, *BT3 = nullptr;
  int *Ad3 = nullptr, *Bd3 = nullptr, *dR3 = nullptr, *dC3 = nullptr;
  unsigned long long *bar3 = nullptr;
  unsigned *keys3 = nullptr;
  T3Dev dev3{};
  // CUDA-event timing of the launches (qap_sa_set_timing)
  struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
  };
  int timing = 0;
  std::vector<TimedLaunch> timed;
};

namespace {

// Device memory of a handle is stream-ordered (cudaMallocAsync/cudaFreeAsync on
// the handle's stream): unlike cudaFree, freeing it never waits for the work
// of other streams, so chains that run side by side (the server, the batch
// set-up) never serialise on each other's allocations.
void dfree(void *p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// Event pair around the launches of one scope, of kernel kind k, on the
// handle's stream while timing is on.
struct LaunchTimer {
  qap_sa *h;
  int k;
  cudaEvent_t a = nullptr, b = nullptr;
  LaunchTimer(qap_sa *h_, int k_) : h(h_), k(k_) {
    if (!h->timing) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      if (a) cudaEventDestroy(a);
      a = b = nullptr;
      cudaGetLastError();
      return;
    }
    cudaEventRecord(a, h->stream);
  }
  ~LaunchTimer() {
    if (!a) return;
    cudaEventRecord(b, h->stream);
    h->timed.push_back({k, a, b});
  }
};

void free_handle(qap_sa *h) {
  if (!h) return;
  cudaStream_t st = h->stream;
  if (st) cudaStreamSynchronize(st);
  dfree(h->A8, st);
  dfree(h->Bp8, st);
  dfree(h->delta, st);
  dfree(h->p, st);
  dfree(h->d, st);
  dfree(h->st, st);
  dfree(h->P, st);
  dfree(h->tiles, st);
  dfree(h->B8, st);
  dfree(h->A3, st);
  if (h->AT3 != h->A3) dfree(h->AT3, st);
  dfree(h->B3, st);
  if (h->BT3 != h->B3) dfree(h->BT3, st);
  dfree(h->Ad3, st);
  dfree(h->Bd3, st);
  dfree(h->dR3, st);
  dfree(h->dC3, st);
  dfree(h->bar3, st);
  dfree(h->keys3, st);
  for (auto &t : h->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  if (h->own_stream && st) cudaStreamDestroy(st);
  delete h;
}

// Threads of the tier-1 CTA: one per tile and one per row at least, 256 at
// least; the kernel is compiled for up to 256 and for up to 640 threads.
int tier1_threads(int N, int ntiles) {
  int nt = ntiles > N ? ntiles : N;
  if (nt < 256) nt = 256;
  return (nt + 31) & ~31;
}

int tier1_fits(int N) {
  const int R = tile_rows(N);
  const int nt = tier1_threads(N, (int)make_tiles(N, R).size());
  if (nt > kT1LargeThreads) return 0;
  return t1_layout(N, row_stride(N)).bytes <= device_smem_optin();
}

int max_n_tier1() {
  static int cached = -1;
  if (cached >= 0) return cached;
  int lo = 2, hi = 1024;
  if (!tier1_fits(lo)) return 0;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (tier1_fits(mid)) lo = mid; else hi = mid - 1;
  }
  cached = lo;
  return lo;
}

// Tier 2: one chain on a cluster of C CTAs of 640 threads, R = 16 tiles.
// Load every kernel of the library now (once per process) and give each the
// device's whole opt-in shared memory as its limit, so that handles of
// different N never lower the limit under one another's launches.  With lazy
// module loading the first launch of a kernel loads its code, and that waits
// for work already running on the device -- a request served on the cluster
// tier while one-SM chains run would stall until they finish.
void preload_kernels() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncAttributes a;
    cudaFuncGetAttributes(&a, setup_pack_kernel);
    cudaFuncGetAttributes(&a, setup_bprime_kernel);
    cudaFuncGetAttributes(&a, setup_gram_kernel);
    cudaFuncGetAttributes(&a, setup_delta_kernel);
    cudaFuncGetAttributes(&a, rebuild_delta_kernel);
    cudaFuncGetAttributes(&a, clear_rebuild_kernel);
    cudaFuncGetAttributes(&a, hot_bprime_kernel);
    cudaFuncGetAttributes(&a, hot_pack_b_kernel);
    cudaFuncGetAttributes(&a, classify_kernel);
    cudaFuncGetAttributes(&a, t3_pack_kernel);
    cudaFuncGetAttributes(&a, t3_perm_kernel);
    cudaFuncGetAttributes(&a, t3_gram_kernel);
    cudaFuncGetAttributes(&a, t3_delta_kernel);
    const int smem = device_smem_optin();
    // the limit covers dynamic shared memory only: the kernel's static part
    // comes off the device's opt-in size
    auto give_all = [smem](const void *k) {
      cudaFuncAttributes fa;
      if (cudaFuncGetAttributes(&fa, k) == cudaSuccess)
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem - (int)fa.sharedSizeBytes);
    };
    give_all((const void *)sa_tier1_kernel<kT1SmallThreads>);
    give_all((const void *)sa_tier1_kernel<kT1LargeThreads>);
    give_all((const void *)sa_batch_kernel);
    give_all((const void *)sa_tier2_kernel);
    give_all((const void *)sa_tier2_batch_kernel);
    give_all((const void *)sa_hot_kernel);
    give_all((const void *)sa_tier3_kernel<false>);
    give_all((const void *)sa_tier3_kernel<true>);
    cudaFuncSetAttribute(sa_tier2_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(sa_tier2_batch_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                         1);
    cudaGetLastError();
    // The kernels that keep Delta in Tensor Memory allocate all 512 columns of
    // the SM's TMEM; a second such CTA on the same SM would wait in
    // tcgen05.alloc for the first to finish -- across the CTAs of a cluster,
    // which wait for each other at cluster barriers, that could never end.
    // Their register use at 640 threads keeps one CTA per SM; check it, and
    // where it does not hold, make every launch of them ask for more than half
    // of the SM's shared memory, which does.
    const void *tmem_kernels[4] = {(const void *)sa_tier1_kernel<kT1LargeThreads>,
                                   (const void *)sa_batch_kernel,
                                   (const void *)sa_tier2_kernel,
                                   (const void *)sa_tier2_batch_kernel};
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    auto ctas_per_sm = [](const void *k, int smem_dyn) {
      int n = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kT1LargeThreads, smem_dyn) !=
          cudaSuccess) {
        cudaGetLastError();
        return -1;
      }
      return n;
    };
    bool one = true;
    for (const void *k : tmem_kernels) one = one && ctas_per_sm(k, 0) <= 1;
    if (!one) {
      g_tmem_min_smem = per_sm / 2 + 1;
      for (const void *k : tmem_kernels) {
        cudaFuncAttributes fa;
        const int dyn = (cudaFuncGetAttributes(&fa, k) == cudaSuccess)
                            ? g_tmem_min_smem - (int)fa.sharedSizeBytes : g_tmem_min_smem;
        if (ctas_per_sm(k, dyn > 0 ? dyn : 0) > 1) g_tmem_ok = false;
      }
    }
    cudaGetLastError();
  });
}

// Dynamic shared memory of a launch of a TMEM-holding kernel: at least what
// keeps it alone on its SM.
int tmem_smem(int want) { return want > g_tmem_min_smem ? want : g_tmem_min_smem; }

int tier2_cluster(int N) {
  const int nt = (int)make_tiles(N, kT2R).size();
  return (nt + kT2Threads - 1) / kT2Threads;
}

int tier2_tpv(int, int) { return kT2Tpv; }

int tier2_bytes(int N, int C) { return t2_layout(N, row_stride(N), C).bytes; }

int tier2_fits(int N) {
  const int C = tier2_cluster(N);
  if (C < 2 || C > kT2MaxCluster || N > kT2MaxN) return 0;
  if (tier2_bytes(N, C) + 64 > device_smem_optin()) return 0;  // 64: static part
  static int ok_for[kT2MaxCluster + 1] = {0};  // 0 unknown, 1 yes, -1 no
  if (ok_for[C] == 0) {
    preload_kernels();
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kT2Threads);
    cfg.dynamicSmemBytes = tier2_bytes(N, C);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    ok_for[C] = (cudaOccupancyMaxActiveClusters(&n, sa_tier2_kernel, &cfg) == cudaSuccess &&
                 n >= 1) ? 1 : -1;
    cudaGetLastError();
  }
  return ok_for[C] > 0;
}


int max_n_tier2() {
  static int cached = -1;
  if (cached >= 0) return cached;
  preload_kernels();
  int best = max_n_tier1();
  for (int N = best + 1; N <= 2048; ++N) {
    if (tier2_cluster(N) > kT2MaxCluster) break;
    if (tier2_fits(N)) best = N;
  }
  cached = best;
  return best;
}

// Tier 3: the largest N whose shared-memory vectors fit one CTA (symmetric
// instances need fewer vectors than general ones).
int max_n_tier3(bool general) {
  const int optin = device_smem_optin();
  int N = 2;
  while (t3_smem_bytes(N + 4, general) + 64 <= optin) N += 4;
  while (t3_smem_bytes(N + 1, general) + 64 <= optin) ++N;
  return N;
}

int max_n_any() {
  static int cached = -1;
  if (cached >= 0) return cached;
  const int t2 = max_n_tier2(), t3 = max_n_tier3(false);
  cached = t2 > t3 ? t2 : t3;
  return cached;
}

// CTAs of a tier-3 grid: one per SM, fewer for small problems (about 256 cells
// of Delta each at least), within what a cooperative launch can keep resident.
int tier3_grid(int N, bool general, int pref) {
  int dev = 0, sms = 1, nb = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void *k = general ? (const void *)sa_tier3_kernel<true> : (const void *)sa_tier3_kernel<false>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kT3Threads,
                                                    t3_smem_bytes(N, general)) != cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  const long long M = (long long)N * (N - 1) / 2;
  long long G = M / 256;
  if (G < 1) G = 1;
  if (G > sms) G = sms;
  if (G > (long long)nb * sms) G = (long long)nb * sms;
  if (pref >= 1 && pref <= (long long)nb * sms) G = pref;
  if (const char *e = getenv("QAPSA_T3_GRID")) {
    const long long x = atoll(e);
    if (x >= 1 && x <= (long long)nb * sms) G = x;
  }
  return (int)G;
}

cudaError_t launch_tier2(const ChainDev &g, unsigned long long it_end, int C,
                         int smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kT2Threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sa_tier2_kernel, g, it_end);
}

// Keep freed stream-ordered memory in the device's default pool instead of
// returning it at every synchronisation (once per device).
void keep_pool_memory() {
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  done[dev] = true;
}

}  // namespace

// Classifies an instance for the choice of tier: symmetry, zero diagonals,
// entries within int8, the largest magnitudes, and whether p0 is a permutation.
__global__ void classify_kernel(const int *A32, const int *B32, const int *p0, int N,
                                int *count, SetupOut *out) {
  int flags = 0, ma = 0, mb = 0;
  const long long NN = (long long)N * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < NN;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx - (long long)i * N);
    const int a = A32[idx], b = B32[idx];
    if (a != A32[(long long)j * N + i] || b != B32[(long long)j * N + i]) flags |= kFlagAsym;
    if (i == j && (a != 0 || b != 0)) flags |= kFlagDiag;
    const int aa = a < 0 ? (a == INT_MIN ? INT_MAX : -a) : a;
    const int ab = b < 0 ? (b == INT_MIN ? INT_MAX : -b) : b;
    ma = max(ma, aa);
    mb = max(mb, ab);
    if (aa > 127) flags |= kFlagRangeA;
    if (ab > 127) flags |= kFlagRangeB;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int v = p0[i];
    if (v < 0 || v >= N) flags |= kFlagPerm;
    else atomicAdd(count + v, 1);
  }
  flags = __reduce_or_sync(0xFFFFFFFFu, flags);
  ma = __reduce_max_sync(0xFFFFFFFFu, ma);
  mb = __reduce_max_sync(0xFFFFFFFFu, mb);
  if ((threadIdx.x & 31) == 0) {
    if (flags) atomicOr(&out->flags, flags);
    atomicMax(&out->max_abs_a, ma);
    atomicMax(&out->max_abs_b, mb);
  }
}

__global__ void classify_perm_kernel(const int *count, int N, SetupOut *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    if (count[i] != 1) atomicOr(&out->flags, kFlagPerm);
}

namespace {

int classify(const int32_t *A32, const int32_t *B32, int32_t N, const int32_t *p032,
             cudaStream_t stream, SetupOut *res) {
  int *count = nullptr;
  SetupOut *so = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&count, sizeof(int) * N, stream);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&so, sizeof(SetupOut), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int) * N, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(so, 0, sizeof(SetupOut), stream);
  if (e == cudaSuccess) {
    const long long NN = (long long)N * N;
    const int blocks = (int)((NN + 255) / 256 < 4096 ? (NN + 255) / 256 : 4096);
    classify_kernel<<<blocks, 256, 0, stream>>>(A32, B32, p032, N, count, so);
    classify_perm_kernel<<<(N + 255) / 256, 256, 0, stream>>>(count, N, so);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, so, sizeof *res, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  dfree(count, stream);
  dfree(so, stream);
  return e == cudaSuccess ? QAP_OK : cuda_fail(e, "classify");
}

// Tier 3 set-up (step (a) of section 2.2): static rows of A, B (and their
// transposes for general instances), Delta_0 from the Gram sums, the Gram
// diagonals, C0, the schedule.  h has its stream and sizes; on failure the
// caller frees h.
int create_tier3(qap_sa *h, const int32_t *A32, const int32_t *B32, const int32_t *p032,
                 const qap_schedule *sc, uint64_t seed, bool general, bool random,
                 const SetupOut &cls) {
  const int N = h->N, M = h->M;
  cudaStream_t stream = h->stream;
  if (N > max_n_tier3(general)) return QAP_E_UNSUPPORTED;
  // Swap costs and the Gram sums behind them stay below 8 N max|A| max|B|.
  if (8.0 * N * (double)cls.max_abs_a * (double)cls.max_abs_b > 2147483647.0)
    return QAP_E_RANGE;
  h->tier = 3;
  h->general = general ? 1 : 0;
  h->random_order = random ? 1 : 0;
  const int SA = t3_np(N);
  const size_t rows = (size_t)N * SA * sizeof(int);
  int *count = nullptr;
  long long *R = nullptr, *C = nullptr;
  SetupOut *so = nullptr;
  auto done = [&](int code) {
    dfree(count, stream);
    dfree(R, stream);
    if (C != R) dfree(C, stream);
    dfree(so, stream);
    return code;
  };
#define CK3(call)                                            \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return done(cuda_fail(e_, #call)); \
  } while (0)
  CK3(cudaMallocAsync((void **)&h->A3, rows, stream));
  CK3(cudaMallocAsync((void **)&h->B3, rows, stream));
  if (general) {
    CK3(cudaMallocAsync((void **)&h->AT3, rows, stream));
    CK3(cudaMallocAsync((void **)&h->BT3, rows, stream));
  } else {
    h->AT3 = h->A3;
    h->BT3 = h->B3;
  }
  CK3(cudaMallocAsync((void **)&h->Ad3, sizeof(int) * N, stream));
  CK3(cudaMallocAsync((void **)&h->Bd3, sizeof(int) * N, stream));
  CK3(cudaMallocAsync((void **)&h->dR3, sizeof(int) * N, stream));
  CK3(cudaMallocAsync((void **)&h->dC3, sizeof(int) * N, stream));
  // two copies of Delta: the state, and the buffer a swap writes during a launch
  CK3(cudaMallocAsync((void **)&h->delta, 2 * sizeof(int) * (size_t)(M > 0 ? M : 1), stream));
  CK3(cudaMallocAsync((void **)&h->p, sizeof(int) * N, stream));
  CK3(cudaMallocAsync((void **)&h->st, sizeof(ChainStatus), stream));
  CK3(cudaMallocAsync((void **)&h->P, sizeof(double) * 8 * 256, stream));
  CK3(cudaMallocAsync((void **)&h->bar3, sizeof(unsigned long long), stream));
  CK3(cudaMallocAsync((void **)&h->keys3, 4 * sizeof(unsigned), stream));
  CK3(cudaMallocAsync((void **)&count, sizeof(int) * N, stream));
  CK3(cudaMallocAsync((void **)&R, sizeof(long long) * (size_t)N * N, stream));
  if (general) CK3(cudaMallocAsync((void **)&C, sizeof(long long) * (size_t)N * N, stream));
  else C = R;
  CK3(cudaMallocAsync((void **)&so, sizeof(SetupOut), stream));
  CK3(cudaMemsetAsync(h->A3, 0, rows, stream));
  CK3(cudaMemsetAsync(h->B3, 0, rows, stream));
  if (general) {
    CK3(cudaMemsetAsync(h->AT3, 0, rows, stream));
    CK3(cudaMemsetAsync(h->BT3, 0, rows, stream));
  }
  CK3(cudaMemsetAsync(count, 0, sizeof(int) * N, stream));
  CK3(cudaMemsetAsync(so, 0, sizeof(SetupOut), stream));
  CK3(cudaMemsetAsync(h->st, 0, sizeof(ChainStatus), stream));
  {
    const long long NN = (long long)N * N;
    const int blocks = (int)((NN + 255) / 256 < 4096 ? (NN + 255) / 256 : 4096);
    t3_pack_kernel<<<blocks, 256, 0, stream>>>(A32, B32, p032, N, SA, h->A3, h->AT3, h->B3,
                                               h->BT3, h->Ad3, h->Bd3, count, h->general, so);
    t3_perm_kernel<<<(N + 255) / 256, 256, 0, stream>>>(p032, N, count, h->p, so);
    dim3 gg((N + 127) / 128, N);
    t3_gram_kernel<<<gg, 128, 0, stream>>>(h->A3, h->AT3, h->B3, h->p, N, SA, h->general, R, C);
    t3_delta_kernel<<<gg, 128, 0, stream>>>(R, C, h->A3, h->B3, h->p, N, SA, h->general,
                                            h->delta, h->dR3, h->dC3, so);
    CK3(cudaGetLastError());
  }
  SetupOut so_h{};
  CK3(cudaMemcpyAsync(&so_h, so, sizeof so_h, cudaMemcpyDeviceToHost, stream));
  CK3(cudaStreamSynchronize(stream));
  done(QAP_OK);
  count = nullptr;
  R = C = nullptr;
  so = nullptr;
  if (so_h.flags & kFlagPerm) return QAP_E_INVAL;

  double T0 = sc->t0, Tf = sc->tf;
  if (sc->flags & QAP_T_RELATIVE) {
    const double mean = so_h.sum_abs_delta > 0 ? (double)so_h.sum_abs_delta / (double)M : 1.0;
    T0 = sc->t0 * mean;
    Tf = sc->tf * T0;
  }
  if (!(T0 > 0.0) || !(Tf > 0.0) || !isfinite(T0) || !isfinite(Tf)) return QAP_E_INVAL;
  build_schedule(&h->sched, T0, Tf, sc->total_iters);
  CK3(cudaMemcpyAsync(h->P, h->sched.P, sizeof h->sched.P, cudaMemcpyHostToDevice, stream));
  {
    ChainStatus st0{};
    st0.cost = so_h.cost0;
    CK3(cudaMemcpyAsync(h->st, &st0, sizeof st0, cudaMemcpyHostToDevice, stream));
  }
  T3Dev &g = h->dev3;
  g.N = N;
  g.M = M;
  g.SA = SA;
  g.general = h->general;
  g.random_order = h->random_order;
  g.G = tier3_grid(N, general, knobs_for(N).t3_grid);
  g.A = h->A3;
  g.AT = h->AT3;
  g.B = h->B3;
  g.BT = h->BT3;
  g.Adiag = h->Ad3;
  g.Bdiag = h->Bd3;
  g.delta = h->delta;
  g.delta2 = h->delta + (M > 0 ? M : 1);
  g.p = h->p;
  g.dR = h->dR3;
  g.dC = h->dC3;
  g.st = h->st;
  g.bar = h->bar3;
  g.keys = h->keys3;
  g.seed = seed;
  g.stream = sc->stream_id;
  g.T0 = T0;
  g.P = h->P;
  g.T0f = (float)T0;
  const double l2r = log2(Tf / T0);
  g.log2a_f = sc->total_iters >= 2 ? (float)(l2r / (double)(sc->total_iters - 1)) : 0.0f;
  g.mrel = (float)(2e-5 + 2e-7 * fabs(l2r) + 8.0 * (double)sc->total_iters * 0x1p-53);
  h->cluster = g.G;
  h->nthreads = kT3Threads;
  h->smem_bytes = t3_smem_bytes(N, general);
  // keep each CTA's share of rows in shared memory when it fits
  g.nvmax = (N + g.G - 1) / g.G + 1;
  g.cache_rows = 0;
  if (!getenv("QAPSA_T3_NOCACHE") &&
      h->smem_bytes + t3_cache_bytes(N, general, g.nvmax) + 64 <= device_smem_optin()) {
    g.cache_rows = 1;
    h->smem_bytes += t3_cache_bytes(N, general, g.nvmax);
  }
  CK3(cudaStreamSynchronize(stream));
  return QAP_OK;
#undef CK3
}

// Common body of the two create entry points; A32/B32/p032 are device
// pointers that stay valid for the duration of the call.
int create_common(const int32_t *A32, const int32_t *B32, int32_t N,
                  const int32_t *p032, const qap_schedule *sc, uint64_t seed,
                  cudaStream_t stream, bool own_stream, qap_sa **out) {
  preload_kernels();
  keep_pool_memory();
  qap_sa *h = new (std::nothrow) qap_sa();
  if (!h) return QAP_E_NOMEM;
  h->N = N;
  h->S = row_stride(N);
  h->M = N * (N - 1) / 2;
  h->stream = stream;
  h->own_stream = own_stream;
  const int S = h->S, M = h->M;
  int rc = QAP_OK;
  int *count = nullptr, *G = nullptr;
  SetupOut *so = nullptr;
  SetupOut so_h{};
  auto fail = [&](int code) {
    dfree(count, stream);
    dfree(G, stream);
    dfree(so, stream);
    free_handle(h);
    return code;
  };
#define CKF(call)                                           \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return fail(cuda_fail(e_, #call)); \
  } while (0)
  // The on-chip tiers take the symmetric, zero-diagonal instances with int8
  // entries in sequential order up to a cluster's capacity; tier 3 the rest.
  {
    SetupOut cls{};
    rc = classify(A32, B32, N, p032, stream, &cls);
    if (rc) return fail(rc);
    if (cls.flags & kFlagPerm) return fail(QAP_E_INVAL);
    const bool random = (sc->flags & QAP_ORDER_RANDOM) != 0;
    const bool general = (cls.flags & (kFlagAsym | kFlagDiag)) != 0;
    const bool wide = (cls.flags & (kFlagRangeA | kFlagRangeB)) != 0;
    const char *et = getenv("QAPSA_TIER");
    const bool force3 = et ? atoi(et) == 3 : knobs_for(N).tier == 3;
    if (random || general || wide || force3 || N > max_n_tier2()) {
      rc = create_tier3(h, A32, B32, p032, sc, seed, general, random, cls);
      if (rc) return fail(rc);
      *out = h;
      return QAP_OK;
    }
  }
  const size_t nS = (size_t)N * S;
  CKF(cudaMallocAsync((void **)&h->A8, nS, stream));
  CKF(cudaMallocAsync((void **)&h->Bp8, nS, stream));
  CKF(cudaMallocAsync((void **)&h->delta, sizeof(int) * (size_t)(M > 0 ? M : 1), stream));
  CKF(cudaMallocAsync((void **)&h->p, sizeof(int) * N, stream));
  CKF(cudaMallocAsync((void **)&h->d, sizeof(int) * N, stream));
  CKF(cudaMallocAsync((void **)&h->st, sizeof(ChainStatus), stream));
  CKF(cudaMallocAsync((void **)&h->P, sizeof(double) * 8 * 256, stream));
  h->tier = N <= max_n_tier1() ? 1 : 2;
  const std::vector<int> tiles = make_tiles(N, h->tier == 1 ? tile_rows(N) : kT2R);
  CKF(cudaMallocAsync((void **)&h->tiles, sizeof(int) * (tiles.size() ? tiles.size() : 1),
                      stream));
  CKF(cudaMemcpyAsync(h->tiles, tiles.data(), sizeof(int) * tiles.size(),
                      cudaMemcpyHostToDevice, stream));
  CKF(cudaMallocAsync((void **)&count, sizeof(int) * N, stream));
  CKF(cudaMallocAsync((void **)&G, sizeof(int) * (size_t)N * N, stream));
  CKF(cudaMallocAsync((void **)&so, sizeof(SetupOut), stream));
  CKF(cudaMemsetAsync(h->A8, 0, nS, stream));
  CKF(cudaMemsetAsync(h->Bp8, 0, nS, stream));
  CKF(cudaMemsetAsync(count, 0, sizeof(int) * N, stream));
  CKF(cudaMemsetAsync(so, 0, sizeof(SetupOut), stream));
  CKF(cudaMemsetAsync(h->st, 0, sizeof(ChainStatus), stream));
  {
    const long long NN = (long long)N * N;
    const int blocks = (int)((NN + 255) / 256 < 4096 ? (NN + 255) / 256 : 4096);
    setup_pack_kernel<<<blocks, 256, 0, stream>>>(A32, B32, p032, N, S, h->A8,
                                                  count, so);
    setup_bprime_kernel<<<blocks, 256, 0, stream>>>(B32, p032, N, S, count,
                                                    h->Bp8, h->p, so);
    dim3 gg((N + 127) / 128, N);
    setup_gram_kernel<<<gg, 128, 0, stream>>>(h->A8, h->Bp8, N, S, G);
    setup_delta_kernel<<<gg, 128, 0, stream>>>(G, h->A8, h->Bp8, N, S,
                                               h->delta, h->d, so);
    CKF(cudaGetLastError());
  }
  CKF(cudaMemcpyAsync(&so_h, so, sizeof so_h, cudaMemcpyDeviceToHost, stream));
  CKF(cudaStreamSynchronize(stream));
  dfree(count, stream);
  count = nullptr;
  dfree(G, stream);
  G = nullptr;
  dfree(so, stream);
  so = nullptr;
  if (so_h.flags & (kFlagAsym | kFlagDiag | kFlagPerm)) return fail(QAP_E_INVAL);
  if (so_h.flags & (kFlagRangeA | kFlagRangeB)) return fail(QAP_E_RANGE);
  // Swap costs and the intermediate sums of the rows-r,s recompute stay
  // below 8 N max|A| max|B| in magnitude; all must fit in int32.
  if (8.0 * N * (double)so_h.max_abs_a * (double)so_h.max_abs_b > 2147483647.0)
    return fail(QAP_E_RANGE);

  // ---- schedule ----
  double T0 = sc->t0, Tf = sc->tf;
  if (sc->flags & QAP_T_RELATIVE) {
    const double mean = so_h.sum_abs_delta > 0
                            ? (double)so_h.sum_abs_delta / (double)M
                            : 1.0;
    T0 = sc->t0 * mean;
    Tf = sc->tf * T0;
  }
  if (!(T0 > 0.0) || !(Tf > 0.0) || !isfinite(T0) || !isfinite(Tf))
    return fail(QAP_E_INVAL);
  build_schedule(&h->sched, T0, Tf, sc->total_iters);
  CKF(cudaMemcpyAsync(h->P, h->sched.P, sizeof h->sched.P,
                      cudaMemcpyHostToDevice, stream));
  {
    ChainStatus st0{};
    st0.cost = so_h.cost0;
    st0.mode = 1;  // start evaluating proposals directly (hot start)
    CKF(cudaMemcpyAsync(h->st, &st0, sizeof st0, cudaMemcpyHostToDevice,
                        stream));
  }
  ChainDev &g = h->dev;
  g.N = N;
  g.S = S;
  g.M = M;
  g.ntiles = (int)tiles.size();
  g.tiles = h->tiles;
  if (h->tier == 1) {
    h->R = tile_rows(N);
    h->nthreads = tier1_threads(N, (int)tiles.size());
    g.tpv = pow2_floor(h->nthreads / N);
    if (g.tpv > 4) g.tpv = 4;  // >= 8 lanes per slice keep the 16-byte loads
                               // of eight consecutive rows conflict-free
  } else {
    h->R = kT2R;
    h->nthreads = kT2Threads;
    h->cluster = tier2_cluster(N);
    g.tpv = tier2_tpv(N, h->cluster);
  }
  g.A = h->A8;
  g.Bp = h->Bp8;
  g.delta = h->delta;
  g.p = h->p;
  g.d = h->d;
  g.st = h->st;
  g.seed = seed;
  g.stream = sc->stream_id;
  g.T0 = T0;
  g.P = h->P;
  g.T0f = (float)T0;
  const double l2r = log2(Tf / T0);
  g.log2a_f = sc->total_iters >= 2 ? (float)(l2r / (double)(sc->total_iters - 1)) : 0.0f;
  // Pre-test margin: covers binary32 rounding of T and -ln u, the byte-table
  // product's drift from T0 alpha^it, and the exponent's rounding.
  g.mrel = (float)(2e-5 + 2e-7 * fabs(l2r) + 8.0 * (double)sc->total_iters * 0x1p-53);
  // Acceptance rate below which the one-SM tier maintains Delta (above it,
  // proposals are evaluated directly): where one accepted swap's O(N^2) update
  // costs as much as evaluating ~2000 proposals directly.  Above warp_lo one
  // warp evaluates them alone (windows of 32..128, no block barrier per
  // accepted swap): from 1 accept in 512 proposals for the 256-thread kernel
  // (one lane per proposal), from 1 in 64 for the 640-thread one (two lanes
  // per proposal, sixteen proposals a pass).  Both from a sweep of whole runs at
  // N = 60..276; the modes change the speed only, never the trajectory.
  {
    const qap_knobs kn = knobs_for(N);
    const char *e = getenv("QAPSA_HYBRID_RATE");
    const float hdef = kn.hybrid_rate >= 0.0f ? kn.hybrid_rate : 5e-4f;
    g.hyb_lo = (h->tier == 1) ? (e ? (float)atof(e) : hdef) : 0.0f;
    if (h->tier == 2) {  // the cluster tier: direct mode at high acceptance as well
      const char *ec = getenv("QAPSA_CLUSTER_HYBRID_RATE");
      const float cdef = kn.cluster_hybrid_rate >= 0.0f ? kn.cluster_hybrid_rate : 2e-3f;
      g.hyb_lo = ec ? (float)atof(ec) : cdef;
    }
    const char *ew = getenv("QAPSA_WARP_RATE");
    float wdef = (h->nthreads <= kT1SmallThreads) ? 1.0f / 512.0f : 1.0f / 64.0f;
    if (kn.warp_rate >= 0.0f) wdef = kn.warp_rate;
    g.warp_lo = (h->tier == 1) ? (ew ? (float)atof(ew) : wdef) : 0.0f;
    // The cluster tier's hot phase on one SM while at least hot_lo of the
    // proposals are accepted, on as many warps (up to the default) as the
    // staged rows leave room for.
    if (h->tier == 2) {
      const char *eh = getenv("QAPSA_HOT");
      const char *el = getenv("QAPSA_HOT_RATE");
      const char *ewp = getenv("QAPSA_HOT_WARPS");
      h->hot_lo = el ? (float)atof(el) : kHotRateDefault;
      const int want = ewp ? atoi(ewp) : kHotWarpsDefault;
      int W = 1;  // a power of two
      while (2 * W <= want && 2 * W <= kHotMaxWarps) W *= 2;
      while (W > 1 && hot_layout(N, S, W).bytes > device_smem_optin()) W /= 2;
      h->hot_warps = W;
      h->hot_smem = hot_layout(N, S, W).bytes;
      h->hot = (eh ? atoi(eh) != 0 : true) && h->hot_lo > 0.0f && g.hyb_lo > 0.0f &&
               h->hot_smem <= device_smem_optin();
      if (h->hot) {
        CKF(cudaMallocAsync((void **)&h->B8, (size_t)N * S, stream));
        hot_pack_b_kernel<<<dim3((S + 255) / 256, N), 256, 0, stream>>>(B32, N, S, h->B8);
        CKF(cudaGetLastError());
      }
    }
  }
  h->layout = t1_layout(N, S);
  h->smem_bytes = h->tier == 1 ? h->layout.bytes : tier2_bytes(N, h->cluster);
  if (h->tier == 2 || h->nthreads > kT1SmallThreads) {
    if (!g_tmem_ok) return fail(QAP_E_UNSUPPORTED);
    h->smem_bytes = tmem_smem(h->smem_bytes);
  }
  CKF(cudaStreamSynchronize(stream));
  *out = h;
  return rc;
#undef CKF
}

int validate_args(const void *A, const void *B, int32_t N, const void *p0,
                  const qap_schedule *sc, qap_sa **out) {
  if (!out) return QAP_E_INVAL;
  *out = nullptr;
  if (!A || !B || !p0 || !sc) return QAP_E_INVAL;
  if (N < 2) return QAP_E_INVAL;
  if (sc->total_iters == 0) return QAP_E_INVAL;
  if (!(sc->t0 > 0.0) || !(sc->tf > 0.0) || !isfinite(sc->t0) || !isfinite(sc->tf))
    return QAP_E_INVAL;
  if (sc->flags & ~(QAP_T_RELATIVE | QAP_ORDER_RANDOM)) return QAP_E_INVAL;
  if (max_n_tier1() == 0) return QAP_E_CUDA;
  if (N > max_n_any()) return QAP_E_UNSUPPORTED;
  return QAP_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// Copies host A, B, p0 to temporary device buffers and runs create_common on
// `st` (owned by the handle if own_stream).
int create_from_host(const int32_t *A, const int32_t *B, int32_t N,
                     const int32_t *p0, const qap_schedule *sched,
                     uint64_t seed, cudaStream_t st, bool own_stream,
                     qap_sa **out) {
  int rc = QAP_OK;
  int32_t *dA = nullptr, *dB = nullptr, *dp = nullptr;
  const size_t nn = sizeof(int32_t) * (size_t)N * N;
  cudaError_t e = cudaMallocAsync((void **)&dA, nn, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&dB, nn, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&dp, sizeof(int32_t) * N, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dA, A, nn, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dB, B, nn, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dp, p0, sizeof(int32_t) * N, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "staging copy");
    dfree(dA, st);
    dfree(dB, st);
    dfree(dp, st);
    cudaStreamSynchronize(st);
    if (own_stream) cudaStreamDestroy(st);
    return rc;
  }
  // create_common synchronises the stream before it returns, and on failure
  // destroys an owned stream together with the partial handle.
  rc = create_common(dA, dB, N, dp, sched, seed, st, own_stream, out);
  // on success create_common has synchronised st; on failure it destroyed an
  // owned st, whose pending work (these frees included) still completes
  cudaStream_t fst = (rc == QAP_OK || !own_stream) ? st : (cudaStream_t)0;
  dfree(dA, fst);
  dfree(dB, fst);
  dfree(dp, fst);
  return rc;
}

}  // namespace

extern "C" {

int qap_sa_create(const int32_t *A, const int32_t *B, int32_t N,
                  const int32_t *p0, const qap_schedule *sched, uint64_t seed,
                  qap_sa **out) {
  int rc = validate_args(A, B, N, p0, sched, out);
  if (rc) return rc;
  cudaStream_t st = nullptr;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  return create_from_host(A, B, N, p0, sched, seed, st, true, out);
}

int qap_sa_create_device(const int32_t *A, const int32_t *B, int32_t N,
                         const int32_t *p0, const qap_schedule *sched,
                         uint64_t seed, void *cuda_stream, qap_sa **out) {
  int rc = validate_args(A, B, N, p0, sched, out);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  bool own = false;
  if (!st) {
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    own = true;
  }
  return create_common(A, B, N, p0, sched, seed, st, own, out);
}

int qap_sa_run_async(qap_sa *h, uint64_t iters) {
  if (!h) return QAP_E_INVAL;
  if (iters > h->sched.I || h->it_host + iters > h->sched.I) return QAP_E_RANGE;
  const unsigned long long end = h->it_host + iters;
  unsigned long long cur = h->it_host;
  while (cur < end) {
    unsigned long long stop = cur + chunk_iters();
    if (stop > end) stop = end;
    if (h->tier == 3) {
      CK(cudaMemsetAsync(h->bar3, 0, sizeof(unsigned long long), h->stream));
      CK(cudaMemsetAsync(h->keys3, 0xFF, 3 * sizeof(unsigned), h->stream));
      T3Dev d3 = h->dev3;
      unsigned long long e3 = stop;
      void *args[] = {&d3, &e3};
      const void *k = h->general ? (const void *)sa_tier3_kernel<true>
                                 : (const void *)sa_tier3_kernel<false>;
      cudaError_t el;
      {
        LaunchTimer t(h, QAP_KT_SA);
        el = cudaLaunchCooperativeKernel(k, dim3(h->dev3.G), dim3(kT3Threads), args,
                                         (size_t)h->smem_bytes, h->stream);
      }
      if (el != cudaSuccess) return cuda_fail(el, "sa_tier3_kernel launch");
    } else if (h->tier == 2) {
      // With the direct mode enabled a launch may leave Delta in global memory
      // stale (it ended in direct mode) or stop early to resume Delta mode:
      // rebuild Delta if flagged, and launch again to the same end (a no-op if
      // the first launch got there).  The second launch starts in Delta mode or
      // at the end, so it never stops early.
      const int rounds = h->dev.hyb_lo > 0.0f ? 2 : 1;
      if (h->hot && h->dev.hyb_lo > 0.0f) {
        // the hot phase first (it returns at once after it has handed the
        // chain over); it leaves B' and Delta in global memory to be rebuilt
        {
          LaunchTimer t(h, QAP_KT_HOT);
          sa_hot_kernel<<<1, 32 * h->hot_warps, h->hot_smem, h->stream>>>(h->dev, h->B8, stop,
                                                                            h->hot_lo);
        }
        LaunchTimer t(h, QAP_KT_AUX);
        hot_bprime_kernel<<<dim3((h->S + 255) / 256, h->N), 256, 0, h->stream>>>(h->dev, h->B8);
        rebuild_delta_kernel<<<dim3((h->N + 127) / 128, h->N), 128, 0, h->stream>>>(h->dev);
        clear_rebuild_kernel<<<1, 1, 0, h->stream>>>(h->st);
      }
      for (int k = 0; k < rounds; ++k) {
        cudaError_t e2;
        {
          LaunchTimer t(h, QAP_KT_SA);
          e2 = launch_tier2(h->dev, stop, h->cluster, h->smem_bytes, h->stream);
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "sa_tier2_kernel launch");
        if (rounds > 1) {
          LaunchTimer t(h, QAP_KT_AUX);
          rebuild_delta_kernel<<<dim3((h->N + 127) / 128, h->N), 128, 0, h->stream>>>(h->dev);
          clear_rebuild_kernel<<<1, 1, 0, h->stream>>>(h->st);
        }
      }
    } else if (h->nthreads <= kT1SmallThreads) {
      LaunchTimer t(h, QAP_KT_SA);
      sa_tier1_kernel<kT1SmallThreads>
          <<<1, h->nthreads, h->layout.bytes, h->stream>>>(h->dev, stop);
    } else {
      LaunchTimer t(h, QAP_KT_SA);
      sa_tier1_kernel<kT1LargeThreads>
          <<<1, h->nthreads, h->smem_bytes, h->stream>>>(h->dev, stop);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sa_tier1_kernel launch");
    cur = stop;
  }
  h->it_host = end;
  return QAP_OK;
}

int qap_sa_inject_barrier_fault(qap_sa *h, int on) {
  if (!h) return QAP_E_INVAL;
  if (h->tier != 3) return QAP_E_UNSUPPORTED;
  h->dev3.bar_skew = on ? 1u : 0u;
  return QAP_OK;
}

int qap_sa_set_timing(qap_sa *h, int on) {
  if (!h) return QAP_E_INVAL;
  cudaStreamSynchronize(h->stream);
  for (auto &t : h->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  h->timed.clear();
  h->timing = on != 0;
  return QAP_OK;
}

int qap_sa_kernel_times(qap_sa *h, double *seconds, uint64_t *launches) {
  if (!h || !seconds || !launches) return QAP_E_INVAL;
  for (int k = 0; k < QAP_KT_COUNT; ++k) {
    seconds[k] = 0.0;
    launches[k] = 0;
  }
  CK(cudaStreamSynchronize(h->stream));
  int rc = QAP_OK;
  for (auto &t : h->timed) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) {
      cudaGetLastError();
      rc = QAP_E_CUDA;
    }
    seconds[t.kind] += ms * 1e-3;
    ++launches[t.kind];
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  h->timed.clear();
  return rc;
}

int qap_sa_sync(qap_sa *h) {
  if (!h) return QAP_E_INVAL;
  CK(cudaStreamSynchronize(h->stream));
  int err = 0;
  CK(cudaMemcpyAsync(&err, &h->st->error, sizeof err, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (err == kT3ErrTimeout) return QAP_E_TIMEOUT;
  return err ? QAP_E_STATE : QAP_OK;
}

int qap_sa_run(qap_sa *h, uint64_t iters) {
  int rc = qap_sa_run_async(h, iters);
  if (rc) return rc;
  return qap_sa_sync(h);
}

int qap_sa_result(qap_sa *h, int32_t *p_out, int64_t *cost,
                  uint64_t *accepts) {
  if (!h) return QAP_E_INVAL;
  ChainStatus st{};
  CK(cudaMemcpyAsync(&st, h->st, sizeof st, cudaMemcpyDeviceToHost, h->stream));
  if (p_out)
    CK(cudaMemcpyAsync(p_out, h->p, sizeof(int32_t) * h->N,
                       cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (st.error) return QAP_E_STATE;
  if (cost) *cost = st.cost;
  if (accepts) *accepts = st.accepts;
  return QAP_OK;
}

int qap_sa_result_device(qap_sa *h, int32_t *p_out, int64_t *cost,
                         uint64_t *accepts) {
  if (!h) return QAP_E_INVAL;
  if (p_out)
    CK(cudaMemcpyAsync(p_out, h->p, sizeof(int32_t) * h->N,
                       cudaMemcpyDeviceToDevice, h->stream));
  if (cost)
    CK(cudaMemcpyAsync(cost, &h->st->cost, sizeof(int64_t),
                       cudaMemcpyDeviceToDevice, h->stream));
  if (accepts)
    CK(cudaMemcpyAsync(accepts, &h->st->accepts, sizeof(uint64_t),
                       cudaMemcpyDeviceToDevice, h->stream));
  return QAP_OK;
}

int qap_sa_get_info(qap_sa *h, qap_sa_info *out) {
  if (!h || !out) return QAP_E_INVAL;
  ChainStatus st{};
  CK(cudaMemcpyAsync(&st, h->st, sizeof st, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  memset(out, 0, sizeof *out);
  out->N = h->N;
  out->tier = h->tier;
  out->iterations = st.it;
  out->accepts = st.accepts;
  out->cost = st.cost;
  out->near_ties = st.near_ties;
  out->exact_evals = st.exact_evals;
  out->windows = st.windows;
  out->T0 = h->sched.T0;
  out->Tf = h->sched.Tf;
  out->alpha = h->sched.alpha;
  out->total_iters = h->sched.I;
  out->smem_bytes = (uint64_t)h->smem_bytes;
  out->direct_iters = st.direct_iters;
  out->direct_accepts = st.direct_accepts;
  out->warp_iters = st.warp_iters;
  out->ctas = h->cluster;
  out->threads = h->nthreads;
  out->hot_iters = st.hot_iters;
  out->hot_accepts = st.hot_accepts;
  return st.error ? QAP_E_STATE : QAP_OK;
}

int qap_sa_delta(qap_sa *h, int32_t *delta_out) {
  if (!h || !delta_out) return QAP_E_INVAL;
  CK(cudaMemcpyAsync(delta_out, h->delta, sizeof(int32_t) * (size_t)h->M,
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return QAP_OK;
}

double qap_sa_temperature(const qap_sa *h, uint64_t it) {
  if (!h) return 0.0;
  return schedule_T(h->sched, it);
}

int qap_sa_near_tie_log(qap_sa *h, uint64_t *it_out, int32_t cap, uint64_t *count) {
  if (!h || cap < 0 || (cap > 0 && !it_out)) return QAP_E_INVAL;
  ChainStatus st{};
  CK(cudaMemcpyAsync(&st, h->st, sizeof st, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const int n = (int)std::min<unsigned>(st.near_log_n, (unsigned)kNearLog);
  for (int k = 0; k < n && k < cap; ++k) it_out[k] = st.near_log[k];
  if (count) *count = st.near_ties;
  return QAP_OK;
}

int qap_sa_accept_probe(qap_sa *h, int32_t n, const uint64_t *it, const uint64_t *it0,
                        const int32_t *delta, int32_t *out) {
  if (!h || n < 0 || (n > 0 && (!it || !it0 || !delta || !out))) return QAP_E_INVAL;
  if (n == 0) return QAP_OK;
  for (int32_t k = 0; k < n; ++k)
    if (it0[k] > it[k] || it[k] - it0[k] >= (uint64_t)kProbeMaxOffset) return QAP_E_RANGE;
  cudaStream_t st = h->stream;
  unsigned long long *d_it = nullptr, *d_it0 = nullptr;
  int *d_delta = nullptr, *d_out = nullptr;
  auto cleanup = [&]() {
    dfree(d_it, st);
    dfree(d_it0, st);
    dfree(d_delta, st);
    dfree(d_out, st);
  };
  cudaError_t e = cudaMallocAsync((void **)&d_it, sizeof(uint64_t) * n, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_it0, sizeof(uint64_t) * n, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_delta, sizeof(int32_t) * n, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_out, sizeof(int32_t) * n, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_it, it, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_it0, it0, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_delta, delta, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    accept_probe_kernel<<<(n + 127) / 128, 128, 0, st>>>(h->dev, n, d_it, d_it0, d_delta, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "qap_sa_accept_probe");
  return QAP_OK;
}

void qap_sa_destroy(qap_sa *h) { free_handle(h); }

int32_t qap_sa_max_n(void) { return max_n_any(); }

int qap_knobs_set(int32_t n_lo, int32_t n_hi, const qap_knobs *k) {
  std::lock_guard<std::mutex> lock(g_knob_mu);
  if (!k) {
    g_knobs.clear();
    return QAP_OK;
  }
  if (n_lo > n_hi || k->reserved != 0 || k->tier < 0 || k->tier > 3 || k->t3_grid < 0)
    return QAP_E_INVAL;
  g_knobs.push_back(KnobRange{n_lo, n_hi, *k});
  return QAP_OK;
}

int qap_tune(int32_t N, uint64_t iters, qap_knobs *best, double *seconds) {
  if (!best || N < 2 || iters < 1) return QAP_E_INVAL;
  if (max_n_tier1() == 0) return QAP_E_CUDA;
  if (N > max_n_any()) return QAP_E_UNSUPPORTED;
  // the instance: uniform symmetric entries in [0, 99], zero diagonal, a random
  // p0 (splitmix64 of a fixed seed: an input generator, nothing of the method)
  uint64_t x = 0x9E3779B97F4A7C15ull ^ (uint64_t)N;
  auto next = [&x]() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  std::vector<int32_t> A((size_t)N * N, 0), B((size_t)N * N, 0), p0(N);
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) {
      A[(size_t)i * N + j] = A[(size_t)j * N + i] = (int32_t)(next() % 100);
      B[(size_t)i * N + j] = B[(size_t)j * N + i] = (int32_t)(next() % 100);
    }
  for (int i = 0; i < N; ++i) p0[i] = i;
  for (int i = N - 1; i > 0; --i) std::swap(p0[i], p0[(size_t)(next() % (uint64_t)(i + 1))]);
  const qap_schedule sc{0.5, 1e-3, iters, QAP_T_RELATIVE, 0};
  // candidates: the default choice first
  std::vector<qap_knobs> cand;
  cand.push_back(default_knobs());
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (N <= max_n_tier1()) {
    const float hs[2] = {2.5e-4f, 1e-3f};
    for (float hr : hs) {
      qap_knobs k = default_knobs();
      k.hybrid_rate = hr;
      cand.push_back(k);
    }
    const float wdef = N <= 180 ? 1.0f / 512.0f : 1.0f / 64.0f;  // the defaults' scale
    const float ws[2] = {0.5f * wdef, 2.0f * wdef};
    for (float wr : ws) {
      qap_knobs k = default_knobs();
      k.warp_rate = wr;
      cand.push_back(k);
    }
  } else if (N <= max_n_tier2()) {
    const float cs[3] = {0.0f, 1e-3f, 4e-3f};
    for (float cr : cs) {
      qap_knobs k = default_knobs();
      k.cluster_hybrid_rate = cr;
      cand.push_back(k);
    }
  }
  if (N > 2 && N <= max_n_tier2()) {
    qap_knobs k = default_knobs();
    k.tier = 3;
    cand.push_back(k);
    k.t3_grid = sms / 2 > 0 ? sms / 2 : 1;
    cand.push_back(k);
  } else if (N > max_n_tier2()) {
    qap_knobs k = default_knobs();
    k.t3_grid = sms / 2 > 0 ? sms / 2 : 1;
    cand.push_back(k);
  }
  double best_s = 1e300;
  int64_t cost0 = 0;
  uint64_t acc0 = 0;
  for (size_t c = 0; c < cand.size(); ++c) {
    t_knob_override = &cand[c];
    qap_sa *h = nullptr;
    int rc = qap_sa_create(A.data(), B.data(), N, p0.data(), &sc, 1, &h);
    t_knob_override = nullptr;
    if (rc) return rc;
    const auto t0 = std::chrono::steady_clock::now();
    rc = qap_sa_run(h, iters);
    const double dt =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int64_t cost = 0;
    uint64_t acc = 0;
    if (!rc) rc = qap_sa_result(h, nullptr, &cost, &acc);
    qap_sa_destroy(h);
    if (rc) return rc;
    if (c == 0) {
      cost0 = cost;
      acc0 = acc;
    } else if (cost != cost0 || acc != acc0) {
      return QAP_E_STATE;  // a knob changed the trajectory: never expected
    }
    if (dt < best_s) {
      best_s = dt;
      *best = cand[c];
    }
  }
  if (seconds) *seconds = best_s;
  return QAP_OK;
}

int32_t qap_sa_max_n_tier(int32_t tier) {
  if (max_n_tier1() == 0) return 0;
  switch (tier) {
    case 1: return max_n_tier1();
    case 2: return max_n_tier2();
    case 3: return max_n_tier3(false);
    case 4: return max_n_tier3(true);
    default: return 0;
  }
}

const char *qap_sa_strerror(int status) {
  switch (status) {
    case QAP_OK: return "ok";
    case QAP_E_INVAL: return "invalid argument";
    case QAP_E_RANGE: return "value out of range";
    case QAP_E_NOMEM: return "out of memory";
    case QAP_E_CUDA: return g_errbuf[0] ? g_errbuf : "CUDA error";
    case QAP_E_TIMEOUT: return "device wait timed out";
    case QAP_E_STATE: return "inconsistent device state";
    case QAP_E_UNSUPPORTED: return "problem size not supported";
    default: return "unknown status";
  }
}

}  // extern "C"

// ------------------------------------------------------------------------- //
// Batch of independent chains.
// ------------------------------------------------------------------------- //
struct qap_batch {
  int count = 0;
  std::vector<qap_sa *> h;
  std::vector<BatchChain> chains;
  cudaStream_t stream = nullptr, stream2 = nullptr;
  BatchChain *d_chains = nullptr;
  int *d_order = nullptr;    // tier-1 chains (one CTA each), then tier-2 chains
  int *d_counter = nullptr;  // [0]: next tier-1 chain, [1]: next tier-2 chain
  int n1 = 0, n2 = 0;        // chains per tier
  int smem = 0, smem2 = 0;
  int grid = 0, cluster2 = 0, grid2 = 0;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void free_batch(qap_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (qap_sa *h : b->h) free_handle(h);
  cudaFree(b->d_chains);
  cudaFree(b->d_order);
  cudaFree(b->d_counter);
  if (b->stream) cudaStreamDestroy(b->stream);
  if (b->stream2) cudaStreamDestroy(b->stream2);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  delete b;
}

}  // namespace

extern "C" {

int qap_batch_create(const qap_problem *probs, int32_t count, qap_batch **out) {
  if (!out) return QAP_E_INVAL;
  *out = nullptr;
  if (!probs || count < 1) return QAP_E_INVAL;
  qap_batch *b = new (std::nothrow) qap_batch();
  if (!b) return QAP_E_NOMEM;
  b->count = count;
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "cudaStreamCreate");
  }
  for (int i = 0; i < count; ++i) {
    const qap_problem &q = probs[i];
    qap_sa *h = nullptr;
    int rc = validate_args(q.A, q.B, q.N, q.p0, &q.sched, &h);
    if (!rc) rc = create_from_host(q.A, q.B, q.N, q.p0, &q.sched, q.seed, b->stream,
                                   false, &h);
    if (rc) {
      free_batch(b);
      return rc;
    }
    b->h.push_back(h);
    if (h->tier == 3) {  // a grid-wide chain cannot share a persistent launch
      free_batch(b);
      return QAP_E_UNSUPPORTED;
    }
    BatchChain bc{};
    bc.g = h->dev;
    bc.it_end = 0;
    bc.R = h->R;
    b->chains.push_back(bc);
    if (h->tier == 1) {
      ++b->n1;
      if (h->smem_bytes > b->smem) b->smem = h->smem_bytes;
    } else {
      ++b->n2;
      if (h->smem_bytes > b->smem2) b->smem2 = h->smem_bytes;
      if (h->cluster > b->cluster2) b->cluster2 = h->cluster;
    }
  }
  // work lists: tier-1 chains then tier-2 chains, each most work (N^2 I) first
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    if (b->h[x]->tier != b->h[y]->tier) return b->h[x]->tier < b->h[y]->tier;
    const double wx = (double)b->h[x]->N * b->h[x]->N * (double)b->h[x]->sched.I;
    const double wy = (double)b->h[y]->N * b->h[y]->N * (double)b->h[y]->sched.I;
    return wx > wy;
  });
  double work1 = 0, work2 = 0;
  for (qap_sa *h : b->h)
    (h->tier == 1 ? work1 : work2) += (double)h->N * h->N * (double)h->sched.I;
  int dev = 0, sms = 0;
  auto fail = [&](cudaError_t err, const char *what) {
    int rc = cuda_fail(err, what);
    free_batch(b);
    return rc;
  };
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return fail(e, "cudaDeviceGetAttribute");
  // SMs for the cluster branch in proportion to its share of the work.
  int sm2 = 0;
  if (b->n2) {
    const int C = b->cluster2;
    sm2 = (int)((double)sms * work2 / (work1 + work2));
    if (b->n1 == 0) sm2 = sms;
    sm2 = (sm2 / C) * C;
    if (sm2 < C) sm2 = C;
    if (sm2 > b->n2 * C) sm2 = b->n2 * C;
    if (b->n1 && sm2 > sms - 1) sm2 = ((sms - 1) / C) * C;
    b->grid2 = sm2;
  }
  b->grid = b->n1 < sms - sm2 ? b->n1 : sms - sm2;
  if (b->n1 && b->grid < 1) b->grid = 1;
  if ((e = cudaMalloc(&b->d_chains, sizeof(BatchChain) * count)) != cudaSuccess)
    return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&b->d_order, sizeof(int) * count)) != cudaSuccess)
    return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&b->d_counter, 2 * sizeof(int))) != cudaSuccess)
    return fail(e, "cudaMalloc");
  if ((e = cudaStreamCreateWithFlags(&b->stream2, cudaStreamNonBlocking)) != cudaSuccess)
    return fail(e, "cudaStreamCreate");
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess)
    return fail(e, "cudaEventCreate");
  if ((e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming)) != cudaSuccess)
    return fail(e, "cudaEventCreate");
  if ((e = cudaMemcpyAsync(b->d_order, order.data(), sizeof(int) * count,
                           cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
    return fail(e, "cudaMemcpyAsync");
  // The whole run is one graph: reset the work counters, then two persistent
  // launches side by side -- one CTA per chain for chains that fit one SM,
  // clusters for the others.
  if (!g_tmem_ok) {
    free_batch(b);
    return QAP_E_UNSUPPORTED;
  }
  if (b->n1) b->smem = tmem_smem(b->smem);
  if (b->n2) b->smem2 = tmem_smem(b->smem2);
  cudaGraph_t graph = nullptr;
  if ((e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return fail(e, "cudaStreamBeginCapture");
  cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(int), b->stream);
  if (b->n2) {
    cudaEventRecord(b->fork, b->stream);
    cudaStreamWaitEvent(b->stream2, b->fork, 0);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = b->cluster2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(b->grid2);
    cfg.blockDim = dim3(kT2Threads);
    cfg.dynamicSmemBytes = b->smem2;
    cfg.stream = b->stream2;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, sa_tier2_batch_kernel, (const BatchChain *)b->d_chains,
                       (const int *)(b->d_order + b->n1), b->n2, b->d_counter + 1);
    cudaEventRecord(b->join, b->stream2);
  }
  if (b->n1)
    sa_batch_kernel<<<b->grid, kBatchThreads, b->smem, b->stream>>>(
        b->d_chains, b->d_order, b->n1, b->d_counter);
  if (b->n2) cudaStreamWaitEvent(b->stream, b->join, 0);
  if ((e = cudaStreamEndCapture(b->stream, &graph)) != cudaSuccess)
    return fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(e, "cudaGraphInstantiate");
  if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
    return fail(e, "cudaStreamSynchronize");
  *out = b;
  return QAP_OK;
}

int qap_batch_run(qap_batch *b, const uint64_t *iters) {
  if (!b) return QAP_E_INVAL;
  for (int i = 0; i < b->count; ++i) {
    qap_sa *h = b->h[i];
    const uint64_t want = iters ? iters[i] : h->sched.I - h->it_host;
    if (want > h->sched.I - h->it_host) return QAP_E_RANGE;
  }
  for (int i = 0; i < b->count; ++i) {
    qap_sa *h = b->h[i];
    const uint64_t want = iters ? iters[i] : h->sched.I - h->it_host;
    b->chains[i].it_end = h->it_host + want;
  }
  CK(cudaMemcpyAsync(b->d_chains, b->chains.data(), sizeof(BatchChain) * b->count,
                     cudaMemcpyHostToDevice, b->stream));
  CK(cudaGraphLaunch(b->exec, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  std::vector<ChainStatus> st(b->count);
  for (int i = 0; i < b->count; ++i)
    CK(cudaMemcpyAsync(&st[i], b->h[i]->st, sizeof(ChainStatus),
                       cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  int rc = QAP_OK;
  for (int i = 0; i < b->count; ++i) {
    b->h[i]->it_host = b->chains[i].it_end;
    if (st[i].error || st[i].it != b->chains[i].it_end) rc = QAP_E_STATE;
  }
  return rc;
}

int qap_batch_result(qap_batch *b, int32_t i, int32_t *p_out, int64_t *cost,
                     uint64_t *accepts) {
  if (!b || i < 0 || i >= b->count) return QAP_E_INVAL;
  return qap_sa_result(b->h[i], p_out, cost, accepts);
}

int qap_batch_get_info(qap_batch *b, int32_t i, qap_sa_info *out) {
  if (!b || i < 0 || i >= b->count) return QAP_E_INVAL;
  return qap_sa_get_info(b->h[i], out);
}

void qap_batch_destroy(qap_batch *b) { free_batch(b); }

}  // extern "C"

// ------------------------------------------------------------------------- //
// Set-up without allocation.
//
// Some callers cannot call cudaMalloc: programs whose device memory is owned
// by another allocator (a framework's caching pool) or fixed by a budget, and
// loops that must not stall on the device-wide synchronisation cudaMalloc and
// cudaFree may imply.  qap_sa_setup_noalloc gives them step (a) of the method
// -- the packed Delta and the cost for a given permutation -- with every
// intermediate (int8 A and B', the Gram matrix, counters) in the file-scope
// array below, which every GPU that loads this library holds until exit.
// ------------------------------------------------------------------------- //
namespace {

constexpr int kNoAllocMaxN = QAP_NOALLOC_MAX_N;
constexpr size_t kNoAllocAlign = 256;
constexpr size_t na_round(size_t x) { return (x + kNoAllocAlign - 1) / kNoAllocAlign * kNoAllocAlign; }
// The row stride of the largest N: every N <= kNoAllocMaxN has a stride no
// larger than this (row_stride is monotone), so its rows fit the array.
constexpr size_t kNaRow = (size_t)row_stride(kNoAllocMaxN);
static_assert(row_stride(kNoAllocMaxN - 1) <= row_stride(kNoAllocMaxN) &&
                  row_stride(kNoAllocMaxN) >= kNoAllocMaxN,
              "row stride of the allocation-free set-up");
constexpr size_t kNaA = 0;
constexpr size_t kNaB = kNaA + na_round((size_t)kNoAllocMaxN * kNaRow);
constexpr size_t kNaG = kNaB + na_round((size_t)kNoAllocMaxN * kNaRow);
constexpr size_t kNaCount = kNaG + na_round(sizeof(int) * (size_t)kNoAllocMaxN * kNoAllocMaxN);
constexpr size_t kNaP = kNaCount + na_round(sizeof(int) * (size_t)kNoAllocMaxN);
constexpr size_t kNaD = kNaP + na_round(sizeof(int) * (size_t)kNoAllocMaxN);
constexpr size_t kNaOut = kNaD + na_round(sizeof(int) * (size_t)kNoAllocMaxN);
constexpr size_t kNoAllocBytes = kNaOut + na_round(sizeof(SetupOut));

}  // namespace

static __device__ __align__(256) unsigned char g_setup_scratch[kNoAllocBytes];

namespace {

std::mutex g_na_mutex;
void *g_na_ptr[64];  // device address of g_setup_scratch, per device

// The host-side name g_setup_scratch is only a stand-in for the device array;
// its device address is looked up once per device, with that device current.
int noalloc_scratch(unsigned char **out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return QAP_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void *ptr = nullptr;
    CK(cudaGetSymbolAddress(&ptr, g_setup_scratch));
    g_na_ptr[dev] = ptr;
  }
  *out = static_cast<unsigned char *>(g_na_ptr[dev]);
  return QAP_OK;
}

}  // namespace

extern "C" int qap_sa_setup_noalloc(const int32_t *A, const int32_t *B,
                                    int32_t N, const int32_t *p,
                                    int32_t *delta_out, int64_t *cost_out,
                                    void *cuda_stream) {
  if (!A || !B || !p || !delta_out || !cost_out || N < 2) return QAP_E_INVAL;
  if (N > kNoAllocMaxN) return QAP_E_RANGE;  // beyond the static array
  unsigned char *base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const int S = row_stride(N);
  if ((size_t)S > kNaRow) return QAP_E_RANGE;  // cannot happen for N <= kNoAllocMaxN
  int8_t *A8 = reinterpret_cast<int8_t *>(base + kNaA);
  int8_t *Bp8 = reinterpret_cast<int8_t *>(base + kNaB);
  int *G = reinterpret_cast<int *>(base + kNaG);
  int *count = reinterpret_cast<int *>(base + kNaCount);
  int *pp = reinterpret_cast<int *>(base + kNaP);
  int *d = reinterpret_cast<int *>(base + kNaD);
  SetupOut *so = reinterpret_cast<SetupOut *>(base + kNaOut);
  // The array keeps the previous call's contents: zero what the kernels
  // accumulate into or read as padding.
  CK(cudaMemsetAsync(A8, 0, (size_t)N * S, stream));
  CK(cudaMemsetAsync(Bp8, 0, (size_t)N * S, stream));
  CK(cudaMemsetAsync(count, 0, sizeof(int) * N, stream));
  CK(cudaMemsetAsync(so, 0, sizeof(SetupOut), stream));
  const long long NN = (long long)N * N;
  const int blocks = (int)((NN + 255) / 256);
  setup_pack_kernel<<<blocks, 256, 0, stream>>>(A, B, p, N, S, A8, count, so);
  setup_bprime_kernel<<<blocks, 256, 0, stream>>>(B, p, N, S, count, Bp8, pp, so);
  dim3 gg((N + 127) / 128, N);
  setup_gram_kernel<<<gg, 128, 0, stream>>>(A8, Bp8, N, S, G);
  setup_delta_kernel<<<gg, 128, 0, stream>>>(G, A8, Bp8, N, S, delta_out, d, so);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(cost_out, &so->cost0, sizeof(int64_t),
                     cudaMemcpyDeviceToDevice, stream));
  SetupOut so_h{};
  CK(cudaMemcpyAsync(&so_h, so, sizeof so_h, cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  if (so_h.flags & (kFlagAsym | kFlagDiag | kFlagPerm)) return QAP_E_INVAL;
  if (so_h.flags & (kFlagRangeA | kFlagRangeB)) return QAP_E_RANGE;
  return QAP_OK;
}

// ------------------------------------------------------------------------- //
// Hooks for the other translation units (qap_internal.h).
// ------------------------------------------------------------------------- //
cudaStream_t qapsa_handle_stream(qap_sa *h) { return h ? h->stream : nullptr; }

void qapsa_keep_delta_mode(qap_sa *h) {
  if (h && h->tier == 2) h->dev.hyb_lo = 0.0f;
}

int qapsa_sms_for(int N) { return N <= max_n_tier1() ? 1 : tier2_cluster(N); }

size_t qapsa_bytes_for(int N) {
  const size_t S = (size_t)row_stride(N), M = (size_t)N * (N - 1) / 2;
  const size_t state = 2 * (size_t)N * S + 4 * M + 8 * (size_t)N + 16384 + 4096;
  const size_t setup_peak = 3 * 4 * (size_t)N * N + 4 * (size_t)N;  // A, B, G staging
  return state + setup_peak;
}
