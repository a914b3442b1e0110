// sa_common.cuh -- device code shared by the SA kernels of libqapsa (sm_103a).
//
// Delta-matrix simulated annealing for the QAP (Paul, arXiv:1208.2675):
//   set-up      : B' (Eq. 3), Delta_0 and C0 (Eq. 1) -- step (a) of section 2.2
//   scan+select : a window of consecutive proposals tested against Eq. (2) in
//                 parallel, the first accepted one in sequential order wins
//                 (section 3 (ii)): warp redux.min + one shared-memory atomicMin
//   update      : p, B' rows/columns r,s (Eq. 3), O(1) update of every Delta
//                 cell off rows r,s, O(N) recompute of rows r,s (section 3 (i),
//                 (ii)); cost += Delta_rs                     -- step (d)
//
// This file: the chain state shared by host and device, Philox4x32-10, the
// binary64 schedule, and the set-up kernels.  The SA loop itself is in
// sa_tier1.cuh.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qapsa {

constexpr unsigned kNone = 0xFFFFFFFFu;
// Near-ties whose iteration index a chain keeps (the count is kept in full).
constexpr int kNearLog = 8;

// Per-chain counters kept in global memory between launches.
struct ChainStatus {
  long long cost;                 // Eq. (1) of the current p
  unsigned long long it;          // iterations done
  unsigned long long accepts;     // accepted swaps
  unsigned long long near_ties;   // |delta + T ln u| < 1e-9 T among binary64 tests
  unsigned long long exact_evals; // acceptance tests decided in binary64
  unsigned long long windows;     // windows scanned
  int error;                      // nonzero: device-detected inconsistency
  int mode;                       // 1: proposals evaluated directly, 0: from Delta
  unsigned long long direct_iters;    // iterations whose proposal was evaluated directly
  unsigned long long direct_accepts;  // accepted swaps among them
  unsigned long long warp_iters;      // direct iterations run by one warp alone
  int need_rebuild;                   // Delta in global memory is stale (cluster
                                      // tier after direct mode): rebuild it
  int hot_off;                        // the hot-phase kernel has handed the chain
                                      // over for good (acceptance fell below its rate)
  unsigned long long hot_iters;       // iterations run by the hot-phase kernel
  unsigned long long hot_accepts;     // accepted swaps among them
  int need_bprime;                    // B' in global memory is stale (after the
                                      // hot-phase kernel): B' = B[p][p] first
  int pad3_;
  unsigned long long near_log[kNearLog];  // iterations of the first near-ties
  unsigned near_log_n;                    // near-ties logged (may exceed kNearLog)
  unsigned pad2_;
};

// Everything one chain's kernels need (passed by value).
struct ChainDev {
  int N;        // problem size
  int S;        // row stride of A and B' in bytes (16 x odd, zero padded)
  int M;        // N(N-1)/2 pairs
  int tpv;      // the host's threads per row for the rows-r,s recompute; the
                // kernels derive their own (the field keeps the parameter
                // layout the kernels were tuned with)
  int ntiles;   // Delta tiles (one per thread of the SA kernel)
  const int *tiles;  // ntiles entries: first row << 16 | first column
  const int8_t *A;   // N*S, constant
  int8_t *Bp;        // N*S, B'[i][j] = B[p(i)][p(j)]
  int *delta;        // M, packed upper triangle in pair order
  int *p;            // N
  int *d;            // N, d_v = sum_k A[v][k] B'[v][k]
  ChainStatus *st;
  unsigned long long seed;
  unsigned stream;
  double T0;         // binary64 schedule
  const double *P;   // [8][256] per-byte factor tables
  float T0f;         // binary32 copies for the approximate pre-test
  float log2a_f;     // log2(alpha)
  float mrel;        // relative margin of the approximate pre-test
  float hyb_lo;      // acceptance rate below which Delta is maintained (0: always)
  float warp_lo;     // acceptance rate from which one warp runs direct mode alone
                     // (0: never)
};

// ------------------------------------------------------------------------- //
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products
// and xors with the key, the key advanced by the Weyl increments in between.
// ------------------------------------------------------------------------- //
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Block of four words covering iterations 4q .. 4q+3 of a chain's stream.
__device__ __forceinline__ uint4 rng_block(unsigned long long seed,
                                           unsigned stream,
                                           unsigned long long q) {
  return philox4x32_10(
      make_uint4((unsigned)q, (unsigned)(q >> 32), stream, 0u),
      make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

__device__ __forceinline__ unsigned word_of(uint4 x, int i) {
  return i == 0 ? x.x : (i == 1 ? x.y : (i == 2 ? x.z : x.w));
}

// T(it) in binary64: T0 times the per-byte factors, high byte first.
__device__ __forceinline__ double temperature(double T0, const double *P,
                                              unsigned long long it) {
  double T = T0;
#pragma unroll
  for (int b = 7; b >= 0; --b)
    T = __dmul_rn(T, __ldg(P + b * 256 + (int)((it >> (8 * b)) & 255u)));
  return T;
}

// Eq. (2) decided in binary64 for a proposal with delta > 0.  A near-tie
// (|delta + T ln u| < 1e-9 T, where CUDA's and another libm's log could decide
// differently) is counted in *near_ties and, if log is not NULL, its iteration
// is recorded in nlog->near_log (one thread per chain passes nlog).
__device__ __noinline__ int exact_accept(unsigned long long seed,
                                         unsigned stream, double T0,
                                         const double *P, int delta,
                                         unsigned long long it,
                                         unsigned long long *near_ties,
                                         ChainStatus *nlog) {
  const uint4 x = rng_block(seed, stream, it >> 2);
  const unsigned xi = word_of(x, (int)(it & 3u));
  const double u = __dmul_rn(__dadd_rn((double)xi, 0.5), 0x1p-32);
  const double T = temperature(T0, P, it);
  const double prod = __dmul_rn(T, log(u));
  if (fabs(__dadd_rn((double)delta, prod)) < __dmul_rn(1e-9, T)) {
    ++*near_ties;
    if (nlog) {
      const unsigned k = nlog->near_log_n++;
      if (k < (unsigned)kNearLog) nlog->near_log[k] = it;
    }
  }
  return (double)delta < -prod;
}


__device__ __forceinline__ int pair_index(const int *rs, int a, int b) {
  const int u = a < b ? a : b, v = a < b ? b : a;
  return rs[u] + (v - u - 1);
}

// ------------------------------------------------------------------------- //
// Set-up kernels (step (a) of section 2.2)
// ------------------------------------------------------------------------- //
enum : int {
  kFlagAsym = 1,
  kFlagDiag = 2,
  kFlagRangeA = 4,
  kFlagRangeB = 8,
  kFlagPerm = 16,
};

struct SetupOut {            // written by the set-up kernels, read by the host
  unsigned long long sum_abs_delta;
  long long cost0;
  int flags;
  int max_abs_a;
  int max_abs_b;
  int pad;
};

// Validates A, B, p0; packs A into int8 rows of stride S; counts p0 values.
__global__ void setup_pack_kernel(const int *A32, const int *B32,
                                  const int *p0, int N, int S, int8_t *A8,
                                  int *count, SetupOut *out) {
  int flags = 0, ma = 0, mb = 0;
  const long long NN = (long long)N * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       idx < NN; idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx - (long long)i * N);
    const int a = A32[idx], b = B32[idx];
    if (a != A32[(long long)j * N + i] || b != B32[(long long)j * N + i])
      flags |= kFlagAsym;
    if (i == j && (a != 0 || b != 0)) flags |= kFlagDiag;
    const int aa = a < 0 ? -a : a, ab = b < 0 ? -b : b;
    ma = max(ma, aa);
    mb = max(mb, ab);
    if (aa > 127) flags |= kFlagRangeA;
    if (ab > 127) flags |= kFlagRangeB;
    A8[(long long)i * S + j] = (int8_t)(aa > 127 ? 0 : a);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += gridDim.x * blockDim.x) {
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

// B'[i][j] = B[p0(i)][p0(j)] (Eq. 3 applied to the whole matrix), p = p0, and
// the permutation check (every location used exactly once).
__global__ void setup_bprime_kernel(const int *B32, const int *p0, int N,
                                    int S, const int *count, int8_t *Bp8,
                                    int *p, SetupOut *out) {
  const long long NN = (long long)N * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       idx < NN; idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx - (long long)i * N);
    int pi = p0[i], pj = p0[j];
    pi = pi < 0 ? 0 : (pi >= N ? N - 1 : pi);  // stay in bounds; rejected later
    pj = pj < 0 ? 0 : (pj >= N ? N - 1 : pj);
    const int b = B32[(long long)pi * N + pj];
    Bp8[(long long)i * S + j] = (int8_t)((b > 127 || b < -127) ? 0 : b);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += gridDim.x * blockDim.x) {
    p[i] = p0[i];
    if (count[i] != 1) atomicOr(&out->flags, kFlagPerm);
  }
}

// G[x][y] = sum_k A[x][k] B'[y][k] (= sum_k A[k][x] B'[k][y] by symmetry).
__global__ void setup_gram_kernel(const int8_t *A8, const int8_t *Bp8, int N,
                                  int S, int *G) {
  const int x = blockIdx.y;
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= N) return;
  const int *ar = reinterpret_cast<const int *>(A8 + (long long)x * S);
  const int *br = reinterpret_cast<const int *>(Bp8 + (long long)y * S);
  int acc = 0;
  for (int w = 0; w < (S >> 2); ++w) acc = __dp4a(__ldg(ar + w), __ldg(br + w), acc);
  G[(long long)x * N + y] = acc;
}

// Delta_uv = 2 (G_uv + G_vu - G_uu - G_vv + 2 A_uv B'_uv) for u < v, which is
// 2 sum_{k not in {u,v}} (A_ku - A_kv)(B'_kv - B'_ku) written through G; the
// diagonal d_v = G_vv; C0 = trace(G) = Eq. (1); and sum |Delta_0|.
__global__ void setup_delta_kernel(const int *G, const int8_t *A8,
                                   const int8_t *Bp8, int N, int S,
                                   int *delta, int *d, SetupOut *out) {
  const int u = blockIdx.y;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long sabs = 0;
  long long c0 = 0;
  if (v < N) {
    if (v == u) {
      const int g = G[(long long)u * N + u];
      d[u] = g;
      c0 = g;
    } else if (v > u) {
      const long long guv = G[(long long)u * N + v], gvu = G[(long long)v * N + u];
      const long long guu = G[(long long)u * N + u], gvv = G[(long long)v * N + v];
      const long long ab = (long long)A8[(long long)u * S + v] * Bp8[(long long)u * S + v];
      const long long dl = 2 * (guv + gvu - guu - gvv + 2 * ab);
      const int rsu = u * N - u * (u + 1) / 2;
      delta[rsu + (v - u - 1)] = (int)dl;
      sabs = (unsigned long long)(dl < 0 ? -dl : dl);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sabs += __shfl_xor_sync(0xFFFFFFFFu, sabs, o);
    c0 += __shfl_xor_sync(0xFFFFFFFFu, c0, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (sabs) atomicAdd(&out->sum_abs_delta, sabs);
    if (c0) atomicAdd(reinterpret_cast<unsigned long long *>(&out->cost0),
                      (unsigned long long)c0);
  }
}

}  // namespace qapsa
