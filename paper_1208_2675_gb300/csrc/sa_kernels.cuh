// sa_kernels.cuh -- device code of libqapsa (sm_103a).
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
// Tier 1 (this file): one CTA of 1024 threads holds Delta (packed upper
// triangle, int32), A and B' (int8, padded rows) in shared memory for the whole
// run; only __syncthreads separates the steps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qapsa {

constexpr int kThreads = 1024;
constexpr unsigned kNone = 0xFFFFFFFFu;

// Per-chain counters kept in global memory between launches.
struct ChainStatus {
  long long cost;                 // Eq. (1) of the current p
  unsigned long long it;          // iterations done
  unsigned long long accepts;     // accepted swaps
  unsigned long long near_ties;   // |delta + T ln u| < 1e-9 T among binary64 tests
  unsigned long long exact_evals; // acceptance tests decided in binary64
  unsigned long long windows;     // windows scanned
  int error;                      // nonzero: device-detected inconsistency
  int pad;
};

// Everything one chain's kernels need (passed by value).
struct ChainDev {
  int N;        // problem size
  int S;        // row stride of A and B' in bytes (multiple of 4, zero padded)
  int M;        // N(N-1)/2 pairs
  int tpv;      // threads per row in the rows-r,s recompute (power of two)
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
__device__ __forceinline__ double temperature(const ChainDev &g,
                                              unsigned long long it) {
  double T = g.T0;
#pragma unroll
  for (int b = 7; b >= 0; --b)
    T = __dmul_rn(T, __ldg(g.P + b * 256 + (int)((it >> (8 * b)) & 255u)));
  return T;
}

// Eq. (2) decided in binary64 for a proposal with delta > 0.
__device__ __noinline__ int exact_accept(const ChainDev &g, int delta,
                                         unsigned long long it,
                                         unsigned long long *near_ties) {
  const uint4 x = rng_block(g.seed, g.stream, it >> 2);
  const unsigned xi = word_of(x, (int)(it & 3u));
  const double u = __dmul_rn(__dadd_rn((double)xi, 0.5), 0x1p-32);
  const double T = temperature(g, it);
  const double prod = __dmul_rn(T, log(u));
  if (fabs(__dadd_rn((double)delta, prod)) < __dmul_rn(1e-9, T)) ++*near_ties;
  return (double)delta < -prod;
}

// Approximate acceptance temperature in binary32 (only for pre-tests whose
// margins cover its error).
__device__ __forceinline__ float temp_f32(const ChainDev &g,
                                          unsigned long long it) {
  return g.T0f * exp2f((float)it * g.log2a_f);
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

// ------------------------------------------------------------------------- //
// Tier-1 SA kernel: one CTA, everything in shared memory.
// ------------------------------------------------------------------------- //
struct SmemLayout {
  int off_delta, off_A, off_B, off_a, off_b, off_d, off_p, off_rs, off_ctl;
  int bytes;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SmemLayout smem_layout(int N, int S, int M) {
  SmemLayout L;
  int o = 0;
  L.off_delta = o; o += align16(4 * M);
  L.off_A = o;     o += align16(N * S);
  L.off_B = o;     o += align16(N * S);
  L.off_a = o;     o += align16(4 * N);
  L.off_b = o;     o += align16(4 * N);
  L.off_d = o;     o += align16(4 * N);
  L.off_p = o;     o += align16(4 * N);
  L.off_rs = o;    o += align16(4 * (N + 1));
  L.off_ctl = o;   o += 64;
  L.bytes = o;
  return L;
}

enum : int { kCtlKey0 = 0, kCtlDr = 3, kCtlDs = 4, kCtlDec = 5 };

__global__ void __launch_bounds__(kThreads, 1)
    sa_cta_kernel(ChainDev g, unsigned long long it_end) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = g.N, S = g.S, M = g.M, NW = g.S >> 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const SmemLayout L = smem_layout(N, S, M);
  int *s_delta = reinterpret_cast<int *>(smem + L.off_delta);
  int8_t *s_A = reinterpret_cast<int8_t *>(smem + L.off_A);
  int8_t *s_B = reinterpret_cast<int8_t *>(smem + L.off_B);
  int *s_a = reinterpret_cast<int *>(smem + L.off_a);
  int *s_b = reinterpret_cast<int *>(smem + L.off_b);
  int *s_d = reinterpret_cast<int *>(smem + L.off_d);
  int *s_p = reinterpret_cast<int *>(smem + L.off_p);
  int *s_rs = reinterpret_cast<int *>(smem + L.off_rs);
  unsigned *s_ctl = reinterpret_cast<unsigned *>(smem + L.off_ctl);

  // ---- load the chain state ----
  for (int i = tid; i < M; i += kThreads) s_delta[i] = g.delta[i];
  {
    const int *gA = reinterpret_cast<const int *>(g.A);
    const int *gB = reinterpret_cast<const int *>(g.Bp);
    int *sA = reinterpret_cast<int *>(s_A);
    int *sB = reinterpret_cast<int *>(s_B);
    for (int i = tid; i < N * NW; i += kThreads) {
      sA[i] = gA[i];
      sB[i] = gB[i];
    }
  }
  for (int i = tid; i < N; i += kThreads) {
    s_p[i] = g.p[i];
    s_d[i] = g.d[i];
  }
  for (int i = tid; i <= N; i += kThreads) s_rs[i] = i * N - i * (i + 1) / 2;
  if (tid < 16) s_ctl[tid] = (tid < 3) ? kNone : 0u;

  unsigned long long it = g.st->it;
  unsigned long long accepts = g.st->accepts;
  long long cost = g.st->cost;
  unsigned long long near_ties = 0, exact_evals = 0, windows = 0;
  int err = 0;
  int mb = (int)(it % (unsigned long long)M);  // it mod M
  int wa = 32;                                 // active warps in the scan
  unsigned wi = 0;                             // window number (key buffer)
  const int tpv = g.tpv;
  const int nvpass = kThreads / tpv;
  const int nv_round = ((N + nvpass - 1) / nvpass) * nvpass;
  __syncthreads();

  while (it < it_end) {
    // ================= scan: one window =================
    const unsigned long long wbase = it & ~3ull;
    int mbw = mb - (int)(it & 3u);
    while (mbw < 0) mbw += M;
    const int TA = wa * 32;
    unsigned long long wend = wbase + 4ull * (unsigned)TA;
    if (wend > it_end) wend = it_end;
    const float Tw = temp_f32(g, wbase), Te = temp_f32(g, wend);
    const float tmax = fmaxf(Tw, Te) * 24.5f;
    const int thr = (tmax < 1.0e9f) ? (int)ceilf(tmax) + 1 : 0x7FFFFFFF;
    unsigned code = kNone;
    if (tid < TA) {
      const unsigned long long ib = wbase + 4ull * (unsigned)tid;
      int m = mbw + 4 * tid;
      if (m >= M) m %= M;
      int dl[4];
      unsigned acc = 0, surv = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int mi = m + i;
        if (mi >= M) mi -= M;
        if (mi >= M) mi %= M;
        const int dv = s_delta[mi];
        dl[i] = dv;
        const unsigned long long itc = ib + i;
        if (itc >= it && itc < wend) {
          if (dv <= 0) acc |= 1u << i;
          else if (dv <= thr) surv |= 1u << i;
        }
      }
      unsigned unc = 0;
      if (surv) {
        const uint4 x = rng_block(g.seed, g.stream, ib >> 2);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (!((surv >> i) & 1u)) continue;
          const float uf = fmaf(__uint2float_rn(word_of(x, i)), 0x1p-32f, 0x1p-33f);
          const float Lf = -logf(uf);
          const float Tf = temp_f32(g, ib + i);
          const float t = Tf * Lf;
          const float mg = g.mrel * t + 1e-6f * Tf;
          const float df = (float)dl[i];
          if (df < t - mg) acc |= 1u << i;
          else if (!(df > t + mg)) unc |= 1u << i;
        }
      }
      const unsigned any = acc | unc;
      if (any) {
        const int f = __ffs(any) - 1;
        code = ((unsigned)(4 * tid + f) << 1) | ((unc >> f) & 1u);
      }
    }
    code = __reduce_min_sync(0xFFFFFFFFu, code);
    if (lane == 0 && code != kNone) atomicMin(s_ctl + kCtlKey0 + (wi % 3u), code);
    __syncthreads();
    code = s_ctl[kCtlKey0 + (wi % 3u)];
    if (tid == 0) s_ctl[kCtlKey0 + ((wi + 2u) % 3u)] = kNone;
    ++wi;
    ++windows;

    if (code == kNone) {  // nothing accepted in [it, wend)
      const int adv = (int)(wend - it);
      mb += adv;
      if (mb >= M) { mb -= M; if (mb >= M) mb %= M; }
      it = wend;
      wa = min(32, wa * 2);
      continue;
    }
    const int j = (int)(code >> 1);
    const unsigned long long itc = wbase + (unsigned)j;
    int mj = mbw + j;
    if (mj >= M) mj %= M;
    const int dlt = s_delta[mj];
    if (code & 1u) {  // undecided by the pre-test: binary64, one thread
      if (tid == 0) {
        ++exact_evals;
        s_ctl[kCtlDec] = (unsigned)exact_accept(g, dlt, itc, &near_ties);
      }
      __syncthreads();
      if (!s_ctl[kCtlDec]) {
        it = itc + 1;
        mb = mj + 1;
        if (mb >= M) mb -= M;
        continue;
      }
    }

    // ================= accept (r, s) =================
    int r;
    {
      const float f2n = (float)(2 * N - 1);
      const float disc = fmaxf(f2n * f2n - 8.0f * (float)mj, 0.0f);
      r = (int)((f2n - sqrtf(disc)) * 0.5f);
      r = max(0, min(r, N - 2));
      while (r > 0 && s_rs[r] > mj) --r;
      while (r < N - 2 && s_rs[r + 1] <= mj) ++r;
    }
    const int s = mj - s_rs[r] + r + 1;
    if (s <= r || s >= N) { err = 1; break; }
    if (j - (int)(it - wbase) < 4 * TA / 8) wa = max(1, wa >> 1);
    it = itc + 1;
    mb = mj + 1;
    if (mb >= M) mb -= M;
    ++accepts;
    if (tid == 0) cost += dlt;

    // ---- staging: a_k = A_rk - A_sk, b_k = B'_sk - B'_rk (B' before the
    // swap), diagonal d_k, swap of B' rows and columns r,s (Eq. 3), p ----
    int dr_part = 0, ds_part = 0;
    if (tid < N) {
      const int k = tid;
      const int Ark = s_A[r * S + k], Ask = s_A[s * S + k];
      const int Brk = s_B[r * S + k], Bsk = s_B[s * S + k];
      const int ak = Ark - Ask, bk = Bsk - Brk;
      s_a[k] = 2 * ak;
      s_b[k] = bk;
      if (k != r && k != s) {
        s_d[k] += ak * bk;
        s_B[r * S + k] = (int8_t)Bsk;
        s_B[s * S + k] = (int8_t)Brk;
        s_B[k * S + r] = (int8_t)Bsk;
        s_B[k * S + s] = (int8_t)Brk;
        dr_part = Ark * Bsk;
        ds_part = Ask * Brk;
      } else if (k == s) {
        dr_part = Ark * Brk;  // A_rs B'_rs
      } else {
        ds_part = Ask * Bsk;  // A_sr B'_sr
      }
      if (k == 0) {
        const int t = s_p[r];
        s_p[r] = s_p[s];
        s_p[s] = t;
      }
    }
    if (warp * 32 < N) {  // warp-uniform: whole warps reduce
      dr_part = __reduce_add_sync(0xFFFFFFFFu, dr_part);
      ds_part = __reduce_add_sync(0xFFFFFFFFu, ds_part);
      if (lane == 0) {
        atomicAdd(reinterpret_cast<int *>(s_ctl + kCtlDr), dr_part);
        atomicAdd(reinterpret_cast<int *>(s_ctl + kCtlDs), ds_part);
      }
    }
    __syncthreads();
    const int dr = (int)s_ctl[kCtlDr], ds = (int)s_ctl[kCtlDs];

    // ---- O(1) update of the cells off rows and columns r,s:
    // Delta_uv += 2 (a_u - a_v)(b_v - b_u).  Rows folded in pairs
    // (R, N-2-R) so that every warp walks N cells. ----
    for (int R = warp; R < (N >> 1); R += kThreads / 32) {
      const int u1 = R, u2 = N - 2 - R, L1 = N - 1 - R;
      const bool two = u2 > R;
      const bool skip1 = (u1 == r) || (u1 == s);
      const bool skip2 = !two || (u2 == r) || (u2 == s);
      if (skip1 && skip2) continue;
      const int a1 = s_a[u1], b1 = s_b[u1];
      const int a2 = two ? s_a[u2] : 0, b2 = two ? s_b[u2] : 0;
      const int base1 = s_rs[u1] - (u1 + 1);
      const int base2 = two ? s_rs[u2] - (u2 + 1) : 0;
      for (int c = lane; c < N; c += 32) {
        const bool p1 = c < L1;
        if (p1 ? skip1 : skip2) continue;
        const int v = p1 ? (R + 1 + c) : c;
        if (v == r || v == s) continue;
        const int au = p1 ? a1 : a2, bu = p1 ? b1 : b2;
        const int addr = (p1 ? base1 : base2) + v;
        s_delta[addr] += (au - s_a[v]) * (s_b[v] - bu);
      }
    }

    // ---- rows r,s from their definition under the new p, through
    // G_xy = <A_x, B'_y>:  Delta_rv = 2 (G_rv + G_vr - d_r - d_v + 2 A_rv B'_rv)
    {
      const int t = tid & (tpv - 1);
      const int *Ar = reinterpret_cast<const int *>(s_A + r * S);
      const int *As = reinterpret_cast<const int *>(s_A + s * S);
      const int *Br = reinterpret_cast<const int *>(s_B + r * S);
      const int *Bs = reinterpret_cast<const int *>(s_B + s * S);
      for (int v = tid / tpv; v < nv_round; v += nvpass) {
        int g1 = 0, g2 = 0, g3 = 0, g4 = 0;
        if (v < N) {
          const int *Av = reinterpret_cast<const int *>(s_A + v * S);
          const int *Bv = reinterpret_cast<const int *>(s_B + v * S);
          for (int w = t; w < NW; w += tpv) {
            const int bv = Bv[w], av = Av[w];
            g1 = __dp4a(Ar[w], bv, g1);
            g2 = __dp4a(As[w], bv, g2);
            g3 = __dp4a(av, Br[w], g3);
            g4 = __dp4a(av, Bs[w], g4);
          }
        }
        for (int o = tpv >> 1; o > 0; o >>= 1) {
          g1 += __shfl_xor_sync(0xFFFFFFFFu, g1, o);
          g2 += __shfl_xor_sync(0xFFFFFFFFu, g2, o);
          g3 += __shfl_xor_sync(0xFFFFFFFFu, g3, o);
          g4 += __shfl_xor_sync(0xFFFFFFFFu, g4, o);
        }
        if (t == 0 && v < N && v != r && v != s) {
          const int dv = s_d[v];
          const int Arv = s_A[r * S + v], Brv = s_B[r * S + v];
          const int Asv = s_A[s * S + v], Bsv = s_B[s * S + v];
          s_delta[pair_index(s_rs, r, v)] = 2 * (g1 + g3 - dr - dv + 2 * Arv * Brv);
          s_delta[pair_index(s_rs, s, v)] = 2 * (g2 + g4 - ds - dv + 2 * Asv * Bsv);
        }
      }
    }
    if (tid == 0) {
      s_delta[mj] = -dlt;
      s_d[r] = dr;
      s_d[s] = ds;
    }
    __syncthreads();
    if (tid == 0) {
      s_ctl[kCtlDr] = 0u;
      s_ctl[kCtlDs] = 0u;
    }
  }

  // ---- write the state back ----
  __syncthreads();
  for (int i = tid; i < M; i += kThreads) g.delta[i] = s_delta[i];
  {
    const int *sB = reinterpret_cast<const int *>(s_B);
    int *gB = reinterpret_cast<int *>(g.Bp);
    for (int i = tid; i < N * NW; i += kThreads) gB[i] = sB[i];
  }
  for (int i = tid; i < N; i += kThreads) {
    g.p[i] = s_p[i];
    g.d[i] = s_d[i];
  }
  if (tid == 0) {
    g.st->it = it;
    g.st->accepts = accepts;
    g.st->cost = cost;
    g.st->near_ties += near_ties;
    g.st->exact_evals += exact_evals;
    g.st->windows += windows;
    if (err) g.st->error = err;
  }
}

}  // namespace qapsa
