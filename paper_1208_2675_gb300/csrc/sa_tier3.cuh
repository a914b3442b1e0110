// sa_tier3.cuh -- tier 3 of the SA loop (Paul, arXiv:1208.2675, sections 2.2
// and 3): one chain on a persistent grid of one CTA per SM, Delta in global
// memory (L2-resident while it fits, HBM beyond), for the instances the
// on-chip tiers do not take: asymmetric A or B or nonzero diagonals (the
// general swap cost), entries beyond int8, random proposal order (section
// 2.1), and N beyond a cluster's on-chip memory.
//
// Where the data lives during a run:
//   Delta   M int32 in pair order (packed upper triangle) in global memory,
//           twice: every accepted swap reads one copy and writes the other,
//           so a CTA still scanning a window after a grid barrier never sees
//           cells another CTA has already moved on to the next swap (the
//           copies change roles at each barrier; at the end of a launch the
//           current copy goes back to the first one).  CTA g owns the pair
//           indices [g M / G, (g + 1) M / G) for the O(1) update;
//   A, A^T, B, B^T  static int32 rows of stride SA (a multiple of 4) in global
//           memory (A^T, B^T only for general instances), read with int4 loads
//           in the rows-r,s recompute and staged into shared memory by TMA bulk
//           copies (cp.async.bulk) for every accepted swap;
//   p, q = p^-1, the diagonals of A and B, the Gram diagonals d_R, d_C, and
//           the staged rows: shared memory of every CTA (each CTA keeps its own
//           copy and updates it identically).
//
// One window of proposals [it, it + wlen):
//   short windows  every CTA evaluates every proposal of the window (Delta
//                  cells read from L2) and finds the same first accepted one --
//                  no communication;
//   long windows   each CTA evaluates the proposals whose cell it owns and
//                  posts its first candidate with a global atomicMin; one grid
//                  barrier, then every CTA reads the minimum.
// An accepted swap (r, s): every CTA stages rows r,s of A (and A^T) and rows
// p(r), p(s) of B (and B^T) into shared memory with cp.async.bulk, forms the
// vectors of the update, updates its own cells in O(1) each
//   Delta_uv += (a_u - a_v)(b_v - b_u) + (c_u - c_v)(e_v - e_u),
//   a_k = A_rk - A_sk, b_k = B'_sk - B'_rk, c_k = A_kr - A_ks, e_k = B'_ks - B'_kr
// (B' before the swap; c = a, e = b for symmetric instances), and recomputes
// the cells (r, v), (s, v) of its share of v from Gram sums over streamed rows:
//   Delta_xy = R_xy + R_yx - R_xx - R_yy + C_xy + C_yx - C_xx - C_yy + corr,
//   R_xy = <A_x, B'_y>, C_xy = <A_.x, B'_.y>, corr from the entries at
//   (x,x), (x,y), (y,x), (y,y) (for symmetric instances 2 (R_xy + R_yx - d_x -
//   d_y) + 4 A_xy B'_xy); then one grid barrier.  The barrier is a monotonic
//   counter with release/acquire and a bounded wait: on expiry the kernel
//   records QAP timeout in the status word and returns.
#pragma once
#include <climits>

#include "sa_tier1.cuh"

namespace qapsa {

constexpr int kT3Threads = 512;
constexpr int kT3Warps = kT3Threads / 32;
constexpr int kT3Kmin = 32;
constexpr int kT3Kred = 1024;        // windows up to this length: every CTA scans it all
constexpr int kT3Kmax = 1 << 16;
constexpr long long kT3WaitCycles = 4000000000ll;  // ~2 s at 2 GHz
constexpr int kT3ErrTimeout = 2;

struct T3Dev {
  int N, M, SA;          // SA: row stride of the static matrices (int32, multiple of 4)
  int general;           // asymmetric / nonzero diagonals: the general forms
  int random_order;      // proposals drawn at random (section 2.1)
  int G;                 // CTAs of the grid
  const int *A, *AT, *B, *BT;  // N x SA each (AT == A and BT == B if !general)
  const int *Adiag, *Bdiag;    // N each
  int *delta;            // M, pair order: the state between launches
  int *delta2;           // M: the second copy, used during a launch
  int *p;                // N
  int *dR, *dC;          // N each: R_vv = <A_v, B'_v>, C_vv = <A_.v, B'_.v>
  ChainStatus *st;
  unsigned long long *bar;  // grid barrier counter (zeroed before each launch)
  unsigned *keys;           // 3 window keys of the long-window scan
  unsigned long long seed;
  unsigned stream;
  double T0;
  const double *P;
  float T0f, log2a_f, mrel;
  int cache_rows;        // this CTA's share of rows of A, B (A^T, B^T) kept in
                         // shared memory for the rows-r,s recompute
  int nvmax;             // rows in a share, at most
  unsigned bar_skew;     // arrivals the grid barrier expects beyond the CTAs'
                         // (0; 1 only to test the bounded wait's expiry)
};

// Shared memory: vectors of NP int32 each, then the control block.
__host__ __device__ inline int t3_np(int N) { return (N + 3) & ~3; }
enum : int {
  kV_p = 0, kV_q, kV_Ad, kV_Bd, kV_dR, kV_dC,
  kV_Ar, kV_As, kV_Acr, kV_Acs,       // rows r,s of A and of A^T (staged by TMA)
  kV_Br, kV_Bs, kV_BTr, kV_BTs,       // rows p(r), p(s) of B and of B^T (staged by TMA)
  kV_Btr, kV_Bts, kV_Bcr, kV_Bcs,     // B'_r., B'_s., B'_.r, B'_.s after the swap
  kV_Atr, kV_Ats, kV_Actr, kV_Acts,   // A_r., A_s., A_.r, A_.s in location order
  kV_a, kV_b, kV_c, kV_e,             // the vectors of the O(1) update
  kV_count
};
// Slot of vector k: symmetric instances use 15 of them (A^T = A, B^T = B, so
// the column vectors alias the row vectors and d_C = d_R).
__host__ __device__ inline int t3_slot(int k, bool gen) {
  if (gen) return k;
  switch (k) {
    case kV_p: return 0;    case kV_q: return 1;    case kV_Ad: return 2;   case kV_Bd: return 3;
    case kV_dR: case kV_dC: return 4;
    case kV_Ar: case kV_Acr: return 5;   case kV_As: case kV_Acs: return 6;
    case kV_Br: case kV_BTr: return 7;   case kV_Bs: case kV_BTs: return 8;
    case kV_Btr: case kV_Bcr: return 9;  case kV_Bts: case kV_Bcs: return 10;
    case kV_Atr: case kV_Actr: return 11; case kV_Ats: case kV_Acts: return 12;
    case kV_a: case kV_c: return 13;     default: return 14;  // kV_b, kV_e
  }
}
__host__ __device__ inline int t3_nvec(bool gen) { return gen ? (int)kV_count : 15; }
constexpr int kT3CtlBytes = 256;
__host__ __device__ inline int t3_smem_bytes(int N, bool gen) {
  return t3_nvec(gen) * 4 * t3_np(N) + kT3CtlBytes;
}
// The cached rows: A_v, B_p(v) (and A^T_v, B^T_p(v)) for the nvmax rows v of a share.
__host__ __device__ inline int t3_cache_bytes(int N, bool gen, int nvmax) {
  return (gen ? 4 : 2) * nvmax * 4 * t3_np(N);
}

// Pair number m of the random order at iteration it: (x M) >> 32, x word 0 of
// Philox4x32-10 at counter (it low, it high, stream, 1).
__device__ __forceinline__ int t3_random_pair(unsigned long long seed, unsigned stream,
                                              unsigned long long it, int M) {
  const uint4 x = philox4x32_10(make_uint4((unsigned)it, (unsigned)(it >> 32), stream, 1u),
                                make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  return (int)(((unsigned long long)x.x * (unsigned long long)(unsigned)M) >> 32);
}

__device__ __forceinline__ int t3_row_start(int N, int u) { return u * N - (u * (u + 1)) / 2; }

// Grid barrier: every CTA adds 1 (release) to a monotonic counter and waits
// (acquire) until it reaches target; the wait is bounded.  Returns false on
// expiry.  Called by every thread of every CTA.
__device__ __forceinline__ bool t3_grid_sync(unsigned long long *bar, unsigned long long &target,
                                             unsigned G, int *s_flag) {
  __syncthreads();
  target += G;
  if (threadIdx.x == 0) {
    __threadfence();
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(bar) : "memory");
    const long long t0 = clock64();
    int ok = 1;
    for (;;) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (clock64() - t0 > kT3WaitCycles) {
        ok = 0;
        break;
      }
    }
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// ---- TMA bulk copies of whole rows into shared memory ----
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Waits for the phase with the given parity; false after ~kT3WaitCycles.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  const long long t0 = clock64();
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kT3WaitCycles) return false;
  }
}
// One row of `bytes` (a multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void tma_row(void *dst, const void *src, unsigned bytes,
                                        unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One chain on the grid, from its state in global memory to iteration it_end.
template <bool GEN>
__device__ void t3_run_chain(const T3Dev &g, unsigned long long it_end, unsigned char *smem) {
  const int N = g.N, M = g.M, SA = g.SA, NP = t3_np(N);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned G = gridDim.x, gb = blockIdx.x;
  int *V = reinterpret_cast<int *>(smem);
  auto vec = [&](int k) { return V + t3_slot(k, GEN) * NP; };
  int *s_p = vec(kV_p), *s_q = vec(kV_q), *s_Ad = vec(kV_Ad), *s_Bd = vec(kV_Bd);
  int *s_dR = vec(kV_dR), *s_dC = GEN ? vec(kV_dC) : vec(kV_dR);
  int *s_Ar = vec(kV_Ar), *s_As = vec(kV_As);
  int *s_Acr = GEN ? vec(kV_Acr) : s_Ar, *s_Acs = GEN ? vec(kV_Acs) : s_As;
  int *s_Br = vec(kV_Br), *s_Bs = vec(kV_Bs), *s_BTr = vec(kV_BTr), *s_BTs = vec(kV_BTs);
  int *s_Btr = vec(kV_Btr), *s_Bts = vec(kV_Bts);
  int *s_Bcr = GEN ? vec(kV_Bcr) : s_Btr, *s_Bcs = GEN ? vec(kV_Bcs) : s_Bts;
  int *s_Atr = vec(kV_Atr), *s_Ats = vec(kV_Ats);
  int *s_Actr = GEN ? vec(kV_Actr) : s_Atr, *s_Acts = GEN ? vec(kV_Acts) : s_Ats;
  int *s_a = vec(kV_a), *s_b = vec(kV_b);
  int *s_c = GEN ? vec(kV_c) : s_a, *s_e = GEN ? vec(kV_e) : s_b;
  unsigned char *ctl = smem + t3_nvec(GEN) * 4 * NP;
  unsigned long long *s_mbar = reinterpret_cast<unsigned long long *>(ctl);       // 8 B
  unsigned *s_wkey = reinterpret_cast<unsigned *>(ctl + 8);                      // 32 warps
  int *s_flag = reinterpret_cast<int *>(ctl + 8 + 4 * 32);                       // barrier ok
  long long *s_sum = reinterpret_cast<long long *>(ctl + 8 + 4 * 48);           // 4 sums

  // ---- state into shared memory ----
  for (int i = tid; i < NP; i += kT3Threads) {
    const bool in = i < N;
    s_p[i] = in ? g.p[i] : 0;
    s_Ad[i] = in ? g.Adiag[i] : 0;
    s_Bd[i] = in ? g.Bdiag[i] : 0;
    s_dR[i] = in ? g.dR[i] : 0;
    if (GEN) s_dC[i] = in ? g.dC[i] : 0;
  }
  if (tid == 0) mbar_init(s_mbar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  for (int i = tid; i < N; i += kT3Threads) s_q[s_p[i]] = i;
  unsigned mbar_phase = 0;
  const bool cache = g.cache_rows != 0;
  int *s_RA = reinterpret_cast<int *>(ctl + kT3CtlBytes);  // [nvmax][NP] each
  int *s_RB = s_RA + g.nvmax * NP;
  int *s_RAT = GEN ? s_RB + g.nvmax * NP : s_RA;
  int *s_RBT = GEN ? s_RAT + g.nvmax * NP : s_RB;

  // this CTA's cells and share of rows
  const long long Mll = M;
  const int lo = (int)((Mll * gb) / G), hi = (int)((Mll * (gb + 1)) / G);
  const int v_lo = (int)(((long long)N * gb) / G), v_hi = (int)(((long long)N * (gb + 1)) / G);
  if (cache) {  // this CTA's share of rows, for the whole launch (B rows follow p)
    __syncthreads();
    for (int i = 0; i < v_hi - v_lo; ++i) {
      const int v = v_lo + i, pv = s_p[v];
      for (int k = tid; k < NP; k += kT3Threads) {
        s_RA[i * NP + k] = __ldg(g.A + (size_t)v * SA + k);
        s_RB[i * NP + k] = __ldg(g.B + (size_t)pv * SA + k);
        if (GEN) {
          s_RAT[i * NP + k] = __ldg(g.AT + (size_t)v * SA + k);
          s_RBT[i * NP + k] = __ldg(g.BT + (size_t)pv * SA + k);
        }
      }
    }
  }

  unsigned long long it = g.st->it;
  unsigned long long accepts = g.st->accepts;
  long long cost = g.st->cost;
  unsigned long long windows = 0, exact = 0, near = 0;
  unsigned long long bar_target = g.bar_skew;
  int err = 0;
  int mb = (int)(it % (unsigned long long)M);
  int K = min(kT3Kmin * 2, M);
  unsigned wi = 0;
  int *Dc = g.delta, *Dn = g.delta2;  // read / written by the current swap
  ChainStatus *nlog = (gb == 0 && tid == 0) ? g.st : nullptr;
  __syncthreads();

  while (it < it_end && !err) {
    // ================= one window =================
    // at most M proposals: a window never wraps onto its own first pair
    const int wlen = (int)min((unsigned long long)min(K, M), it_end - it);
    const bool partitioned = wlen > kT3Kred;
    // integer pre-filter: -ln u <= 22.9, so delta > 24.5 T rejects whatever u is
    const float Tw = g.T0f * exp2f(u64_to_f32(it) * g.log2a_f);
    const float Te = Tw * exp2f((float)wlen * g.log2a_f);
    const float tmax = fmaxf(Tw, Te) * 24.5f;
    const int thr = (tmax < 1.0e9f) ? (int)ceilf(tmax) + 1 : 0x7FFFFFFF;
    unsigned best = kNone;
    // proposals j in blocks of four aligned to Philox blocks: j = 4 t' - (it & 3) + w
    const int o = (int)(it & 3u);
    const int nblk = (wlen + o + 3) >> 2;
    for (int bq = tid; bq < nblk; bq += kT3Threads) {
      int dv[4];
      unsigned live = 0;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int j = 4 * bq + w - o;
        dv[w] = 0;
        if (j < 0 || j >= wlen) continue;
        int m;
        if (g.random_order) {
          m = t3_random_pair(g.seed, g.stream, it + (unsigned)j, M);
        } else {
          m = mb + j;
          if (m >= M) m -= M;
        }
        if (partitioned && (m < lo || m >= hi)) continue;
        dv[w] = __ldcg(Dc + m);
        live |= 1u << w;
      }
      if (!live) continue;
      unsigned acc = 0, unc = 0, need = 0;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        if (!((live >> w) & 1u)) continue;
        if (dv[w] <= 0) acc |= 1u << w;
        else if (dv[w] <= thr) need |= 1u << w;
      }
      if (need && !(acc & ((need & (0u - need)) - 1u))) {  // an earlier accept decides
        const unsigned long long q = ((it - (unsigned)o) >> 2) + (unsigned)bq;
        const uint4 x = rng_block(g.seed, g.stream, q);
        const float Tq = g.T0f * exp2f(u64_to_f32(q << 2) * g.log2a_f);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          if (!((need >> w) & 1u)) continue;
          const float2 b = accept_interval(g.mrel, Tq * exp2f((float)w * g.log2a_f),
                                           word_of(x, w));
          const float df = (float)dv[w];
          if (df < b.x) acc |= 1u << w;
          else if (!(df > b.y)) unc |= 1u << w;
        }
      }
      const unsigned any = acc | unc;
      if (any) {
        const int w = __ffs(any) - 1;
        const unsigned key = ((unsigned)(4 * bq + w - o) << 1) | ((unc >> w) & 1u);
        best = min(best, key);
      }
    }
    const unsigned wmin = __reduce_min_sync(0xFFFFFFFFu, best);
    if (lane == 0) s_wkey[warp] = wmin;
    __syncthreads();
    unsigned code = kNone;
#pragma unroll
    for (int w = 0; w < kT3Warps; ++w) code = min(code, s_wkey[w]);
    ++windows;
    if (partitioned) {
      unsigned *key = g.keys + (wi % 3u);
      if (tid == 0) {
        if (code != kNone) atomicMin(key, code);
        if (gb == 0) g.keys[(wi + 1u) % 3u] = kNone;  // two windows old: read by all
      }
      if (!t3_grid_sync(g.bar, bar_target, G, s_flag)) {
        err = kT3ErrTimeout;
        break;
      }
      code = __ldcg(key);
      ++wi;
    }
    __syncthreads();  // s_wkey is rewritten by the next window
    if (code == kNone) {
      it += (unsigned)wlen;
      mb = (int)(((long long)mb + wlen) % Mll);
      K = min(2 * K, min(M, g.random_order ? kT3Kred : kT3Kmax));
      continue;
    }
    const int j = (int)(code >> 1);
    int m;
    if (g.random_order) {
      m = t3_random_pair(g.seed, g.stream, it + (unsigned)j, M);
    } else {
      m = mb + j;
      if (m >= M) m -= M;
    }
    const int dlt = __ldcg(Dc + m);
    if (code & 1u) {  // undecided by the binary32 pre-test: binary64, the same everywhere
      unsigned long long nt = 0;
      const int dec = exact_accept(g.seed, g.stream, g.T0, g.P, dlt, it + (unsigned)j, &nt,
                                   nlog);
      ++exact;
      near += nt;
      if (!dec) {
        it += (unsigned)j + 1;
        mb = (int)(((long long)mb + j + 1) % Mll);
        continue;
      }
    }
    // ================= accept the swap (r, s) =================
    int r, s;
    decode_pair(N, m, r, s);
    if (r < 0 || r >= s || s >= N) {
      err = 1;
      break;
    }
    if (j < K / 8) K = max(min(kT3Kmin, M), K / 2);
    it += (unsigned)j + 1;
    mb = (int)(((long long)mb + j + 1) % Mll);
    ++accepts;
    cost += dlt;

    // ---- p, q after the swap; rows r,s of A, A^T and p(r), p(s) of B, B^T
    //      (both before and after: p'(r) = p(s), p'(s) = p(r)) by TMA ----
    const int pr = s_p[r], ps = s_p[s];  // before the swap
    __syncthreads();                     // every thread has read s_p[r], s_p[s]
    if (tid == 0) {
      s_p[r] = ps;
      s_p[s] = pr;
      s_q[ps] = r;
      s_q[pr] = s;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const unsigned rowb = 4u * (unsigned)SA;
      mbar_expect_tx(s_mbar, (GEN ? 8u : 4u) * rowb);
      tma_row(s_Ar, g.A + (size_t)r * SA, rowb, s_mbar);
      tma_row(s_As, g.A + (size_t)s * SA, rowb, s_mbar);
      tma_row(s_Br, g.B + (size_t)ps * SA, rowb, s_mbar);  // row p'(r) of B
      tma_row(s_Bs, g.B + (size_t)pr * SA, rowb, s_mbar);  // row p'(s) of B
      if (GEN) {
        tma_row(s_Acr, g.AT + (size_t)r * SA, rowb, s_mbar);
        tma_row(s_Acs, g.AT + (size_t)s * SA, rowb, s_mbar);
        tma_row(s_BTr, g.BT + (size_t)ps * SA, rowb, s_mbar);
        tma_row(s_BTs, g.BT + (size_t)pr * SA, rowb, s_mbar);
      }
    }
    const bool staged = mbar_wait(s_mbar, mbar_phase);
    mbar_phase ^= 1u;
    if (!staged) {
      err = kT3ErrTimeout;
      break;
    }
    __syncthreads();  // p', q' visible
    // B'_x. and B'_.x after the swap (facility order); A rows in location order;
    // the vectors of the O(1) update (k outside {r, s}: B' before the swap of
    // row r is B' after it of row s, and so on)
    for (int k = tid; k < NP; k += kT3Threads) {
      if (cache) {  // rows r and s of the share now hold rows p'(r), p'(s) of B
        if (r >= v_lo && r < v_hi) {
          s_RB[(r - v_lo) * NP + k] = s_Br[k];
          if (GEN) s_RBT[(r - v_lo) * NP + k] = s_BTr[k];
        }
        if (s >= v_lo && s < v_hi) {
          s_RB[(s - v_lo) * NP + k] = s_Bs[k];
          if (GEN) s_RBT[(s - v_lo) * NP + k] = s_BTs[k];
        }
      }
      if (k < N) {
        const int pk = s_p[k], qk = s_q[k];
        const int btr = s_Br[pk], bts = s_Bs[pk];
        s_Btr[k] = btr;
        s_Bts[k] = bts;
        s_Atr[k] = s_Ar[qk];
        s_Ats[k] = s_As[qk];
        s_a[k] = s_Ar[k] - s_As[k];
        s_b[k] = btr - bts;
        if (GEN) {
          const int bcr = s_BTr[pk], bcs = s_BTs[pk];
          s_Bcr[k] = bcr;
          s_Bcs[k] = bcs;
          s_Actr[k] = s_Acr[qk];
          s_Acts[k] = s_Acs[qk];
          s_c[k] = s_Acr[k] - s_Acs[k];
          s_e[k] = bcr - bcs;
        }
      } else {
        s_Btr[k] = s_Bts[k] = s_Atr[k] = s_Ats[k] = s_a[k] = s_b[k] = 0;
        if (GEN) s_Bcr[k] = s_Bcs[k] = s_Actr[k] = s_Acts[k] = s_c[k] = s_e[k] = 0;
      }
    }
    __syncthreads();
    // ---- Gram diagonals (O(1) off r,s; warps 0-3 take the four dot products
    //      of d_R(r), d_R(s), d_C(r), d_C(s)) and the O(1) update of this CTA's
    //      cells off rows and columns r,s, eight loads in flight per thread ----
    for (int k = tid; k < N; k += kT3Threads) {
      if (k != r && k != s) {
        s_dR[k] += s_c[k] * s_e[k];
        if (GEN) s_dC[k] += s_a[k] * s_b[k];
      }
    }
    if (warp < (GEN ? 4 : 2)) {
      const int *x = warp == 0 ? s_Ar : (warp == 1 ? s_As : (warp == 2 ? s_Acr : s_Acs));
      const int *y = warp == 0 ? s_Btr : (warp == 1 ? s_Bts : (warp == 2 ? s_Bcr : s_Bcs));
      long long acc = 0;
      for (int k = lane; k < N; k += 32) acc += (long long)x[k] * y[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
      if (lane == 0) s_sum[warp] = acc;
    }
    {
      int u = 0, vv = 0;
      if (lo + tid < hi) decode_pair(N, lo + tid, u, vv);
      for (int base = lo + tid; base < hi; base += 8 * kT3Threads) {
        int dl[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int mm = base + i * kT3Threads;
          dl[i] = mm < hi ? __ldcg(Dc + mm) : 0;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int mm = base + i * kT3Threads;
          if (mm >= hi) break;
          while (mm >= t3_row_start(N, u + 1)) ++u;  // rows of this thread's cells ascend
          const int v = mm - t3_row_start(N, u) + u + 1;
          if (u == r || u == s || v == r || v == s) {
            if (u == r && v == s) __stcg(Dn + mm, -dlt);  // the rest: rows r,s below
            continue;
          }
          int d = dl[i];
          d += (s_a[u] - s_a[v]) * (s_b[v] - s_b[u]);
          d += (s_c[u] - s_c[v]) * (s_e[v] - s_e[u]);  // symmetric: c = a, e = b
          __stcg(Dn + mm, d);
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      s_dR[r] = (int)s_sum[0];
      s_dR[s] = (int)s_sum[1];
      if (GEN) {
        s_dC[r] = (int)s_sum[2];
        s_dC[s] = (int)s_sum[3];
      }
    }
    __syncthreads();
    // ---- cells (r, v) and (s, v) of this CTA's share of v: one warp a row ----
    for (int v = v_lo + warp; v < v_hi; v += kT3Warps) {
      if (v == r || v == s) continue;
      const int pv = s_p[v];
      const int iv = v - v_lo;
      const int4 *Av = reinterpret_cast<const int4 *>(cache ? s_RA + iv * NP : g.A + (size_t)v * SA);
      const int4 *Bv = reinterpret_cast<const int4 *>(cache ? s_RB + iv * NP : g.B + (size_t)pv * SA);
      const int4 *ATv =
          reinterpret_cast<const int4 *>(cache ? s_RAT + iv * NP : g.AT + (size_t)v * SA);
      const int4 *BTv =
          reinterpret_cast<const int4 *>(cache ? s_RBT + iv * NP : g.BT + (size_t)pv * SA);
      const int4 *atr = reinterpret_cast<const int4 *>(s_Atr);
      const int4 *ats = reinterpret_cast<const int4 *>(s_Ats);
      const int4 *btr = reinterpret_cast<const int4 *>(s_Btr);
      const int4 *bts = reinterpret_cast<const int4 *>(s_Bts);
      const int4 *actr = reinterpret_cast<const int4 *>(s_Actr);
      const int4 *acts = reinterpret_cast<const int4 *>(s_Acts);
      const int4 *bcr = reinterpret_cast<const int4 *>(s_Bcr);
      const int4 *bcs = reinterpret_cast<const int4 *>(s_Bcs);
      int Rrv = 0, Rsv = 0, Rvr = 0, Rvs = 0, Crv = 0, Csv = 0, Cvr = 0, Cvs = 0;
      for (int c = lane; c < (NP >> 2); c += 32) {
        const int4 bv = cache ? Bv[c] : __ldg(Bv + c), av = cache ? Av[c] : __ldg(Av + c);
        int4 x = atr[c];
        Rrv += x.x * bv.x + x.y * bv.y + x.z * bv.z + x.w * bv.w;
        x = ats[c];
        Rsv += x.x * bv.x + x.y * bv.y + x.z * bv.z + x.w * bv.w;
        x = btr[c];
        Rvr += av.x * x.x + av.y * x.y + av.z * x.z + av.w * x.w;
        x = bts[c];
        Rvs += av.x * x.x + av.y * x.y + av.z * x.z + av.w * x.w;
        if (GEN) {
          const int4 btv = cache ? BTv[c] : __ldg(BTv + c);
          const int4 atv = cache ? ATv[c] : __ldg(ATv + c);
          x = actr[c];
          Crv += x.x * btv.x + x.y * btv.y + x.z * btv.z + x.w * btv.w;
          x = acts[c];
          Csv += x.x * btv.x + x.y * btv.y + x.z * btv.z + x.w * btv.w;
          x = bcr[c];
          Cvr += atv.x * x.x + atv.y * x.y + atv.z * x.z + atv.w * x.w;
          x = bcs[c];
          Cvs += atv.x * x.x + atv.y * x.y + atv.z * x.z + atv.w * x.w;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        Rrv += __shfl_xor_sync(0xFFFFFFFFu, Rrv, off);
        Rsv += __shfl_xor_sync(0xFFFFFFFFu, Rsv, off);
        Rvr += __shfl_xor_sync(0xFFFFFFFFu, Rvr, off);
        Rvs += __shfl_xor_sync(0xFFFFFFFFu, Rvs, off);
        if (GEN) {
          Crv += __shfl_xor_sync(0xFFFFFFFFu, Crv, off);
          Csv += __shfl_xor_sync(0xFFFFFFFFu, Csv, off);
          Cvr += __shfl_xor_sync(0xFFFFFFFFu, Cvr, off);
          Cvs += __shfl_xor_sync(0xFFFFFFFFu, Cvs, off);
        }
      }
      if (lane == 0) {
        const int Avv = s_Ad[v], Bvv = s_Bd[pv];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int x = t ? s : r;
          const int Rxy = t ? Rsv : Rrv, Ryx = t ? Rvs : Rvr;
          const int *Ax = t ? s_As : s_Ar;      // row x of A
          const int *Bx = t ? s_Bts : s_Btr;    // row x of B' (after the swap)
          int val;
          if (GEN) {
            const int Cxy = t ? Csv : Crv, Cyx = t ? Cvs : Cvr;
            const int *Acx = t ? s_Acs : s_Acr;  // column x of A
            const int *Bcx = t ? s_Bcs : s_Bcr;  // column x of B'
            const int Axx = s_Ad[x], Bxx = s_Bd[s_p[x]];
            const int Axy = Ax[v], Ayx = Acx[v], Bxy = Bx[v], Byx = Bcx[v];
            val = Rxy + Ryx - s_dR[x] - s_dR[v] + Cxy + Cyx - s_dC[x] - s_dC[v] -
                  (Axx - Ayx) * (Byx - Bxx) - (Axy - Avv) * (Bvv - Bxy) -
                  (Axx - Axy) * (Bxy - Bxx) - (Ayx - Avv) * (Bvv - Byx) +
                  (Axx - Avv) * (Bvv - Bxx) + (Axy - Ayx) * (Byx - Bxy);
          } else {
            val = 2 * (Rxy + Ryx - s_dR[x] - s_dR[v]) + 4 * Ax[v] * Bx[v];
          }
          const int uu = min(x, v), ww = max(x, v);
          __stcg(Dn + t3_row_start(N, uu) + (ww - uu - 1), val);
        }
      }
    }
    if (!t3_grid_sync(g.bar, bar_target, G, s_flag)) {
      err = kT3ErrTimeout;
      break;
    }
    int *const t = Dc;  // every cell of Dn has been written: it becomes current
    Dc = Dn;
    Dn = t;
  }

  // ---- the current copy of this CTA's cells back into g.delta (no CTA reads
  //      g.delta while it is the other copy; all CTAs swapped equally often) ----
  if (Dc != g.delta && !err)
    for (int mm = lo + tid; mm < hi; mm += kT3Threads) __stcg(g.delta + mm, __ldcg(Dc + mm));

  // ---- state back to global memory (every CTA holds the same copy) ----
  if (gb == 0) {
    for (int i = tid; i < N; i += kT3Threads) {
      g.p[i] = s_p[i];
      g.dR[i] = s_dR[i];
      if (GEN) g.dC[i] = s_dC[i];
    }
    if (tid == 0) {
      g.st->it = it;
      g.st->accepts = accepts;
      g.st->cost = cost;
      g.st->windows += windows;
      g.st->exact_evals += exact;
      g.st->near_ties += near;
      if (err) g.st->error = err;
    }
  } else if (err && tid == 0) {
    g.st->error = err;
  }
}

template <bool GEN>
__global__ void __launch_bounds__(kT3Threads, 1) sa_tier3_kernel(T3Dev g, unsigned long long it_end) {
  extern __shared__ __align__(16) unsigned char smem[];
  t3_run_chain<GEN>(g, it_end, smem);
}

// ------------------------------------------------------------------------- //
// Set-up of tier 3 (step (a) of section 2.2 for general instances)
// ------------------------------------------------------------------------- //
// Static rows: A, A^T, B, B^T padded to stride SA; diagonals; validation.
__global__ void t3_pack_kernel(const int *A32, const int *B32, const int *p0, int N, int SA,
                               int *A, int *AT, int *B, int *BT, int *Ad, int *Bd, int *count,
                               int general, SetupOut *out) {
  int ma = 0, mb = 0, flags = 0;
  const long long NN = (long long)N * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < NN;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx - (long long)i * N);
    const int a = A32[idx], b = B32[idx];
    A[(long long)i * SA + j] = a;
    B[(long long)i * SA + j] = b;
    if (general) {
      AT[(long long)j * SA + i] = a;
      BT[(long long)j * SA + i] = b;
    }
    if (i == j) {
      Ad[i] = a;
      Bd[i] = b;
    }
    const int aa = a < 0 ? (a == INT_MIN ? INT_MAX : -a) : a;
    const int ab = b < 0 ? (b == INT_MIN ? INT_MAX : -b) : b;
    ma = max(ma, aa);
    mb = max(mb, ab);
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

__global__ void t3_perm_kernel(const int *p0, int N, const int *count, int *p, SetupOut *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    p[i] = p0[i];
    if (count[i] != 1) atomicOr(&out->flags, kFlagPerm);
  }
}

// R[x][y] = <A_x, B'_y> and C[x][y] = <A_.x, B'_.y> (B' = B[p][p]), 64-bit
// products summed in int64 (the host has checked the int32 bound of the sums).
// One thread per (x, y); A^T rows are A's columns.
__global__ void t3_gram_kernel(const int *A, const int *AT, const int *B, const int *p, int N,
                               int SA, int general, long long *R, long long *C) {
  const int x = blockIdx.y;
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= N) return;
  const int py = p[y];
  long long r = 0, c = 0;
  for (int k = 0; k < N; ++k) {
    const int pk = __ldg(p + k);
    r += (long long)__ldg(A + (size_t)x * SA + k) * __ldg(B + (size_t)py * SA + pk);
    if (general)
      c += (long long)__ldg(AT + (size_t)x * SA + k) * __ldg(B + (size_t)pk * SA + py);
  }
  R[(size_t)x * N + y] = r;
  C[(size_t)x * N + y] = general ? c : r;
}

// Delta_xy for x < y from the Gram sums (the general form; the symmetric form
// for symmetric instances), the diagonals d_R, d_C, the cost C0 = trace(R)
// (Eq. 1) and sum |Delta_0|.
__global__ void t3_delta_kernel(const long long *R, const long long *C, const int *A, const int *B,
                                const int *p, int N, int SA, int general, int *delta, int *dR,
                                int *dC, SetupOut *out) {
  const int x = blockIdx.y;
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long sabs = 0;
  long long c0 = 0;
  if (y < N) {
    if (y == x) {
      dR[x] = (int)R[(size_t)x * N + x];
      dC[x] = (int)C[(size_t)x * N + x];
      c0 = R[(size_t)x * N + x];
    } else if (y > x) {
      auto Rv = [&](int a, int b) { return R[(size_t)a * N + b]; };
      auto Cv = [&](int a, int b) { return C[(size_t)a * N + b]; };
      auto Av = [&](int a, int b) { return (long long)A[(size_t)a * SA + b]; };
      auto Bp = [&](int a, int b) { return (long long)B[(size_t)p[a] * SA + p[b]]; };
      long long d;
      if (general) {
        d = Rv(x, y) + Rv(y, x) - Rv(x, x) - Rv(y, y) + Cv(x, y) + Cv(y, x) - Cv(x, x) -
            Cv(y, y) - (Av(x, x) - Av(y, x)) * (Bp(y, x) - Bp(x, x)) -
            (Av(x, y) - Av(y, y)) * (Bp(y, y) - Bp(x, y)) -
            (Av(x, x) - Av(x, y)) * (Bp(x, y) - Bp(x, x)) -
            (Av(y, x) - Av(y, y)) * (Bp(y, y) - Bp(y, x)) +
            (Av(x, x) - Av(y, y)) * (Bp(y, y) - Bp(x, x)) +
            (Av(x, y) - Av(y, x)) * (Bp(y, x) - Bp(x, y));
      } else {
        d = 2 * (Rv(x, y) + Rv(y, x) - Rv(x, x) - Rv(y, y)) + 4 * Av(x, y) * Bp(x, y);
      }
      delta[t3_row_start(N, x) + (y - x - 1)] = (int)d;
      sabs = (unsigned long long)(d < 0 ? -d : d);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sabs += __shfl_xor_sync(0xFFFFFFFFu, sabs, o);
    c0 += __shfl_xor_sync(0xFFFFFFFFu, c0, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (sabs) atomicAdd(&out->sum_abs_delta, sabs);
    if (c0) atomicAdd(reinterpret_cast<unsigned long long *>(&out->cost0), (unsigned long long)c0);
  }
}

}  // namespace qapsa
