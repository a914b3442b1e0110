// sa_tier1.cuh -- tier 1 of the SA loop (Paul, arXiv:1208.2675, sections 2.2
// and 3): one CTA runs the whole chain.
//
// Where the data lives during a run:
//   Delta  thread t owns an R x 4 tile of the upper triangle (rows
//          u0..u0+R-1, columns v0..v0+3), in its registers (256 threads, up
//          to 255 registers each) or, in the 640-thread kernels, in its own
//          Tensor Memory lane, moved to registers 4 rows at a time; the O(1)
//          update of a cell is three integer ops;
//   A, B'  shared memory, int8, rows of stride S = 16 x odd bytes (conflict-free
//          128-bit loads in the rows-r,s recompute);
//   a, b, d, p, the two recomputed rows, per-warp winner slots: shared memory.
//
// With Delta maintained (low acceptance) one accepted swap costs three block
// barriers:
//   scan    every thread tests its tile's cells that fall in the window
//           [it, it + K) of the cyclic proposal order against Eq. (2);
//           redux.min per warp, atomicMin across warps      -> barrier
//   stage   a_k = A_rk - A_sk, b_k = B'_sk - B'_rk (B' before the swap),
//           d_k, the row/column swap of B' (Eq. 3), p        -> barrier
//   update  O(1) update of every tile cell; rows r,s from their definition
//           through dp4a dot products into shared memory     -> barrier
// and the recomputed rows are copied into the owning tiles at the top of the
// next scan (each thread touches only its own tile there).  At higher
// acceptance the proposals are evaluated directly (t1_run_chain), by the whole
// CTA (two barriers per accepted swap) or, while many are accepted, by one
// warp alone (t1_warp_run, no block barrier).
#pragma once
#include "sa_common.cuh"
#include "sa_tmem.cuh"

namespace qapsa {

struct T1Layout {
  int off_A, off_B, off_a, off_b, off_d, off_p, off_nr, off_ns, off_slot, off_ctl;
  int off_tt;
  int bytes;
};

// Proposals of the next window whose Eq. (2) thresholds are prepared during
// the update phase of an accepted swap.
constexpr int kTabMax = 512;

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

// Vectors are padded so that tiles at the edge may read a few entries past N.
__host__ __device__ inline int t1_vec_len(int N) { return ((N + 15) & ~15) + 16; }

__host__ __device__ inline T1Layout t1_layout(int N, int S) {
  T1Layout L;
  const int NP = t1_vec_len(N);
  int o = 0;
  L.off_A = o;    o += align16(N * S);
  L.off_B = o;    o += align16(N * S);
  L.off_a = o;    o += 4 * NP;
  L.off_b = o;    o += 4 * NP;
  L.off_d = o;    o += 4 * NP;
  L.off_p = o;    o += 4 * NP;
  L.off_nr = o;   o += 4 * NP;
  L.off_ns = o;   o += 4 * NP;
  L.off_slot = o; o += 16 * 32;
  L.off_ctl = o;  o += 128;
  L.off_tt = o;   o += 8 * kTabMax;
  L.bytes = o;
  return L;
}

// Tile height of the register tiles of Delta, and the two thread counts the
// one-CTA kernel is compiled for: 256 (up to 255 registers per thread) for
// problems whose tiles fit, 640 (96 registers) above.
constexpr int kT1R = 16;
constexpr int kT1SmallThreads = 256;
constexpr int kT1LargeThreads = 640;

// s_ctl words: three window keys, the d_r / d_s sums of even accepts, the
// binary64 verdict, the d_r / d_s sums of odd accepts, then (from word 8,
// 8-byte aligned) thread 0's 64-bit counters.
enum : int { kT1Key0 = 0, kT1Dr = 3, kT1Ds = 4, kT1Dec = 5, kT1Dr1 = 6, kT1Ds1 = 7 };
enum : int { kC64Accepts = 0, kC64Cost = 1, kC64Near = 2, kC64Exact = 3, kC64Windows = 4,
              kC64DirIt = 5, kC64DirAcc = 6, kC64WarpIt = 7 };
// s_ctl words 24..31: the chain position handed between the CTA and the
// warp-only direct mode.
constexpr int kT1Pos = 24;
// Iterations per block of the mode decisions (Delta / direct / warp-only).
constexpr int kHybBlock = 16384;
// Longest window of the warp-only direct mode.
constexpr int kWarpMaxK = 128;

__device__ __forceinline__ float u64_to_f32(unsigned long long x) {
  return __uint2float_rn((unsigned)(x >> 32)) * 4294967296.0f +
         __uint2float_rn((unsigned)x);
}

// Pair index of (u, v), u < v, in the row-major enumeration of pairs r < s.
__device__ __forceinline__ int pidx(int N, int u, int v) {
  return u * N - (u * (u + 1)) / 2 + (v - u - 1);
}

// (r, s) = pair number m of the row-major enumeration of pairs r < s.
__device__ __forceinline__ void decode_pair(int N, int m, int &r, int &s) {
  const float f2n = (float)(2 * N - 1);
  int q = (int)((f2n - sqrtf(fmaxf(f2n * f2n - 8.0f * (float)m, 0.0f))) * 0.5f);
  q = max(0, min(q, N - 2));
  while (q > 0 && q * N - (q * (q + 1)) / 2 > m) --q;
  while (q < N - 2 && (q + 1) * N - ((q + 1) * (q + 2)) / 2 <= m) ++q;
  r = q;
  s = m - (q * N - (q * (q + 1)) / 2) + q + 1;
}

// The pair after (r, s) in the cyclic enumeration.
__device__ __forceinline__ void next_pair(int N, int &r, int &s) {
  if (++s >= N) {
    if (++r >= N - 1) r = 0;
    s = r + 1;
  }
}

// Does the closed interval [lo, hi] of pair indices meet the window, which
// starts at pair a and covers len <= M consecutive pairs, wrapping at M?
__device__ __forceinline__ bool meets_window(int lo, int hi, int a, int len,
                                             int M) {
  const int end = a + len - 1;
  if (end < M) return lo <= end && hi >= a;
  return hi >= a || lo <= end - M;
}

// Binary32 pre-test interval for a proposal made at temperature ~Tc with
// random word x: accept for sure if delta < lo, reject for sure if
// delta > hi, otherwise decide in binary64.  t = Tc * (-ln u) and the margin
// covers the binary32 errors of Tc, ln u and (float)delta (mrel relative,
// 1e-6 Tc absolute).  A non-finite t gives NaN bounds: undecided.
__device__ __forceinline__ float2 accept_interval(float mrel, float Tc,
                                                  unsigned x) {
  const float uf = fmaf(__uint2float_rn(x), 0x1p-32f, 0x1p-33f);
  const float t = Tc * -logf(uf);
  const float mg = mrel * t + 1e-6f * Tc;
  return make_float2(t - mg, t + mg);
}

// Pre-test of up to four cells of one tile row that fall outside the prepared
// table (long windows at low temperature, where survivors are rare).  Returns
// the accepted cells in bits 0-3 and the undecided ones in bits 4-7.
__device__ __noinline__ unsigned pretest_cells(unsigned long long seed,
                                               unsigned stream, float log2a,
                                               float mrel,
                                               unsigned long long it, float Tw,
                                               int j0, int j1, int j2, int j3,
                                               int d0, int d1, int d2, int d3,
                                               unsigned mask) {
  const int jj[4] = {j0, j1, j2, j3};
  const int dd[4] = {d0, d1, d2, d3};
  unsigned long long qc = ~0ull;
  uint4 xb = make_uint4(0, 0, 0, 0);
  unsigned out = 0;
  for (int c = 0; c < 4; ++c) {
    if (!((mask >> c) & 1u)) continue;
    const unsigned long long itc = it + (unsigned)jj[c];
    if ((itc >> 2) != qc) {
      qc = itc >> 2;
      xb = rng_block(seed, stream, qc);
    }
    const float Tc = Tw * exp2f((float)jj[c] * log2a);
    const float2 b = accept_interval(mrel, Tc, word_of(xb, (int)(itc & 3u)));
    const float df = (float)dd[c];
    if (df < b.x) out |= 1u << c;
    else if (!(df > b.y)) out |= 16u << c;
  }
  return out;
}

// Delta of the cells of one tile from their definition under the current p,
// through G_xy = <A_x, B'_y>: Delta_uv = 2 (G_uv + G_vu - d_u - d_v + 2 A_uv B'_uv).
template <int R>
__device__ __forceinline__ void t1_rebuild_tile(int (&D)[R][4], int u0, int v0,
                                                int N, int S, const int8_t *s_A,
                                                const int8_t *s_B, const int *s_d) {
  const int NC = S >> 4;
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int u = u0 + i, v = v0 + c;
      if (!(u < v && v < N)) continue;
      const int4 *Au = reinterpret_cast<const int4 *>(s_A + u * S);
      const int4 *Bu = reinterpret_cast<const int4 *>(s_B + u * S);
      const int4 *Av = reinterpret_cast<const int4 *>(s_A + v * S);
      const int4 *Bv = reinterpret_cast<const int4 *>(s_B + v * S);
      int guv = 0, gvu = 0;
      for (int k = 0; k < NC; ++k) {
        const int4 a = Au[k], b = Bv[k], a2 = Av[k], b2 = Bu[k];
        guv = __dp4a(a.x, b.x, guv); guv = __dp4a(a.y, b.y, guv);
        guv = __dp4a(a.z, b.z, guv); guv = __dp4a(a.w, b.w, guv);
        gvu = __dp4a(a2.x, b2.x, gvu); gvu = __dp4a(a2.y, b2.y, gvu);
        gvu = __dp4a(a2.z, b2.z, gvu); gvu = __dp4a(a2.w, b2.w, gvu);
      }
      D[i][c] = 2 * (guv + gvu - s_d[u] - s_d[v] + 2 * (int)s_A[u * S + v] * (int)s_B[u * S + v]);
    }
}

// The same for rows uq .. uq+3 of a tile (cells that are no pair get 0).
__device__ __forceinline__ void t1_rebuild_piece(int (&Dq)[16], int uq, int v0, int N,
                                                 int S, const int8_t *s_A,
                                                 const int8_t *s_B, const int *s_d) {
  const int NC = S >> 4;
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int u = uq + ii, v = v0 + c;
      Dq[4 * ii + c] = 0;
      if (!(u < v && v < N)) continue;
      const int4 *Au = reinterpret_cast<const int4 *>(s_A + u * S);
      const int4 *Bu = reinterpret_cast<const int4 *>(s_B + u * S);
      const int4 *Av = reinterpret_cast<const int4 *>(s_A + v * S);
      const int4 *Bv = reinterpret_cast<const int4 *>(s_B + v * S);
      int guv = 0, gvu = 0;
      for (int k = 0; k < NC; ++k) {
        const int4 a = Au[k], b = Bv[k], a2 = Av[k], b2 = Bu[k];
        guv = __dp4a(a.x, b.x, guv); guv = __dp4a(a.y, b.y, guv);
        guv = __dp4a(a.z, b.z, guv); guv = __dp4a(a.w, b.w, guv);
        gvu = __dp4a(a2.x, b2.x, gvu); gvu = __dp4a(a2.y, b2.y, gvu);
        gvu = __dp4a(a2.z, b2.z, gvu); gvu = __dp4a(a2.w, b2.w, gvu);
      }
      Dq[4 * ii + c] =
          2 * (guv + gvu - s_d[u] - s_d[v] + 2 * (int)s_A[u * S + v] * (int)s_B[u * S + v]);
    }
}

struct WarpPos {
  unsigned it_lo, it_hi;
  int mb, cr, cs, blk_it, blk_acc, err;
};

// Byte i (0..3) of a packed word of int8 values, sign-extended.
__device__ __forceinline__ int s8_of(int w, int i) {
  return static_cast<int8_t>(static_cast<unsigned>(w) >> (8 * i));
}

// Product of 16 int8 pairs (two 16-byte chunks) added to acc.
__device__ __forceinline__ int dot16x(int4 x, int4 y, int acc) {
  acc = __dp4a(x.x, y.x, acc);
  acc = __dp4a(x.y, y.y, acc);
  acc = __dp4a(x.z, y.z, acc);
  return __dp4a(x.w, y.w, acc);
}

// Direct mode run by the calling warp alone, with no block barrier: while
// proposals are accepted often, an accepted swap then costs a few hundred
// cycles of one warp.  Lane l evaluates proposal it + j, j = l, l + 32, ... of a
// window of up to kWarpMaxK proposals -- delta = 2 (<A_r, B'_s> + <A_s, B'_r>
// - d_r - d_s + 2 A_rs B'_rs) by dp4a, its Eq. (2) pre-test from its own
// Philox block -- the first accepted one is found with a warp reduction, and
// the swap is applied to B', d and p by the lanes together.  The chain
// position comes from and goes back to *pos; returns at it_end, at the end of
// the current block of kHybBlock iterations, or on an inconsistency.  Counters
// go to c64 (lane 0).
//
// LPP lanes evaluate one proposal (the dot products split over them), so a pass
// takes 32 / LPP proposals.  The loop is a function of its own, not inlined,
// and a kernel calls one instantiation only: one warp runs it alone for
// thousands of iterations and it must stay small in the instruction cache
// (with all three instantiations reachable from one kernel the warp mode ran
// three times slower).
template <int LPP>
__device__ __noinline__ void t1_warp_run(int N, int S, int M, unsigned long long seed,
                                            unsigned stream, double T0, const double *P,
                                            float T0f, float log2a_f, float mrel,
                                            unsigned long long it_end,
                                            const int8_t *s_A, int8_t *s_B, int *s_d,
                                            int *s_p, unsigned long long *c64,
                                            WarpPos *pos, ChainStatus *st) {
  const unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const int NC = S >> 4;
  __syncwarp();
  unsigned long long it = ((unsigned long long)pos->it_hi << 32) | pos->it_lo;
  int mb = pos->mb, cr = pos->cr, cs = pos->cs;
  int blk_it = pos->blk_it, blk_acc = pos->blk_acc, err = 0;
  // counters of this call (lane 0 adds them to c64 at the end)
  unsigned long long n_it = 0, n_acc = 0, n_win = 0, n_exact = 0;
  long long d_cost = 0;
  const int kmax = min(M, kWarpMaxK);
  int K = min(32, kmax);
  constexpr int lpp = LPP;  // lanes per proposal
  constexpr int ppp = 32 / LPP;
  const int sub = lane & (LPP - 1);
  // Rolling table of Eq. (2) pre-test intervals in registers: lane l holds
  // those of Philox block q0 + l (iterations 4 (q0 + l) .. + 3), computed as the
  // prepared table computes them; a proposal fetches its own by shuffles.
  unsigned long long q0 = ~0ull;
  float2 tb0 = make_float2(0.f, 0.f), tb1 = tb0, tb2 = tb0, tb3 = tb0;
  while (it < it_end && blk_it < kHybBlock) {
    const int wlen = (int)min((unsigned long long)K, it_end - it);
    unsigned best = kNone;
    int brs = 0, bdv = 0;
    for (int j0 = 0; j0 < wlen; j0 += ppp) {
      {
        const unsigned long long qa = (it + (unsigned)j0) >> 2;
        if (qa < q0 || ((it + (unsigned)(j0 + ppp - 1)) >> 2) >= q0 + 32) {  // refill
          q0 = qa;
          const unsigned long long q = q0 + (unsigned)lane;
          const uint4 x = rng_block(seed, stream, q);
          const float Tq = T0f * exp2f(u64_to_f32(q << 2) * log2a_f);
          tb0 = accept_interval(mrel, Tq, x.x);
          tb1 = accept_interval(mrel, Tq * exp2f(log2a_f), x.y);
          tb2 = accept_interval(mrel, Tq * exp2f(2.0f * log2a_f), x.z);
          tb3 = accept_interval(mrel, Tq * exp2f(3.0f * log2a_f), x.w);
        }
      }
      const int j = j0 + lane / lpp;
      float2 b;
      {
        const unsigned long long itc = it + (unsigned)j;
        const int src = (int)((itc >> 2) - q0) & 31, w = (int)(itc & 3u);
        const float x0 = __shfl_sync(FULL, tb0.x, src), y0 = __shfl_sync(FULL, tb0.y, src);
        const float x1 = __shfl_sync(FULL, tb1.x, src), y1 = __shfl_sync(FULL, tb1.y, src);
        const float x2 = __shfl_sync(FULL, tb2.x, src), y2 = __shfl_sync(FULL, tb2.y, src);
        const float x3 = __shfl_sync(FULL, tb3.x, src), y3 = __shfl_sync(FULL, tb3.y, src);
        b.x = w == 0 ? x0 : (w == 1 ? x1 : (w == 2 ? x2 : x3));
        b.y = w == 0 ? y0 : (w == 1 ? y1 : (w == 2 ? y2 : y3));
      }
      int r = cr, s = cs + j, g1 = 0, g2 = 0;
      if (j < wlen) {
        while (s >= N) {  // on into the next rows of the cyclic order
          const int o = s - N;
          if (++r >= N - 1) r = 0;
          s = r + 1 + o;
        }
        const int4 *Ar4 = reinterpret_cast<const int4 *>(s_A + r * S);
        const int4 *As4 = reinterpret_cast<const int4 *>(s_A + s * S);
        const int4 *Br4 = reinterpret_cast<const int4 *>(s_B + r * S);
        const int4 *Bs4 = reinterpret_cast<const int4 *>(s_B + s * S);
#pragma unroll 4
        for (int c = sub; c < NC; c += lpp) {
          g1 = dot16x(Ar4[c], Bs4[c], g1);
          g2 = dot16x(As4[c], Br4[c], g2);
        }
      }
      for (int o = 1; o < lpp; o <<= 1) {
        g1 += __shfl_xor_sync(FULL, g1, o);
        g2 += __shfl_xor_sync(FULL, g2, o);
      }
      if (j < wlen && sub == 0) {
        const int dv = 2 * (g1 + g2 - s_d[r] - s_d[s] +
                            2 * (int)s_A[r * S + s] * (int)s_B[r * S + s]);
        const float df = (float)dv;
        const unsigned acc = (dv <= 0 || df < b.x) ? 1u : 0u;
        const unsigned unc = (!acc && !(df > b.y)) ? 1u : 0u;
        if (acc | unc) {
          best = ((unsigned)j << 1) | unc;
          brs = (r << 16) | s;
          bdv = dv;
        }
      }
      if (__any_sync(FULL, best != kNone)) break;  // later passes come later in order
    }
    const unsigned wmin = __reduce_min_sync(FULL, best);
    ++n_win;
    if (wmin == kNone) {
      it += (unsigned)wlen;
      mb += wlen;
      if (mb >= M) mb -= M;
      decode_pair(N, mb, cr, cs);
      blk_it += wlen;
      n_it += (unsigned)wlen;
      K = min(2 * K, kmax);
      continue;
    }
    const int wl = __ffs(__ballot_sync(FULL, best == wmin)) - 1;
    const int j = (int)(wmin >> 1);
    const int rs = __shfl_sync(FULL, brs, wl);
    const int dlt = __shfl_sync(FULL, bdv, wl);
    const int r = rs >> 16, s = rs & 0xFFFF;
    if (wmin & 1u) {  // undecided by the binary32 pre-test: binary64
      int dec = 0;
      if (lane == 0) {
        ++n_exact;
        dec = exact_accept(seed, stream, T0, P, dlt, it + (unsigned)j, &c64[kC64Near], st);
      }
      dec = __shfl_sync(FULL, dec, 0);
      if (!dec) {
        it += (unsigned)j + 1;
        mb += j + 1;
        if (mb >= M) mb -= M;
        cr = r;
        cs = s;
        next_pair(N, cr, cs);
        blk_it += j + 1;
        n_it += (unsigned)j + 1;
        continue;
      }
    }
    if (r < 0 || r >= s || s >= N) {
      err = 1;
      break;
    }
    // ---- accept the swap (r, s) ----
    if (j < K / 8) K = max(min(32, kmax), K / 2);
    it += (unsigned)j + 1;
    mb += j + 1;
    if (mb >= M) mb -= M;
    cr = r;
    cs = s;
    next_pair(N, cr, cs);
    blk_it += j + 1;
    ++blk_acc;
    n_it += (unsigned)j + 1;
    ++n_acc;
    d_cost += dlt;
    // B' rows and columns r,s (Eq. 3); d_k += (A_rk - A_sk)(B'_sk - B'_rk);
    // d_r, d_s of the new p.  A lane takes four consecutive k: one 32-bit word
    // of rows r,s of A and B' and one int4 of d; rows r and s of B' trade their
    // words except the bytes of columns r,s; columns r,s are stored by byte.
    int dr_part = 0, ds_part = 0;
    for (int kb = 0; kb < N; kb += 128) {
      const int k0 = kb + 4 * lane;
      const bool live = k0 < N;
      const int kr = live ? k0 : 0;
      const int ar = *reinterpret_cast<const int *>(s_A + r * S + kr);
      const int as = *reinterpret_cast<const int *>(s_A + s * S + kr);
      const int br = *reinterpret_cast<const int *>(s_B + r * S + kr);
      const int bs = *reinterpret_cast<const int *>(s_B + s * S + kr);
      int4 dq = *reinterpret_cast<const int4 *>(s_d + kr);
      int dd[4] = {dq.x, dq.y, dq.z, dq.w};
      unsigned keep = 0;  // bytes of columns r and s: they stay
      if (r >= k0 && r < k0 + 4) keep |= 0xFFu << (8 * (r - k0));
      if (s >= k0 && s < k0 + 4) keep |= 0xFFu << (8 * (s - k0));
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = k0 + i;
        if (!live || k >= N) break;
        const int Ark = s8_of(ar, i), Ask = s8_of(as, i);
        const int Brk = s8_of(br, i), Bsk = s8_of(bs, i);
        if (k != r && k != s) {
          dd[i] += (Ark - Ask) * (Bsk - Brk);
          s_B[k * S + r] = (int8_t)Bsk;
          s_B[k * S + s] = (int8_t)Brk;
          dr_part += Ark * Bsk;
          ds_part += Ask * Brk;
        } else if (k == s) {
          dr_part += Ark * Brk;  // A_rs B'_rs
        } else {
          ds_part += Ask * Bsk;  // A_sr B'_sr
        }
      }
      if (live) {
        *reinterpret_cast<int *>(s_B + r * S + k0) =
            (int)(((unsigned)bs & ~keep) | ((unsigned)br & keep));
        *reinterpret_cast<int *>(s_B + s * S + k0) =
            (int)(((unsigned)br & ~keep) | ((unsigned)bs & keep));
        *reinterpret_cast<int4 *>(s_d + k0) = make_int4(dd[0], dd[1], dd[2], dd[3]);
      }
    }
    const int dr = __reduce_add_sync(FULL, dr_part), ds = __reduce_add_sync(FULL, ds_part);
    __syncwarp();
    if (lane == 0) {
      s_d[r] = dr;
      s_d[s] = ds;
      const int t = s_p[r];
      s_p[r] = s_p[s];
      s_p[s] = t;
    }
    __syncwarp();
  }
  if (lane == 0) {
    pos->it_lo = (unsigned)it;
    pos->it_hi = (unsigned)(it >> 32);
    pos->mb = mb;
    pos->cr = cr;
    pos->cs = cs;
    pos->blk_it = blk_it;
    pos->blk_acc = blk_acc;
    pos->err = err;
    c64[kC64Accepts] += n_acc;
    c64[kC64Cost] += (unsigned long long)d_cost;
    c64[kC64Windows] += n_win;
    c64[kC64Exact] += n_exact;
    c64[kC64DirIt] += n_it;
    c64[kC64WarpIt] += n_it;
    c64[kC64DirAcc] += n_acc;
  }
  __syncwarp();
}

// Mode decisions at the end of a block of kHybBlock iterations (every thread
// alike): Delta mode below g.hyb_lo, direct mode above 4 g.hyb_lo once in
// Delta mode, and within direct mode one warp alone from g.warp_lo up.
__device__ __forceinline__ void t1_block_end(const ChainDev &g, int &mode, bool &rebuild,
                                             int &warp_mode, int &blk_it, int &blk_acc) {
  if (blk_it < kHybBlock) return;
  if (mode == 1 && (float)blk_acc < g.hyb_lo * (float)blk_it) {
    mode = 0;  // few accepts: maintain Delta from here on
    rebuild = true;
  } else if (mode == 0 && g.hyb_lo > 0.0f && (float)blk_acc > 4.0f * g.hyb_lo * (float)blk_it) {
    mode = 1;  // many accepts again: evaluate proposals directly
  }
  warp_mode = (mode == 1 && g.warp_lo > 0.0f && (float)blk_acc >= g.warp_lo * (float)blk_it);
  blk_it = blk_acc = 0;
}

// One chain, run by the whole CTA from its state in global memory to iteration
// it_end and written back.  `smem` holds at least t1_layout(N, S).bytes.
//
// Two ways to obtain the swap cost of a proposal, chosen by the measured
// acceptance rate (the trajectory is the same either way: delta is the same
// exact integer):
//   Delta mode   the maintained matrix (section 2.2): a proposal costs one
//                register read, an accepted swap the O(N^2) update;
//   direct mode  delta = 2 (<A_r, B'_s> + <A_s, B'_r> - d_r - d_s + 2 A_rs B'_rs)
//                evaluated for every proposal of the window (four threads per
//                proposal, dp4a), and an accepted swap only moves p, B' and d.
// While many proposals are accepted (high temperature) direct mode is far
// cheaper; the kernel switches to Delta mode, rebuilding Delta, once the
// acceptance rate of a block of 16384 iterations drops below g.hyb_lo.
//
// TM: the tiles live in TMEM at address tb (this thread's lane, 4R columns)
// instead of registers; every TMEM access below is reached by whole warps.
// WLPP: lanes per proposal of the warp-only direct mode.
template <int R, bool TM, int WLPP>
__device__ __forceinline__ void t1_run_chain(const ChainDev &g,
                                             unsigned long long it_end,
                                             unsigned char *smem, unsigned tb) {
  const int N = g.N, S = g.S, M = g.M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = blockDim.x;
  const T1Layout L = t1_layout(N, S);
  int8_t *s_A = reinterpret_cast<int8_t *>(smem + L.off_A);
  int8_t *s_B = reinterpret_cast<int8_t *>(smem + L.off_B);
  int *s_a = reinterpret_cast<int *>(smem + L.off_a);
  int *s_b = reinterpret_cast<int *>(smem + L.off_b);
  int *s_d = reinterpret_cast<int *>(smem + L.off_d);
  int *s_p = reinterpret_cast<int *>(smem + L.off_p);
  int *s_nr = reinterpret_cast<int *>(smem + L.off_nr);
  int *s_ns = reinterpret_cast<int *>(smem + L.off_ns);
  int4 *s_slot = reinterpret_cast<int4 *>(smem + L.off_slot);
  unsigned *s_ctl = reinterpret_cast<unsigned *>(smem + L.off_ctl);
  float2 *s_tt = reinterpret_cast<float2 *>(smem + L.off_tt);

  // ---- chain state into shared memory and registers ----
  {
    const int4 *gA = reinterpret_cast<const int4 *>(g.A);
    const int4 *gB = reinterpret_cast<const int4 *>(g.Bp);
    int4 *sA = reinterpret_cast<int4 *>(s_A);
    int4 *sB = reinterpret_cast<int4 *>(s_B);
    for (int i = tid; i < (N * S) >> 4; i += nthreads) {
      sA[i] = gA[i];
      sB[i] = gB[i];
    }
  }
  const int NP = t1_vec_len(N);
  for (int i = tid; i < NP; i += nthreads) {
    s_p[i] = i < N ? g.p[i] : 0;
    s_d[i] = i < N ? g.d[i] : 0;
    s_a[i] = 0;
    s_b[i] = 0;
  }
  if (tid < 8) s_ctl[tid] = (tid < 3) ? kNone : 0u;

  const bool has_tile = tid < g.ntiles;
  int u0 = 0, v0 = 0;
  if (has_tile) {
    const int t = g.tiles[tid];
    u0 = t >> 16;
    v0 = t & 0xFFFF;
  }
  // Cell (u0+i, v0+c) is a pair iff u0+i < v0+c < N.
  int D[TM ? 1 : R][4];  // the register tiles (unused with TM)
  int tm_lo = 0x7FFFFFFF, tm_hi = -1;
  if constexpr (TM) {
#pragma unroll 1
    for (int q = 0; q < R / 4; ++q) {
      int Dq[16];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int u = u0 + 4 * q + ii, v = v0 + c;
          Dq[4 * ii + c] = 0;
          if (has_tile && u < v && v < N) {
            const int m = pidx(N, u, v);
            Dq[4 * ii + c] = g.delta[m];
            tm_lo = min(tm_lo, m);
            tm_hi = max(tm_hi, m);
          }
        }
      tmem_st16(tb + 16 * q, Dq);
    }
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int u = u0 + i, v = v0 + c;
        D[i][c] = 0;
        if (has_tile && u < v && v < N) {
          const int m = pidx(N, u, v);
          D[i][c] = g.delta[m];
          tm_lo = min(tm_lo, m);
          tm_hi = max(tm_hi, m);
        }
      }
  }

  unsigned long long *c64 = reinterpret_cast<unsigned long long *>(s_ctl + 8);
  if (tid == 0) {
    c64[kC64Accepts] = g.st->accepts;
    c64[kC64Cost] = (unsigned long long)g.st->cost;
    c64[kC64Near] = 0;
    c64[kC64Exact] = 0;
    c64[kC64Windows] = 0;
    c64[kC64DirIt] = 0;
    c64[kC64DirAcc] = 0;
    c64[kC64WarpIt] = 0;
  }
  unsigned long long it = g.st->it;
  int err = 0;
  int mb = (int)(it % (unsigned long long)M);  // pair index of iteration it
  int cr, cs;                                   // that pair, (cr, cs)
  decode_pair(N, mb, cr, cs);
  int K = min(1024, M);                         // window length
  (void)K;
  unsigned wi = 0;
  int pend_r = -1, pend_s = -1;
  unsigned long long tab_it = 0;  // first iteration covered by s_tt
  int tab_len = 0;                // entries of s_tt that are valid
  int mode = (g.hyb_lo > 0.0f) ? g.st->mode : 0;
  int blk_it = 0, blk_acc = 0;    // iterations and accepts of the current block
  int warp_mode = (mode == 1 && g.warp_lo > 0.0f);  // direct mode by one warp alone
  bool rebuild = false;           // Delta registers to be recomputed
  // Direct mode: d of the last swap's r and s, taken from the reduction while
  // s_d[r], s_d[s] are being written (one barrier fewer per accepted swap).
  int ov_r = -1, ov_s = -1, ov_dr = 0, ov_ds = 0;
  unsigned nacc = 0;  // accepted swaps in this launch: d_r, d_s sums alternate
  const int per_pass = nthreads >> 2;  // proposals evaluated at once, direct mode
  int tpv = 1;  // threads per row in the rows-r,s recompute: <= 4 keeps >= 8
                // lanes per slice, so 16-byte loads of 8 rows are conflict-free
  while (tpv < 4 && 2 * tpv * N <= nthreads) tpv *= 2;
  const int lpt = 32 / tpv;  // lanes per dot-product slice
  const int t_sl = lane / lpt, v_l = lane - t_sl * lpt;
  const int vslots = (nthreads >> 5) * lpt;
  const int NC = S >> 4;  // 16-byte chunks per row
  __syncthreads();

  for (;;) {
    // ---- rows/columns r,s recomputed by the previous accept -> the tiles ----
    if constexpr (TM) {
      if (pend_r >= 0) {
        const int r = pend_r, s = pend_s;
        const bool col_hit = has_tile && ((r >= v0 && r < v0 + 4) || (s >= v0 && s < v0 + 4));
#pragma unroll 1
        for (int q = 0; q < R / 4; ++q) {
          const int uq = u0 + 4 * q;
          const bool row_hit =
              has_tile && ((r >= uq && r < uq + 4) || (s >= uq && s < uq + 4));
          if (!__any_sync(0xFFFFFFFFu, row_hit || col_hit)) continue;
          int Dq[16];
          tmem_ld16(tb + 16 * q, Dq);
          if (row_hit) {
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
              const int u = uq + ii;
              if (u == r || u == s) {
                const int *src = (u == r) ? s_nr : s_ns;
#pragma unroll
                for (int c = 0; c < 4; ++c) Dq[4 * ii + c] = src[v0 + c];
              }
            }
          }
          if (col_hit) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int v = v0 + c;
              if (v == r || v == s) {
                const int *src = (v == r) ? s_nr : s_ns;
#pragma unroll
                for (int ii = 0; ii < 4; ++ii) Dq[4 * ii + c] = src[uq + ii];
              }
            }
          }
          tmem_st16(tb + 16 * q, Dq);
        }
      }
    } else {
      if (pend_r >= 0 && has_tile) {
        const int r = pend_r, s = pend_s;
        if ((r >= u0 && r < u0 + R) || (s >= u0 && s < u0 + R)) {
#pragma unroll
          for (int i = 0; i < R; ++i) {
            const int u = u0 + i;
            if (u == r || u == s) {
              const int *src = (u == r) ? s_nr : s_ns;
#pragma unroll
              for (int c = 0; c < 4; ++c) D[i][c] = src[v0 + c];
            }
          }
        }
        if ((r >= v0 && r < v0 + 4) || (s >= v0 && s < v0 + 4)) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int v = v0 + c;
            if (v == r || v == s) {
              const int *src = (v == r) ? s_nr : s_ns;
#pragma unroll
              for (int i = 0; i < R; ++i) D[i][c] = src[u0 + i];
            }
          }
        }
      }
    }
    pend_r = -1;
    // Delta registers from their definition: after a switch to Delta mode, and
    // before the state is stored if Delta was not being maintained.
    const bool last = it >= it_end || err;
    if constexpr (TM) {
      if (rebuild || (last && mode == 1)) {
#pragma unroll 1
        for (int q = 0; q < R / 4; ++q) {
          int Dq[16];
          t1_rebuild_piece(Dq, u0 + 4 * q, v0, has_tile ? N : 0, S, s_A, s_B, s_d);
          tmem_st16(tb + 16 * q, Dq);
        }
      }
    } else if (has_tile && (rebuild || (last && mode == 1))) {
      t1_rebuild_tile<R>(D, u0, v0, N, S, s_A, s_B, s_d);
    }
    rebuild = false;
    if (last) break;

    if (mode == 1 && warp_mode) {
      // ================= warp-only direct mode, to the block's end =================
      WarpPos *pos = reinterpret_cast<WarpPos *>(s_ctl + kT1Pos);
      if (tid == 0) {
        pos->it_lo = (unsigned)it;
        pos->it_hi = (unsigned)(it >> 32);
        pos->mb = mb;
        pos->cr = cr;
        pos->cs = cs;
        pos->blk_it = blk_it;
        pos->blk_acc = blk_acc;
        pos->err = 0;
      }
      if (warp == 0)
        t1_warp_run<WLPP>(N, S, M, g.seed, g.stream, g.T0, g.P, g.T0f, g.log2a_f, g.mrel,
                          it_end, s_A, s_B, s_d, s_p, c64, pos, g.st);
      __syncthreads();
      it = ((unsigned long long)pos->it_hi << 32) | pos->it_lo;
      mb = pos->mb;
      cr = pos->cr;
      cs = pos->cs;
      blk_it = pos->blk_it;
      blk_acc = pos->blk_acc;
      err = pos->err;
      __syncthreads();  // every thread has read the position before it is reused
      tab_len = 0;      // the prepared thresholds are for an older position
      ov_r = ov_s = -1;
      t1_block_end(g, mode, rebuild, warp_mode, blk_it, blk_acc);
      continue;
    }

    // ================= scan one window =================
    // Window = iterations it .. it + wlen - 1, wlen <= M, so the proposal at
    // offset j is pair (mb + j) mod M and every pair occurs at most once.
    const int wlen = (int)min((unsigned long long)K, it_end - it);
    // offset of this window in the prepared table (none if it lies outside)
    const int jt0 = (it >= tab_it && it - tab_it < (unsigned long long)tab_len)
                        ? (int)(it - tab_it) : kTabMax;
    // Integer pre-filter for proposals beyond the table: -ln u <= 22.9 for
    // u >= 2^-33, so delta > 24.5 T (T the window's largest binary32
    // temperature) is rejected whatever u is.
    float Tw = 0.0f;
    int thr = 0;
    if (jt0 + wlen > tab_len) {
      Tw = g.T0f * exp2f(u64_to_f32(it) * g.log2a_f);
      const float Te = Tw * exp2f((float)wlen * g.log2a_f);
      const float tmax = fmaxf(Tw, Te) * 24.5f;
      thr = (tmax < 1.0e9f) ? (int)ceilf(tmax) + 1 : 0x7FFFFFFF;
    }
    unsigned best = kNone;
    int bu = 0, bv = 0, bd = 0;
    if (mode == 1) {
      // ---- direct evaluation: four threads per proposal ----
      const int sub = tid & 3;
      for (int jb = 0; jb < wlen; jb += per_pass) {
        const int j = jb + (tid >> 2);
        int r = cr, s = cs + j, g1 = 0, g2 = 0;
        if (j < wlen) {
          if (s >= N) {  // beyond the window's first row
            int m = mb + j;
            if (m >= M) m -= M;
            decode_pair(N, m, r, s);
          }
          const int4 *Ar4 = reinterpret_cast<const int4 *>(s_A + r * S);
          const int4 *As4 = reinterpret_cast<const int4 *>(s_A + s * S);
          const int4 *Br4 = reinterpret_cast<const int4 *>(s_B + r * S);
          const int4 *Bs4 = reinterpret_cast<const int4 *>(s_B + s * S);
          for (int c = sub; c < NC; c += 4) {
            const int4 a = Ar4[c], b = Bs4[c];
            g1 = __dp4a(a.x, b.x, g1); g1 = __dp4a(a.y, b.y, g1);
            g1 = __dp4a(a.z, b.z, g1); g1 = __dp4a(a.w, b.w, g1);
            const int4 a2 = As4[c], b2 = Br4[c];
            g2 = __dp4a(a2.x, b2.x, g2); g2 = __dp4a(a2.y, b2.y, g2);
            g2 = __dp4a(a2.z, b2.z, g2); g2 = __dp4a(a2.w, b2.w, g2);
          }
        }
        g1 += __shfl_xor_sync(0xFFFFFFFFu, g1, 1);
        g2 += __shfl_xor_sync(0xFFFFFFFFu, g2, 1);
        g1 += __shfl_xor_sync(0xFFFFFFFFu, g1, 2);
        g2 += __shfl_xor_sync(0xFFFFFFFFu, g2, 2);
        if (sub == 0 && j < wlen) {
          const int dr_ = (r == ov_r) ? ov_dr : (r == ov_s ? ov_ds : s_d[r]);
          const int ds_ = (s == ov_r) ? ov_dr : (s == ov_s ? ov_ds : s_d[s]);
          const int dv = 2 * (g1 + g2 - dr_ - ds_ +
                              2 * (int)s_A[r * S + s] * (int)s_B[r * S + s]);
          unsigned acc = 0, unc = 0;
          const int jt = jt0 + j;
          if (dv <= 0) {
            acc = 1;
          } else if (jt < tab_len) {
            const float2 b = s_tt[jt];
            const float df = (float)dv;
            if (df < b.x) acc = 1;
            else if (!(df > b.y)) unc = 1;
          } else if (dv <= thr) {
            const unsigned o = pretest_cells(g.seed, g.stream, g.log2a_f, g.mrel, it, Tw,
                                             j, 0, 0, 0, dv, 0, 0, 0, 1u);
            acc = o & 1u;
            unc = (o >> 4) & 1u;
          }
          if (acc | unc) {
            const unsigned key = ((unsigned)j << 1) | unc;
            if (key < best) {
              best = key;
              bu = r;
              bv = s;
              bd = dv;
            }
          }
        }
      }
    } else if constexpr (TM) {
      const bool scan_me = has_tile && meets_window(tm_lo, tm_hi, mb, wlen, M);
      if (__any_sync(0xFFFFFFFFu, scan_me)) {
#pragma unroll 1
        for (int q = 0; q < R / 4; ++q) {
          unsigned rows = 0;  // rows of this 4-row piece with a cell in the window
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) {
            const int u = u0 + 4 * q + ii;
            if (scan_me && u < N - 1 && u < v0 + 3) {
              const int mrow = u * N - (u * (u + 1)) / 2 - u - 1;
              const int vlo = max(v0, u + 1), vhi = min(v0 + 3, N - 1);
              if (meets_window(mrow + vlo, mrow + vhi, mb, wlen, M)) rows |= 1u << ii;
            }
          }
          if (!__any_sync(0xFFFFFFFFu, rows != 0u)) continue;
          int Dq[16];
          tmem_ld16(tb + 16 * q, Dq);
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) {
            if (!((rows >> ii) & 1u)) continue;
            const int u = u0 + 4 * q + ii;
            const int mrow = u * N - (u * (u + 1)) / 2 - u - 1;
            int jc[4];
            unsigned acc = 0, unc = 0, slow = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              int j = mrow + v0 + c - mb;
              if (j < 0) j += M;
              jc[c] = j;
              const int v = v0 + c;
              if (v > u && v < N && j < wlen) {
                const int dv = Dq[4 * ii + c];
                const int jt = jt0 + j;
                if (dv <= 0) {
                  acc |= 1u << c;
                } else if (jt < tab_len) {
                  const float2 b = s_tt[jt];
                  const float df = (float)dv;
                  if (df < b.x) acc |= 1u << c;
                  else if (!(df > b.y)) unc |= 1u << c;
                } else if (dv <= thr) {
                  slow |= 1u << c;
                }
              }
            }
            if (slow) {
              const unsigned o = pretest_cells(g.seed, g.stream, g.log2a_f, g.mrel, it, Tw,
                                               jc[0], jc[1], jc[2], jc[3], Dq[4 * ii + 0],
                                               Dq[4 * ii + 1], Dq[4 * ii + 2],
                                               Dq[4 * ii + 3], slow);
              acc |= o & 15u;
              unc |= o >> 4;
            }
            const unsigned any = acc | unc;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              if ((any >> c) & 1u) {
                const unsigned key = ((unsigned)jc[c] << 1) | ((unc >> c) & 1u);
                if (key < best) {
                  best = key;
                  bu = u;
                  bv = v0 + c;
                  bd = Dq[4 * ii + c];
                }
              }
            }
          }
        }
      }
    } else if (has_tile && meets_window(tm_lo, tm_hi, mb, wlen, M)) {
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int u = u0 + i;
        if (u >= N - 1 || u >= v0 + 3) continue;  // no pair u < v in this row
        const int mrow = u * N - (u * (u + 1)) / 2 - u - 1;  // pidx(u,v) = mrow + v
        const int vlo = max(v0, u + 1), vhi = min(v0 + 3, N - 1);
        if (!meets_window(mrow + vlo, mrow + vhi, mb, wlen, M)) continue;
        int jc[4];
        unsigned acc = 0, unc = 0, slow = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          int j = mrow + v0 + c - mb;
          if (j < 0) j += M;
          jc[c] = j;
          const int v = v0 + c;
          if (v > u && v < N && j < wlen) {
            const int dv = D[i][c];
            const int jt = jt0 + j;
            if (dv <= 0) {
              acc |= 1u << c;
            } else if (jt < tab_len) {
              const float2 b = s_tt[jt];
              const float df = (float)dv;
              if (df < b.x) acc |= 1u << c;
              else if (!(df > b.y)) unc |= 1u << c;
            } else if (dv <= thr) {
              slow |= 1u << c;
            }
          }
        }
        if (slow) {
          const unsigned o = pretest_cells(g.seed, g.stream, g.log2a_f, g.mrel,
                                           it, Tw, jc[0], jc[1], jc[2], jc[3],
                                           D[i][0], D[i][1], D[i][2], D[i][3], slow);
          acc |= o & 15u;
          unc |= o >> 4;
        }
        const unsigned any = acc | unc;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if ((any >> c) & 1u) {
            const unsigned key = ((unsigned)jc[c] << 1) | ((unc >> c) & 1u);
            if (key < best) {
              best = key;
              bu = u;
              bv = v0 + c;
              bd = D[i][c];
            }
          }
        }
      }
    }
    const unsigned wmin = __reduce_min_sync(0xFFFFFFFFu, best);
    if (wmin != kNone && best == wmin) {
      s_slot[warp] = make_int4((int)best, bu, bv, bd);
      atomicMin(s_ctl + kT1Key0 + (wi % 3u),
                (((best >> 1) << 5 | (unsigned)warp) << 1) | (best & 1u));
    }
    __syncthreads();
    const unsigned code = s_ctl[kT1Key0 + (wi % 3u)];
    if (tid == 0) {
      s_ctl[kT1Key0 + ((wi + 2u) % 3u)] = kNone;
      ++c64[kC64Windows];
    }
    ov_r = ov_s = -1;  // s_d[r], s_d[s] are current after this barrier
    ++wi;

    if (code == kNone) {  // nothing accepted in the window
      mb += wlen;
      if (mb >= M) mb -= M;
      decode_pair(N, mb, cr, cs);
      if (tid == 0 && mode == 1) c64[kC64DirIt] += (unsigned)wlen;
      it += (unsigned)wlen;
      K = min(K * 2, mode == 1 ? min(M, 4 * per_pass) : M);
      blk_it += wlen;
      t1_block_end(g, mode, rebuild, warp_mode, blk_it, blk_acc);
      continue;
    }
    const int j = (int)(code >> 6);
    const int4 sl = s_slot[(code >> 1) & 31u];
    const int r = sl.y, s = sl.z, dlt = sl.w;
    if (code & 1u) {  // undecided by the binary32 pre-test: binary64
      if (tid == 0) {
        ++c64[kC64Exact];
        s_ctl[kT1Dec] =
            (unsigned)exact_accept(g.seed, g.stream, g.T0, g.P, dlt,
                                   it + (unsigned)j, &c64[kC64Near], g.st);
      }
      __syncthreads();
      if (!s_ctl[kT1Dec]) {
        if (tid == 0 && mode == 1) c64[kC64DirIt] += (unsigned)j + 1;
        it += (unsigned)j + 1;
        mb += j + 1;
        if (mb >= M) mb -= M;
        cr = r;
        cs = s;
        next_pair(N, cr, cs);
        continue;
      }
    }

    // ================= accept the swap (r, s) =================
    if (r < 0 || r >= s || s >= N) {
      err = 1;
      continue;
    }
    if (j < K / 8) K = max(64, K / 2);
    K = min(K, mode == 1 ? min(M, 4 * per_pass) : M);
    blk_it += j + 1;
    ++blk_acc;
    if (tid == 0 && mode == 1) {
      c64[kC64DirIt] += (unsigned)j + 1;
      ++c64[kC64DirAcc];
    }
    it += (unsigned)j + 1;
    mb += j + 1;
    if (mb >= M) mb -= M;
    cr = r;
    cs = s;
    next_pair(N, cr, cs);
    if (tid == 0) {
      ++c64[kC64Accepts];
      c64[kC64Cost] += (unsigned long long)(long long)dlt;
    }

    // ---- stage: a, b from B' before the swap; d; swap B' rows/cols; p ----
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
    if (warp * 32 < N) {
      dr_part = __reduce_add_sync(0xFFFFFFFFu, dr_part);
      ds_part = __reduce_add_sync(0xFFFFFFFFu, ds_part);
      if (lane == 0) {
        atomicAdd(reinterpret_cast<int *>(s_ctl + ((nacc & 1u) ? kT1Dr1 : kT1Dr)), dr_part);
        atomicAdd(reinterpret_cast<int *>(s_ctl + ((nacc & 1u) ? kT1Ds1 : kT1Ds)), ds_part);
      }
    }
    if (tid == 0) {  // the other pair: last read before the previous window's
                     // barrier, next written after this stage's barrier
      s_ctl[(nacc & 1u) ? kT1Dr : kT1Dr1] = 0u;
      s_ctl[(nacc & 1u) ? kT1Ds : kT1Ds1] = 0u;
    }
    // ---- thresholds of the next window [it, it + tab_len), one Philox
    //      block per thread, on the last warps (free during the stage) ----
    tab_it = it;
    tab_len = min(K, kTabMax);
    {
      const int o = (int)(it & 3u);
      const int nblk = (tab_len + o + 3) >> 2;
      const int qb = nthreads - 1 - tid;  // the last warps do this: they have
                                          // the least of the other work
      if (qb < nblk) {
        const unsigned long long q = (it >> 2) + (unsigned)qb;
        const uint4 x = rng_block(g.seed, g.stream, q);
        const float Tq = g.T0f * exp2f(u64_to_f32(q << 2) * g.log2a_f);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int jt = 4 * qb + w - o;
          if (jt >= 0 && jt < tab_len)
            s_tt[jt] = accept_interval(g.mrel, Tq * exp2f((float)w * g.log2a_f),
                                       word_of(x, w));
        }
      }
    }

    __syncthreads();
    const int dr = (int)s_ctl[(nacc & 1u) ? kT1Dr1 : kT1Dr];
    const int ds = (int)s_ctl[(nacc & 1u) ? kT1Ds1 : kT1Ds];
    ++nacc;

    if (mode == 0) {
    // ---- rows r,s under the new p through G_xy = <A_x, B'_y>:
    //      Delta_rv = 2 (G_rv + G_vr - d_r - d_v + 2 A_rv B'_rv) ----
    {
      const int4 *Ar4 = reinterpret_cast<const int4 *>(s_A + r * S);
      const int4 *As4 = reinterpret_cast<const int4 *>(s_A + s * S);
      const int4 *Br4 = reinterpret_cast<const int4 *>(s_B + r * S);
      const int4 *Bs4 = reinterpret_cast<const int4 *>(s_B + s * S);
      for (int vb = 0; vb < N; vb += vslots) {
        const int v = vb + warp * lpt + v_l;
        int g1 = 0, g2 = 0, g3 = 0, g4 = 0;
        if (v < N) {
          const int4 *Av4 = reinterpret_cast<const int4 *>(s_A + v * S);
          const int4 *Bv4 = reinterpret_cast<const int4 *>(s_B + v * S);
#pragma unroll 1
          for (int c = t_sl; c < NC; c += tpv) {
            const int4 bv = Bv4[c];
            int4 x = Ar4[c];
            g1 = __dp4a(x.x, bv.x, g1); g1 = __dp4a(x.y, bv.y, g1);
            g1 = __dp4a(x.z, bv.z, g1); g1 = __dp4a(x.w, bv.w, g1);
            x = As4[c];
            g2 = __dp4a(x.x, bv.x, g2); g2 = __dp4a(x.y, bv.y, g2);
            g2 = __dp4a(x.z, bv.z, g2); g2 = __dp4a(x.w, bv.w, g2);
            const int4 av = Av4[c];
            x = Br4[c];
            g3 = __dp4a(av.x, x.x, g3); g3 = __dp4a(av.y, x.y, g3);
            g3 = __dp4a(av.z, x.z, g3); g3 = __dp4a(av.w, x.w, g3);
            x = Bs4[c];
            g4 = __dp4a(av.x, x.x, g4); g4 = __dp4a(av.y, x.y, g4);
            g4 = __dp4a(av.z, x.z, g4); g4 = __dp4a(av.w, x.w, g4);
          }
        }
        for (int o = lpt; o < 32; o <<= 1) {
          g1 += __shfl_xor_sync(0xFFFFFFFFu, g1, o);
          g2 += __shfl_xor_sync(0xFFFFFFFFu, g2, o);
          g3 += __shfl_xor_sync(0xFFFFFFFFu, g3, o);
          g4 += __shfl_xor_sync(0xFFFFFFFFu, g4, o);
        }
        if (t_sl == 0 && v < N && v != r && v != s) {
          const int dv = s_d[v];
          const int Arv = s_A[r * S + v], Brv = s_B[r * S + v];
          const int Asv = s_A[s * S + v], Bsv = s_B[s * S + v];
          s_nr[v] = 2 * (g1 + g3 - dr - dv + 2 * Arv * Brv);
          s_ns[v] = 2 * (g2 + g4 - ds - dv + 2 * Asv * Bsv);
        }
      }
    }
    // ---- O(1) update of every tile cell: Delta_uv += 2 (a_u - a_v)(b_v - b_u);
    //      cells in rows/columns r,s are overwritten from s_nr/s_ns later ----
    if constexpr (TM) {
      if (__any_sync(0xFFFFFFFFu, has_tile)) {
        const int4 av = *reinterpret_cast<const int4 *>(s_a + v0);
        const int4 bv = *reinterpret_cast<const int4 *>(s_b + v0);
#pragma unroll 1
        for (int q = 0; q < R / 4; ++q) {
          int Dq[16];
          tmem_ld16(tb + 16 * q, Dq);
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) {
            const int au = s_a[u0 + 4 * q + ii], bu_ = s_b[u0 + 4 * q + ii];
            Dq[4 * ii + 0] += (au - av.x) * (bv.x - bu_);
            Dq[4 * ii + 1] += (au - av.y) * (bv.y - bu_);
            Dq[4 * ii + 2] += (au - av.z) * (bv.z - bu_);
            Dq[4 * ii + 3] += (au - av.w) * (bv.w - bu_);
          }
          tmem_st16(tb + 16 * q, Dq);
        }
      }
    } else {
      if (has_tile) {
        const int4 av = *reinterpret_cast<const int4 *>(s_a + v0);
        const int4 bv = *reinterpret_cast<const int4 *>(s_b + v0);
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const int au = s_a[u0 + i], bu_ = s_b[u0 + i];
          D[i][0] += (au - av.x) * (bv.x - bu_);
          D[i][1] += (au - av.y) * (bv.y - bu_);
          D[i][2] += (au - av.z) * (bv.z - bu_);
          D[i][3] += (au - av.w) * (bv.w - bu_);
        }
      }
    }
    }
    if (mode == 0) {
      if (tid == 0) {
        s_nr[s] = -dlt;
        s_ns[r] = -dlt;
        s_d[r] = dr;
        s_d[s] = ds;
      }
      __syncthreads();
      pend_r = r;
      pend_s = s;
    } else {
      // no barrier: the next window reads d_r, d_s from these registers while
      // thread 0 stores them; the accumulators are cleared after its barrier
      ov_r = r;
      ov_s = s;
      ov_dr = dr;
      ov_ds = ds;
      if (tid == 0) {
        s_d[r] = dr;
        s_d[s] = ds;
      }
    }
    t1_block_end(g, mode, rebuild, warp_mode, blk_it, blk_acc);
  }

  // ---- state back to global memory ----
  if constexpr (TM) {
#pragma unroll 1
    for (int q = 0; q < R / 4; ++q) {
      int Dq[16];
      tmem_ld16(tb + 16 * q, Dq);
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int u = u0 + 4 * q + ii, v = v0 + c;
          if (has_tile && u < v && v < N) g.delta[pidx(N, u, v)] = Dq[4 * ii + c];
        }
    }
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int u = u0 + i, v = v0 + c;
        if (has_tile && u < v && v < N) g.delta[pidx(N, u, v)] = D[i][c];
      }
  }
  __syncthreads();
  {
    const int4 *sB = reinterpret_cast<const int4 *>(s_B);
    int4 *gB = reinterpret_cast<int4 *>(g.Bp);
    for (int i = tid; i < (N * S) >> 4; i += nthreads) gB[i] = sB[i];
  }
  for (int i = tid; i < N; i += nthreads) {
    g.p[i] = s_p[i];
    g.d[i] = s_d[i];
  }
  if (tid == 0) {
    g.st->it = it;
    g.st->accepts = c64[kC64Accepts];
    g.st->cost = (long long)c64[kC64Cost];
    g.st->near_ties += c64[kC64Near];
    g.st->exact_evals += c64[kC64Exact];
    g.st->windows += c64[kC64Windows];
    g.st->direct_iters += c64[kC64DirIt];
    g.st->direct_accepts += c64[kC64DirAcc];
    g.st->warp_iters += c64[kC64WarpIt];
    g.st->mode = mode;
    if (err) g.st->error = err;
  }
}

template <int BOUND>
__global__ void __launch_bounds__(BOUND, 1)
    sa_tier1_kernel(ChainDev g, unsigned long long it_end) {
  extern __shared__ __align__(16) unsigned char smem[];
  if constexpr (BOUND > kT1SmallThreads) {  // 96 registers a thread: tiles in TMEM;
                                            // long rows: 2 lanes per proposal
    __shared__ unsigned s_tmem;
    const unsigned tb = tile_tmem_acquire(&s_tmem, 4 * kT1R);
    t1_run_chain<kT1R, true, 2>(g, it_end, smem, tb);
    tile_tmem_release(&s_tmem);
  } else {
    t1_run_chain<kT1R, false, 1>(g, it_end, smem, 0u);
  }
}

// ------------------------------------------------------------------------- //
// Batch of independent chains (no counterpart in the paper's single-chain
// method; the paper mentions repeated runs of the heuristic only in passing).  A persistent
// grid: every CTA takes the next chain from a work list (longest first) with
// one atomic, runs it to its iteration target with the tier-1 code, and takes
// the next, until the list is empty.
// ------------------------------------------------------------------------- //
struct BatchChain {
  ChainDev g;
  unsigned long long it_end;
  int R;
  int pad;
};

constexpr int kBatchThreads = 640;

__global__ void __launch_bounds__(kBatchThreads, 1)
    sa_batch_kernel(const BatchChain *__restrict__ chains,
                    const int *__restrict__ order, int n, int *counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_next;
  __shared__ unsigned s_tmem;
  const unsigned tb = tile_tmem_acquire(&s_tmem, 4 * kT1R);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    __syncthreads();
    const int k = s_next;
    if (k >= n) break;
    const BatchChain &bc = chains[order[k]];
    t1_run_chain<kT1R, true, 1>(bc.g, bc.it_end, smem, tb);
  }
  tile_tmem_release(&s_tmem);
}

}  // namespace qapsa
