// sa_tier2.cuh -- tier 2 of the SA loop (Paul, arXiv:1208.2675, sections 2.2
// and 3): one chain on a thread-block cluster of C CTAs (C <= 16), for N above
// what one SM holds (up to 1136).
//
// Where the data lives during a run:
//   Delta  Tensor Memory of the cluster: the R x 4 tiles of the upper triangle
//          are split into C contiguous ranges, one per CTA (<= 640 tiles each);
//          thread t keeps its tile in its own TMEM lane, 4R columns, and moves
//          it to registers 4 or 8 rows (16 or 32 cells) at a time;
//   A, B'  shared memory of the cluster: CTA c holds the int8 rows v of its
//          slice [c*NV, (c+1)*NV) of both matrices (row stride S), loaded once
//          per launch; B' rows are written back at the end;
//   a, b, d, p, the recomputed rows, rows r,s of A and B', the threshold
//          table: shared memory of every CTA (each CTA keeps its own copy and
//          updates it identically).
//
// While many proposals are accepted (block acceptance above g.hyb_lo) the
// chain runs in direct mode instead: Delta is not maintained, each CTA
// evaluates the window's proposals whose second row lies in its slice, and an
// accepted swap only updates d, p and B'; the tiles are rebuilt from their
// definition when Delta mode resumes and before the state is stored.
//
// In Delta mode one accepted swap costs two cluster barriers and one CTA barrier:
//   scan    each CTA tests its tiles in the window; warp winners post
//           atomicMin(code) into every CTA's key word (DSMEM)  -> cluster barrier
//   stage   (every CTA) rows r,s of A and of B' before the swap are read from
//           the CTAs that own them (DSMEM) into local copies, and a_k, b_k,
//           d_k, d_r, d_s formed from them                     -> CTA barrier
//   finish  rows r,s of this slice from dot products over local shared memory
//           plus O(1) corrections for the swap, posted into every CTA (DSMEM,
//           16-byte stores); O(1) update of the TMEM cells    -> cluster barrier
// and at the top of the next scan each CTA swaps columns r,s of its B' rows (and
// rewrites rows r,s if it owns them) and copies the recomputed rows into its
// TMEM tiles.  All control decisions are computed identically in every CTA from
// the same data, so the CTAs never diverge and every barrier is reached by all.
// The barriers are hardware cluster barriers: there is no software spin-wait.
#pragma once
#include <cooperative_groups.h>

#include "sa_tier1.cuh"
#include "sa_tmem.cuh"

namespace qapsa {

namespace cg = cooperative_groups;

constexpr int kT2Threads = 640;
constexpr int kT2R = 16;
constexpr int kT2MaxCluster = 16;
constexpr int kT2Tpv = 8;      // the host's ChainDev::tpv (the kernels do not read it)
constexpr int kT2MaxN = 1136;  // 16 CTAs x 640 tiles of 16 x 4 hold N <= 1136

// Shared memory of one CTA.  Everything but the slices of A and B' sits at
// fixed offsets sized for kT2MaxN, so that the compiler addresses it from the
// base with immediates instead of holding a pointer per array in registers.
constexpr int kT2NP = ((kT2MaxN + 15) & ~15) + 16;  // vector length bound
constexpr int kT2MaxS = 1136;                       // row stride bound, 16 x odd
constexpr int kT2OffCtl = 0;
constexpr int kT2OffSlot = 128;
constexpr int kT2OffTt = kT2OffSlot + 16 * 32 * kT2MaxCluster;
constexpr int kT2OffVa = kT2OffTt + 8 * kTabMax;
constexpr int kT2OffVb = kT2OffVa + 4 * kT2NP;
constexpr int kT2OffVd = kT2OffVb + 4 * kT2NP;
constexpr int kT2OffVp = kT2OffVd + 4 * kT2NP;
constexpr int kT2OffVnr = kT2OffVp + 4 * kT2NP;
constexpr int kT2OffVns = kT2OffVnr + 4 * kT2NP;
constexpr int kT2OffRowAr = kT2OffVns + 4 * kT2NP;  // row r of A
constexpr int kT2OffRowAs = kT2OffRowAr + kT2MaxS;  // row s of A
constexpr int kT2OffRowBr = kT2OffRowAs + kT2MaxS;  // row r of B' before the swap
constexpr int kT2OffRowBs = kT2OffRowBr + kT2MaxS;  // row s of B' before the swap
constexpr int kT2OffRowWa = kT2OffRowBs + kT2MaxS;  // direct mode: row cr of A
constexpr int kT2OffRowWb = kT2OffRowWa + kT2MaxS;  // direct mode: row cr of B'
constexpr int kT2OffSlice = kT2OffRowWb + kT2MaxS;  // this CTA's rows of A, then of B'

struct T2Layout {
  int NV;  // rows of A and B' per CTA
  int bytes;
};

// Shared-memory size of one CTA of a C-CTA cluster (S: row stride, a multiple
// of 16 bytes, <= kT2MaxS).
__host__ __device__ inline T2Layout t2_layout(int N, int S, int C) {
  T2Layout L;
  L.NV = (((N + C - 1) / C) + 3) & ~3;  // a multiple of 4: rows are posted in fours
  L.bytes = kT2OffSlice + 2 * L.NV * S;
  return L;
}

// Sums of 16 values over the 32 lanes of a warp in 16 shuffles: lane l returns
// the total of v[((l >> 3) & 3) * 4 + ((l >> 1) & 3)] (lanes l and l ^ 1 alike).
// v is consumed.
__device__ __forceinline__ int reduce_scatter16(int (&v)[16], int lane) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool hi = lane & 16;
    const int send = hi ? v[i] : v[i + 8], keep = hi ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool hi = lane & 8;
    const int send = hi ? v[i] : v[i + 4], keep = hi ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = lane & 4;
    const int send = hi ? v[i] : v[i + 2], keep = hi ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 4);
  }
  {
    const bool hi = lane & 2;
    const int send = hi ? v[0] : v[1], keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 2);
  }
  return v[0] + __shfl_xor_sync(0xFFFFFFFFu, v[0], 1);
}

__device__ __forceinline__ int dot16(int4 x, int4 y, int acc) {
  acc = __dp4a(x.x, y.x, acc);
  acc = __dp4a(x.y, y.y, acc);
  acc = __dp4a(x.z, y.z, acc);
  return __dp4a(x.w, y.w, acc);
}

// Mode decisions of the cluster tier at the end of a block of kHybBlock
// iterations (every thread of every CTA alike): to direct mode above
// 4 g.hyb_lo, back to Delta mode (Delta rebuilt first) below g.hyb_lo where
// allow_back.  With the host's rebuild a launch stops to resume Delta mode, and
// only one that started in direct mode may stop: the host queues two launches
// per piece of a run, and the second starts in Delta mode or at the end.
__device__ __forceinline__ void t2_block_end(const ChainDev &g, int &mode, bool &rebuild,
                                             bool allow_back, int &blk_it, int &blk_acc,
                                             int mb, int &cr, int &cs, int &wrow) {
  if (blk_it < kHybBlock) return;
  if (mode == 1 && (float)blk_acc < g.hyb_lo * (float)blk_it) {
    if (allow_back) {
      mode = 0;
      rebuild = true;  // in the tiles, or (host rebuild) by stopping the launch
    }
  } else if (mode == 0 && g.hyb_lo > 0.0f && (float)blk_acc > 4.0f * g.hyb_lo * (float)blk_it) {
    mode = 1;
    decode_pair(g.N, mb, cr, cs);
    wrow = -1;
  }
  blk_it = blk_acc = 0;
}

// Delta of the calling thread's tile from its definition into its TMEM cells,
// Delta_uv = 2 (<A_u, B'_v> + <A_v, B'_u> - d_u - d_v + 2 A_uv B'_uv), from the
// rows of A and B' in global memory (every CTA has written its B' rows there)
// and d.  Every thread of the cluster calls it (the TMEM stores are
// warp-collective), from one call site: when Delta mode resumes and before the
// state is stored after direct mode.
__device__ __forceinline__ void t2_rebuild_tile(const int8_t *A, const int8_t *Bp, const int *d,
                                             int N, int S, int u0, int v0, bool has_tile,
                                             unsigned tb) {
  const int NC = S >> 4;
#pragma unroll 1
  for (int q = 0; q < kT2R / 4; ++q) {
    int Dq[16];
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int u = u0 + 4 * q + ii, v = v0 + c;
        int val = 0;
        if (has_tile && u < v && v < N) {
          const int4 *Au = reinterpret_cast<const int4 *>(A + (size_t)u * S);
          const int4 *Bu = reinterpret_cast<const int4 *>(Bp + (size_t)u * S);
          const int4 *Av = reinterpret_cast<const int4 *>(A + (size_t)v * S);
          const int4 *Bv = reinterpret_cast<const int4 *>(Bp + (size_t)v * S);
          int guv = 0, gvu = 0;
          for (int k = 0; k < NC; ++k) {
            guv = dot16(__ldg(Au + k), __ldcg(Bv + k), guv);
            gvu = dot16(__ldg(Av + k), __ldcg(Bu + k), gvu);
          }
          val = 2 * (guv + gvu - d[u] - d[v] +
                     2 * (int)A[(size_t)u * S + v] * (int)__ldcg(Bp + (size_t)u * S + v));
        }
        Dq[4 * ii + c] = val;
      }
    tmem_st16(tb + 16 * q, Dq);
  }
}

// One chain on the calling cluster.  Every CTA of the cluster must call it with
// the same arguments.
// tb: TMEM address of the calling thread's tile (lane group of its warp,
// first of the warp's 4R columns).  HostRebuild: when Delta mode must resume
// after direct mode the launch stops and the host's queued rebuild_delta_kernel
// and second launch continue (the single-chain kernel); otherwise the tiles
// are rebuilt inside the kernel (the persistent batch kernel).
template <bool HostRebuild>
__device__ __forceinline__ void t2_run_chain(const ChainDev &g,
                                             unsigned long long it_end,
                                             unsigned char *smem, unsigned tb) {
  constexpr int R = kT2R;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int N = g.N, S = g.S, M = g.M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = blockDim.x;
  const T2Layout L = t2_layout(N, S, C);
  const int NV = L.NV;
  int8_t *s_A = reinterpret_cast<int8_t *>(smem + kT2OffSlice);
  int8_t *s_B = s_A + NV * S;
  int *s_a = reinterpret_cast<int *>(smem + kT2OffVa);
  int *s_b = reinterpret_cast<int *>(smem + kT2OffVb);
  int *s_d = reinterpret_cast<int *>(smem + kT2OffVd);
  int *s_p = reinterpret_cast<int *>(smem + kT2OffVp);
  int *s_nr = reinterpret_cast<int *>(smem + kT2OffVnr);
  int *s_ns = reinterpret_cast<int *>(smem + kT2OffVns);
  int8_t *a_r = reinterpret_cast<int8_t *>(smem + kT2OffRowAr);
  int8_t *a_s = reinterpret_cast<int8_t *>(smem + kT2OffRowAs);
  int8_t *o_r = reinterpret_cast<int8_t *>(smem + kT2OffRowBr);
  int8_t *o_s = reinterpret_cast<int8_t *>(smem + kT2OffRowBs);
  int8_t *w_a = reinterpret_cast<int8_t *>(smem + kT2OffRowWa);
  int8_t *w_b = reinterpret_cast<int8_t *>(smem + kT2OffRowWb);
  int4 *s_slot = reinterpret_cast<int4 *>(smem + kT2OffSlot);
  unsigned *s_ctl = reinterpret_cast<unsigned *>(smem + kT2OffCtl);
  float2 *s_tt = reinterpret_cast<float2 *>(smem + kT2OffTt);
  unsigned long long *c64 = reinterpret_cast<unsigned long long *>(s_ctl + 8);
  const int sv_lo = rank * NV, sv_hi = min(N, sv_lo + NV);

  const int NP = t1_vec_len(N);
  for (int i = tid; i < NP; i += nthreads) {
    s_p[i] = i < N ? g.p[i] : 0;
    s_d[i] = i < N ? g.d[i] : 0;
    s_a[i] = 0;
    s_b[i] = 0;
  }
  {  // this CTA's rows of A and B'
    const int n4 = max(0, sv_hi - sv_lo) * (S >> 4);
    const int4 *gA4 = reinterpret_cast<const int4 *>(g.A + (size_t)sv_lo * S);
    const int4 *gB4 = reinterpret_cast<const int4 *>(g.Bp + (size_t)sv_lo * S);
    int4 *lA4 = reinterpret_cast<int4 *>(s_A);
    int4 *lB4 = reinterpret_cast<int4 *>(s_B);
    for (int i = tid; i < n4; i += nthreads) {
      lA4[i] = __ldg(gA4 + i);
      lB4[i] = gB4[i];
    }
  }
  if (tid < 8) s_ctl[tid] = (tid < 3) ? kNone : 0u;
  if (tid == 0) {
    c64[kC64Accepts] = g.st->accepts;
    c64[kC64Cost] = (unsigned long long)g.st->cost;
    c64[kC64Near] = 0;
    c64[kC64Exact] = 0;
    c64[kC64Windows] = 0;
  }

  // ---- this CTA's tiles and slice ----
  const int TP = (g.ntiles + C - 1) / C;
  const int my_tile = rank * TP + tid;
  const bool has_tile = tid < TP && my_tile < g.ntiles;
  int u0 = 0, v0 = 0;
  if (has_tile) {
    const int t = g.tiles[my_tile];
    u0 = t >> 16;
    v0 = t & 0xFFFF;
  }
  // Modes, as in the one-SM tier: 1 = proposals evaluated directly (Delta not
  // maintained), 0 = read from Delta; the tiles are rebuilt from their
  // definition when Delta mode resumes and before the state is stored.
  int mode = (g.hyb_lo > 0.0f) ? g.st->mode : 0;
  const bool allow_back = !HostRebuild || mode == 1;
  bool tiles_valid = (mode == 0);  // the TMEM tiles hold Delta of the current p
  int tm_lo = 0x7FFFFFFF, tm_hi = -1;
#pragma unroll 1
  for (int q = 0; q < R / 4; ++q) {  // cells to TMEM, 4 rows at a time
    int Dq[16];
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int u = u0 + 4 * q + ii, v = v0 + c;
        Dq[4 * ii + c] = 0;
        if (has_tile && u < v && v < N) {
          const int m = pidx(N, u, v);
          if (tiles_valid) Dq[4 * ii + c] = g.delta[m];
          tm_lo = min(tm_lo, m);
          tm_hi = max(tm_hi, m);
        }
      }
    if (tiles_valid) tmem_st16(tb + 16 * q, Dq);
  }
  const int NC = S >> 4;  // 16-byte chunks of a row

  unsigned long long it = g.st->it;
  int err = 0;
  int mb = (int)(it % (unsigned long long)M);
  int K = min(1024, M);
  unsigned wi = 0;
  int pend_r = -1, pend_s = -1;
  unsigned long long tab_it = 0;
  int tab_len = 0;
  int blk_it = 0, blk_acc = 0;  // iterations and accepts of the current block
  bool rebuild = false;         // Delta mode resumes: tiles from their definition first
  int cr = 0, cs = 1;  // direct mode: pair of iteration it
  int wrow = -1;       // direct mode: the row staged in w_a, w_b
  if (mode == 1) decode_pair(N, mb, cr, cs);
  if (tid == 0) {
    c64[kC64DirIt] = 0;
    c64[kC64DirAcc] = 0;
  }
  // every CTA's B' rows to global memory, then every thread's tile from its
  // definition (all threads of the cluster together)
  auto rebuild_tiles = [&]() {
    __syncthreads();  // this CTA's B' swap of the loop top is complete
    const int n4 = max(0, sv_hi - sv_lo) * (S >> 4);
    int4 *gB4 = reinterpret_cast<int4 *>(g.Bp + (size_t)sv_lo * S);
    const int4 *lB4 = reinterpret_cast<const int4 *>(s_B);
    for (int i = tid; i < n4; i += nthreads) gB4[i] = lB4[i];
    __threadfence();
    cluster.sync();  // every CTA's rows written
    t2_rebuild_tile(g.A, g.Bp, s_d, N, S, u0, v0, has_tile, tb);
    cluster.sync();  // every CTA has read them
    tiles_valid = true;
  };
  cluster.sync();  // every CTA initialised before any remote write

  bool last = false;
  for (;;) {  // segments: a rebuild of the tiles between them, out of the window loop
  for (;;) {
    if (pend_r >= 0) {
      const int r = pend_r, s = pend_s;
      // ---- B' swap of the previous accept (Eq. 3), this CTA's rows ----
      for (int v = sv_lo + tid; v < sv_hi; v += nthreads) {
        if (v == r || v == s) continue;
        int8_t *row = s_B + (v - sv_lo) * S;
        const int8_t t = row[r];
        row[r] = row[s];
        row[s] = t;
      }
      if (r >= sv_lo && r < sv_hi) {  // new row r = old row s, columns r,s swapped
        int8_t *row = s_B + (r - sv_lo) * S;
        for (int k = tid; k < N; k += nthreads)
          row[k] = (k == r) ? o_s[s] : (k == s ? o_s[r] : o_s[k]);
      }
      if (s >= sv_lo && s < sv_hi) {  // new row s = old row r, columns r,s swapped
        int8_t *row = s_B + (s - sv_lo) * S;
        for (int k = tid; k < N; k += nthreads)
          row[k] = (k == r) ? o_r[s] : (k == s ? o_r[r] : o_r[k]);
      }
      // ---- recomputed rows/columns r,s -> the TMEM cells (warp-collective),
      //      8 rows at a time (Delta mode) ----
      const bool col_hit = has_tile && ((r >= v0 && r < v0 + 4) || (s >= v0 && s < v0 + 4));
#pragma unroll 1
      for (int h = 0; h < R / 8 && mode == 0 && !rebuild; ++h) {
        const int uh = u0 + 8 * h;
        const bool row_hit = has_tile && ((r >= uh && r < uh + 8) || (s >= uh && s < uh + 8));
        if (!__any_sync(0xFFFFFFFFu, row_hit || col_hit)) continue;
        int Dh[32];
        tmem_ld32(tb + 32 * h, Dh);
        if (row_hit) {
#pragma unroll
          for (int ii = 0; ii < 8; ++ii) {
            const int u = uh + ii;
            if (u == r || u == s) {
              const int *src = (u == r) ? s_nr : s_ns;
#pragma unroll
              for (int c = 0; c < 4; ++c) Dh[4 * ii + c] = src[v0 + c];
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
              for (int ii = 0; ii < 8; ++ii) Dh[4 * ii + c] = src[uh + ii];
            }
          }
        }
        tmem_st32(tb + 32 * h, Dh);
      }
    }
    pend_r = -1;
    last = it >= it_end || err;
    if (last || rebuild) break;

    // ================= scan one window =================
    // direct mode: the window stays in row cr (pairs (cr, cs .. N-1))
    const int wlen = (int)min((unsigned long long)(mode == 1 ? min(K, N - cs) : K), it_end - it);
    const int jt0 = (it >= tab_it && it - tab_it < (unsigned long long)tab_len)
                        ? (int)(it - tab_it) : kTabMax;
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
      // ---- direct mode: each CTA evaluates the proposals (cr, s) whose row s
      //      lies in its slice, eight lanes a proposal:
      //      delta = 2 (<A_r, B'_s> + <A_s, B'_r> - d_r - d_s + 2 A_rs B'_rs) ----
      if (wrow != cr) {  // a new row (the same decision in every CTA): from the
                         // CTA that owns it, once every CTA's loop-top swap is done
        cluster.sync();
        const int q = cr / NV;
        const int *ra = cluster.map_shared_rank(
            reinterpret_cast<const int *>(s_A + (cr - q * NV) * S), q);
        const int *rb = cluster.map_shared_rank(
            reinterpret_cast<const int *>(s_B + (cr - q * NV) * S), q);
        for (int w = tid; w < (S >> 2); w += nthreads) {
          reinterpret_cast<int *>(w_a)[w] = ra[w];
          reinterpret_cast<int *>(w_b)[w] = rb[w];
        }
        wrow = cr;
      }
      __syncthreads();  // window row staged; this CTA's B' swap of the loop top done
      const int jlo = max(0, sv_lo - cs), jhi = min(wlen, sv_hi - cs);
      const int per_pass = nthreads >> 3;  // eight lanes a proposal
      for (int jb = jlo; jb < jhi; jb += per_pass) {  // the same passes in every warp
        const int j = jb + (tid >> 3), sub = tid & 7;
        const bool live = j < jhi;
        int g1 = 0, g2 = 0;
        if (live) {
          const int s = cs + j;
          const int4 *As4 = reinterpret_cast<const int4 *>(s_A + (s - sv_lo) * S);
          const int4 *Bs4 = reinterpret_cast<const int4 *>(s_B + (s - sv_lo) * S);
          const int4 *Ar4 = reinterpret_cast<const int4 *>(w_a);
          const int4 *Br4 = reinterpret_cast<const int4 *>(w_b);
          for (int c = sub; c < NC; c += 8) {
            g1 = dot16(Ar4[c], Bs4[c], g1);
            g2 = dot16(As4[c], Br4[c], g2);
          }
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
          g1 += __shfl_xor_sync(0xFFFFFFFFu, g1, o);
          g2 += __shfl_xor_sync(0xFFFFFFFFu, g2, o);
        }
        if (live && sub == 0) {
          const int s = cs + j;
          const int dv = 2 * (g1 + g2 - s_d[cr] - s_d[s] + 2 * (int)w_a[s] * (int)w_b[s]);
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
            const unsigned o = pretest_cells(g.seed, g.stream, g.log2a_f, g.mrel, it, Tw, j,
                                             0, 0, 0, dv, 0, 0, 0, 1u);
            acc = o & 1u;
            unc = (o >> 4) & 1u;
          }
          const unsigned key = ((unsigned)j << 1) | unc;
          if ((acc | unc) && key < best) {
            best = key;
            bu = cr;
            bv = s;
            bd = dv;
          }
        }
      }
    }
    const bool scan_me = mode == 0 && has_tile && meets_window(tm_lo, tm_hi, mb, wlen, M);
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
                                             Dq[4 * ii + 1], Dq[4 * ii + 2], Dq[4 * ii + 3],
                                             slow);
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
    {
      const unsigned wmin = __reduce_min_sync(0xFFFFFFFFu, best);
      if (wmin != kNone && best == wmin) {
        const int slot = rank * 32 + warp;
        const unsigned code =
            (((((best >> 1) << 4) | (unsigned)rank) << 5 | (unsigned)warp) << 1) |
            (best & 1u);
        for (int q = 0; q < C; ++q) {
          int4 *rs = cluster.map_shared_rank(s_slot, q);
          rs[slot] = make_int4((int)best, bu, bv, bd);
          unsigned *rk = cluster.map_shared_rank(s_ctl, q);
          atomicMin(rk + kT1Key0 + (wi % 3u), code);
        }
      }
    }
    cluster.sync();
    const unsigned code = s_ctl[kT1Key0 + (wi % 3u)];
    if (tid == 0) {
      s_ctl[kT1Key0 + ((wi + 2u) % 3u)] = kNone;
      if (rank == 0) ++c64[kC64Windows];
    }
    ++wi;

    if (code == kNone) {
      mb += wlen;
      if (mb >= M) mb -= M;
      it += (unsigned)wlen;
      K = min(K * 2, M);
      if (mode == 1) {
        if (tid == 0 && rank == 0) c64[kC64DirIt] += (unsigned)wlen;
        decode_pair(N, mb, cr, cs);
      }
      blk_it += wlen;
      t2_block_end(g, mode, rebuild, allow_back, blk_it, blk_acc, mb, cr, cs, wrow);
      continue;
    }
    const int j = (int)(code >> 10);  // code = j | rank (4 bits) | warp (5) | undecided (1)
    const int4 sl = s_slot[(code >> 1) & 511u];
    const int r = sl.y, s = sl.z, dlt = sl.w;
    if (code & 1u) {  // every CTA decides the same binary64 test
      unsigned long long nt = 0;
      const int dec = exact_accept(g.seed, g.stream, g.T0, g.P, dlt, it + (unsigned)j, &nt,
                                   (tid == 0 && rank == 0) ? g.st : nullptr);
      if (tid == 0 && rank == 0) {
        ++c64[kC64Exact];
        c64[kC64Near] += nt;
      }
      cluster.sync();  // every CTA has read the winner's slot before any posts again
      if (!dec) {
        it += (unsigned)j + 1;
        mb += j + 1;
        if (mb >= M) mb -= M;
        if (mode == 1) {
          if (tid == 0 && rank == 0) c64[kC64DirIt] += (unsigned)j + 1;
          decode_pair(N, mb, cr, cs);
        }
        blk_it += j + 1;
        t2_block_end(g, mode, rebuild, allow_back, blk_it, blk_acc, mb, cr, cs, wrow);
        continue;
      }
    }
    if (r < 0 || r >= s || s >= N) {
      err = 1;
      continue;
    }
    if (j < K / 8) K = max(64, K / 2);
    K = min(K, M);
    it += (unsigned)j + 1;
    mb += j + 1;
    if (mb >= M) mb -= M;
    if (tid == 0 && rank == 0) {
      ++c64[kC64Accepts];
      c64[kC64Cost] += (unsigned long long)(long long)dlt;
      if (mode == 1) {
        c64[kC64DirIt] += (unsigned)j + 1;
        ++c64[kC64DirAcc];
      }
    }
    blk_it += j + 1;
    ++blk_acc;
    // direct mode: the row of the next window, old contents, fetched below
    int ncr = r, ncs = s;
    next_pair(N, ncr, ncs);
    if (mode == 1) tiles_valid = false;

    // ---- stage (every CTA): rows r,s of A and of B' before the swap from
    //      the CTAs that own them; a, b, d, d_r, d_s from them ----
    {
      const int qr = r / NV, qs = s / NV;
      const int *Ar = cluster.map_shared_rank(
          reinterpret_cast<const int *>(s_A + (r - qr * NV) * S), qr);
      const int *As = cluster.map_shared_rank(
          reinterpret_cast<const int *>(s_A + (s - qs * NV) * S), qs);
      const int *Br = cluster.map_shared_rank(
          reinterpret_cast<const int *>(s_B + (r - qr * NV) * S), qr);
      const int *Bs = cluster.map_shared_rank(
          reinterpret_cast<const int *>(s_B + (s - qs * NV) * S), qs);
      int *lAr = reinterpret_cast<int *>(a_r), *lAs = reinterpret_cast<int *>(a_s);
      int *lBr = reinterpret_cast<int *>(o_r), *lBs = reinterpret_cast<int *>(o_s);
      const int SW = S >> 2;
      int dr_part = 0, ds_part = 0;
      if (mode == 1) {  // row ncr of A and B' before the swap
        const int qn = ncr / NV;
        const int *Na = cluster.map_shared_rank(
            reinterpret_cast<const int *>(s_A + (ncr - qn * NV) * S), qn);
        const int *Nb = cluster.map_shared_rank(
            reinterpret_cast<const int *>(s_B + (ncr - qn * NV) * S), qn);
        for (int w = tid; w < SW; w += nthreads) {
          reinterpret_cast<int *>(w_a)[w] = Na[w];
          reinterpret_cast<int *>(w_b)[w] = Nb[w];
        }
      }
      for (int w = tid; w < SW; w += nthreads) {
        const int ar = Ar[w], as = As[w], br = Br[w], bs = Bs[w];
        lAr[w] = ar;
        lAs[w] = as;
        lBr[w] = br;
        lBs[w] = bs;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int k = 4 * w + i;
          if (k < N) {
            const int Ark = s8_of(ar, i), Ask = s8_of(as, i);
            const int Brk = s8_of(br, i), Bsk = s8_of(bs, i);
            const int ak = Ark - Ask, bk = Bsk - Brk;
            s_a[k] = 2 * ak;
            s_b[k] = bk;
            if (k != r && k != s) {
              s_d[k] += ak * bk;
              dr_part += Ark * Bsk;
              ds_part += Ask * Brk;
            } else if (k == s) {
              dr_part += Ark * Brk;
            } else {
              ds_part += Ask * Bsk;
            }
          }
        }
      }
      if (tid == 0) {
        const int t = s_p[r];
        s_p[r] = s_p[s];
        s_p[s] = t;
      }
      dr_part = __reduce_add_sync(0xFFFFFFFFu, dr_part);
      ds_part = __reduce_add_sync(0xFFFFFFFFu, ds_part);
      if (lane == 0 && (dr_part | ds_part)) {
        atomicAdd(reinterpret_cast<int *>(s_ctl + kT1Dr), dr_part);
        atomicAdd(reinterpret_cast<int *>(s_ctl + kT1Ds), ds_part);
      }
    }
    __syncthreads();  // rows r,s, a, b, d, d_r, d_s complete

    if (mode == 1) {
      // ---- the next window's row under the new p: B'new_x = B'_pi(x) with
      //      columns r,s exchanged (pi swaps r and s); A is constant ----
      if (ncr == r || ncr == s) {
        const int8_t *src = (ncr == r) ? o_s : o_r;
        for (int k = tid; k < S; k += nthreads)
          w_b[k] = (k == r) ? src[s] : (k == s ? src[r] : src[k]);
      } else if (tid == 0) {
        const int8_t t = w_b[r];
        w_b[r] = w_b[s];
        w_b[s] = t;
      }
      wrow = ncr;
    }

    // ---- rows r,s of this slice under the new p, from dot products on B'
    //      before the swap plus the O(1) terms the swap changes:
    //      <A_r, B'new_v> = <A_r, B_v> + A_rs (B_vr - B_vs),
    //      <A_v, B'new_r> = <A_v, B_s> + (A_vs - A_vr) B_rs, and symmetrically.
    //      Warp w takes slice rows vq .. vq+3 (vq = sv_lo + 4w, then 4 x warps on),
    //      its lanes the 16-byte chunks, so rows r,s of A and B' are read once
    //      per four slice rows; the four results are posted into every CTA as
    //      one 16-byte store per row of values ----
    {
      const int dr = (int)s_ctl[kT1Dr], ds = (int)s_ctl[kT1Ds];
      const int Ars = a_r[s], Brs = o_r[s];
      const int4 *Ar4 = reinterpret_cast<const int4 *>(a_r);
      const int4 *As4 = reinterpret_cast<const int4 *>(a_s);
      const int4 *Br4 = reinterpret_cast<const int4 *>(o_r);
      const int4 *Bs4 = reinterpret_cast<const int4 *>(o_s);
      const int nw = nthreads >> 5;
      for (int vq = sv_lo + 4 * warp; vq < sv_hi && mode == 0; vq += 4 * nw) {
        const int nk = min(4, sv_hi - vq);
        int gk[16];  // [k][<A_r,B_v>, <A_s,B_v>, <A_v,B_s>, <A_v,B_r>], v = vq + k
#pragma unroll
        for (int i = 0; i < 16; ++i) gk[i] = 0;
        for (int c = lane; c < NC; c += 32) {
          const int4 ar = Ar4[c], as = As4[c], br = Br4[c], bs = Bs4[c];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (k < nk) {
              const int row = (vq + k - sv_lo) * S;
              const int4 bv = reinterpret_cast<const int4 *>(s_B + row)[c];
              const int4 av = reinterpret_cast<const int4 *>(s_A + row)[c];
              gk[4 * k + 0] = dot16(ar, bv, gk[4 * k + 0]);
              gk[4 * k + 1] = dot16(as, bv, gk[4 * k + 1]);
              gk[4 * k + 2] = dot16(av, bs, gk[4 * k + 2]);
              gk[4 * k + 3] = dot16(av, br, gk[4 * k + 3]);
            }
          }
        }
        const int tot = reduce_scatter16(gk, lane);
        const int kb = lane & ~7;  // lanes kb .. kb+7 hold row k = lane >> 3
        const int G1 = __shfl_sync(0xFFFFFFFFu, tot, kb);
        const int G2 = __shfl_sync(0xFFFFFFFFu, tot, kb + 2);
        const int G3 = __shfl_sync(0xFFFFFFFFu, tot, kb + 4);
        const int G4 = __shfl_sync(0xFFFFFFFFu, tot, kb + 6);
        const int v = vq + (lane >> 3);
        int nr = 0, ns = 0;
        if (v < sv_hi) {
          if (v == s) {
            nr = -dlt;  // Delta_rs of the new p
          } else if (v == r) {
            ns = -dlt;
          } else {
            const int Avr = a_r[v], Avs = a_s[v];
            const int Bvr = o_r[v], Bvs = o_s[v];
            const int dv = s_d[v];
            nr = 2 * (G1 + Ars * (Bvr - Bvs) + G3 + (Avs - Avr) * Brs - dr - dv +
                      2 * Avr * Bvs);
            ns = 2 * (G2 - Ars * (Bvr - Bvs) + G4 - (Avs - Avr) * Brs - ds - dv +
                      2 * Avs * Bvr);
          }
        }
        const int4 nq = make_int4(__shfl_sync(0xFFFFFFFFu, nr, 0), __shfl_sync(0xFFFFFFFFu, nr, 8),
                                  __shfl_sync(0xFFFFFFFFu, nr, 16), __shfl_sync(0xFFFFFFFFu, nr, 24));
        const int4 sq = make_int4(__shfl_sync(0xFFFFFFFFu, ns, 0), __shfl_sync(0xFFFFFFFFu, ns, 8),
                                  __shfl_sync(0xFFFFFFFFu, ns, 16), __shfl_sync(0xFFFFFFFFu, ns, 24));
        if (lane < C) {  // vq is a multiple of 4: 16-byte aligned
          *reinterpret_cast<int4 *>(cluster.map_shared_rank(s_nr, lane) + vq) = nq;
          *reinterpret_cast<int4 *>(cluster.map_shared_rank(s_ns, lane) + vq) = sq;
        }
      }
    }
    // ---- thresholds of the next window ----
    tab_it = it;
    tab_len = min(K, kTabMax);
    {
      const int o = (int)(it & 3u);
      const int nblk = (tab_len + o + 3) >> 2;
      const int qb = nthreads - 1 - tid;
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
    // ---- O(1) update of the TMEM cells (warp-collective), 8 rows at a time ----
    if (mode == 0 && __any_sync(0xFFFFFFFFu, has_tile)) {
      const int4 av = *reinterpret_cast<const int4 *>(s_a + v0);
      const int4 bv = *reinterpret_cast<const int4 *>(s_b + v0);
#pragma unroll 1
      for (int h = 0; h < R / 8; ++h) {
        int Dh[32];
        tmem_ld32(tb + 32 * h, Dh);
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
          const int au = s_a[u0 + 8 * h + ii], bu_ = s_b[u0 + 8 * h + ii];
          Dh[4 * ii + 0] += (au - av.x) * (bv.x - bu_);
          Dh[4 * ii + 1] += (au - av.y) * (bv.y - bu_);
          Dh[4 * ii + 2] += (au - av.z) * (bv.z - bu_);
          Dh[4 * ii + 3] += (au - av.w) * (bv.w - bu_);
        }
        tmem_st32(tb + 32 * h, Dh);
      }
    }
    if (tid == 0) {
      s_d[r] = (int)s_ctl[kT1Dr];
      s_d[s] = (int)s_ctl[kT1Ds];
    }
    cluster.sync();  // rows r,s delivered everywhere; B' reads of this accept done
    if (tid == 0) {
      s_ctl[kT1Dr] = 0u;
      s_ctl[kT1Ds] = 0u;
    }
    pend_r = r;
    pend_s = s;
    if (mode == 1) {
      cr = ncr;
      cs = ncs;
    }
    t2_block_end(g, mode, rebuild, allow_back, blk_it, blk_acc, mb, cr, cs, wrow);
  }
    // tiles from their definition (the loop top's B' swap done): Delta mode
    // resumes, or the state is about to be stored and Delta was not maintained
    if constexpr (HostRebuild) {
      break;  // Delta in global memory is rebuilt by the host's queued kernel
    } else {
      if (rebuild || !tiles_valid) {
        rebuild_tiles();
        rebuild = false;
      }
      if (last) break;
    }
  }

  // ---- state back to global memory (Delta if the tiles hold it) ----
#pragma unroll 1
  for (int q = 0; q < R / 4 && tiles_valid; ++q) {
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
  __syncthreads();
  {
    const int n4 = max(0, sv_hi - sv_lo) * (S >> 4);
    int4 *gB4 = reinterpret_cast<int4 *>(g.Bp + (size_t)sv_lo * S);
    const int4 *lB4 = reinterpret_cast<const int4 *>(s_B);
    for (int i = tid; i < n4; i += nthreads) gB4[i] = lB4[i];
  }
  if (rank == 0) {
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
      g.st->mode = mode;
      if (!tiles_valid) g.st->need_rebuild = 1;  // host rebuild only (else valid)
      if (err) g.st->error = err;
    }
  }
  cluster.sync();  // no CTA leaves while others may still address its memory
}

// Delta of every pair from its definition under the chain's current B' and d in
// global memory, Delta_uv = 2 (<A_u, B'_v> + <A_v, B'_u> - d_u - d_v + 2 A_uv B'_uv),
// if the last single-chain cluster launch left it stale (grid:
// ceil(N / blockDim) x N).
__global__ void rebuild_delta_kernel(ChainDev g) {
  if (!g.st->need_rebuild) return;
  const int N = g.N, S = g.S;
  const int u = blockIdx.y, v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v <= u || v >= N) return;
  const int4 *Au = reinterpret_cast<const int4 *>(g.A + (size_t)u * S);
  const int4 *Bu = reinterpret_cast<const int4 *>(g.Bp + (size_t)u * S);
  const int4 *Av = reinterpret_cast<const int4 *>(g.A + (size_t)v * S);
  const int4 *Bv = reinterpret_cast<const int4 *>(g.Bp + (size_t)v * S);
  int guv = 0, gvu = 0;
  for (int c = 0; c < (S >> 4); ++c) {
    guv = dot16(__ldg(Au + c), Bv[c], guv);
    gvu = dot16(__ldg(Av + c), Bu[c], gvu);
  }
  g.delta[pidx(N, u, v)] = 2 * (guv + gvu - g.d[u] - g.d[v] +
                                2 * (int)g.A[(size_t)u * S + v] * (int)g.Bp[(size_t)u * S + v]);
}

// Delta in global memory is current again (after rebuild_delta_kernel).
__global__ void clear_rebuild_kernel(ChainStatus *st) {
  st->need_rebuild = 0;
  st->need_bprime = 0;
}

__global__ void __launch_bounds__(kT2Threads, 1)
    sa_tier2_kernel(ChainDev g, unsigned long long it_end) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_tmem;
  const unsigned tb = tile_tmem_acquire(&s_tmem, 4 * kT2R);
  t2_run_chain<true>(g, it_end, smem, tb);
  tile_tmem_release(&s_tmem);
}

// Batch of large chains: each cluster takes chains from a work list.
__global__ void __launch_bounds__(kT2Threads, 1)
    sa_tier2_batch_kernel(const BatchChain *__restrict__ chains,
                          const int *__restrict__ order, int n, int *counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_next;
  __shared__ unsigned s_tmem;
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned tb = tile_tmem_acquire(&s_tmem, 4 * kT2R);
  for (;;) {
    cluster.sync();
    if (cluster.block_rank() == 0 && threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    cluster.sync();
    const int k = *cluster.map_shared_rank(&s_next, 0);
    cluster.sync();  // every CTA has read the index before it can change
    if (k >= n) break;
    const BatchChain &bc = chains[order[k]];
    t2_run_chain<false>(bc.g, bc.it_end, smem, tb);
  }
  tile_tmem_release(&s_tmem);
}

}  // namespace qapsa
