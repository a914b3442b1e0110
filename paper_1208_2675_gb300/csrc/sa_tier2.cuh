// sa_tier2.cuh -- tier 2 of the SA loop (Paul, arXiv:1208.2675, sections 2.2
// and 3): one chain on a thread-block cluster of C CTAs (C <= 16), for N above
// what one SM holds (up to ~1100).
//
// Where the data lives during a run:
//   Delta  registers of the cluster: the R x 4 tiles of the upper triangle are
//          split into C contiguous ranges, one per CTA (<= 640 tiles each);
//   A, B'  global memory (int8 rows of stride S, L2-resident); CTA c owns the
//          rows v of its slice [c*NV, (c+1)*NV) for the rows-r,s recompute and
//          for the column swaps of B';
//   a, b, d, p, the two recomputed rows, the threshold table: shared memory of
//          every CTA (each CTA keeps its own copy and updates it identically).
//
// One accepted swap costs two cluster barriers:
//   scan    each CTA tests its tiles in the window; warp winners post
//           atomicMin(code) into every CTA's key word (DSMEM)  -> cluster barrier
//   stage   (every CTA) a_k, b_k, d_k from rows r,s of B' before the swap
//           || dot products of the rows-r,s recompute for this CTA's slice,
//           on B' before the swap                            -> CTA barrier
//   finish  rows r,s of this slice = dot products + O(1) corrections for the
//           swap, posted into every CTA (DSMEM); O(1) update of the register
//           cells                                            -> cluster barrier
// and at the top of the next scan each CTA swaps columns r,s of its B' rows (and
// rewrites rows r,s if it owns them) and copies the recomputed rows into its
// registers.  All control decisions are computed identically in every CTA from
// the same data, so the CTAs never diverge and every barrier is reached by all.
// The barriers are hardware cluster barriers: there is no software spin-wait.
#pragma once
#include <cooperative_groups.h>

#include "sa_tier1.cuh"

namespace qapsa {

namespace cg = cooperative_groups;

constexpr int kT2Threads = 640;
constexpr int kT2R = 16;
constexpr int kT2MaxCluster = 16;

struct T2Layout {
  int off_a, off_b, off_d, off_p, off_nr, off_ns, off_or, off_os, off_slot, off_ctl, off_tt;
  int bytes;
};

__host__ __device__ inline T2Layout t2_layout(int N) {
  const int NP = t1_vec_len(N);
  T2Layout L;
  int o = 0;
  L.off_a = o;    o += 4 * NP;
  L.off_b = o;    o += 4 * NP;
  L.off_d = o;    o += 4 * NP;
  L.off_p = o;    o += 4 * NP;
  L.off_nr = o;   o += 4 * NP;
  L.off_ns = o;   o += 4 * NP;
  L.off_or = o;   o += align16(NP);           // row r of B' before the swap
  L.off_os = o;   o += align16(NP);           // row s of B' before the swap
  L.off_slot = o; o += 16 * 32 * kT2MaxCluster;
  L.off_ctl = o;  o += 128;
  L.off_tt = o;   o += 8 * kTabMax;
  L.bytes = o;
  return L;
}

// One chain on the calling cluster.  Every CTA of the cluster must call it with
// the same arguments.
__device__ __forceinline__ void t2_run_chain(const ChainDev &g,
                                             unsigned long long it_end,
                                             unsigned char *smem) {
  constexpr int R = kT2R;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int N = g.N, S = g.S, M = g.M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = blockDim.x;
  const T2Layout L = t2_layout(N);
  int *s_a = reinterpret_cast<int *>(smem + L.off_a);
  int *s_b = reinterpret_cast<int *>(smem + L.off_b);
  int *s_d = reinterpret_cast<int *>(smem + L.off_d);
  int *s_p = reinterpret_cast<int *>(smem + L.off_p);
  int *s_nr = reinterpret_cast<int *>(smem + L.off_nr);
  int *s_ns = reinterpret_cast<int *>(smem + L.off_ns);
  int8_t *s_or = reinterpret_cast<int8_t *>(smem + L.off_or);
  int8_t *s_os = reinterpret_cast<int8_t *>(smem + L.off_os);
  int4 *s_slot = reinterpret_cast<int4 *>(smem + L.off_slot);
  unsigned *s_ctl = reinterpret_cast<unsigned *>(smem + L.off_ctl);
  float2 *s_tt = reinterpret_cast<float2 *>(smem + L.off_tt);
  unsigned long long *c64 = reinterpret_cast<unsigned long long *>(s_ctl + 8);
  const int8_t *gA = g.A;
  int8_t *gB = g.Bp;

  const int NP = t1_vec_len(N);
  for (int i = tid; i < NP; i += nthreads) {
    s_p[i] = i < N ? g.p[i] : 0;
    s_d[i] = i < N ? g.d[i] : 0;
    s_a[i] = 0;
    s_b[i] = 0;
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
  int D[R][4];
  int tm_lo = 0x7FFFFFFF, tm_hi = -1;
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
  const int NV = (N + C - 1) / C;
  const int sv_lo = rank * NV, sv_hi = min(N, sv_lo + NV);
  const int tpv = g.tpv, lpt = 32 / tpv;
  const int t_sl = lane / lpt, v_l = lane - t_sl * lpt;
  const int vslots = (nthreads >> 5) * lpt;
  const int NC = S >> 4;

  unsigned long long it = g.st->it;
  int err = 0;
  int mb = (int)(it % (unsigned long long)M);
  int K = min(1024, M);
  unsigned wi = 0;
  int pend_r = -1, pend_s = -1;
  unsigned long long tab_it = 0;
  int tab_len = 0;
  cluster.sync();  // every CTA initialised before any remote write

  for (;;) {
    if (pend_r >= 0) {
      const int r = pend_r, s = pend_s;
      // ---- B' swap of the previous accept (Eq. 3), this CTA's rows ----
      for (int v = sv_lo + tid; v < sv_hi; v += nthreads) {
        if (v == r || v == s) continue;
        int8_t *row = gB + (size_t)v * S;
        const int8_t t = row[r];
        row[r] = row[s];
        row[s] = t;
      }
      if (r >= sv_lo && r < sv_hi)  // new row r = old row s, columns r,s swapped
        for (int k = tid; k < N; k += nthreads)
          gB[(size_t)r * S + k] = (k == r) ? s_os[s] : (k == s ? s_os[r] : s_os[k]);
      if (s >= sv_lo && s < sv_hi)  // new row s = old row r, columns r,s swapped
        for (int k = tid; k < N; k += nthreads)
          gB[(size_t)s * S + k] = (k == r) ? s_or[s] : (k == s ? s_or[r] : s_or[k]);
      // ---- recomputed rows/columns r,s -> registers ----
      if (has_tile) {
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
    if (it >= it_end || err) break;

    // ================= scan one window =================
    const int wlen = (int)min((unsigned long long)K, it_end - it);
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
    if (has_tile && meets_window(tm_lo, tm_hi, mb, wlen, M)) {
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int u = u0 + i;
        if (u >= N - 1 || u >= v0 + 3) continue;
        const int mrow = u * N - (u * (u + 1)) / 2 - u - 1;
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
      continue;
    }
    const int j = (int)(code >> 10);  // code = j | rank (4 bits) | warp (5) | undecided (1)
    const int4 sl = s_slot[(code >> 1) & 511u];
    const int r = sl.y, s = sl.z, dlt = sl.w;
    if (code & 1u) {  // every CTA decides the same binary64 test
      unsigned long long nt = 0;
      const int dec = exact_accept(g.seed, g.stream, g.T0, g.P, dlt, it + (unsigned)j, &nt);
      if (tid == 0 && rank == 0) {
        ++c64[kC64Exact];
        c64[kC64Near] += nt;
      }
      cluster.sync();  // every CTA has read the winner's slot before any posts again
      if (!dec) {
        it += (unsigned)j + 1;
        mb += j + 1;
        if (mb >= M) mb -= M;
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
    }

    // ---- stage (every CTA): a, b, d from rows r,s of B' before the swap;
    //      N may exceed the CTA's threads ----
    int dr_part = 0, ds_part = 0;
    for (int k = tid; k < N; k += nthreads) {
      const int Ark = __ldg(gA + (size_t)r * S + k), Ask = __ldg(gA + (size_t)s * S + k);
      const int Brk = __ldcg(gB + (size_t)r * S + k), Bsk = __ldcg(gB + (size_t)s * S + k);
      s_or[k] = (int8_t)Brk;
      s_os[k] = (int8_t)Bsk;
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
      if (k == 0) {
        const int t = s_p[r];
        s_p[r] = s_p[s];
        s_p[s] = t;
      }
    }
    dr_part = __reduce_add_sync(0xFFFFFFFFu, dr_part);
    ds_part = __reduce_add_sync(0xFFFFFFFFu, ds_part);
    if (lane == 0 && (dr_part | ds_part)) {
      atomicAdd(reinterpret_cast<int *>(s_ctl + kT1Dr), dr_part);
      atomicAdd(reinterpret_cast<int *>(s_ctl + kT1Ds), ds_part);
    }
    // ---- dot products of this slice on B' before the swap ----
    // slots: v = sv_lo + vb + warp * lpt + v_l for vb = 0, vslots, ...
    constexpr int kMaxPass = 2;
    int G1[kMaxPass], G2[kMaxPass], G3[kMaxPass], G4[kMaxPass];
    {
      const int4 *Ar4 = reinterpret_cast<const int4 *>(gA + (size_t)r * S);
      const int4 *As4 = reinterpret_cast<const int4 *>(gA + (size_t)s * S);
      const int4 *Br4 = reinterpret_cast<const int4 *>(gB + (size_t)r * S);
      const int4 *Bs4 = reinterpret_cast<const int4 *>(gB + (size_t)s * S);
#pragma unroll
      for (int ps = 0; ps < kMaxPass; ++ps) {
        const int v = sv_lo + ps * vslots + warp * lpt + v_l;
        int g1 = 0, g2 = 0, g3 = 0, g4 = 0;
        if (ps * vslots < sv_hi - sv_lo && v < sv_hi) {
          const int4 *Av4 = reinterpret_cast<const int4 *>(gA + (size_t)v * S);
          const int4 *Bv4 = reinterpret_cast<const int4 *>(gB + (size_t)v * S);
#pragma unroll 2
          for (int c = t_sl; c < NC; c += tpv) {
            const int4 bv = Bv4[c];
            int4 x = __ldg(Ar4 + c);
            g1 = __dp4a(x.x, bv.x, g1); g1 = __dp4a(x.y, bv.y, g1);
            g1 = __dp4a(x.z, bv.z, g1); g1 = __dp4a(x.w, bv.w, g1);
            x = __ldg(As4 + c);
            g2 = __dp4a(x.x, bv.x, g2); g2 = __dp4a(x.y, bv.y, g2);
            g2 = __dp4a(x.z, bv.z, g2); g2 = __dp4a(x.w, bv.w, g2);
            const int4 av = __ldg(Av4 + c);
            x = __ldcg(Bs4 + c);
            g3 = __dp4a(av.x, x.x, g3); g3 = __dp4a(av.y, x.y, g3);
            g3 = __dp4a(av.z, x.z, g3); g3 = __dp4a(av.w, x.w, g3);
            x = __ldcg(Br4 + c);
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
        G1[ps] = g1;
        G2[ps] = g2;
        G3[ps] = g3;
        G4[ps] = g4;
      }
    }
    __syncthreads();  // a, b, d, d_r, d_s and the staged rows are complete
    const int dr = (int)s_ctl[kT1Dr], ds = (int)s_ctl[kT1Ds];

    // ---- rows r,s of this slice under the new p, from the dot products on
    //      B' before the swap plus the O(1) terms the swap changes:
    //      <A_r, B'new_v> = <A_r, B_v> + A_rs (B_vr - B_vs),
    //      <A_v, B'new_r> = <A_v, B_s> + (A_vs - A_vr) B_rs, and symmetrically ----
    {
      const int Ars = __ldg(gA + (size_t)r * S + s);
      const int Brs = s_or[s];
#pragma unroll
      for (int ps = 0; ps < kMaxPass; ++ps) {
        const int v = sv_lo + ps * vslots + warp * lpt + v_l;
        if (t_sl == 0 && ps * vslots < sv_hi - sv_lo && v < sv_hi && v != r && v != s) {
          const int Avr = __ldg(gA + (size_t)r * S + v), Avs = __ldg(gA + (size_t)s * S + v);
          const int Bvr = s_or[v], Bvs = s_os[v];
          const int dv = s_d[v];
          const int nr = 2 * (G1[ps] + Ars * (Bvr - Bvs) + G3[ps] + (Avs - Avr) * Brs -
                              dr - dv + 2 * Avr * Bvs);
          const int ns = 2 * (G2[ps] - Ars * (Bvr - Bvs) + G4[ps] - (Avs - Avr) * Brs -
                              ds - dv + 2 * Avs * Bvr);
          for (int q = 0; q < C; ++q) {
            cluster.map_shared_rank(s_nr, q)[v] = nr;
            cluster.map_shared_rank(s_ns, q)[v] = ns;
          }
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
    // ---- O(1) update of the register cells ----
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
    if (tid == 0) {
      s_nr[s] = -dlt;
      s_ns[r] = -dlt;
      s_d[r] = dr;
      s_d[s] = ds;
    }
    cluster.sync();  // rows r,s delivered everywhere; B' reads of this accept done
    if (tid == 0) {
      s_ctl[kT1Dr] = 0u;
      s_ctl[kT1Ds] = 0u;
    }
    pend_r = r;
    pend_s = s;
  }

  // ---- state back to global memory ----
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int u = u0 + i, v = v0 + c;
      if (has_tile && u < v && v < N) g.delta[pidx(N, u, v)] = D[i][c];
    }
  __syncthreads();
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
      if (err) g.st->error = err;
    }
  }
  cluster.sync();  // no CTA leaves while others may still address its memory
}

__global__ void __launch_bounds__(kT2Threads, 1)
    sa_tier2_kernel(ChainDev g, unsigned long long it_end) {
  extern __shared__ __align__(16) unsigned char smem[];
  t2_run_chain(g, it_end, smem);
}

// Batch of large chains: each cluster takes chains from a work list.
__global__ void __launch_bounds__(kT2Threads, 1)
    sa_tier2_batch_kernel(const BatchChain *__restrict__ chains,
                          const int *__restrict__ order, int n, int *counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_next;
  cg::cluster_group cluster = cg::this_cluster();
  for (;;) {
    cluster.sync();
    if (cluster.block_rank() == 0 && threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    cluster.sync();
    const int k = *cluster.map_shared_rank(&s_next, 0);
    if (k >= n) {
      cluster.sync();
      return;
    }
    const BatchChain &bc = chains[order[k]];
    t2_run_chain(bc.g, bc.it_end, smem);
  }
}

}  // namespace qapsa
