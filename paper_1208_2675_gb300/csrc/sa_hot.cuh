// sa_hot.cuh -- the hot phase of a cluster-tier chain (Paul, arXiv:1208.2675,
// sections 2.2 and 3): while many proposals are accepted, one CTA on one SM
// evaluates them directly from the constant matrices A and B and the
// permutation p, and maintains B' = B[p][p] (Eq. 3) only for the row it is
// sweeping.
//
// The cluster kernel pays two cluster barriers and an exchange of rows over
// distributed shared memory for every accepted swap, and a chain that keeps B'
// in memory writes two bytes into every row of B' per accepted swap.  Both set
// the pace while one proposal in three to one in a few hundred is accepted.
// This kernel reads the swap cost of proposal (r, s) as
//   delta = 2 (<A~_r, B_p(s)> + <A_s, B'_r> - d_r - d_s + 2 A_rs B'_rs),
//   A~_r[m] = A[r][q(m)] (q = p^-1), so <A~_r, B_p(s)> = <A_r, B'_s>,
//   B'_r[k] = B[p(r)][p(k)],  d_v = <A_v, B'_v>,
// with A~_r, B'_r, A_r, d, p, q in shared memory.  The proposals of the cyclic
// order run along row r (s = r+1 .. N-1) before moving to row r+1, so A~_r and
// B'_r serve a whole row; each proposal needs rows A_s and B_p(s) of the
// constant matrices, which the kernel streams from global memory (L2) with
// cp.async into a ring of shared-memory slots a pass ahead.  A staged row stays
// valid across accepted swaps of its row sweep: an accepted (r, s*) changes p
// only at r and s*, and the rows still to come have s > s*.
//
//   pass    group g (eight lanes; four groups a warp) takes proposal s of the
//           window [s_cur, s_cur + K) with s = g mod P (P = 4 W): its rows
//           are in slot s mod 2P, and it keeps the copies of s + P issued.
//           The Philox word of the proposal and its binary32 interval for
//           Eq. (2) come from a table that a warp with no proposal in the pass
//           fills for the iterations after it (the group draws them itself when
//           the table has no entry).  The first accepted (or undecided)
//           proposal in sequential order: redux.min per warp, one CTA barrier.
//   accept  (r, s*), from the staged rows of s*: d_k += (A_rk - A_s*k)(B'_s*k
//           - B'_rk) off r, s*; the new B'_r (a gather of B_p(s*) by the new p)
//           into the second buffer; d_r, d_s* by a reduction; two entries of
//           A~_r; then p, q.  One CTA barrier.
//   row     A_r, B_p(r) copied in, A~_r and B'_r gathered through q and p.
//
// Delta and B' in global memory are not maintained: the kernel flags both for
// the host's kernels (B' = B[p][p], then Delta) before the cluster kernel
// resumes.  It runs blocks of kHybBlock iterations and hands the chain over
// for good at the end of the first block whose acceptance rate is below
// hot_lo (below the cluster tier's switch rate g.hyb_lo, in Delta mode).  The
// trajectory is the sequential method's: the same proposals, the same
// decisions.  Symmetric instances with zero diagonals only (the cluster tier's).
#pragma once
#include "sa_tier1.cuh"

namespace qapsa {

constexpr int kHotPPW = 4;        // proposals (groups) per warp
constexpr int kHotLPP = 8;        // lanes per proposal
constexpr int kHotMaxWarps = 16;  // a power of two, as W must be
constexpr int kHotWarpsDefault = 8;
constexpr int kHotTab = 256;      // entries of the table of Eq. (2) intervals
// From whole-piece timings of the N = 1024 schedule, seconds per 1e8
// iterations at acceptance 0.019 / 0.012 / 0.007: this kernel 8.3 / 7.3 /
// 6.7; the cluster kernel maintaining Delta 18.8 / 11.8 / 7.2 (about 10 us per
// accepted swap), in its direct mode 13.7 / - / 5.7.  The kernel keeps the
// chain down to 0.009, the cluster's direct mode takes it from there.
constexpr float kHotRateDefault = 0.009f;

struct HotLayout {
  int off_p, off_q, off_d;                      // int32 vectors
  int off_Ar, off_At, off_Bt0, off_Bt1, off_Br; // int8 rows of S bytes
  int off_key, off_slot, off_red, off_ctl, off_tab;
  int off_ring;                                 // 2P slots of (A_s, B_p(s))
  int bytes;
};

__host__ __device__ inline HotLayout hot_layout(int N, int S, int W) {
  HotLayout L;
  const int NP = t1_vec_len(N);
  const int P = kHotPPW * W;
  int o = 0;
  L.off_p = o;    o += 4 * NP;
  L.off_q = o;    o += 4 * NP;
  L.off_d = o;    o += 4 * NP;
  L.off_Ar = o;   o += S;
  L.off_At = o;   o += S;
  L.off_Bt0 = o;  o += S;
  L.off_Bt1 = o;  o += S;
  L.off_Br = o;   o += S;
  L.off_key = o;  o += 4 * 2 * kHotMaxWarps;
  L.off_slot = o; o += 8 * 2 * kHotMaxWarps;
  L.off_red = o;  o += 8 * kHotMaxWarps;
  L.off_ctl = o;  o += 16;
  o = align16(o);
  L.off_tab = o;  o += 16 * kHotTab;
  L.off_ring = o; o += 2 * P * 2 * S;
  L.bytes = o;
  return L;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
// All but the most recent group of the calling thread's copies are complete.
__device__ __forceinline__ void cp_async_wait_prior() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// The binary32 interval of Eq. (2) for the proposal made at iteration itc.
__device__ __forceinline__ float2 hot_interval(const ChainDev &g, unsigned long long itc) {
  const uint4 x = rng_block(g.seed, g.stream, itc >> 2);
  const float Tc = g.T0f * exp2f(u64_to_f32(itc) * g.log2a_f);
  return accept_interval(g.mrel, Tc, word_of(x, (int)(itc & 3u)));
}

// g: the chain (A with rows of stride S; g.Bp, g.delta not used); B8: the
// constant B with rows of stride S; hot_lo: the acceptance rate below which
// the kernel hands the chain over.  One CTA of 32 W threads, W a power of two
// up to kHotMaxWarps, with hot_layout(N, S, W).bytes of dynamic shared memory.
__global__ void __launch_bounds__(32 * kHotMaxWarps, 1)
    sa_hot_kernel(ChainDev g, const int8_t *__restrict__ B8, unsigned long long it_end,
                  float hot_lo) {
  extern __shared__ __align__(16) unsigned char smem[];
  {
    const ChainStatus *st = g.st;
    if (g.hyb_lo <= 0.0f || hot_lo <= 0.0f || st->mode == 0 || st->hot_off || st->error ||
        st->it >= it_end)
      return;
  }
  const unsigned FULL = 0xFFFFFFFFu;
  const int N = g.N, S = g.S, M = g.M, NC = S >> 4;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthreads = blockDim.x, W = nthreads >> 5;
  const int P = kHotPPW * W;    // proposals a pass covers at most (a power of two)
  const int R = 2 * P;          // ring slots
  const HotLayout L = hot_layout(N, S, W);
  int *s_p = reinterpret_cast<int *>(smem + L.off_p);
  int *s_q = reinterpret_cast<int *>(smem + L.off_q);
  int *s_d = reinterpret_cast<int *>(smem + L.off_d);
  int8_t *s_Ar = reinterpret_cast<int8_t *>(smem + L.off_Ar);  // A_r
  int8_t *s_At = reinterpret_cast<int8_t *>(smem + L.off_At);  // A~_r
  int8_t *s_Bt = reinterpret_cast<int8_t *>(smem + L.off_Bt0); // B'_r (current buffer)
  int8_t *s_Bn = reinterpret_cast<int8_t *>(smem + L.off_Bt1); // B'_r (next buffer)
  int8_t *s_Br = reinterpret_cast<int8_t *>(smem + L.off_Br);  // B_p(r)
  unsigned *s_key = reinterpret_cast<unsigned *>(smem + L.off_key);
  int2 *s_slot = reinterpret_cast<int2 *>(smem + L.off_slot);
  int2 *s_red = reinterpret_cast<int2 *>(smem + L.off_red);
  int *s_dec = reinterpret_cast<int *>(smem + L.off_ctl);
  // interval of the proposal at iteration i in entry i mod kHotTab: (lo, hi,
  // the low 32 bits of i, unused)
  float4 *s_tab = reinterpret_cast<float4 *>(smem + L.off_tab);
  int8_t *s_ring = reinterpret_cast<int8_t *>(smem + L.off_ring);
  const int8_t *gA = g.A;

  const int NP = t1_vec_len(N);
  for (int i = tid; i < NP; i += nthreads) {
    s_p[i] = i < N ? g.p[i] : 0;
    s_d[i] = i < N ? g.d[i] : 0;
  }
  for (int k = N + tid; k < S; k += nthreads) s_Bn[k] = 0;  // padding of the second buffer
  for (int i = tid; i < kHotTab; i += nthreads)
    s_tab[i] = make_float4(0.0f, 0.0f, __uint_as_float(~(unsigned)i), 0.0f);  // no entry
  __syncthreads();
  for (int i = tid; i < N; i += nthreads) s_q[s_p[i]] = i;

  unsigned long long it = g.st->it;
  const unsigned long long it_start = it;
  int r, s_cur;  // the row being swept and the next proposal's column
  decode_pair(N, (int)(it % (unsigned long long)M), r, s_cur);
  // thread 0's counters
  unsigned long long n_acc = 0, n_pass = 0, n_exact = 0, n_near = 0;
  long long d_cost = 0;
  int blk_it = 0, blk_acc = 0, mode = 1, err = 0;
  bool handover = false;
  unsigned par = 0;
  int K = min(32, P);  // proposals evaluated in a pass (adapted like a window)
  int dR = 0;          // d_r of the row being swept
  const int grp = lane >> 3, sub = lane & (kHotLPP - 1);
  const int G = warp * kHotPPW + grp;  // this group's residue of s mod P
  int nx = 0;                          // the group's next s not yet issued

  // copies of the rows of proposal s into its slot (by the eight lanes of its group)
  auto issue = [&](int s) {
    int8_t *dst = s_ring + (size_t)(s & (R - 1)) * (2 * S);
    const int8_t *srcA = gA + (size_t)s * S;
    const int8_t *srcB = B8 + (size_t)s_p[s] * S;
    for (int c = sub; c < NC; c += kHotLPP) {
      cp_async16(dst + 16 * c, srcA + 16 * c);
      cp_async16(dst + S + 16 * c, srcB + 16 * c);
    }
  };
  bool new_row = true;

  while (it < it_end) {
    if (new_row) {
      // ================= start of row r at column s_cur =================
      __syncthreads();  // A~_r, B'_r, p, q and the slots of the previous row settled
      const int8_t *ra = gA + (size_t)r * S;
      const int8_t *rb = B8 + (size_t)s_p[r] * S;
      for (int c = tid; c < 2 * NC; c += nthreads) {
        if (c < NC) cp_async16(s_Ar + 16 * c, ra + 16 * c);
        else cp_async16(s_Br + 16 * (c - NC), rb + 16 * (c - NC));
      }
      // this group's first proposal of the row and the one a pass later
      const int s0 = s_cur + ((G - s_cur) & (P - 1));
      if (s0 < N) issue(s0);
      if (s0 + P < N) issue(s0 + P);
      nx = s0 + 2 * P;
      cp_async_commit();
      cp_async_wait_all();
      __syncthreads();
      for (int k = tid; k < S; k += nthreads) {
        s_At[k] = k < N ? s_Ar[s_q[k]] : (int8_t)0;
        s_Bt[k] = k < N ? s_Br[s_p[k]] : (int8_t)0;
      }
      dR = s_d[r];
      new_row = false;
      __syncthreads();
    }
    // ================= one pass: proposals s_cur .. s_cur + plen - 1 =================
    const int plen = (int)min((unsigned long long)min(K, N - s_cur), it_end - it);
    const int j = (G - s_cur) & (P - 1);  // this group's offset in the pass
    const int sg = s_cur + j;             // and its proposal
    const bool live = j < plen;
    // keep the group's next proposal staged a pass ahead
    while (nx <= sg + P && nx < N) {
      issue(nx);
      nx += P;
    }
    cp_async_commit();
    float2 bnd = make_float2(0.0f, 0.0f);
    int dsg = 0;
    if (__any_sync(FULL, live)) {
      // Eq. (2) interval of this proposal (from the table when an idle warp
      // has drawn it) and d_s while the copies complete
      if (live && sub == 0) {
        const unsigned long long itc = it + (unsigned)j;
        const float4 e = s_tab[itc & (kHotTab - 1)];
        if (__float_as_uint(e.z) == (unsigned)itc) {
          bnd = make_float2(e.x, e.y);
        } else {
          bnd = hot_interval(g, itc);
          s_tab[itc & (kHotTab - 1)] = make_float4(bnd.x, bnd.y, __uint_as_float((unsigned)itc), 0.0f);
        }
        dsg = s_d[sg];
      }
    } else {
      // an idle warp: the first idle one draws the intervals of the 128
      // iterations after the pass (the next passes' windows lie in them)
      int first_idle = -1;
      for (int w = 0; w < W && first_idle < 0; ++w) {
        const int jmin = (4 * w - s_cur) & (P - 1);  // offsets of its groups: jmin .. jmin+3 mod P
        bool any_live = false;
#pragma unroll
        for (int gg = 0; gg < kHotPPW; ++gg) any_live |= ((jmin + gg) & (P - 1)) < plen;
        if (!any_live) first_idle = w;
      }
      if (warp == first_idle) {
        const unsigned long long a = it + (unsigned)plen;
        const unsigned long long q = (a >> 2) + (unsigned)lane;
        const uint4 x = rng_block(g.seed, g.stream, q);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const unsigned long long itc = (q << 2) + (unsigned)w;
          if (itc < a) continue;  // inside this pass: its groups draw them
          const float Tc = g.T0f * exp2f(u64_to_f32(itc) * g.log2a_f);
          const float2 b = accept_interval(g.mrel, Tc, word_of(x, w));
          s_tab[itc & (kHotTab - 1)] = make_float4(b.x, b.y, __uint_as_float((unsigned)itc), 0.0f);
        }
      }
    }
    cp_async_wait_prior();  // the copies of proposal sg (issued a pass or more ago)
    __syncwarp();
    int g1 = 0, g2 = 0;
    int ab = 0;  // A_rs B'_rs, loaded with the rows
    if (live) {
      if (sub == 0) ab = (int)s_Ar[sg] * (int)s_Bt[sg];
      const int8_t *slot = s_ring + (size_t)(sg & (R - 1)) * (2 * S);
      const int4 *As4 = reinterpret_cast<const int4 *>(slot);
      const int4 *Bs4 = reinterpret_cast<const int4 *>(slot + S);
      const int4 *At4 = reinterpret_cast<const int4 *>(s_At);
      const int4 *Bt4 = reinterpret_cast<const int4 *>(s_Bt);
      int a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
#pragma unroll 3
      for (int c = sub; c < NC; c += kHotLPP) {
        const int4 x = At4[c], y = Bs4[c], u = As4[c], v = Bt4[c];
        a0 = __dp4a(x.x, y.x, a0);  // <A~_r, B_p(s)> = <A_r, B'_s>
        a1 = __dp4a(x.y, y.y, a1);
        a2 = __dp4a(x.z, y.z, a2);
        a3 = __dp4a(x.w, y.w, a3);
        b0 = __dp4a(u.x, v.x, b0);  // <A_s, B'_r>
        b1 = __dp4a(u.y, v.y, b1);
        b2 = __dp4a(u.z, v.z, b2);
        b3 = __dp4a(u.w, v.w, b3);
      }
      g1 = (a0 + a1) + (a2 + a3);
      g2 = (b0 + b1) + (b2 + b3);
    }
    int gs = g1 + g2;
#pragma unroll
    for (int o = 1; o < kHotLPP; o <<= 1) gs += __shfl_xor_sync(FULL, gs, o);
    unsigned best = kNone;
    int dv = 0;
    if (live && sub == 0) {
      dv = 2 * (gs - dR - dsg + 2 * ab);
      const float df = (float)dv;
      unsigned acc = 0, unc = 0;
      if (dv <= 0 || df < bnd.x) acc = 1u;
      else if (!(df > bnd.y)) unc = 1u;
      if (acc | unc) best = ((unsigned)j << 1) | unc;
    }
    const unsigned wmin = __reduce_min_sync(FULL, best);
    if (best != kNone && best == wmin) s_slot[par * kHotMaxWarps + warp] = make_int2(sg, dv);
    if (lane == 0) s_key[par * kHotMaxWarps + warp] = wmin;
    __syncthreads();  // keys, slots, the table (and thread 0's d, p, q of the last swap)
    const unsigned code =
        __reduce_min_sync(FULL, lane < W ? s_key[par * kHotMaxWarps + lane] : kNone);
    const unsigned pp = par;
    par ^= 1u;
    if (tid == 0) ++n_pass;

    if (code == kNone) {
      it += (unsigned)plen;
      s_cur += plen;
      blk_it += plen;
      K = min(2 * K, P);
    } else {
      const int jw = (int)(code >> 1);
      const int s_old = s_cur;
      // the winner's warp: its group is (s_old + jw) mod P
      const int2 sl = s_slot[pp * kHotMaxWarps + ((s_old + jw) & (P - 1)) / kHotPPW];
      const int ss = sl.x, dlt = sl.y;
      bool take = true;
      if (code & 1u) {  // undecided by the binary32 pre-test: binary64
        if (tid == 0) {
          ++n_exact;
          *s_dec = exact_accept(g.seed, g.stream, g.T0, g.P, dlt, it + (unsigned)jw, &n_near,
                                g.st);
        }
        __syncthreads();
        take = *s_dec != 0;
      }
      if (ss != s_old + jw || ss <= r || ss >= N) {
        err = 1;
        break;
      }
      it += (unsigned)jw + 1;
      s_cur = ss + 1;
      blk_it += jw + 1;
      if (take) {
        // ================= accept the swap (r, ss) =================
        if (jw < K / 8) K = max(4, K / 2);
        ++blk_acc;
        if (tid == 0) {
          ++n_acc;
          d_cost += dlt;
        }
        const int8_t *slot = s_ring + (size_t)(ss & (R - 1)) * (2 * S);
        const int8_t *As = slot, *Bps = slot + S;  // A_ss and B_p(ss)
        const int pr = s_p[r], ps = s_p[ss];
        int dr_part = 0, ds_part = 0;
        // four columns k0 .. k0+3 a thread: words of A_r, A_ss, B'_r, four of p
        // and d; the padding columns (k >= N) keep B'_r = 0 and d unchanged
        for (int k0 = 4 * tid; k0 < N; k0 += 4 * nthreads) {
          const int4 p4 = *reinterpret_cast<const int4 *>(s_p + k0);
          const int arw = *reinterpret_cast<const int *>(s_Ar + k0);
          const int asw = *reinterpret_cast<const int *>(As + k0);
          const int btw = *reinterpret_cast<const int *>(s_Bt + k0);
          const int4 dq = *reinterpret_cast<const int4 *>(s_d + k0);
          const int pk[4] = {p4.x, p4.y, p4.z, p4.w};
          int dd[4] = {dq.x, dq.y, dq.z, dq.w};
          unsigned bn = 0;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int k = k0 + c;
            if (k >= N) break;
            const bool off = k != r && k != ss;
            // the new B'_r[k] = B[p'(r)][p'(k)], p'(r) = p(ss), p' = p swapped at r, ss
            const int gk = Bps[off ? pk[c] : (k == r ? ps : pr)];
            bn |= ((unsigned)gk & 0xFFu) << (8 * c);
            const int ark = s8_of(arw, c), ask = s8_of(asw, c), btk = s8_of(btw, c);
            // the new B'_ss[k] = B[p(r)][p'(k)]: the old B'_r at k with r, ss exchanged
            const int bto = off ? btk : (int)s_Bt[k == r ? ss : r];
            dr_part += ark * gk;
            ds_part += ask * bto;
            if (off) dd[c] += (ark - ask) * (gk - btk);  // the old B'_ss,k is gk here
          }
          *reinterpret_cast<unsigned *>(s_Bn + k0) = bn;
          *reinterpret_cast<int4 *>(s_d + k0) = make_int4(dd[0], dd[1], dd[2], dd[3]);
        }
        if (tid == 0) {  // A~_r[m] = A[r][q'(m)]: q'(p(r)) = ss, q'(p(ss)) = r
          s_At[pr] = s_Ar[ss];
          s_At[ps] = s_Ar[r];
        }
        dr_part = __reduce_add_sync(FULL, dr_part);
        ds_part = __reduce_add_sync(FULL, ds_part);
        if (lane == 0) s_red[warp] = make_int2(dr_part, ds_part);
        __syncthreads();  // d, the new B'_r, A~_r, the partial sums
        // every warp sums the W partial sums at once (lane w loads warp w's)
        const int2 v = lane < W ? s_red[lane] : make_int2(0, 0);
        const int dr = __reduce_add_sync(FULL, v.x);
        const int ds = __reduce_add_sync(FULL, v.y);
        dR = dr;
        int8_t *t = s_Bt;
        s_Bt = s_Bn;
        s_Bn = t;
        if (tid == 0) {  // read again only after the next pass's barrier
          s_d[r] = dr;
          s_d[ss] = ds;
          s_p[r] = ps;
          s_p[ss] = pr;
          s_q[ps] = r;
          s_q[pr] = ss;
        }
      }
    }
    if (s_cur >= N) {  // the row is done: the next row of the cyclic order
      if (++r >= N - 1) r = 0;
      s_cur = r + 1;
      new_row = true;
    }
    // ---- block end: hand over below hot_lo, in Delta mode below g.hyb_lo ----
    if (blk_it >= kHybBlock) {
      if ((float)blk_acc < g.hyb_lo * (float)blk_it) {
        mode = 0;
        handover = true;
      } else if ((float)blk_acc < hot_lo * (float)blk_it) {
        handover = true;
      }
      blk_it = blk_acc = 0;
      if (handover) break;
    }
  }

  // ---- state back to global memory; B' and Delta are rebuilt by the host's kernels ----
  cp_async_wait_all();
  __syncthreads();
  for (int i = tid; i < N; i += nthreads) {
    g.p[i] = s_p[i];
    g.d[i] = s_d[i];
  }
  if (tid == 0) {
    ChainStatus *st = g.st;
    st->it = it;
    st->accepts += n_acc;
    st->cost += d_cost;
    st->near_ties += n_near;
    st->exact_evals += n_exact;
    st->windows += n_pass;
    st->direct_iters += it - it_start;
    st->direct_accepts += n_acc;
    st->hot_iters += it - it_start;
    st->hot_accepts += n_acc;
    st->mode = mode;
    st->need_rebuild = 1;
    st->need_bprime = 1;
    if (handover) st->hot_off = 1;
    if (err) st->error = err;
  }
}

// B'[x][y] = B[p(x)][p(y)] (Eq. 3) from the constant B and the current p, if
// the hot-phase kernel left B' in global memory stale (grid: ceil(S / blockDim)
// x N; the padding columns are zero).
__global__ void hot_bprime_kernel(ChainDev g, const int8_t *__restrict__ B8) {
  if (!g.st->need_bprime) return;
  const int N = g.N, S = g.S;
  const int x = blockIdx.y, y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= S) return;
  g.Bp[(size_t)x * S + y] = y < N ? B8[(size_t)g.p[x] * S + g.p[y]] : (int8_t)0;
}

// B as int8 rows of stride S (zero padding), for the hot-phase kernel
// (grid: ceil(S / blockDim) x N; the entries have been checked to fit int8).
__global__ void hot_pack_b_kernel(const int *B32, int N, int S, int8_t *B8) {
  const int x = blockIdx.y, y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= S) return;
  B8[(size_t)x * S + y] = y < N ? (int8_t)B32[(size_t)x * N + y] : (int8_t)0;
}

}  // namespace qapsa
