/*
 * qap_oracle.c -- plain CPU oracle for Delta-matrix simulated annealing (SA)
 * on the quadratic assignment problem, after G. Paul, "A GPU implementation of
 * the Simulated Annealing Heuristic for the Quadratic Assignment Problem"
 * (arXiv:1208.2675).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  The product
 * (the CUDA library under paper_1208_2675_gb300/) never loads it and shares no
 * code, header, table or helper with it.
 *
 * Written to be read against the paper, not to be fast:
 *   - one thread, no blocking, no vector tricks;
 *   - Delta is a full N x N int64 matrix;
 *   - B is always indexed through the permutation, B[p[i]][p[j]]: the oracle
 *     keeps no B' matrix (Eq. 3 is a GPU data-layout device of the paper, not
 *     part of what the method computes);
 *   - floating point is IEEE binary64; build with -ffp-contract=off.
 *
 * What each function follows:
 *   orc_cost                Eq. (1), section 1.
 *   orc_swap_cost_change    C(p o (r s)) - C(p) by Eq. (1) twice (brute force).
 *   orc_delta_entry         closed form of the same change for symmetric,
 *                           zero-diagonal A and B (derived from Eq. (1); the
 *                           paper cites Taillard for it and prints no formula).
 *   orc_delta_entry_general the same change for any A and B (asymmetric,
 *                           nonzero diagonals): the general swap cost, derived
 *                           from Eq. (1) the same way.
 *   orc_philox4x32_10       Philox4x32-10 of Salmon et al., SC'11 ("Parallel
 *                           random numbers: as easy as 1, 2, 3").
 *   orc_uniform             the uniform r of Eq. (2), section 2.1.
 *   orc_sched_*             geometric cooling, lowered at every iteration (sec. 2.1).
 *   orc_chain_run           the Delta-matrix approach, steps (a)-(e) of
 *                           section 2.2, with the acceptance test of Eq. (2);
 *                           or the traditional SA of section 2.1 (delta from
 *                           scratch for every proposal).
 *
 * Each side counts the binary64 tests of Eq. (2) with |delta + T ln u| below
 * 1e-9 T ("near-ties", where two libm logs could decide differently) and logs
 * the iterations of the first ones (orc_chain_set_near_log).
 *
 * Readings where the paper is silent (each is stated where it is used):
 *   R1 proposals: sequential cyclic enumeration of pairs r<s, row-major,
 *      pair(it) = pair number (it mod M), M = N(N-1)/2 (sec. 2.1, sec. 3(ii)).
 *   R2 r of Eq. (2): u = (x + 0.5) * 2^-32 with x the 32-bit Philox word for
 *      iteration it; a word exists for every iteration, used or not.
 *   R3 acceptance: delta <= 0 is always accepted (e^0 = 1 > r for r < 1);
 *      otherwise accept iff (double)delta < -(T(it) * log(u)).
 *   R4 cooling: T(it) = T0 * alpha^it evaluated as a product of per-byte
 *      tables built by repeated squaring (orc_sched_build).
 *   R5 relative temperatures: T0 = t0 * (sum_{r<s} |Delta0_rs|) / M,
 *      Tf = tf * T0; an instance with Delta0 == 0 everywhere uses t0, tf as
 *      absolute temperatures.
 *   R6 random proposal order (section 2.1 allows drawing the pair at random), chosen with
 *      orc_chain_set_order: the pair proposed at iteration it is pair number
 *      m = (x * M) >> 32 of the row-major enumeration, x word 0 of
 *      Philox4x32-10(counter = (it low, it high, stream, 1), key = seed).
 *   R7 general instances: when A or B is not symmetric with a zero diagonal,
 *      the swap costs and their update use the general forms
 *      (orc_delta_entry_general, orc_apply_swap), else the symmetric ones.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Eq. (1): C = sum_i sum_j A[i][j] * B[p(i)][p(j)].                          */
/* ------------------------------------------------------------------------ */
EXPORT int64_t orc_cost(int32_t N, const int32_t *A, const int32_t *B,
                        const int32_t *p) {
  int64_t c = 0;
  for (int32_t i = 0; i < N; ++i)
    for (int32_t j = 0; j < N; ++j)
      c += (int64_t)A[(int64_t)i * N + j] *
           (int64_t)B[(int64_t)p[i] * N + p[j]];
  return c;
}

/* Brute force: the cost change of exchanging the locations of facilities r
 * and s, evaluated as Eq. (1) after the exchange minus Eq. (1) before it. */
EXPORT int64_t orc_swap_cost_change(int32_t N, const int32_t *A,
                                    const int32_t *B, const int32_t *p,
                                    int32_t r, int32_t s) {
  int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  memcpy(q, p, sizeof(int32_t) * (size_t)N);
  int32_t t = q[r];
  q[r] = q[s];
  q[s] = t;
  int64_t d = orc_cost(N, A, B, q) - orc_cost(N, A, B, p);
  free(q);
  return d;
}

/* Closed form of the same change for symmetric A, B with zero diagonal.
 * Only terms of Eq. (1) with i or j in {r, s} change; pairing (r,k) with
 * (k,r) and (s,k) with (k,s) through the symmetry, and noting that the
 * (r,s)/(s,r) terms cancel, leaves
 *   Delta_rs = 2 * sum_{k not in {r,s}} (A[k][r] - A[k][s]) *
 *                                      (B[p(k)][p(s)] - B[p(k)][p(r)]).     */
EXPORT int64_t orc_delta_entry(int32_t N, const int32_t *A, const int32_t *B,
                               const int32_t *p, int32_t r, int32_t s) {
  int64_t acc = 0;
  for (int32_t k = 0; k < N; ++k) {
    if (k == r || k == s) continue;
    int64_t a = (int64_t)A[(int64_t)k * N + r] - A[(int64_t)k * N + s];
    int64_t b = (int64_t)B[(int64_t)p[k] * N + p[s]] -
                B[(int64_t)p[k] * N + p[r]];
    acc += a * b;
  }
  return 2 * acc;
}

/* The same change for any A and B.  Write B'[x][y] = B[p(x)][p(y)].  The
 * terms of Eq. (1) with neither index in {r, s} do not change; those with one
 * index in {r, s} give, for every other k, the row and the column sums below;
 * the four terms with both indices in {r, s} give the first two products:
 *   Delta_rs = (A[r][r] - A[s][s]) (B'[s][s] - B'[r][r])
 *            + (A[r][s] - A[s][r]) (B'[s][r] - B'[r][s])
 *            + sum_{k not in {r,s}} (A[r][k] - A[s][k]) (B'[s][k] - B'[r][k])
 *                                 + (A[k][r] - A[k][s]) (B'[k][s] - B'[k][r]). */
EXPORT int64_t orc_delta_entry_general(int32_t N, const int32_t *A,
                                       const int32_t *B, const int32_t *p,
                                       int32_t r, int32_t s) {
#define ORC_A(i, j) ((int64_t)A[(int64_t)(i) * N + (j)])
#define ORC_BP(i, j) ((int64_t)B[(int64_t)p[i] * N + p[j]])
  int64_t d = (ORC_A(r, r) - ORC_A(s, s)) * (ORC_BP(s, s) - ORC_BP(r, r)) +
              (ORC_A(r, s) - ORC_A(s, r)) * (ORC_BP(s, r) - ORC_BP(r, s));
  for (int32_t k = 0; k < N; ++k) {
    if (k == r || k == s) continue;
    d += (ORC_A(r, k) - ORC_A(s, k)) * (ORC_BP(s, k) - ORC_BP(r, k)) +
         (ORC_A(k, r) - ORC_A(k, s)) * (ORC_BP(k, s) - ORC_BP(k, r));
  }
#undef ORC_A
#undef ORC_BP
  return d;
}

/* 1 if A and B are both symmetric with a zero diagonal (the instance family of
 * section 4), for which orc_delta_entry holds. */
static int orc_is_symmetric_family(int32_t N, const int32_t *A, const int32_t *B) {
  for (int32_t i = 0; i < N; ++i) {
    if (A[(int64_t)i * N + i] != 0 || B[(int64_t)i * N + i] != 0) return 0;
    for (int32_t j = i + 1; j < N; ++j)
      if (A[(int64_t)i * N + j] != A[(int64_t)j * N + i] ||
          B[(int64_t)i * N + j] != B[(int64_t)j * N + i])
        return 0;
  }
  return 1;
}

/* Step (a) of section 2.2: the matrix of the costs of every possible swap
 * under the current assignment p.  Full symmetric N x N, zero diagonal. */
EXPORT void orc_delta_matrix(int32_t N, const int32_t *A, const int32_t *B,
                             const int32_t *p, int64_t *D) {
  for (int32_t r = 0; r < N; ++r) {
    D[(int64_t)r * N + r] = 0;
    for (int32_t s = r + 1; s < N; ++s) {
      int64_t d = orc_delta_entry(N, A, B, p, r, s);
      D[(int64_t)r * N + s] = d;
      D[(int64_t)s * N + r] = d;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  One round maps the      */
/* counter (c0,c1,c2,c3) with key (k0,k1) to                                   */
/*   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));         */
/* the key is advanced by the Weyl constants between rounds.                   */
/* ------------------------------------------------------------------------ */
EXPORT void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                              uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* R2: the 32-bit word for iteration `it` of stream `stream` under `seed`:
 * counter = (it/4 low, it/4 high, stream, 0), key = (seed low, seed high),
 * word it mod 4 of the block. */
EXPORT uint32_t orc_rand_word(uint64_t seed, uint32_t stream, uint64_t it) {
  uint64_t blk = it / 4u;
  uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)(blk >> 32), stream, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[it % 4u];
}

/* The uniform r of Eq. (2): (x + 0.5) / 2^32, strictly inside (0, 1) and
 * exact in binary64. */
EXPORT double orc_uniform(uint64_t seed, uint32_t stream, uint64_t it) {
  return ((double)orc_rand_word(seed, stream, it) + 0.5) * 0x1p-32;
}

/* ------------------------------------------------------------------------ */
/* R4: geometric cooling T(it) = T0 * alpha^it, alpha = (Tf/T0)^(1/(I-1)).     */
/* alpha^it is formed without pow/exp per iteration so that any two programs   */
/* that follow these steps get the same binary64 value:                        */
/*   q[0] = alpha, q[i] = q[i-1] * q[i-1]                 (alpha^(2^i))        */
/*   P[b][v] = product over set bits i of v, ascending, of q[8b + i],          */
/*             starting from 1.0                          (alpha^(v * 256^b))  */
/*   T(it) = T0 * P[7][byte 7 of it] * ... * P[0][byte 0 of it], multiplied    */
/*           left to right (high byte first).                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  double T0, Tf, alpha;
  uint64_t I;
  double q[64];
  double P[8][256];
} orc_sched;

static void orc_sched_build(orc_sched *S, double T0, double Tf, uint64_t I) {
  S->T0 = T0;
  S->Tf = Tf;
  S->I = I;
  S->alpha = (I >= 2) ? pow(Tf / T0, 1.0 / (double)(I - 1)) : 1.0;
  S->q[0] = S->alpha;
  for (int i = 1; i < 64; ++i) S->q[i] = S->q[i - 1] * S->q[i - 1];
  for (int b = 0; b < 8; ++b) {
    for (int v = 0; v < 256; ++v) {
      double x = 1.0;
      for (int i = 0; i < 8; ++i)
        if ((v >> i) & 1) x = x * S->q[8 * b + i];
      S->P[b][v] = x;
    }
  }
}

static double orc_sched_T(const orc_sched *S, uint64_t it) {
  double T = S->T0;
  for (int b = 7; b >= 0; --b) T = T * S->P[b][(it >> (8 * b)) & 0xFFu];
  return T;
}

/* ------------------------------------------------------------------------ */
/* One SA chain.                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t N;
  int64_t M;
  int32_t *A, *B, *p;
  int64_t *D;       /* full symmetric Delta, N x N */
  int64_t cost;     /* Eq. (1) of p, kept as cost += delta on accept */
  uint64_t it;      /* iterations done so far */
  uint64_t accepts; /* accepted swaps so far */
  uint64_t near_ties;
  uint64_t seed;
  uint32_t stream;
  int32_t cur_r, cur_s; /* pair(it mod M) */
  orc_sched S;
  int check;            /* brute-force check after every accepted swap */
  int64_t check_failures;
  uint64_t *log;        /* iteration index of each accepted swap */
  uint64_t log_cap, log_n;
  uint64_t *nlog;       /* iteration index of each near-tie (R3) */
  uint64_t nlog_cap;
  int32_t general;      /* R7: the general swap-cost forms are in use */
  int32_t random_order; /* R6: proposals drawn at random */
} orc_chain;

static void orc_pair_of(int32_t N, int64_t m, int32_t *r, int32_t *s) {
  int32_t row = 0;
  while (m >= (int64_t)(N - 1 - row)) {
    m -= (N - 1 - row);
    ++row;
  }
  *r = row;
  *s = row + 1 + (int32_t)m;
}

EXPORT orc_chain *orc_chain_create(int32_t N, const int32_t *A,
                                   const int32_t *B, const int32_t *p0,
                                   double t0, double tf, uint64_t total_iters,
                                   int32_t relative, uint64_t seed,
                                   uint32_t stream) {
  if (N < 2) return NULL;
  orc_chain *c = (orc_chain *)calloc(1, sizeof(orc_chain));
  size_t n2 = (size_t)N * (size_t)N;
  c->N = N;
  c->M = (int64_t)N * (N - 1) / 2;
  c->A = (int32_t *)malloc(sizeof(int32_t) * n2);
  c->B = (int32_t *)malloc(sizeof(int32_t) * n2);
  c->p = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  c->D = (int64_t *)malloc(sizeof(int64_t) * n2);
  memcpy(c->A, A, sizeof(int32_t) * n2);
  memcpy(c->B, B, sizeof(int32_t) * n2);
  memcpy(c->p, p0, sizeof(int32_t) * (size_t)N);
  /* Step (a): initial Delta and the cost of Eq. (1). */
  c->general = !orc_is_symmetric_family(N, c->A, c->B);
  if (c->general) {
    for (int32_t r = 0; r < N; ++r) {
      c->D[(int64_t)r * N + r] = 0;
      for (int32_t s = r + 1; s < N; ++s) {
        int64_t d = orc_delta_entry_general(N, c->A, c->B, c->p, r, s);
        c->D[(int64_t)r * N + s] = d;
        c->D[(int64_t)s * N + r] = d;
      }
    }
  } else {
    orc_delta_matrix(N, c->A, c->B, c->p, c->D);
  }
  c->cost = orc_cost(N, c->A, c->B, c->p);
  double T0 = t0, Tf = tf;
  if (relative) { /* R5 */
    int64_t sum = 0;
    for (int32_t r = 0; r < N; ++r)
      for (int32_t s = r + 1; s < N; ++s) {
        int64_t d = c->D[(int64_t)r * N + s];
        sum += d < 0 ? -d : d;
      }
    double mean = (sum > 0) ? (double)sum / (double)c->M : 1.0;
    T0 = t0 * mean;
    Tf = tf * T0;
  }
  orc_sched_build(&c->S, T0, Tf, total_iters);
  c->seed = seed;
  c->stream = stream;
  c->it = 0;
  c->cur_r = 0;
  c->cur_s = 1;
  return c;
}

EXPORT void orc_chain_destroy(orc_chain *c) {
  if (!c) return;
  free(c->A);
  free(c->B);
  free(c->p);
  free(c->D);
  free(c->log);
  free(c->nlog);
  free(c);
}

EXPORT void orc_chain_set_check(orc_chain *c, int32_t on) { c->check = on; }

/* R6: 1 = proposals drawn at random, 0 = sequential cyclic order (default). */
EXPORT void orc_chain_set_order(orc_chain *c, int32_t random_order) {
  c->random_order = random_order ? 1 : 0;
}

EXPORT int32_t orc_chain_is_general(const orc_chain *c) { return c->general; }
EXPORT int64_t orc_chain_check_failures(const orc_chain *c) {
  return c->check_failures;
}

EXPORT void orc_chain_set_log(orc_chain *c, uint64_t cap) {
  free(c->log);
  c->log = cap ? (uint64_t *)malloc(sizeof(uint64_t) * cap) : NULL;
  c->log_cap = cap;
  c->log_n = 0;
}

EXPORT uint64_t orc_chain_get_log(const orc_chain *c, uint64_t *out,
                                  uint64_t cap) {
  uint64_t n = c->log_n < cap ? c->log_n : cap;
  if (n) memcpy(out, c->log, sizeof(uint64_t) * n);
  return c->log_n;
}

/* The iteration indices of the first near-ties (cap of them are kept; the
 * count, near_ties, is kept in full). */
EXPORT void orc_chain_set_near_log(orc_chain *c, uint64_t cap) {
  free(c->nlog);
  c->nlog = cap ? (uint64_t *)malloc(sizeof(uint64_t) * cap) : NULL;
  c->nlog_cap = cap;
}

EXPORT uint64_t orc_chain_get_near_log(const orc_chain *c, uint64_t *out,
                                       uint64_t cap) {
  uint64_t n = c->near_ties < c->nlog_cap ? c->near_ties : c->nlog_cap;
  if (n > cap) n = cap;
  if (n) memcpy(out, c->nlog, sizeof(uint64_t) * n);
  return c->near_ties;
}

EXPORT void orc_chain_schedule(const orc_chain *c, double *T0, double *Tf,
                               double *alpha) {
  *T0 = c->S.T0;
  *Tf = c->S.Tf;
  *alpha = c->S.alpha;
}

EXPORT double orc_chain_temperature(const orc_chain *c, uint64_t it) {
  return orc_sched_T(&c->S, it);
}

EXPORT void orc_chain_state(const orc_chain *c, int32_t *p_out, int64_t *cost,
                            uint64_t *accepts, uint64_t *it,
                            uint64_t *near_ties) {
  memcpy(p_out, c->p, sizeof(int32_t) * (size_t)c->N);
  *cost = c->cost;
  *accepts = c->accepts;
  *it = c->it;
  *near_ties = c->near_ties;
}

EXPORT void orc_chain_delta(const orc_chain *c, int64_t *D_out) {
  memcpy(D_out, c->D, sizeof(int64_t) * (size_t)c->N * (size_t)c->N);
}

/* R3: the test of Eq. (2) for the proposal made at iteration `it`. */
static int orc_accept(orc_chain *c, int64_t delta, uint64_t it) {
  if (delta <= 0) return 1;
  double u = orc_uniform(c->seed, c->stream, it);
  double T = orc_sched_T(&c->S, it);
  double prod = T * log(u);
  if (fabs((double)delta + prod) < 1e-9 * T) {
    if (c->nlog && c->near_ties < c->nlog_cap) c->nlog[c->near_ties] = it;
    c->near_ties++;
  }
  return (double)delta < -prod;
}

/* R3 for a given (delta, it) under the chain's schedule and random stream:
 * 1 if the proposal is accepted.  Changes nothing but the near-tie count. */
EXPORT int32_t orc_chain_accepts(orc_chain *c, int64_t delta, uint64_t it) {
  return orc_accept(c, delta, it);
}

/* Step (d) of section 2.2 for the accepted swap (r, s) with cost change delta:
 * update p, and update Delta to the swap costs under the new p.
 *  - A cell (u,v) with {u,v} and {r,s} disjoint changes in O(1): only the
 *    k = r and k = s terms of its sum see different B entries, giving
 *      Delta_uv += 2 (A_ru - A_rv - A_su + A_sv)
 *                   (B_{p(s)p(v)} - B_{p(s)p(u)} - B_{p(r)p(v)} + B_{p(r)p(u)})
 *    with p the assignment BEFORE the swap.
 *  - A cell in row or column r or s is recomputed from its definition with the
 *    assignment AFTER the swap. */
static void orc_apply_swap(orc_chain *c, int32_t r, int32_t s, int64_t delta) {
  const int32_t N = c->N;
  const int32_t *A = c->A, *B = c->B;
  int32_t *p = c->p;
  int64_t *D = c->D;
  const int32_t pr = p[r], ps = p[s];
  for (int32_t u = 0; u < N; ++u) {
    if (u == r || u == s) continue;
    for (int32_t v = u + 1; v < N; ++v) {
      if (v == r || v == s) continue;
      int64_t a = (int64_t)A[(int64_t)r * N + u] - A[(int64_t)r * N + v] -
                  A[(int64_t)s * N + u] + A[(int64_t)s * N + v];
      int64_t b = (int64_t)B[(int64_t)ps * N + p[v]] -
                  B[(int64_t)ps * N + p[u]] - B[(int64_t)pr * N + p[v]] +
                  B[(int64_t)pr * N + p[u]];
      D[(int64_t)u * N + v] += 2 * a * b;
      D[(int64_t)v * N + u] = D[(int64_t)u * N + v];
    }
  }
  p[r] = ps;
  p[s] = pr;
  c->cost += delta;
  for (int32_t v = 0; v < N; ++v) {
    if (v != r) {
      int64_t d = orc_delta_entry(N, A, B, p, r, v);
      D[(int64_t)r * N + v] = d;
      D[(int64_t)v * N + r] = d;
    }
    if (v != s) {
      int64_t d = orc_delta_entry(N, A, B, p, s, v);
      D[(int64_t)s * N + v] = d;
      D[(int64_t)v * N + s] = d;
    }
  }
  c->accepts++;
}

/* The same step for general A and B (R7).  A cell (u,v) disjoint from {r,s}
 * sees different B entries only in the k = r and k = s terms of its row sum
 * and of its column sum (orc_delta_entry_general), which gives, with p the
 * assignment BEFORE the swap and B'[x][y] = B[p(x)][p(y)],
 *   Delta_uv += (A[r][u] - A[r][v] - A[s][u] + A[s][v])
 *               (B'[s][v] - B'[s][u] - B'[r][v] + B'[r][u])
 *             + (A[u][r] - A[v][r] - A[u][s] + A[v][s])
 *               (B'[v][s] - B'[u][s] - B'[v][r] + B'[u][r]);
 * with A, B symmetric the two products are equal (the symmetric form).  Cells
 * in rows or columns r, s are recomputed from the definition after the swap. */
static void orc_apply_swap_general(orc_chain *c, int32_t r, int32_t s, int64_t delta) {
  const int32_t N = c->N;
  const int32_t *A = c->A, *B = c->B;
  int32_t *p = c->p;
  int64_t *D = c->D;
#define ORC_A(i, j) ((int64_t)A[(int64_t)(i) * N + (j)])
#define ORC_BP(i, j) ((int64_t)B[(int64_t)p[i] * N + p[j]])
  for (int32_t u = 0; u < N; ++u) {
    if (u == r || u == s) continue;
    for (int32_t v = u + 1; v < N; ++v) {
      if (v == r || v == s) continue;
      int64_t a1 = ORC_A(r, u) - ORC_A(r, v) - ORC_A(s, u) + ORC_A(s, v);
      int64_t b1 = ORC_BP(s, v) - ORC_BP(s, u) - ORC_BP(r, v) + ORC_BP(r, u);
      int64_t a2 = ORC_A(u, r) - ORC_A(v, r) - ORC_A(u, s) + ORC_A(v, s);
      int64_t b2 = ORC_BP(v, s) - ORC_BP(u, s) - ORC_BP(v, r) + ORC_BP(u, r);
      D[(int64_t)u * N + v] += a1 * b1 + a2 * b2;
      D[(int64_t)v * N + u] = D[(int64_t)u * N + v];
    }
  }
#undef ORC_A
#undef ORC_BP
  const int32_t t = p[r];
  p[r] = p[s];
  p[s] = t;
  c->cost += delta;
  for (int32_t v = 0; v < N; ++v) {
    if (v != r) {
      int64_t d = orc_delta_entry_general(N, A, B, p, r, v);
      D[(int64_t)r * N + v] = d;
      D[(int64_t)v * N + r] = d;
    }
    if (v != s) {
      int64_t d = orc_delta_entry_general(N, A, B, p, s, v);
      D[(int64_t)s * N + v] = d;
      D[(int64_t)v * N + s] = d;
    }
  }
  c->accepts++;
}

/* R6: the pair proposed at iteration it under random order. */
static void orc_random_pair(const orc_chain *c, uint64_t it, int32_t *r, int32_t *s) {
  uint32_t ctr[4] = {(uint32_t)it, (uint32_t)(it >> 32), c->stream, 1u};
  uint32_t key[2] = {(uint32_t)c->seed, (uint32_t)(c->seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  int64_t m = (int64_t)(((uint64_t)out[0] * (uint64_t)c->M) >> 32);
  orc_pair_of(c->N, m, r, s);
}

/* The pair the chain proposes at iteration it (R1 or R6); for sequential order
 * this is pair number it mod M. */
EXPORT void orc_chain_proposal(const orc_chain *c, uint64_t it, int32_t *r, int32_t *s) {
  if (c->random_order)
    orc_random_pair(c, it, r, s);
  else
    orc_pair_of(c->N, (int64_t)(it % (uint64_t)c->M), r, s);
}

static void orc_check_state(orc_chain *c) {
  const int32_t N = c->N;
  if (orc_cost(N, c->A, c->B, c->p) != c->cost) c->check_failures++;
  for (int32_t r = 0; r < N; ++r)
    for (int32_t s = r + 1; s < N; ++s)
      if (orc_swap_cost_change(N, c->A, c->B, c->p, r, s) !=
          c->D[(int64_t)r * N + s])
        c->check_failures++;
}

static void orc_advance_cursor(orc_chain *c) {
  c->cur_s++;
  if (c->cur_s == c->N) {
    c->cur_r++;
    c->cur_s = c->cur_r + 1;
    if (c->cur_r == c->N - 1) {
      c->cur_r = 0;
      c->cur_s = 1;
    }
  }
}

/* Steps (b)-(e) of section 2.2 for `iters` more iterations.  With
 * `traditional` set, delta is computed from scratch by Eq. (1) for every
 * proposal (section 2.1) and Delta is not used. */
EXPORT int32_t orc_chain_run(orc_chain *c, uint64_t iters,
                             int32_t traditional) {
  const int32_t N = c->N;
  orc_pair_of(N, (int64_t)(c->it % (uint64_t)c->M), &c->cur_r, &c->cur_s);
  uint64_t end = c->it + iters;
  for (; c->it < end; c->it++) {
    int32_t r = c->cur_r, s = c->cur_s;
    orc_advance_cursor(c);
    if (c->random_order) orc_random_pair(c, c->it, &r, &s);
    int64_t delta = traditional
                        ? orc_swap_cost_change(N, c->A, c->B, c->p, r, s)
                        : c->D[(int64_t)r * N + s];
    if (!orc_accept(c, delta, c->it)) continue;
    if (c->log && c->log_n < c->log_cap) c->log[c->log_n] = c->it;
    if (c->log) c->log_n++;
    if (traditional) {
      int32_t t = c->p[r];
      c->p[r] = c->p[s];
      c->p[s] = t;
      c->cost += delta;
      c->accepts++;
    } else {
      if (c->general)
        orc_apply_swap_general(c, r, s, delta);
      else
        orc_apply_swap(c, r, s, delta);
      if (c->check) orc_check_state(c);
    }
  }
  return 0;
}
