"""The identities the cluster tier's hot-phase kernel evaluates (reading R12),
checked on the CPU against Eq. (1) by brute force.

The kernel never forms B' = B[p][p]; it reads the swap cost of proposal (r, s)
as 2 (<A~_r, B_p(s)> + <A_s, B'_r> - d_r - d_s + 2 A_rs B'_rs) with
A~_r[m] = A[r][q(m)] (q = p^-1), B'_r[k] = B[p(r)][p(k)] and d_v = <A_v, B'_v>,
and after an accepted swap (r, s) it updates, from the row B_p(s) alone:
  B'_r(new)[k] = B_p(s)[p'(k)],  p' = p with r, s exchanged;
  d_k += (A_rk - A_sk)(B'_sk - B'_rk) for k off r, s (B' before the swap);
  d_r = <A_r, B'_r(new)>,  d_s = <A_s, B'_r(old) with entries r, s exchanged>;
  A~_r[p(r)] = A_rs, A~_r[p(s)] = A_rr.
This restates those steps in numpy and compares every quantity with its
definition after each step of random sweeps along rows (symmetric instances
with a zero diagonal, the cluster tier's family).
"""
import numpy as np
import pytest


def cost(A, B, p):  # Eq. (1)
    return int((A * B[np.ix_(p, p)]).sum())


def swap_cost(A, B, p, r, s):
    q = p.copy()
    q[r], q[s] = q[s], q[r]
    return cost(A, B, q) - cost(A, B, p)


def sym(rng, N, lo, hi):
    M = rng.integers(lo, hi, (N, N))
    M = np.triu(M, 1)
    return M + M.T


@pytest.mark.parametrize("N,seed", [(2, 1), (3, 2), (7, 3), (16, 4), (23, 5)])
def test_row_sweep_identities_match_the_definitions(N, seed):
    rng = np.random.default_rng([seed, N, 0xB07])
    A, B = sym(rng, N, -9, 10), sym(rng, N, -9, 10)
    p = rng.permutation(N)
    d = np.array([int(A[v] @ B[p[v]][p]) for v in range(N)])
    checked = 0
    for sweep in range(3 * N):
        r = sweep % max(1, N - 1)
        if N < 2:
            break
        q = np.argsort(p)
        Ar, At, Bt, dR = A[r].copy(), A[r][q].copy(), B[p[r]][p].copy(), d[r]
        for s in range(r + 1, N):
            Bps, As = B[p[s]], A[s]
            dv = 2 * (int(At @ Bps) + int(As @ Bt) - dR - d[s] + 2 * Ar[s] * Bt[s])
            assert dv == swap_cost(A, B, p, r, s)
            checked += 1
            if rng.random() < 0.4:  # accept, whatever the criterion says
                pr, ps = p[r], p[s]
                Bn, dn = np.zeros(N, np.int64), d.copy()
                dr = ds = 0
                for k in range(N):
                    off = k != r and k != s
                    gk = Bps[p[k] if off else (ps if k == r else pr)]
                    Bn[k] = gk
                    bto = Bt[k if off else (s if k == r else r)]
                    dr += Ar[k] * gk
                    ds += As[k] * bto
                    if off:
                        dn[k] += (Ar[k] - As[k]) * (gk - Bt[k])
                At[pr], At[ps] = Ar[s], Ar[r]
                dn[r], dn[s] = dr, ds
                p[r], p[s] = ps, pr
                d, dR, Bt = dn, dr, Bn
                q = np.argsort(p)
                assert np.array_equal(At, A[r][q])
                assert np.array_equal(Bt, B[p[r]][p])
                assert np.array_equal(d, [int(A[v] @ B[p[v]][p]) for v in range(N)])
    assert checked >= 3 * (N - 1)
