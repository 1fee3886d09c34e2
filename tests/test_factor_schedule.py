"""Model check of the task schedule of the eigen stage's factor launch (CPU).

The launch computes the blocked Cholesky factor A = L L^T of A = M + tau I,
the inverse factor X = L^-1 and T = A^-1 = X^T X as tile tasks that CTAs claim
from one counter; each task waits only for per-tile state words (see
`k_factor` in csrc/k_eig.cu).  This test replays that schedule on small
matrices with tiles of 4: the same task kinds, claim order, wait conditions and
state updates, executed by a pool of W simulated CTAs that each hold one
claimed task and run whichever held task has its conditions met (chosen at
random).  It checks that

  * no pool of at least G + 1 CTAs (G chains) ever stalls: every condition a
    held task waits for is eventually met (the schedule needs no
    co-residency);
  * each read-modify-write finds its tile in exactly the state the conditions
    promise (no update is lost or applied twice);
  * the result is A^-1 to rounding, for single problems and batches of
    problems of different sizes.

It exercises the design, not the CUDA code; the GPU tests check the kernel's
results against the oracle.
"""
import math
import random

import numpy as np
import pytest

BS = 4  # tile size of the model (32 on the GPU)
LAG = 1  # steps by which the inverse-factor tasks trail the Cholesky tasks in claim order


def tri_index(u):
    r = int((math.sqrt(8.0 * u + 1.0) - 1.0) * 0.5)
    while (r + 1) * (r + 2) // 2 <= u:
        r += 1
    while r * (r + 1) // 2 > u:
        r -= 1
    return r, u - r * (r + 1) // 2


def trail_pair(k, t, u):
    """Pair u of a trailing update over t remaining blocks, column by column."""
    a, b = tri_index(t * (t + 1) // 2 - 1 - u)
    return k + 1 + (t - 1 - b), k + 1 + (t - 1 - a)


def _blk(M, i, j):
    return M[i * BS:(i + 1) * BS, j * BS:(j + 1) * BS]


def _set(M, i, j, v):
    M[i * BS:(i + 1) * BS, j * BS:(j + 1) * BS] = v


def run_schedule(nbs, W, G, lag, seed):
    rng = np.random.default_rng(seed)
    K = max(nbs)
    probs = []
    for nb in nbs:
        n = nb * BS
        Gm = rng.standard_normal((n, n))
        A = Gm @ Gm.T + n * np.eye(n)
        probs.append(dict(nb=nb, A=A, F1=A.copy(), F2=np.zeros((n, n)), T=np.full((n, n), np.nan),
                          Dinv=np.zeros((nb, BS, BS)), SA=np.zeros((nb, nb), int), SX=np.zeros((nb, nb), int),
                          ST=np.zeros((nb, nb), int)))

    # claim order: the chains, then per step P, T, S(k - lag), U(k - lag), R(k - lag), then the tail
    def seg(kind, k):
        out = []
        for p, P in enumerate(probs):
            nb = P["nb"]
            if kind == "P":
                cnt = max(0, nb - k - 3)
            elif kind == "T":
                t = max(0, nb - k - 2)
                cnt = t * (t + 1) // 2
            elif not (0 <= k < nb):
                cnt = 0
            elif kind == "S":
                cnt = k + 1
            elif kind == "U":
                cnt = max(0, nb - k - 2) * (k + 1)
            else:
                cnt = (k + 1) * (k + 2) // 2
            out += [(kind, p, k, l) for l in range(cnt)]
        return out

    tasks = [("C", c, 0, 0) for c in range(G)]
    for k in range(K):
        tasks += seg("P", k) + seg("T", k) + seg("S", k - lag) + seg("U", k - lag) + seg("R", k - lag)
    for m in range(lag):
        kk = K - lag + m
        tasks += seg("S", kk) + seg("U", kk) + seg("R", kk)

    def chain(c):
        mine = [q for q in range(len(probs)) if q % G == c]
        for k in range(K):
            for q in mine:
                P = probs[q]
                nb, SA, F1, Dv = P["nb"], P["SA"], P["F1"], P["Dinv"]
                if k >= nb:
                    continue
                b1 = k + 1 < nb
                conds = []
                if k >= 2:
                    conds.append(lambda SA=SA, k=k: SA[k, k] >= k - 1)
                if b1 and k >= 2:
                    conds.append(lambda SA=SA, k=k: SA[k + 1, k] >= k - 1)
                if b1 and k >= 3:
                    conds.append(lambda SA=SA, k=k: SA[k + 1, k - 1] >= k - 2)
                if b1 and k >= 2:
                    conds.append(lambda SA=SA, k=k: SA[k + 1, k - 2] >= k - 1)
                yield conds
                Y = _blk(F1, k, k).copy()
                if k >= 1:
                    Ls = _blk(F1, k, k - 1).copy()
                    Y -= Ls @ Ls.T
                if b1:
                    if k >= 1:  # the second block below the diagonal of the previous column
                        w = _blk(F1, k + 1, k - 1).copy()
                        if k >= 2:
                            w -= _blk(F1, k + 1, k - 2) @ _blk(F1, k - 1, k - 2).T
                        assert SA[k + 1, k - 1] == max(k - 2, 0)
                        _set(F1, k + 1, k - 1, w @ Dv[k - 1].T)
                        SA[k + 1, k - 1] = k
                    W1 = _blk(F1, k + 1, k).copy()
                    if k >= 1:
                        W1 -= _blk(F1, k + 1, k - 1) @ Ls.T
                assert SA[k, k] == max(k - 1, 0)
                Dv[k] = np.linalg.inv(np.linalg.cholesky(Y))
                SA[k, k] = k + 1
                if b1:
                    assert SA[k + 1, k] == max(k - 1, 0)
                    _set(F1, k + 1, k, W1 @ Dv[k].T)
                    SA[k + 1, k] = k + 1

    def task(t):
        kind, p, k, l = t
        if kind == "C":
            yield from chain(p)
            return
        P = probs[p]
        nb, SA, SX, ST, F1, F2, Dv = P["nb"], P["SA"], P["SX"], P["ST"], P["F1"], P["F2"], P["Dinv"]
        if kind == "P":  # tile (i, k), i >= k + 3
            i = k + 3 + l
            conds = [lambda: SA[k, k] >= k + 1]
            if k > 0:
                conds += [lambda: SA[i, k - 1] >= k, lambda: SA[k, k - 1] >= k, lambda: SA[i, k] >= k - 1]
            yield conds
            a = _blk(F1, i, k).copy()
            if k > 0:
                a -= _blk(F1, i, k - 1) @ _blk(F1, k, k - 1).T
            assert SA[i, k] == max(k - 1, 0)
            _set(F1, i, k, a @ Dv[k].T)
            SA[i, k] = k + 1
        elif kind == "T":  # A_ij -= L_ik L_jk^T, j >= k + 2
            i, j = trail_pair(k + 1, nb - k - 2, l)
            yield [lambda: SA[i, k] >= k + 1, lambda: SA[j, k] >= k + 1, lambda: SA[i, j] >= k]
            assert SA[i, j] == k
            _set(F1, i, j, _blk(F1, i, j) - _blk(F1, i, k) @ _blk(F1, j, k).T)
            SA[i, j] = k + 1
        elif kind == "S":  # row k of X = L^-1
            j = l
            conds = [lambda: SA[k, k] >= k + 1]
            if j < k:
                conds += [lambda: SA[k, k - 1] >= k, lambda: SX[k - 1, j] >= k - j, lambda: SX[k, j] >= k - 1 - j]
            yield conds
            if j < k:
                assert SX[k, j] == k - 1 - j
                cur = _blk(F2, k, j) - _blk(F1, k, k - 1) @ _blk(F2, k - 1, j)
            else:
                cur = np.eye(BS)
            _set(F2, k, j, Dv[k] @ cur)
            SX[k, j] = k - j + 1
        elif kind == "U":  # X_ij -= L_ik X_kj, i >= k + 2
            i, j = k + 2 + l // (k + 1), l % (k + 1)
            yield [lambda: SX[k, j] >= k - j + 1, lambda: SA[i, k] >= k + 1, lambda: SX[i, j] >= k - j]
            assert SX[i, j] == k - j
            _set(F2, i, j, _blk(F2, i, j) - _blk(F1, i, k) @ _blk(F2, k, j))
            SX[i, j] = k - j + 1
        else:  # R: row k's share of T_ij
            i, j = tri_index(l)
            yield [lambda: SX[k, i] >= k - i + 1, lambda: SX[k, j] >= k - j + 1, lambda: ST[i, j] >= k - i]
            assert ST[i, j] == k - i
            c = _blk(F2, k, i).T @ _blk(F2, k, j)
            _set(P["T"], i, j, c if k == i else _blk(P["T"], i, j) + c)
            if k == nb - 1 and i != j:
                _set(P["T"], j, i, _blk(P["T"], i, j).T)
            ST[i, j] = k - i + 1

    rnd = random.Random(seed)
    nxt, running = 0, []
    while nxt < len(tasks) or running:
        while len(running) < W and nxt < len(tasks):
            gen = task(tasks[nxt])
            nxt += 1
            try:
                running.append([gen, next(gen)])
            except StopIteration:
                pass
        ready = [r for r in running if all(c() for c in r[1])]
        assert ready, "the schedule stalled"
        r = rnd.choice(ready)
        try:
            r[1] = next(r[0])
        except StopIteration:
            running.remove(r)
    worst = 0.0
    for P in probs:
        assert not np.isnan(P["T"]).any()
        Ai = np.linalg.inv(P["A"])
        worst = max(worst, float(np.abs(P["T"] - Ai).max() / np.abs(Ai).max()))
    return worst


@pytest.mark.parametrize("nbs", [[1], [2], [3], [5], [8], [1, 3], [4, 2, 6], [7, 7, 1, 2]])
def test_schedule_never_stalls_and_gives_the_inverse(nbs):
    for G in sorted({1, len(nbs)}):
        for W in (G + 1, G + 2, G + 5, 64):
            assert run_schedule(nbs, W, G, LAG, seed=sum(nbs) * 7 + W + G) <= 1e-13


def test_trail_pairs_enumerate_the_trailing_block_column_first():
    for nb in (3, 6, 9):
        for k in range(nb - 1):
            t = nb - k - 2
            pairs = [trail_pair(k + 1, t, u) for u in range(t * (t + 1) // 2)]
            assert sorted(pairs) == sorted((i, j) for i in range(k + 2, nb) for j in range(k + 2, i + 1))
            if pairs:
                assert pairs[0] == (k + 2, k + 2)
