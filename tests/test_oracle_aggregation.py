"""Pins of the oracle's aggregation rules (§5.2 and §5.3 use an AMG of each block; the build restates it
as smoothed aggregation with a deterministic distance-2 maximal independent set).

The rules under test:
  * strength: j is strong for i when max(|a_ij|, |a_ji|) >= theta * sqrt(|a_ii a_jj|) (per node, |a| is
    the sum over the nc components); rows with no strong connection are not aggregated;
  * priority key of row i on level l: (splitmix64((l << 32) | i) >> 33, i), compared as one integer;
  * synchronous rounds: an undecided row becomes a root when its key is the largest among the undecided
    rows within strong-graph distance 2; rows within distance 2 of a new root become decided;
  * phase 1: a strong neighbour of a root joins the root's aggregate; aggregates are numbered in root order;
  * phase 2: a remaining row joins the aggregate of its strongest phase-1 neighbour, ties to the smaller
    aggregate id.

The expected aggregates of the first graph were worked out by hand from these rules (the derivation is
in the comments); the random graphs are compared with a direct Python restatement of the same rules."""
import numpy as np
import pytest

import oracle


def key(i, level):
    h = oracle.lib().or_splitmix64((level << 32) | i)  # splitmix64 is pinned by its published vector
    return ((h >> 33) << 32) | i


def csr_from_edges(n, edges, nc=1):
    """Symmetric matrix with unit diagonal and -w on each edge (i, j, w); nc identical components."""
    rows = [dict() for _ in range(n)]
    for i in range(n):
        rows[i][i] = 1.0
    for i, j, w in edges:
        rows[i][j] = -w
        rows[j][i] = -w
    rp, ci, v = [0], [], []
    for i in range(n):
        for j in sorted(rows[i]):
            ci.append(j)
            v.extend([rows[i][j]] * nc)
        rp.append(len(ci))
    return np.array(rp), np.array(ci), np.array(v)


def test_hand_worked_graph():
    # Level-0 keys of rows 0..16 in decreasing order: 0, 13, 6, 9, 8, 2, 12, 1, 15, 4, 14, 7, 5, 16, 11, 3, 10.
    order = sorted(range(17), key=lambda i: key(i, 0), reverse=True)
    assert order == [0, 13, 6, 9, 8, 2, 12, 1, 15, 4, 14, 7, 5, 16, 11, 3, 10]
    # Three paths R - M - X - M' - R' with the six largest keys on the R's, so the roots are exactly
    # {0, 2, 6, 8, 9, 13} after one round, numbered 0..5 in row order: agg(0)=0, agg(2)=1, agg(6)=2,
    # agg(8)=3, agg(9)=4, agg(13)=5.  Every M joins its root in phase 1; every X is at distance 2 from two
    # roots and is left for phase 2.
    edges = [
        # path A: 13 - 16 - 12 - 1 - 0, weights 0.5 (12-16) against 0.3 (12-1); the edge 12-0 is weak
        # (0.05 < theta).  Phase 2 puts 12 with its strongest neighbour 16, i.e. aggregate 5, although
        # 1 comes first in row 12, is the weaker neighbour, and leads to the smaller aggregate id 0.  A rule
        # that took the weak edge would put 12 next to root 0 (aggregate 0 in phase 1).
        (13, 16, 0.4), (16, 12, 0.5), (12, 1, 0.3), (1, 0, 0.4), (12, 0, 0.05),
        # path B1: 9 - 3 - 10 - 15 - 2, equal weights at 10: the tie goes to the smaller aggregate id,
        # agg(2) = 1 through 15, although 3 (aggregate 4) comes first in row 10.
        (9, 3, 0.4), (3, 10, 0.4), (10, 15, 0.4), (15, 2, 0.4),
        # path B2: 6 - 4 - 7 - 14 - 8, equal weights at 7: the smaller id, agg(6) = 2, comes first in
        # row 7, so a rule keeping the last of equal weights (aggregate 3) is caught here.
        (6, 4, 0.4), (4, 7, 0.4), (7, 14, 0.4), (14, 8, 0.4),
    ]
    rp, ci, v = csr_from_edges(17, edges)
    # row 5: only a weak coupling, to row 11; row 11: an identity row.  Neither is aggregated.
    rows = [list(zip(ci[rp[i]:rp[i + 1]], v[rp[i]:rp[i + 1]])) for i in range(17)]
    rows[5] = sorted(rows[5] + [(11, -0.05)])
    rp = np.cumsum([0] + [len(r) for r in rows])
    ci = np.array([c for r in rows for c, _ in r])
    v = np.array([x for r in rows for _, x in r])
    agg, root, na = oracle.aggregate(rp, ci, v, theta=0.08, level=0)
    expect_root = {0, 2, 6, 8, 9, 13}
    assert set(np.flatnonzero(root)) == expect_root
    assert na == 6
    expect = [0, 0, 1, 4, 2, -1, 2, 2, 3, 4, 1, -1, 5, 5, 3, 1, 5]
    assert agg.tolist() == expect


@pytest.mark.parametrize("level,expect_root", [(0, 0), (1, 12), (2, 3)])
def test_root_is_the_largest_key_of_the_level(level, expect_root):
    # a star: every row lies within distance 2 of every other, so the single root is the row with the
    # largest key of that level (the keys differ per level: 0, 12 and 3 for levels 0, 1, 2; the smallest
    # keys are on rows 10, 10 and 15)
    n = 17
    rp, ci, v = csr_from_edges(n, [(16, i, 0.3) for i in range(16)])
    assert max(range(n), key=lambda i: key(i, level)) == expect_root
    agg, root, na = oracle.aggregate(rp, ci, v, level=level)
    assert np.flatnonzero(root).tolist() == [expect_root]
    assert na == 1 and np.all(agg == 0)


def reference_aggregate(n, nc, rp, ci, v, theta, level):
    """The aggregation rules restated directly (dense graph, breadth-first distances)."""
    A = np.zeros((n, n))
    present = np.zeros((n, n), bool)
    for i in range(n):
        for q in range(rp[i], rp[i + 1]):
            A[i, ci[q]] = np.abs(v[q * nc:(q + 1) * nc]).sum()
            present[i, ci[q]] = True
    nz_off = np.array([any(v[q * nc + c] != 0.0 for q in range(rp[i], rp[i + 1]) if ci[q] != i for c in range(nc))
                       for i in range(n)])
    d = np.diag(A)
    S = np.zeros((n, n), bool)
    for i in range(n):
        for j in range(n):
            if i != j and present[i, j] and nz_off[i] and nz_off[j]:
                t = max(A[i, j], A[j, i])
                if t > 0 and t >= theta * np.sqrt(d[i] * d[j]):
                    S[i, j] = True
    W = np.where(S, np.maximum(A, A.T) / np.sqrt(np.outer(d, d)), 0.0)
    dist2 = S | (S.astype(int) @ S.astype(int) > 0)
    np.fill_diagonal(dist2, False)
    state = np.where(S.any(axis=1), 0, 3)  # 0 undecided, 1 root, 2 covered, 3 not aggregated
    keys = [key(i, level) for i in range(n)]
    while (state == 0).any():
        und = state == 0
        new = [i for i in range(n) if und[i] and all(keys[i] > keys[j] for j in np.flatnonzero(dist2[i] & und))]
        for i in new:
            state[i] = 1
        for i in range(n):
            if state[i] == 0 and any(dist2[i, r] for r in new):
                state[i] = 2
    roots = np.flatnonzero(state == 1)
    agg = -np.ones(n, int)
    agg[roots] = np.arange(len(roots))
    ph1 = agg.copy()
    for i in range(n):
        if state[i] == 2:
            rs = [r for r in roots if S[i, r]]
            if rs:
                ph1[i] = agg[rs[0]]
    out = ph1.copy()
    for i in range(n):
        if state[i] == 2 and ph1[i] < 0:
            cands = [(-W[i, j], ph1[j]) for j in np.flatnonzero(S[i]) if ph1[j] >= 0]
            out[i] = min(cands)[1]
    return out, state == 1


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_match_the_rules(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(8, 40))
    nc = int(rng.choice([1, 3]))
    rows = [dict() for _ in range(n)]
    for i in range(n):
        rows[i][i] = rng.uniform(0.5, 2.0, nc)
    for _ in range(int(rng.integers(n, 3 * n))):
        i, j = rng.integers(0, n, 2)
        if i == j:
            continue
        # a mix of strong and weak couplings; repeated weights make phase-2 ties
        w = rng.choice([0.01, 0.2, 0.2, 0.5, rng.uniform(0.0, 0.6)])
        rows[i][j] = -w * rng.uniform(0.5, 1.0, nc) if nc == 3 else -np.array([w])
        if rng.uniform() < 0.8:
            rows[j][i] = rows[i][j]
    rp, ci, v = [0], [], []
    for i in range(n):
        for j in sorted(rows[i]):
            ci.append(j)
            v.extend(rows[i][j].tolist())
        rp.append(len(ci))
    rp, ci, v = np.array(rp), np.array(ci), np.array(v)
    level = int(rng.integers(0, 4))
    agg, root, na = oracle.aggregate(rp, ci, v, nc=nc, theta=0.08, level=level)
    ragg, rroot = reference_aggregate(n, nc, rp, ci, v, 0.08, level)
    assert np.array_equal(root, rroot)
    assert agg.tolist() == ragg.tolist()
    assert na == rroot.sum()
