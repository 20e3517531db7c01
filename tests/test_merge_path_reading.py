"""Pins the reading behind the warp-parallel SolveOT1D (Alg. 1) and SolveMOT (Alg. 3) walks on the CPU.

The GPU kernel takes Alg. 1's branch "point i is exhausted first" as A_i <= B_j
(A, B the partial sums of the two histograms), splits the resulting merge of the
two partial-sum sequences into equal shares found by binary search, and links
the shares' potentials through affine maps x -> c + sigma x (sigma = +-1) of
their starting i-potential.  This test restates that scheme in plain Python
(FP64) and checks it against the oracle's sequential walk, which tracks the
untransported masses directly, on random, ragged and zero-weight inputs and on
any number of shares.  It exercises the reading, not the kernel."""
import numpy as np
import pytest

from oracle import fw1d as W


def merge_i(A, n, B, m, s):
    lo, hi = max(0, s - (m - 1)), min(s, n - 1)
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if (s - mid >= m - 1) or not (B[s - mid] < A[mid - 1]):
            lo = mid
        else:
            hi = mid - 1
    return lo


def merge_path_walk(x, a, y, b, p, shares):
    n, m = len(x), len(y)
    A, B = np.cumsum(a), np.cumsum(b)
    steps = (n - 1) + (m - 1)
    C = lambda i, j: abs(x[i] - y[j]) ** p

    def advance_i(i, j):
        return i < n - 1 and (j == m - 1 or not (B[j] < A[i]))

    starts, maps = [], []
    for ell in range(shares):
        s0, s1 = ell * steps // shares, (ell + 1) * steps // shares
        i0 = merge_i(A, n, B, m, s0)
        j0 = s0 - i0
        cR, sgR, cS, sgS = 0.0, 1.0, C(i0, j0), -1.0
        i, j = i0, j0
        for _ in range(s0, s1):
            if advance_i(i, j):
                i += 1
                cR, sgR = C(i, j) - cS, -sgS
            else:
                j += 1
                cS, sgS = C(i, j) - cR, -sgR
        starts.append((s0, s1, i0, j0))
        maps.append((cR, sgR))
    f, g = np.zeros(n), np.zeros(m)
    r0 = 0.0
    for ell in range(shares):
        s0, s1, i0, j0 = starts[ell]
        ri, sj = r0, C(i0, j0) - r0
        if ell == 0:
            g[0] = sj
        i, j = i0, j0
        for _ in range(s0, s1):
            if advance_i(i, j):
                i += 1
                ri = C(i, j) - sj
                f[i] = ri
            else:
                j += 1
                sj = C(i, j) - ri
                g[j] = sj
        c, sg = maps[ell]
        r0 = c + sg * r0
    return f, g


@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("shares", [1, 3, 32])
def test_merge_path_walk_equals_sequential_walk(seed, shares):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 50)), int(rng.integers(1, 50))
    p = [1.0, 1.5, 2.0][seed % 3]
    x = np.sort(rng.normal(size=n))
    y = np.sort(rng.normal(0.3, 0.8, size=m))
    a = rng.exponential(size=n)
    b = rng.exponential(size=m)
    if n > 3:
        a[n // 3] = 0.0
    if m > 3:
        b[m // 2] = 0.0
    b *= a.sum() / b.sum()  # balanced, as between the re-weighted histograms
    _, f_ref, g_ref = W.solve_ot_1d(x, a, y, b, p)
    f, g = merge_path_walk(x, a, y, b, p, shares)
    scale = 1.0 + float(np.abs(x[:, None] - y[None, :]).max() ** p)
    assert np.abs(f - f_ref.numpy()).max() <= 1e-12 * scale
    assert np.abs(g - g_ref.numpy()).max() <= 1e-12 * scale


# ---- the K-way form (SolveMOT, Alg. 3) -------------------------------------------------------
from oracle import mmot1d as MM


def _mm_cost(z, w):
    b = sum(wk * zk for wk, zk in zip(w, z))
    return sum(wk * (zk - b) ** 2 for wk, zk in zip(w, z)), b


def _state_at(E, s):
    """Counts of events per measure before the event of rank s in (value, measure, index) order."""
    K = len(E)
    total = sum(len(e) for e in E)
    if s >= total:
        return [len(e) for e in E]
    for k in range(K):
        lo, hi = 0, len(E[k]) - 1
        while lo <= hi:
            i = (lo + hi) // 2
            v = E[k][i]
            cnt = [int(np.searchsorted(E[q], v, side="right" if q < k else "left")) for q in range(K)]
            r = i + sum(cnt[q] for q in range(K) if q != k)
            if r == s:
                return [i if q == k else cnt[q] for q in range(K)]
            lo, hi = (i + 1, hi) if r < s else (lo, i - 1)
    raise AssertionError("no event of rank s")


def kway_merge_path_walk(xs, al, w, shares):
    K, N = len(xs), [len(x) for x in xs]
    A = [np.cumsum(a) for a in al]
    E = [a[:-1] for a in A]
    steps = sum(n - 1 for n in N)
    f = [np.zeros(n) for n in N]
    sh = [(l * steps // shares, (l + 1) * steps // shares) for l in range(shares)]

    def pick(idx):
        return min((k for k in range(K) if idx[k] < N[k] - 1), key=lambda k: (A[k][idx[k]], k))

    D = []
    for s0, s1 in sh:  # first walk: each measure's summed cost change over the share
        idx = _state_at(E, s0)
        z = [xs[k][idx[k]] for k in range(K)]
        C, _ = _mm_cost(z, w)
        d = [0.0] * K
        for _ in range(s0, s1):
            p = pick(idx)
            idx[p] += 1
            z[p] = xs[p][idx[p]]
            Cn, _ = _mm_cost(z, w)
            d[p] += Cn - C
            C = Cn
        D.append(d)
    cur = [_mm_cost([x[0] for x in xs], w)[0]] + [0.0] * (K - 1)
    f[0][0] = cur[0]
    bary = []
    for (s0, s1), d in zip(sh, D):  # second walk: the potentials and the plan's positive masses
        idx = _state_at(E, s0)
        prev = max([A[k][idx[k] - 1] for k in range(K) if idx[k] > 0] + [0.0])
        z = [xs[k][idx[k]] for k in range(K)]
        C, b = _mm_cost(z, w)
        c = list(cur)
        for _ in range(s0, s1):
            p = pick(idx)
            v = A[p][idx[p]]
            if v - prev > 0:
                bary.append((b, v - prev))
            prev = v
            idx[p] += 1
            z[p] = xs[p][idx[p]]
            Cn, b = _mm_cost(z, w)
            c[p] += Cn - C
            C = Cn
            f[p][idx[p]] = c[p]
        cur = [cur[k] + d[k] for k in range(K)]
    last = max([e[-1] for e in E if len(e)] + [0.0])
    if A[0][-1] - last > 0:
        bary.append((_mm_cost([x[-1] for x in xs], w)[1], A[0][-1] - last))
    return f, bary


@pytest.mark.parametrize("seed", range(30))
@pytest.mark.parametrize("shares", [1, 5, 32])
def test_kway_merge_path_walk_equals_sequential_solvemot(seed, shares):
    rng = np.random.default_rng(1000 + seed)
    K = int(rng.integers(2, 6))
    N = [int(rng.integers(1, 30)) for _ in range(K)]
    xs = [np.sort(rng.normal(size=n)) for n in N]
    al = [rng.exponential(size=n) for n in N]
    tot = al[0].sum()
    al = [a * tot / a.sum() for a in al]  # balanced, as the re-weighted measures
    w = list(rng.dirichlet(np.ones(K)))
    plan, fs = MM.solve_mot_1d(xs, al, w)
    f, bary = kway_merge_path_walk(xs, al, w, shares)
    for k in range(K):
        assert np.abs(fs[k].numpy() - f[k]).max() <= 1e-12 * (1.0 + sum(np.ptp(x) ** 2 for x in xs))
    ref = [(_mm_cost([xs[k][i] for k, i in enumerate(t)], w)[1], m) for t, m in plan if m > 0]
    assert len(ref) == len(bary)
    for (b1, m1), (b2, m2) in zip(ref, bary):
        assert abs(b1 - b2) <= 1e-12 and abs(m1 - m2) <= 1e-12 * tot
