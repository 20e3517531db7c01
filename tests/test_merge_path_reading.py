"""Pins the reading behind the warp-parallel SolveOT1D walk (Alg. 1) on the CPU.

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
