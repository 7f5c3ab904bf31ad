"""Host-side model of how the blocked dense LU (the exact check path of
Sec. 3's block determinants) applies a panel's row swaps to the columns right
of the panel: the LU_NB swaps k <-> ipiv[k] of one panel (partial pivoting,
LAPACK getrf order) are folded into one permutation of the rows they touch,
(destination rows, source rows), which a warp per column gathers and then
scatters.  The model follows the device function's steps; the test checks it
against the swaps applied one after another, and that a panel touches at most
2 LU_NB rows (the size of the device buffers).
"""
import numpy as np
import pytest

NB = 32


def panel_permutation(ipiv, k0, nbe):
    """(rows, src): position i of the list receives the value that row src[i]
    held before the panel.  Rows k0..k0+nbe-1 come first, then every pivot
    row outside them, in order of first use."""
    rows = [k0 + t for t in range(nbe)]
    src = list(rows)
    for t in range(nbe):
        p = ipiv[k0 + t]
        q = rows.index(p) if p in rows else -1
        if q < 0:
            q = len(rows)
            rows.append(p)
            src.append(p)
        src[t], src[q] = src[q], src[t]
    return rows, src


def sequential(col, ipiv, k0, nbe):
    out = np.array(col, copy=True)
    for t in range(nbe):
        k, p = k0 + t, ipiv[k0 + t]
        out[k], out[p] = out[p], out[k]
    return out


@pytest.mark.parametrize("n,k0", [(192, 0), (192, 160), (3072, 32 * 40), (200, 192), (33, 0)])
@pytest.mark.parametrize("seed", range(4))
def test_gathered_permutation_equals_sequential_swaps(n, k0, seed):
    rng = np.random.default_rng(seed)
    nbe = min(NB, n - k0)
    for trial in range(25):
        ipiv = np.zeros(n, dtype=np.int64)
        mode = trial % 3
        for t in range(nbe):
            k = k0 + t
            if mode == 0:  # anywhere below
                ipiv[k] = rng.integers(k, n)
            elif mode == 1:  # inside the panel's own rows
                ipiv[k] = rng.integers(k, min(n, k0 + nbe))
            else:  # often no swap, sometimes the same far row again
                ipiv[k] = k if rng.random() < 0.5 else min(n - 1, k0 + nbe + rng.integers(0, 3))
        col = rng.standard_normal(n)
        rows, src = panel_permutation(ipiv, k0, nbe)
        assert len(rows) <= 2 * NB
        assert sorted(rows) == sorted(src)  # a permutation of the touched rows
        gathered = np.array(col, copy=True)
        vals = [col[s] for s in src]
        for r, v in zip(rows, vals):
            gathered[r] = v
        assert np.array_equal(gathered, sequential(col, ipiv, k0, nbe))


def test_model_detects_swaps_applied_in_reverse():
    """Folding the swaps in the opposite order gives another permutation, so
    the comparison above would catch it."""
    ipiv = np.arange(64)
    ipiv[0], ipiv[1] = 40, 40
    col = np.arange(64, dtype=float)
    rev = np.array(col, copy=True)
    for t in (1, 0):
        rev[t], rev[ipiv[t]] = rev[ipiv[t]], rev[t]
    assert not np.array_equal(rev, sequential(col, ipiv, 0, 2))
    rows, src = panel_permutation(ipiv, 0, 2)
    g = np.array(col, copy=True)
    for r, s in zip(rows, [col[s] for s in src]):
        g[r] = s
    assert np.array_equal(g, sequential(col, ipiv, 0, 2))
