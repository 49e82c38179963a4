"""Host-side checks of two structural facts the factorisation kernel relies
on when it skips work (cholesky.cu, the walker and the diagonal tile).

* The walker's TRSM(j+1, j) multiplies by Linv_jj^T, whose upper part is
  stored as exact zeros. Output column block b therefore needs only the
  contraction chunks m < 16 (b + 1). Its UPDATE(j+1, j+1, j) is symmetric,
  and only the lower part is read, so only the 16x16 blocks a >= b are
  formed. With the kernel's thread layout (row ty + 16 a, column
  tx + 16 b), the kept terms and blocks must cover every nonzero term and
  every entry that is read.
* The diagonal tile is factorised by Gaussian elimination in LDL^T form
  over [A | I], 4 columns per step. Rows i <= k get zero multipliers at
  step k. Skipping their updates must leave L and L^-1 unchanged, and
  both must be right (L L^T = A, L^-1 L = I).

No GPU: numpy, with the kernel's index sets and step order.
"""
import numpy as np
import pytest

NB = 64


def _kept_trsm(mc, b):
    return b >= mc


def test_walker_trsm_chunks_cover_every_nonzero_term():
    # Y = Linv_jj: Y[c][m] != 0 only for m <= c; the term (c, m) is summed
    # iff chunk m // 16 is kept for column block c // 16
    for c in range(NB):
        for m in range(NB):
            kept = _kept_trsm(m // 16, c // 16)
            if m <= c:
                assert kept, (c, m)
    # and the skipped share is 6 of 16 chunk-block pairs
    pairs = [(mc, b) for mc in range(4) for b in range(4)]
    assert sum(not _kept_trsm(mc, b) for mc, b in pairs) == 6


def test_walker_trsm_restricted_sum_equals_full_sum_bit_for_bit():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((NB, NB)).astype(np.float32)
    Y = np.tril(rng.standard_normal((NB, NB))).astype(np.float32)   # upper part exactly zero
    full = np.zeros((NB, NB), np.float32)
    part = np.zeros((NB, NB), np.float32)
    cols = np.arange(NB)
    for m in range(NB):   # the kernel's order: ascending m for every output
        term = X[:, m:m + 1] * Y[None, :, m]                # [r][c] = X[r][m] Y[c][m]
        full = (full + term).astype(np.float32)
        keep = _kept_trsm(m // 16, cols // 16)
        part = np.where(keep[None, :], (part + term).astype(np.float32), part)
    assert np.array_equal(full, part)


def test_walker_update_lower_blocks_cover_what_potrf_reads():
    # thread (tx, ty) forms rows ty + 16 a and columns tx + 16 b for the
    # blocks a >= b; POTRF reads the lower part, column <= row
    formed = np.zeros((NB, NB), bool)
    for ty in range(16):
        for tx in range(16):
            for a in range(4):
                for b in range(a + 1):
                    formed[ty + 16 * a, tx + 16 * b] = True
    assert formed[np.tril_indices(NB)].all()
    assert formed.sum() == 10 * 256


def _ldlt_sweep(A, W=4, skip_final_rows=False):
    """The diagonal tile's elimination as the kernel performs it. Returns
    (L, Linv) and the largest |c| seen on rows <= k."""
    n = A.shape[0]
    a = A.copy()
    y = np.eye(n)
    piv = np.zeros(n)
    worst_done = 0.0
    for k in range(0, n, W):
        K = slice(k, k + W)
        V = a[:, K].copy()                       # columns K as they stand
        Z = y[K, :].copy()                       # rows K of Y as they stand
        E = V[K, :].copy()                       # pivot block, lower part used
        Ld = np.eye(W)
        p = np.zeros(W)
        for nn in range(W):                      # right-looking LDL^T of E
            p[nn] = E[nn, nn]
            for m in range(nn + 1, W):
                Ld[m, nn] = E[m, nn] / p[nn]
            for m in range(nn + 1, W):
                for o in range(nn + 1, m + 1):
                    E[m, o] -= Ld[m, nn] * E[o, nn]
        piv[K] = p
        for i in range(n):
            if skip_final_rows and i <= k:
                continue
            u = np.zeros(W)
            for m in range(W):
                u[m] = V[i, m] - sum(Ld[m, q] * u[q] for q in range(m))
            c = np.zeros(W)
            for m in range(W - 1, -1, -1):
                c[m] = u[m] / p[m] if i > k + m else 0.0
                c[m] -= sum(c[q] * Ld[q, m] for q in range(m + 1, W))
            if i <= k:
                worst_done = max(worst_done, float(np.abs(c).max()))
            # A[i][j] -= c . V[j, :] for j beyond the block; the block's own
            # columns take u (the finished L' entries)
            a[i, k + W:] -= V[k + W:, :] @ c
            a[i, K] = u
            y[i, :] -= c @ Z
    d = np.sqrt(piv)
    L = np.tril(a, -1) / d[None, :] + np.diag(d)
    Linv = np.tril(y) / d[:, None]
    return L, Linv, worst_done


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_diagonal_tile_rows_at_or_above_k_have_zero_multipliers(seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((NB, NB))
    A = G @ G.T / NB + np.eye(NB)
    L, Linv, worst = _ldlt_sweep(A)
    assert worst == 0.0
    np.testing.assert_allclose(L @ L.T, A, rtol=0, atol=1e-12 * np.abs(A).max())
    np.testing.assert_allclose(Linv @ L, np.eye(NB), rtol=0, atol=1e-12)
    L2, Linv2, _ = _ldlt_sweep(A, skip_final_rows=True)
    assert np.array_equal(L, L2)
    assert np.array_equal(Linv, Linv2)
