"""The block schedules of the CUDA factorisation drivers, restated in numpy
and checked against the CPU oracle on the CPU.

The library's drivers (csrc/factor.cu) order their GEMMs and small kernels
in ways the oracle does not: gs2 (Eq. 3) by a 2 x 2 recursion with n^3
flops, and the Cholesky of each diagonal block (Eq. 2) over sub-panels of
32 rows.  These tests replay the same block algebra with numpy on small
sizes, ragged halves and several recursion depths, so that an error in the
identities themselves (a sign, a half-step, a transposed factor) shows up
without a GPU; the GPU parity tests then check the kernels against the
oracle elementwise.  CPU only."""
import numpy as np
import pytest

import inputs
import oracle


def _sygst_rec(A, U, NB, leaf_blocks=4):
    """C = U^-T A U^-1 from A's lower triangle, in the library's recursion:
    C11 recursively; Y = A21 U11^-1; P = U12^T C11; Z = Y - P/2;
    A22 -= Z U12 + U12^T Z^T (lower); C22 recursively; C21 = U22^-T (Z - P/2).
    Leaves (at most leaf_blocks outer blocks) use the direct form."""
    n = A.shape[0]
    if n <= leaf_blocks * NB:
        L = np.tril(A)
        A[:] = L + np.tril(L, -1).T
        Ui = np.linalg.inv(U)
        A[:] = Ui.T @ A @ Ui
        return
    nbk = -(-n // NB)
    n1 = ((nbk + 1) // 2) * NB
    A11, A21, A22 = A[:n1, :n1], A[n1:, :n1], A[n1:, n1:]
    U11, U12, U22 = U[:n1, :n1], U[:n1, n1:], U[n1:, n1:]
    _sygst_rec(A11, U11, NB, leaf_blocks)
    A21[:] = A21 @ np.linalg.inv(U11)                      # Y
    P = U12.T @ A11
    A21 -= 0.5 * P                                         # Z
    M = A21 @ U12
    A22[:] = np.tril(A22 - M - M.T) + np.triu(A22, 1)      # lower triangle only
    A21 -= 0.5 * P                                         # W
    A22[np.triu_indices(A22.shape[0], 1)] = np.nan         # the upper triangle is never read
    _sygst_rec(A22, U22, NB, leaf_blocks)
    A21[:] = np.linalg.inv(U22).T @ A21
    A[:n1, n1:] = A21.T


@pytest.mark.parametrize("n,NB", [(7, 1), (37, 4), (64, 4), (101, 8), (300, 16)])
def test_sygst_recursion_matches_oracle(n, NB):
    A, B, _ = (t.numpy() for t in inputs.make_pencil(n, seed=n + NB))
    U = oracle.potrf(B)
    Co = oracle.sygst(A, U)
    W = A.copy()
    W[np.triu_indices(n, 1)] = np.nan
    _sygst_rec(W, U, NB)
    assert np.isfinite(W).all()
    assert np.abs(W - Co).max() <= 1e-12 * np.abs(Co).max()


def test_sygst_recursion_depth():
    """n = 300 with outer blocks of 16 recurses three levels before the
    leaves of at most 64 rows; the flops of the recursion fall below the
    direct form's 4n^3/3 (the reason for it)."""
    def flops(n, NB):
        if n <= 4 * NB:
            return 4 * n ** 3 / 3, 0
        n1 = ((-(-n // NB) + 1) // 2) * NB
        n2 = n - n1
        f1, d1 = flops(n1, NB)
        f2, d2 = flops(n2, NB)
        return f1 + f2 + n2 * n1 ** 2 + 2 * n2 * n1 ** 2 + 2 * n1 * n2 ** 2 + n1 * n2 ** 2, 1 + max(d1, d2)
    f, depth = flops(300, 16)
    assert depth == 3
    f, _ = flops(16384, 512)
    assert f < 0.78 * (4 * 16384 ** 3 / 3)


def _chol_subpanels(D, PW=32):
    """Upper Cholesky of a diagonal block over sub-panels of PW rows, as the
    library's k_chol_sub / k_chol_panel / k_chol_update launches do."""
    D = np.triu(D.copy())
    kb = D.shape[0]
    for p0 in range(0, kb, PW):
        p1 = min(kb, p0 + PW)
        S = D[p0:p1, p0:p1]
        Upp = np.linalg.cholesky(np.triu(S) + np.triu(S, 1).T).T   # the one-warp sub-block
        D[p0:p1, p0:p1] = Upp
        if p1 < kb:
            D[p0:p1, p1:] = np.linalg.solve(Upp.T, D[p0:p1, p1:])   # the panel rows
            D[p1:, p1:] -= np.triu(D[p0:p1, p1:].T @ D[p0:p1, p1:])  # rank-PW update, upper
    return D


@pytest.mark.parametrize("kb", [1, 31, 32, 33, 60, 128, 160])
def test_chol_subpanels_match_oracle(kb):
    B = inputs.make_pencil(max(kb, 2), seed=kb)[1].numpy()[:kb, :kb]
    U = _chol_subpanels(B)
    assert np.abs(U - oracle.potrf(B)).max() <= 1e-12 * np.abs(U).max()
