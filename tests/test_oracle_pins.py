"""Pins for the CPU oracle against facts fixed by the paper and by mathematics,
not by the oracle itself: exact golden pencils (Eq. 1-4), closed forms,
textbook/library routines on special cases, invariants, brute force.

CPU only; no GPU or CUDA library involved."""
import numpy as np
import pytest
import scipy.linalg as sla

import inputs
import oracle


def _spd(n, seed):
    r = np.random.default_rng(seed)
    G = r.standard_normal((n, n))
    return G @ G.T / n + np.eye(n)


def _sym(n, seed, scale=1.0):
    r = np.random.default_rng(seed)
    M = r.standard_normal((n, n)) * scale
    return M + M.T


# ---------------------------------------------------------------- Eq. 2 ----
def test_potrf_golden_exact(golden4):
    A, B, U, lam = golden4
    assert np.array_equal(oracle.potrf(B), U)


def test_potrf_reconstructs_and_matches_library():
    B = _spd(97, 1)
    U = oracle.potrf(B)
    assert np.allclose(np.tril(U, -1), 0.0)
    assert np.abs(U.T @ U - B).max() < 1e-13
    L = np.linalg.cholesky(B)
    assert np.abs(U - L.T).max() < 1e-13


def test_potrf_reports_first_bad_pivot():
    B = np.diag([1.0, 2.0, -1.0, 4.0])
    with pytest.raises(oracle.NotSPD) as ei:
        oracle.potrf(B)
    assert ei.value.index == 3
    B = _spd(20, 2)
    B[11, 11] = -100.0
    with pytest.raises(oracle.NotSPD) as ei:
        oracle.potrf(B)
    assert ei.value.index == 12


# ---------------------------------------------------------------- Eq. 3 ----
def test_sygst_golden_exact(golden4):
    A, B, U, lam = golden4
    C = oracle.sygst(A, U)
    H = 0.5 * np.array([[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]], dtype=float)
    assert np.abs(C - H @ np.diag(lam) @ H.T).max() < 1e-14


def test_sygst_matches_explicit_inverse_and_reads_lower_only():
    n = 83
    A = _sym(n, 3)
    B = _spd(n, 4)
    U = np.linalg.cholesky(B).T
    Ui = np.linalg.inv(U)
    Cref = Ui.T @ A @ Ui
    Ain = A.copy()
    Ain[np.triu_indices(n, 1)] = np.nan  # upper triangle must not be read
    C = oracle.sygst(Ain, U)
    assert np.array_equal(C, C.T)
    assert np.abs(C - Cref).max() < 1e-11 * np.abs(Cref).max()


# ---------------------------------------------------------------- Eq. 4 ----
def test_backsolve_matches_library():
    n, s = 71, 5
    U = np.triu(np.random.default_rng(5).standard_normal((n, n))) + 5 * np.eye(n)
    Y = np.random.default_rng(6).standard_normal((n, s))
    X = oracle.backsolve(U, Y)
    assert np.abs(U @ X - Y).max() < 1e-12
    assert np.abs(X - sla.solve_triangular(U, Y, lower=False)).max() < 1e-12


# ------------------------------------------------- Section 2.2 (TD) -------
def test_tridiag_is_orthogonal_similarity():
    n = 60
    C = _sym(n, 7)
    d, e, R, tau = oracle.tridiag(C)
    Q = oracle.apply_q(R, tau, np.eye(n))
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-13
    assert np.abs(Q.T @ C @ Q - T).max() < 1e-12 * np.abs(C).max()


def test_tql_eigenvalues_match_library_and_vectors_are_eigenvectors():
    for m, seed in ((1, 0), (2, 1), (57, 2), (200, 3)):
        d, e = (t.numpy() for t in inputs.make_tridiagonal(m, seed))
        w, Z = oracle.tql(d, e, vectors=True)
        assert np.all(np.diff(w) >= 0)
        if m > 1:
            ref = sla.eigvalsh_tridiagonal(d, e)
        else:
            ref = d
        assert np.abs(w - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
        T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        assert np.abs(T @ Z - Z * w).max() < 1e-11 * np.abs(d).max()
        assert np.abs(Z.T @ Z - np.eye(m)).max() < 1e-12


def test_sturm_count_matches_eigenvalue_count():
    d, e = (t.numpy() for t in inputs.make_tridiagonal(150, 11))
    w = sla.eigvalsh_tridiagonal(d, e)
    for x in np.linspace(w[0] - 1, w[-1] + 1, 37):
        assert oracle.sturm_count(d, e, x) == int(np.sum(w < x))
    # midpoints between consecutive eigenvalues give exact counts 1..m-1
    for i in range(0, 149, 7):
        assert oracle.sturm_count(d, e, 0.5 * (w[i] + w[i + 1])) == i + 1


@pytest.mark.parametrize("clustered", [False, True])
def test_inverse_iteration_vectors(clustered):
    d, e = (t.numpy() for t in inputs.make_tridiagonal(120, 13, clustered=clustered))
    w = sla.eigvalsh_tridiagonal(d, e)
    lam = w[:30]
    Z = oracle.tri_invit(d, e, lam)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.abs(T @ Z - Z * lam).max() < 1e-9 * np.abs(d).max()
    assert np.abs(Z.T @ Z - np.eye(30)).max() < 1e-9


# ------------------------------------------------------ brute force (P3) --
def test_jacobi_matches_library():
    for n in (2, 5, 33, 64):
        C = _sym(n, 20 + n)
        w, V = oracle.jacobi(C)
        ref = np.linalg.eigvalsh(C)
        assert np.abs(w - ref).max() < 1e-12 * np.abs(ref).max()
        assert np.abs(C @ V - V * w).max() < 1e-11 * np.abs(ref).max()
        assert np.abs(V.T @ V - np.eye(n)).max() < 1e-12


def test_full_route_agrees_with_jacobi_on_explicit_c():
    n = 48
    A = _sym(n, 31)
    B = _spd(n, 32)
    w, X = oracle.gsyeig(A, B, n)
    U = np.linalg.cholesky(B).T
    Ui = np.linalg.inv(U)
    wj, Vj = oracle.jacobi(Ui.T @ A @ Ui)
    assert np.abs(w - wj).max() < 1e-11 * np.abs(wj).max()
    Xj = Ui @ Vj
    # eigenvalues are simple here: vectors agree up to sign
    for c in range(n):
        sgn = np.sign(X[:, c] @ B @ Xj[:, c])
        assert np.abs(X[:, c] - sgn * Xj[:, c]).max() < 1e-8


# --------------------------------------------------------- whole route ----
def test_golden_pencil_eigenpairs(golden4):
    A, B, U, lam = golden4
    w, X = oracle.gsyeig(A, B, 4)
    assert np.abs(w - lam).max() < 1e-13
    H = 0.5 * np.array([[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]], dtype=float)
    Xref = np.linalg.solve(U, H)
    for c in range(4):
        sgn = np.sign(X[:, c] @ B @ Xref[:, c])
        assert np.abs(X[:, c] - sgn * Xref[:, c]).max() < 1e-13


def test_known_spectrum_config_n512():
    A, B, lam = (t.numpy() for t in inputs.make_pencil(512, 0))
    s = 10
    for vec in ("ql", "invit"):
        w, X = oracle.gsyeig(A, B, s, vectors=vec)
        assert np.max(np.abs(w - lam[:s]) / lam[:s]) < 1e-10
        assert np.abs(X.T @ B @ X - np.eye(s)).max() < 1e-10
        R = A @ X - (B @ X) * w
        nA, nB = np.linalg.norm(A, 2), np.linalg.norm(B, 2)
        eta = np.linalg.norm(R, axis=0) / ((nA + np.abs(w) * nB) * np.linalg.norm(X, axis=0))
        assert eta.max() < 1e-14


def test_largest_and_smallest():
    A, B, lam = (t.numpy() for t in inputs.make_pencil(300, 3))
    w, X = oracle.gsyeig(A, B, 7, which="largest")
    assert np.max(np.abs(w - lam[-7:]) / lam[-7:]) < 1e-11
    w, X = oracle.gsyeig(A, B, 7, which="smallest")
    assert np.max(np.abs(w - lam[:7]) / lam[:7]) < 1e-10


def test_inverse_problem_relation():
    """Section 3.1's inverse problem, as the GPU route's reading uses it: with
    A and B positive definite, the s largest pairs (mu, y) of B y = mu A y
    (y^T A y = 1) give the s smallest pairs of (A, B) as lambda = 1/mu in
    reverse order and x = y / sqrt(mu) (then x^T B x = 1)."""
    n, s = 400, 9
    A, B, lam = (t.numpy() for t in inputs.make_pencil(n, 12))
    assert lam.min() > 0
    mu, Y = oracle.gsyeig(B, A, s, which="largest")  # roles swapped: A is the SPD matrix factored
    assert np.abs(Y.T @ A @ Y - np.eye(s)).max() < 1e-10
    w_inv = 1.0 / mu[::-1]
    X_inv = Y[:, ::-1] / np.sqrt(mu[::-1])
    w, X = oracle.gsyeig(A, B, s)
    assert np.max(np.abs(w_inv - w) / w) < 1e-10
    assert np.max(np.abs(w_inv - lam[:s]) / lam[:s]) < 1e-10
    assert np.abs(X_inv.T @ B @ X_inv - np.eye(s)).max() < 1e-10
    # the same vectors up to sign (the constructed spectrum has no clusters at the bottom)
    assert np.abs(np.abs(np.sum(X_inv * (B @ X), axis=0)) - 1.0).max() < 1e-8


def test_standard_problem_special_case():
    n = 90
    A = _sym(n, 41)
    w, X = oracle.gsyeig(A, np.eye(n), 12)
    ref_w, ref_V = np.linalg.eigh(A)
    assert np.abs(w - ref_w[:12]).max() < 1e-12 * np.abs(ref_w).max()
    assert np.abs(np.abs(X.T @ ref_V[:, :12]) - np.eye(12)).max() < 1e-10


def test_diagonal_pencil_closed_form():
    a = np.array([3.0, -1.0, 8.0, 0.5, 2.0, 10.0])
    b = np.array([1.0, 2.0, 4.0, 0.25, 8.0, 5.0])
    w, X = oracle.gsyeig(np.diag(a), np.diag(b), 6)
    assert np.abs(w - np.sort(a / b)).max() < 1e-14
    # eigenvectors are scaled unit vectors e_i / sqrt(b_i)
    order = np.argsort(a / b, kind="stable")
    for c, i in enumerate(order):
        assert abs(abs(X[i, c]) - 1 / np.sqrt(b[i])) < 1e-14


def test_two_by_two_closed_form():
    A = np.array([[2.0, 1.0], [1.0, -3.0]])
    B = np.array([[4.0, 1.0], [1.0, 3.0]])
    # det(A - l B) = 0: (detB) l^2 - (a11 b22 + a22 b11 - 2 a12 b12) l + detA = 0
    qa = B[0, 0] * B[1, 1] - B[0, 1] ** 2
    qb = -(A[0, 0] * B[1, 1] + A[1, 1] * B[0, 0] - 2 * A[0, 1] * B[0, 1])
    qc = A[0, 0] * A[1, 1] - A[0, 1] ** 2
    disc = np.sqrt(qb * qb - 4 * qa * qc)
    roots = np.sort([(-qb - disc) / (2 * qa), (-qb + disc) / (2 * qa)])
    w, X = oracle.gsyeig(A, B, 2)
    assert np.abs(w - roots).max() < 1e-14


def test_block_diagonal_pencil():
    blocks = [(np.array([[2.0, 1.0], [1.0, 2.0]]), np.eye(2)),
              (np.array([[5.0, 0.0], [0.0, 7.0]]), np.array([[1.0, 0.0], [0.0, 7.0]]))]
    A = sla.block_diag(*[b[0] for b in blocks])
    B = sla.block_diag(*[b[1] for b in blocks])
    w, X = oracle.gsyeig(A, B, 4)
    assert np.abs(w - np.array([1.0, 1.0, 3.0, 5.0])).max() < 1e-14
    assert np.abs(X.T @ B @ X - np.eye(4)).max() < 1e-14


def test_subspace_angle_helper_detects_rotation():
    """The parity tests' eigenvector metric: zero for identical bases, the
    rotation angle for a basis rotated by a known angle."""
    from tests import _checks

    n = 40
    B = np.eye(n)
    X = np.eye(n)[:, :3]
    w = np.array([1.0, 2.0, 3.0])
    lam = np.arange(1.0, n + 1)
    ang, _ = _checks.max_subspace_angle(B, X, X, w, lam, 40.0, 1e-12)
    assert ang < 1e-15
    t = 1e-6
    Y = X.copy()
    Y[:, 1] = np.cos(t) * X[:, 1] + np.sin(t) * np.eye(n)[:, 10]
    ang, _ = _checks.max_subspace_angle(B, Y, X, w, lam, 40.0, 1e-12)
    assert abs(ang - np.sin(t)) < 1e-12


# ---- the warm-start network's oracle (oracle/mlp.py) -----------------------

def test_mlp_oracle_bf16_rounding_known_values():
    """bf16 keeps 8 significant bits: ties go to the even neighbour."""
    from oracle import mlp

    x = np.array([1.0, 1 + 2.0**-8, 1 + 3 * 2.0**-8, 1 + 2.0**-8 + 2.0**-20, -2.5, 3.14159, 0.0, 2.0**-130])
    want = np.array([1.0, 1.0, 1 + 2.0**-6, 1 + 2.0**-7, -2.5, 3.140625, 0.0, 2.0**-130])
    assert np.array_equal(mlp.bf16_round(x), want)


def test_mlp_oracle_identity_network():
    """n_in = H = n_out, W = I, b = 0 and X >= 0: both ReLUs pass X through, Y = X."""
    from oracle import mlp

    n = 16
    I = np.eye(n).ravel()
    p = np.concatenate([I, np.zeros(n), I, np.zeros(n), I, np.zeros(n)])
    X = np.random.default_rng(1).uniform(0, 1, (5, n))
    Y, _, _ = mlp.forward(p, X, n, n, n, bf16=False)
    assert np.array_equal(Y, X)


def test_mlp_oracle_gradient_matches_finite_differences():
    """Back-propagation of the FP64 network against central differences of
    the loss in every parameter (a dropped term, a wrong transpose or a
    wrong ReLU mask fails this)."""
    from oracle import mlp

    r = np.random.default_rng(2)
    n_in, H, n_out, batch = 5, 16, 3, 7
    P = H * n_in + H + H * H + H + n_out * H + n_out
    p = r.standard_normal(P) * 0.5
    X = r.standard_normal((batch, n_in))
    T = r.standard_normal((batch, n_out))
    wo = np.array([2.0, 0.5, 1.0])
    _, g = mlp.loss_and_grad(p, X, T, n_in, H, n_out, wo, bf16=False)
    h = 1e-6
    num = np.empty(P)
    for i in range(P):
        e = np.zeros(P)
        e[i] = h
        lp, _ = mlp.loss_and_grad(p + e, X, T, n_in, H, n_out, wo, bf16=False)
        lm, _ = mlp.loss_and_grad(p - e, X, T, n_in, H, n_out, wo, bf16=False)
        num[i] = (lp - lm) / (2 * h)
    assert np.abs(num - g).max() <= 1e-6 * max(1.0, np.abs(g).max())


def test_mlp_oracle_adam_first_step_closed_form():
    """From zero moments the bias-corrected first step is lr g / (|g| + eps)."""
    from oracle import mlp

    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p1, m, v = mlp.adam(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, 0.01)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_pencil_sequence_spectrum_is_lambda_of_t():
    """The sequence generator's low-rank update reproduces A(t) = U^T Q(t)
    diag(lam(t)) Q(t)^T U: the generalized eigenvalues of (A(t), B) are
    lam0 + t d (scipy's generalized symmetric eigensolver as the check)."""
    import scipy.linalg

    import inputs

    seq = inputs.PencilSequence(96, seed=4, dt=0.05)
    for k in (0, 3, 17):
        A, B, lam = seq.pencil(k)
        w = scipy.linalg.eigh(A.numpy(), B.numpy(), eigvals_only=True)
        assert np.abs(w - lam.numpy()).max() <= 1e-9 * 1000


def test_structured_pencil_spectrum_is_lambda():
    """The O(n^2) stand-in pencil (reflector Q, banded U): its generalized
    eigenvalues are the drawn lambda (scipy's generalized eigensolver)."""
    import scipy.linalg

    import inputs

    import torch

    A, B, lam = inputs.make_pencil_structured(160, seed=3, reflectors=5, band=3)
    assert torch.equal(A, A.T) and torch.equal(B, B.T)
    w = scipy.linalg.eigh(A.numpy(), B.numpy(), eigvals_only=True)
    assert np.abs(w - lam.numpy()).max() <= 1e-9 * 1000
    assert np.linalg.eigvalsh(B.numpy()).min() > 0.5
