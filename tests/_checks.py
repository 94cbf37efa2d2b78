"""Accuracy measures used by the parity tests (numpy, float64, host side).

eta_i: normwise backward error of the pair (lambda_i, x_i) of the pencil
(A, B):  ||A x - lambda B x||_2 / ((||A||_2 + |lambda| ||B||_2) ||x||_2).
The paper's own Frobenius ratios (Tables 3 and 7) are reported alongside.
"""
import numpy as np


def norm2_est(M: np.ndarray, iters: int = 30, seed: int = 0) -> float:
    """Largest singular value of a symmetric M by power iteration."""
    v = np.random.default_rng(seed).standard_normal(M.shape[0])
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = M @ v
        lam = np.linalg.norm(w)
        if lam == 0.0:
            return 0.0
        v = w / lam
    return float(lam)


def eta(A, B, w, X, nA=None, nB=None) -> np.ndarray:
    nA = norm2_est(A) if nA is None else nA
    nB = norm2_est(B) if nB is None else nB
    R = A @ X - (B @ X) * w
    return np.linalg.norm(R, axis=0) / ((nA + np.abs(w) * nB) * np.linalg.norm(X, axis=0))


def b_orth_err(B, X) -> float:
    s = X.shape[1]
    return float(np.abs(X.T @ B @ X - np.eye(s)).max())


def paper_metrics(A, B, w, X):
    """Table 3 / 7: ||I - X^T B X||_F / ||B||_F and ||A X - B X L||_F / max(||A||_F, ||B||_F)."""
    s = X.shape[1]
    o = np.linalg.norm(np.eye(s) - X.T @ B @ X) / np.linalg.norm(B)
    r = np.linalg.norm(A @ X - (B @ X) * w) / max(np.linalg.norm(A), np.linalg.norm(B))
    return float(o), float(r)


def clusters(w: np.ndarray, thresh: float):
    """Maximal runs of indices whose consecutive gaps are below thresh."""
    out, start = [], 0
    for i in range(1, len(w) + 1):
        if i == len(w) or w[i] - w[i - 1] >= thresh:
            out.append((start, i))
            start = i
    return out


def max_subspace_angle(B, Xa, Xb, w, w_all_ref, cnorm: float, res_bound: float):
    """Largest principal angle, in the B inner product, between the
    cluster subspaces spanned by Xa and Xb, together with the bound it is
    held to.  Clusters are runs of consecutive gaps below 1e-6 ||C||.  The
    bound is the Davis-Kahan sin-theta bound with residual res_bound
    (absolute, standard-form), res_bound / gap_ext, floored at 1e-9;
    gap_ext is the distance from the cluster to the rest of the reference
    spectrum.  Returns (angle, bound) for the cluster with the largest ratio."""
    worst, worst_lim = 0.0, 1.0
    for a, b in clusters(w, 1e-6 * cnorm):
        # sin of the largest angle from the B-orthogonal residual of the
        # projection (no cancellation, unlike 1 - cos^2)
        Xa_c, Xb_c = Xa[:, a:b], Xb[:, a:b]
        R = Xa_c - Xb_c @ (Xb_c.T @ B @ Xa_c)
        ev = np.linalg.eigvalsh(R.T @ B @ R)
        ang = float(np.sqrt(max(0.0, ev.max())))
        lo, hi = w[a], w[b - 1]
        others = w_all_ref[(w_all_ref < lo - 1e-6 * cnorm) | (w_all_ref > hi + 1e-6 * cnorm)]
        gap = float(np.min(np.minimum(np.abs(others - lo), np.abs(others - hi)))) if len(others) else cnorm
        lim = max(1e-9, res_bound / max(gap, 1e-300))
        if ang / lim > worst / worst_lim:
            worst, worst_lim = ang, lim
    return worst, worst_lim
