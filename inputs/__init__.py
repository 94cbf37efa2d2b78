"""Seeded synthetic pencils (A, B) with a known generalized spectrum.

Shared by the oracle tests, the GPU parity tests, the smoke check and the
benchmark.  It holds none of the solver's arithmetic: it only draws random
numbers and calls library routines (QR, Cholesky, matmul) to build inputs.

Construction (the workloads stand in for the paper's molecular-dynamics and
DFT pencils of Section 3, n ~ 10^4 - 10^5, whose matrices are not public):

  * G ~ N(0, 1) n-by-n,             B = G G^T / n + I        (SPD, spectrum in ~[1, 5])
  * H ~ N(0, 1) n-by-n, H = Q R,    Q <- Q diag(sign(diag R)) (Haar orthogonal)
  * lambda_i ~ Uniform(0, 1000), sorted ascending
  * U = chol(B) (upper, B = U^T U),  C = Q diag(lambda) Q^T,  A = U^T C U

so that the generalized eigenvalues of (A, B) are lambda by construction and
the eigenvectors are X = U^-1 Q.  Random draws come from a CPU
``torch.Generator`` seeded with ``seed``, in the order G, H, lambda; the
algebra runs in float64 on ``device``.  A and B are exactly symmetric, so
their row-major storage is also their column-major storage.
"""
from __future__ import annotations

import torch


def draw(n: int, seed: int = 0):
    """The raw draws (G, H, lambda) as float64 CPU tensors."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    G = torch.randn(n, n, generator=g, dtype=torch.float64)
    H = torch.randn(n, n, generator=g, dtype=torch.float64)
    lam = torch.rand(n, generator=g, dtype=torch.float64) * 1000.0
    lam, _ = torch.sort(lam)
    return G, H, lam


def make_pencil(n: int, seed: int = 0, device: str | torch.device = "cpu", lam=None, B_identity: bool = False):
    """Return (A, B, lam) on ``device``: A = U^T Q diag(lam) Q^T U, B = U^T U.

    ``lam`` overrides the drawn spectrum (sorted ascending, length n);
    ``B_identity`` makes B = I (the standard problem as a special case).
    """
    G, H, lam0 = draw(n, seed)
    dev = torch.device(device)
    G = G.to(dev)
    H = H.to(dev)
    lam = lam0.to(dev) if lam is None else torch.as_tensor(lam, dtype=torch.float64).to(dev)
    if B_identity:
        B = torch.eye(n, dtype=torch.float64, device=dev)
    else:
        B = G @ G.T
        B /= n
        B += torch.eye(n, dtype=torch.float64, device=dev)
        B = 0.5 * (B + B.T)
    del G
    Q, R = torch.linalg.qr(H)
    del H
    Q *= torch.sign(torch.diagonal(R)).unsqueeze(0)
    del R
    C = (Q * lam.unsqueeze(0)) @ Q.T
    del Q
    U = torch.linalg.cholesky(B).T  # upper
    A = U.T @ C
    del C
    A = A @ U
    del U
    A = 0.5 * (A + A.T)
    return A.contiguous(), B.contiguous(), lam


def make_vector(n: int, seed: int = 0, device="cpu", cols: int | None = None):
    """A seeded N(0, 1) vector (or n-by-cols block) in float64."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed) + 7919)
    shape = (n,) if cols is None else (cols, n)
    v = torch.randn(*shape, generator=g, dtype=torch.float64)
    if cols is not None:
        v = v.T  # column-major n-by-cols view backed by a contiguous cols-by-n buffer
    return v.to(device)


def make_tridiagonal(m: int, seed: int = 0, clustered: bool = False):
    """A seeded symmetric tridiagonal (d, e) of order m; ``clustered`` repeats
    blocks so that eigenvalues come in tight groups."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed) + 104729)
    d = torch.rand(m, generator=g, dtype=torch.float64) * 1000.0
    e = torch.randn(max(m - 1, 0), generator=g, dtype=torch.float64) * 10.0
    if clustered and m >= 8:
        k = m // 4
        d[k : 2 * k] = d[:k]
        e[k : 2 * k - 1] = e[: k - 1]
        e[k - 1] = 1e-9
        if 2 * k - 1 < m - 1:
            e[2 * k - 1] = 1e-9
    return d, e
