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


class PencilSequence:
    """A seeded sequence of related pencils with a known spectrum: B is fixed
    (as in make_pencil) and, for t = dt k,

        A(t) = U^T Q(t) diag(lam(t)) Q(t)^T U,   lam(t) = lam0 + t d,
        Q(t) = H_r(t) ... H_1(t) Q0,   H_j(t) = I - 2 v_j(t) v_j(t)^T,
        v_j(t) = (v_j0 + t v_j1) / ||v_j0 + t v_j1||,

    with Q0 Haar, lam0 ~ U(0, 1000), d, v_j0, v_j1 ~ N(0, 1) (drawn in the
    order G, H, lam0, d, v0, v1 from a CPU generator seeded with seed).  The
    generalized eigenvalues of (A(t), B) are lam(t).  The reflectors enter
    through their compact WY form H(t) = I - W Y^T, so that with the
    precomputed A0 = U^T C0 U and A1 = U^T D0 U (C0 = Q0 diag(lam0) Q0^T,
    D0 = Q0 diag(d) Q0^T) each A(t) costs O(n^2 r):

        A(t) = A0 + t A1 - F P^T - P F^T + P (Y^T G) P^T,
        P = U^T W,  G = (C0 + t D0) Y,  F = U^T G.

    The stand-in for the related problems of a DFT self-consistency cycle.
    """

    def __init__(self, n: int, seed: int = 0, device="cpu", reflectors: int = 8, dt: float = 0.005):
        g = torch.Generator(device="cpu")
        g.manual_seed(int(seed))
        dev = torch.device(device)
        self.n, self.dt, self.device = n, dt, dev
        G = torch.randn(n, n, generator=g, dtype=torch.float64)
        H = torch.randn(n, n, generator=g, dtype=torch.float64)
        self.lam0 = torch.rand(n, generator=g, dtype=torch.float64).mul_(1000.0).to(dev)
        self.d = torch.randn(n, generator=g, dtype=torch.float64).to(dev)
        self.v0 = torch.randn(n, reflectors, generator=g, dtype=torch.float64).to(dev)
        self.v1 = torch.randn(n, reflectors, generator=g, dtype=torch.float64).to(dev)
        G = G.to(dev)
        B = G @ G.T
        B /= n
        B += torch.eye(n, dtype=torch.float64, device=dev)
        self.B = (0.5 * (B + B.T)).contiguous()
        del G, B
        self.U = torch.linalg.cholesky(self.B).T.contiguous()  # upper, B = U^T U
        Q, R = torch.linalg.qr(H.to(dev))
        Q *= torch.sign(torch.diagonal(R)).unsqueeze(0)
        del R, H
        self.C0 = (Q * self.lam0.unsqueeze(0)) @ Q.T
        self.D0 = (Q * self.d.unsqueeze(0)) @ Q.T
        del Q
        self.A0 = self.U.T @ (self.C0 @ self.U)
        self.A1 = self.U.T @ (self.D0 @ self.U)

    def lam(self, k: int):
        """lam(t_k), ascending."""
        return torch.sort(self.lam0 + (self.dt * k) * self.d).values

    def pencil(self, k: int):
        """(A(t_k), B, lam(t_k) ascending); A is a new tensor, B the shared one."""
        t = self.dt * k
        V = self.v0 + t * self.v1
        V = V / V.norm(dim=0, keepdim=True)
        W = 2.0 * V[:, :1]
        Y = V[:, :1].clone()
        for j in range(1, V.shape[1]):
            v = V[:, j : j + 1]
            Y = torch.cat([Y, v - Y @ (W.T @ v)], dim=1)
            W = torch.cat([W, 2.0 * v], dim=1)
        P = self.U.T @ W
        Gm = self.C0 @ Y + t * (self.D0 @ Y)
        F = self.U.T @ Gm
        A = self.A0 + t * self.A1 - F @ P.T - P @ F.T + P @ (Y.T @ Gm) @ P.T
        A = 0.5 * (A + A.T)
        return A.contiguous(), self.B, self.lam(k)


def make_pencil_structured(n: int, seed: int = 0, device="cpu", reflectors: int = 16, band: int = 8,
                           dtype=torch.float64):
    """A dense pencil with a known spectrum, built in O(n^2 (r + w)) work for
    orders where the construction of make_pencil (a Haar Q and G G^T, about
    6 n^3 flops) is out of reach (n = 65536: ~30 minutes of GB300 FP64):

      * lambda_i ~ Uniform(0, 1000), sorted (as make_pencil);
      * Q = H_r ... H_1, H_j = I - 2 v_j v_j^T, v_j ~ N(0, 1) normalised
        (r = 16 reflectors: a dense orthogonal matrix, not Haar);
      * B = U^T U with U = I + N, N strictly upper triangular with `band`
        nonzero superdiagonals of N(0, 0.05 / band) entries (kappa(B) ~ 1);
      * C = Q diag(lambda) Q^T (each reflector a symmetric rank-2 update in
        place), A = U^T C U.

    The generalized eigenvalues are lambda by construction.  Draws from a CPU
    generator seeded with seed, in the order lambda, v, N.  A and B are dense
    n x n, exactly symmetric.  Returns (A, B, lambda)."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    dev = torch.device(device)
    lam = torch.sort(torch.rand(n, generator=g, dtype=torch.float64) * 1000.0).values
    V = torch.randn(n, reflectors, generator=g, dtype=torch.float64)
    V /= V.norm(dim=0, keepdim=True)
    Nd = torch.randn(band, n, generator=g, dtype=torch.float64) * (0.05 / band)
    lam, V, Nd = lam.to(dev), V.to(dev), Nd.to(dev)
    C = torch.diag(lam)
    for j in range(reflectors):
        v = V[:, j]
        u = C @ v
        y = 2.0 * u - (2.0 * torch.dot(v, u)) * v
        C.addr_(v, y, alpha=-1.0)  # H C H = C - v y^T - y v^T
        C.addr_(y, v, alpha=-1.0)
    # M = C U (columns: M[:, j] = C[:, j] + sum_d C[:, j - d] N[j - d, j])
    A = C.clone()
    for d in range(1, band + 1):
        A[:, d:].addcmul_(C[:, :-d], Nd[d - 1, d:].unsqueeze(0))
    del C
    # A = U^T M (rows: A[i, :] = M[i, :] + sum_d N[i - d, i] M[i - d, :]); M rows i - d read before row i changes
    M = A.clone()
    for d in range(1, band + 1):
        A[d:, :].addcmul_(M[:-d, :], Nd[d - 1, d:].unsqueeze(1))
    del M
    A = 0.5 * (A + A.T) if n <= 8192 else _symmetrize_inplace(A)
    # B = U^T U = I + N + N^T + N^T N
    B = torch.eye(n, dtype=torch.float64, device=dev)
    for d in range(1, band + 1):
        B.diagonal(d).add_(Nd[d - 1, d:])
        B.diagonal(-d).add_(Nd[d - 1, d:])
    # N^T N: entry (i, j) = sum_k N[k, i] N[k, j]; with band w it is banded of width w
    Nm = torch.zeros(band + 1, n, dtype=torch.float64, device=dev)  # Nm[d, j] = N[j - d, j]
    Nm[1:, :] = Nd
    for di in range(1, band + 1):
        for dj in range(1, band + 1):
            # k = i - di = j - dj  =>  j = i - di + dj
            off = dj - di
            if off >= 0:
                i = torch.arange(di, n - off, device=dev)
                B[i, i + off] += Nm[di, i] * Nm[dj, i + off]
                if off > 0:
                    B[i + off, i] += Nm[di, i] * Nm[dj, i + off]
    return A.contiguous(), B.contiguous(), lam


def _symmetrize_inplace(A, blk: int = 4096):
    """A <- (A + A^T) / 2 block by block (no n x n temporary)."""
    n = A.shape[0]
    for i in range(0, n, blk):
        for j in range(i, n, blk):
            a = A[i:i + blk, j:j + blk]
            b = A[j:j + blk, i:i + blk]
            m = 0.5 * (a + b.T)
            a.copy_(m)
            b.copy_(m.T)
    return A
