"""Writes pencil4_exact.txt: a 4-by-4 pencil whose generalized eigenvalues are
known exactly.  Eq. 3 says (A, B) and C = U^-T A U^-1 share eigenvalues when
B = U^T U; so A = U^T C U with C = H diag(1, 2, 3, 4) H^T (H the orthogonal,
symmetric Hadamard matrix / 2) has eigenvalues 1, 2, 3, 4 and eigenvectors
X = U^-1 H.  Every entry is a dyadic rational, so the file is exact in
binary floating point.  Pure rational arithmetic; uses no solver code."""
from fractions import Fraction as F
import os

n = 4
H = [[F(s, 2) for s in row] for row in [[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]]]
U = [[F(x) for x in r] for r in [[1, 1, 0, 0], [0, 2, 1, 0], [0, 0, 1, 1], [0, 0, 0, 2]]]
lam = [F(1), F(2), F(3), F(4)]


def mm(X, Y):
    return [[sum(X[i][k] * Y[k][j] for k in range(n)) for j in range(n)] for i in range(n)]


def tr(X):
    return [[X[j][i] for j in range(n)] for i in range(n)]


L = [[lam[i] if i == j else F(0) for j in range(n)] for i in range(n)]
A = mm(tr(U), mm(mm(H, mm(L, tr(H))), U))
B = mm(tr(U), U)
out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pencil4_exact.txt")
with open(out, "w") as f:
    f.write("# Exact 4x4 symmetric-definite pencil (Eq. 1) built as A = U^T C U, B = U^T U (Eq. 2, 3)\n")
    f.write("# with C = H diag(1,2,3,4) H^T, H = Hadamard/2; generalized eigenvalues are exactly 1 2 3 4.\n")
    f.write("# Written by make_pencil4_exact.py (rational arithmetic only).\n")
    for name, M in (("A", A), ("B", B), ("U", U)):
        for r in M:
            f.write(name + " " + " ".join(str(x) for x in r) + "\n")
    f.write("lambda " + " ".join(str(x) for x in lam) + "\n")
