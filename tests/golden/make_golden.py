"""Write exact rational least-squares fixtures (tests/golden/*.txt).

The paper prints no worked example, so each fixture is an exact construction
from the definitions it relies on (Eq. opt:lls, Eq. qr_lls, Eq. recqr):

  * W = (I - S)(I + S)^{-1} with S skew-symmetric and rational is an exactly
    orthogonal rational m x m matrix (Cayley transform).
  * Q = W[:, :n], R rational upper triangular with positive diagonal,
    A = Q R: then (Q, R) is THE reduced QR of A with positive diagonal.
  * b = A x + W[:, n:] c: the second term is orthogonal to range(A), so x is
    the exact least-squares solution and r = W[:, n:] c the exact residual.

Everything is computed in Python Fractions; no oracle or GPU code is called.
Each file stores m, n and the exact entries of A, R, Q, x, b, r as p/q strings.
Run: python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import random
from fractions import Fraction as F

HERE = os.path.dirname(os.path.abspath(__file__))


def mat_mul(X, Y):
    return [[sum(X[i][k] * Y[k][j] for k in range(len(Y))) for j in range(len(Y[0]))]
            for i in range(len(X))]


def mat_inv(X):
    n = len(X)
    M = [row[:] + [F(int(i == j)) for j in range(n)] for i, row in enumerate(X)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [v / piv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [row[n:] for row in M]


def cayley(m, rnd):
    S = [[F(0)] * m for _ in range(m)]
    for i in range(m):
        for j in range(i + 1, m):
            v = F(rnd.randint(-3, 3), rnd.randint(1, 3))
            S[i][j], S[j][i] = v, -v
    I = [[F(int(i == j)) for j in range(m)] for i in range(m)]
    ImS = [[I[i][j] - S[i][j] for j in range(m)] for i in range(m)]
    IpS = [[I[i][j] + S[i][j] for j in range(m)] for i in range(m)]
    return mat_mul(ImS, mat_inv(IpS))


def make(name, m, n, seed):
    rnd = random.Random(seed)
    W = cayley(m, rnd)
    Q = [row[:n] for row in W]
    R = [[F(0)] * n for _ in range(n)]
    for i in range(n):
        R[i][i] = F(rnd.randint(1, 6), rnd.randint(1, 2))
        for j in range(i + 1, n):
            R[i][j] = F(rnd.randint(-5, 5), rnd.randint(1, 4))
    A = mat_mul(Q, R)
    x = [F(rnd.randint(-4, 4), rnd.randint(1, 3)) for _ in range(n)]
    c = [F(rnd.randint(-2, 2), rnd.randint(1, 5)) for _ in range(m - n)]
    Ax = [sum(A[i][j] * x[j] for j in range(n)) for i in range(m)]
    r = [sum(W[i][n + k] * c[k] for k in range(m - n)) for i in range(m)]
    b = [Ax[i] + r[i] for i in range(m)]
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        f.write(f"# exact construction (Eq. recqr / Eq. qr_lls): A = Q R, b = A x + r, r orthogonal to range(A)\n")
        f.write(f"# generated by tests/golden/make_golden.py, seed {seed}\n")
        f.write(f"m {m}\nn {n}\n")
        for tag, M in (("A", A), ("R", R), ("Q", Q)):
            for i, row in enumerate(M):
                f.write(f"{tag} {i} " + " ".join(str(v) for v in row) + "\n")
        f.write("x " + " ".join(str(v) for v in x) + "\n")
        f.write("b " + " ".join(str(v) for v in b) + "\n")
        f.write("r " + " ".join(str(v) for v in r) + "\n")


if __name__ == "__main__":
    make("lls_exact_6x3.txt", 6, 3, seed=5)
    make("lls_exact_9x4.txt", 9, 4, seed=7)
    make("lls_exact_5x1.txt", 5, 1, seed=11)
