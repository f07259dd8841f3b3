"""Oracle: Lanczos for the lowest eigenpair of a symmetric linear operator.

Sec. 9.3 of arXiv 2401.01921 (the LinOp paragraph): the Lanczos solver needs
only the action of the operator on a vector (a LinOp), which here is the
H_eff*psi network contraction; it returns the lowest eigenvalues and
eigenvectors.  The paper defers the details to the user guide, so the steps
are the textbook ones (Golub & Van Loan, Matrix Computations, Sec. 10.1;
Parlett, The Symmetric Eigenvalue Problem, Ch. 13):

1. v_0 = psi / ||psi||, beta_0 = 0.
2. for j = 0..K-1: w = H v_j; alpha_j = <v_j, w>; w -= alpha_j v_j + beta_j v_{j-1};
   full reorthogonalisation against v_0..v_j by classical Gram-Schmidt, done
   twice; beta_{j+1} = ||w||; stop if beta_{j+1} < 1e-14 * max(|alpha_i|, beta_i);
   v_{j+1} = w / beta_{j+1}.
3. the lowest eigenvalue of the tridiagonal T (diagonal alpha, off-diagonal
   beta) by Sturm-sequence bisection (count of negative pivots of T - x I)
   until the bracket stops shrinking; its eigenvector y by inverse iteration;
   the Ritz vector is V y (sign: largest |component| of y positive).

Parity: pinned by dense ``numpy.linalg.eigh`` of the operator (independent
library routine) and, through the H_eff network, by the closed-form ground
energies of the open Heisenberg chain for N = 2 and N = 4 sites
(tests/test_oracle_lanczos.py).
"""
from __future__ import annotations

import numpy as np


def sturm_count(alpha, beta, x) -> int:
    """Number of eigenvalues of T below x (negative pivots of the LDL^T of T - xI)."""
    cnt = 0
    d = 1.0
    tiny = 1e-300
    for j in range(len(alpha)):
        b2 = beta[j] * beta[j] if j > 0 else 0.0
        d = (alpha[j] - x) - (b2 / d if j > 0 else 0.0)
        if d == 0.0:
            d = -tiny
        if d < 0:
            cnt += 1
    return cnt


def lowest_eig_bisect(alpha, beta) -> float:
    """Lowest eigenvalue of the symmetric tridiagonal T; beta[j] couples j-1 and j."""
    k = len(alpha)
    r = [abs(beta[j]) if j > 0 else 0.0 for j in range(k)]
    lo = min(alpha[j] - r[j] - (abs(beta[j + 1]) if j + 1 < k else 0.0) for j in range(k))
    hi = max(alpha[j] + r[j] + (abs(beta[j + 1]) if j + 1 < k else 0.0) for j in range(k))
    while True:
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            return hi
        if sturm_count(alpha, beta, mid) >= 1:
            hi = mid
        else:
            lo = mid


def tridiag_eigvec(alpha, beta, lam, iters: int = 3) -> np.ndarray:
    """Eigenvector of T for eigenvalue lam by inverse iteration (Thomas solve)."""
    k = len(alpha)
    shift = lam - 1e-13 * max(1.0, abs(lam))
    y = np.ones(k) / np.sqrt(k)
    for _ in range(iters):
        a = np.array(alpha, dtype=np.float64) - shift
        b = np.array([beta[j] for j in range(1, k)], dtype=np.float64)
        c = b.copy()
        rhs = y.copy()
        for j in range(1, k):
            piv = a[j - 1] if a[j - 1] != 0 else 1e-300
            m = b[j - 1] / piv
            a[j] -= m * c[j - 1]
            rhs[j] -= m * rhs[j - 1]
        x = np.zeros(k)
        x[k - 1] = rhs[k - 1] / (a[k - 1] if a[k - 1] != 0 else 1e-300)
        for j in range(k - 2, -1, -1):
            x[j] = (rhs[j] - c[j] * x[j + 1]) / (a[j] if a[j] != 0 else 1e-300)
        y = x / np.linalg.norm(x)
    if y[np.argmax(np.abs(y))] < 0:
        y = -y
    return y


def lanczos(apply, v0: np.ndarray, nsteps: int, stop_rel: float = 1e-14):
    """Returns (lowest eigenvalue, Ritz vector, alpha list, beta list, matvec count)."""
    v = v0 / np.linalg.norm(v0)
    V = [v]
    alpha, beta = [], [0.0]
    for j in range(nsteps):
        w = apply(V[j])
        a = float(np.dot(V[j], w))
        alpha.append(a)
        w = w - a * V[j]
        if j > 0:
            w = w - beta[j] * V[j - 1]
        for _ in range(2):
            c = np.array([np.dot(u, w) for u in V])
            for cu, u in zip(c, V):
                w = w - cu * u
        b = float(np.linalg.norm(w))
        # negligible against the scale of T seen so far (max |alpha| and max beta): with
        # alpha identically zero, as for the XX chain from a Neel state, max |alpha| alone
        # would never stop an exhausted Krylov space
        if j == nsteps - 1 or b < stop_rel * max(max(abs(x) for x in alpha), max(beta)):
            break
        beta.append(b)
        V.append(w / b)
    k = len(alpha)
    lam = lowest_eig_bisect(alpha, beta[:k])
    y = tridiag_eigvec(alpha, beta[:k], lam)
    x = np.zeros_like(v0, dtype=np.float64)
    for yi, u in zip(y, V[:k]):
        x = x + yi * u
    return lam, x, alpha, beta[1:k], k
