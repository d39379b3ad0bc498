"""Partial-pivoting LU (oracle side).

The paper writes every LU as MATLAB's builtin ``lu`` (Sec. 2, "lu(.)"):
``[L, U, P] = lu(Y)`` gives P Y = L U with L unit lower trapezoidal and U
upper trapezoidal (Alg. rlu step 3, Alg. bpowerlu steps 4 and 6), and the
two-output form ``[L, ~] = lu(X)`` gives the *permuted* factor P^T L, whose
rows line up with the rows of X (Alg. basicpoweriteration step 4 writes
L = P^T L explicitly; Alg. gpowerlu uses the two-output form).

Readings (the paper is silent on them):
* pivot of column j: the entry of largest magnitude among the rows not yet
  pivoted, ties going to the row that comes first in the current (swapped)
  row order -- the rule of LAPACK's getf2 behind MATLAB's ``lu``;
* multipliers as LAPACK's getf2 / getrf2 form them (the LU behind MATLAB's
  ``lu``): a_ij times the reciprocal 1 / u_jj when |u_jj| is at least the
  smallest normal number, else a_ij / u_jj;
* a column whose candidates are all exactly zero is skipped: no swap, no
  division, its multipliers stay 0, and ``info`` records the first such
  column (1-based), as LAPACK does.

Pinned by: exact rational elimination on small inputs (Python fractions),
scipy.linalg.lu (LAPACK getrf) pivots on random panels, and P X = L U.
"""
import numpy as np

_SMALLEST_NORMAL = np.finfo(np.float64).tiny      # 2^-1022


def getrf(X):
    """Right-looking LU with row swaps.

    Returns (perm, L, U, info) with X[perm] = L @ U, perm[pos] = original row
    index at position pos, L m x r unit lower trapezoidal, U r x n upper
    trapezoidal, r = min(m, n)."""
    A = np.array(X, dtype=np.float64, order="C", copy=True)
    m, n = A.shape
    r = min(m, n)
    perm = np.arange(m)
    info = 0
    for j in range(r):
        i = j + int(np.argmax(np.abs(A[j:, j])))
        if A[i, j] != 0.0:
            if i != j:
                A[[j, i], :] = A[[i, j], :]
                perm[[j, i]] = perm[[i, j]]
            piv = A[j, j]
            if abs(piv) >= _SMALLEST_NORMAL:
                A[j + 1:, j] = A[j + 1:, j] * (1.0 / piv)
            else:
                A[j + 1:, j] = A[j + 1:, j] / piv
        elif info == 0:
            info = j + 1
        if j + 1 < n and j + 1 < m:
            A[j + 1:, j + 1:] -= np.outer(A[j + 1:, j], A[j, j + 1:])
    L = np.tril(A[:, :r], -1) + np.eye(m, r)
    U = np.triu(A[:r, :])
    return perm, L, U, info


def lu_full(Y):
    """[L, U, P] = lu(Y): returns (perm, L, U, info) with Y[perm] = L U."""
    return getrf(Y)


def lu_permuted_L(X):
    """[L, ~] = lu(X): the permuted unit lower factor P^T L (m x r)."""
    perm, L, _, _ = getrf(X)
    Lp = np.empty_like(L)
    Lp[perm, :] = L
    return Lp
