"""Error measures used by the paper's experiments (oracle side).

* relative Frobenius error ||A - A_k||_F / ||A||_F (Eq. error), with
  A_k = P^T L U Q for the LU factorisations;
* the Eckart-Young optimum sqrt(sum_{i>k} sigma_i^2) (Eq. ey) and the
  smallest rank that meets a relative tolerance (Sec. 6.4, "Truncated SVD");
* the sine of the largest principal angle between two column spaces, used
  to compare ranges (Thm. acc:t, and the Remark that re-orthogonalisation
  leaves the range unchanged in exact arithmetic).
"""
import numpy as np


def rel_lu_error(A, p, q, L, U):
    A = np.asarray(A, dtype=np.float64)
    R = A[np.asarray(p)][:, np.asarray(q)] - L @ U
    return float(np.linalg.norm(R) / np.linalg.norm(A))


def eckart_young_error(sigma, k):
    """Relative optimal rank-k Frobenius error from the singular values."""
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    return float(np.sqrt(np.sum(s2[k:]) / np.sum(s2)))


def eckart_young_rank(sigma, eps):
    """Smallest k with relative optimal Frobenius error <= eps."""
    s2 = np.sort(np.asarray(sigma, dtype=np.float64))[::-1] ** 2
    total = np.sum(s2)
    tail = total - np.concatenate([[0.0], np.cumsum(s2)])   # tail[k] = sum_{i>k}
    tail = np.maximum(tail, 0.0)
    ok = np.sqrt(tail / total) <= eps
    return int(np.argmax(ok)) if ok.any() else len(s2)


def max_principal_sine(X, Y):
    """sin of the largest principal angle between range(X) and range(Y)
    (equal column counts): ||(I - Qx Qx^T) Qy||_2."""
    Qx, _ = np.linalg.qr(np.asarray(X, dtype=np.float64))
    Qy, _ = np.linalg.qr(np.asarray(Y, dtype=np.float64))
    Rm = Qy - Qx @ (Qx.T @ Qy)
    return float(np.linalg.norm(Rm, 2))
