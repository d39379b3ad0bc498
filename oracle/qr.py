"""Economy QR (oracle side).

The paper writes ``[V, ~] = qr(A^T V)`` (Alg. gpowerlu, last step of the
power iteration; Alg. basicpoweriteration2 step 5) for "an orthonormal basis"
of an n x l matrix.  Reading used: the economy (thin) QR, n x l Q with
orthonormal columns, made unique by R_ii >= 0 (columns of Q and rows of R are
negated where Householder gives R_ii < 0).

Method: textbook Householder triangularisation (Golub & Van Loan, Alg. 5.2.1)
followed by backward accumulation of the first l columns of Q.

Pinned by: Q^T Q = I, Q R = X, R upper triangular with R_ii >= 0, and
numpy.linalg.qr with the same sign normalisation.
"""
import numpy as np


def qr_economy(X):
    """Returns (Q, R): X = Q R, Q n x l orthonormal columns, R l x l, R_ii >= 0."""
    R = np.array(X, dtype=np.float64, copy=True)
    n, l = R.shape
    if n < l:
        raise ValueError("qr_economy needs rows >= columns")
    vs = []
    for j in range(l):
        x = R[j:, j].copy()
        normx = np.linalg.norm(x)
        if normx == 0.0:
            vs.append(None)
            continue
        alpha = -normx if x[0] >= 0.0 else normx
        v = x
        v[0] -= alpha
        vnorm = np.linalg.norm(v)
        if vnorm == 0.0:
            vs.append(None)
            continue
        v /= vnorm
        R[j:, j:] -= 2.0 * np.outer(v, v @ R[j:, j:])
        vs.append(v)
    Rout = np.triu(R[:l, :])
    Q = np.zeros((n, l))
    Q[:l, :l] = np.eye(l)
    for j in range(l - 1, -1, -1):
        v = vs[j]
        if v is None:
            continue
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    sign = np.where(np.diag(Rout) < 0.0, -1.0, 1.0)
    Q = Q * sign[None, :]
    Rout = Rout * sign[:, None]
    return Q, Rout
