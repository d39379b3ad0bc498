"""Products with a sparse A held in compressed sparse rows (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The sparse runtime
experiment of Sec. 6 runs the algorithms on MATLAB ``sprand`` matrices; the
only operation that changes is the product with A or A^T, which here is the
plain definition over the stored entries:

  (A X)(i, :)   = sum over t in row i of   val[t] X(col[t], :)
  (A^T Z)(j, :) = sum over t with col[t] = j of   val[t] Z(row(t), :)

Both are computed from the CSR of A alone (the transposed product scatters
by column), in float64.  ``SparsePassCounter`` offers the interface of
``PassCounter`` so that every algorithm of ``oracle.powerlu`` runs on it
unchanged.  Pinned by the ``-m "not gpu"`` tests against the dense product
of the same matrix and against scipy.sparse.
"""
import numpy as np

# entries handled per chunk, so that a product never holds more than about
# this many rows of X at once
_CHUNK = 1 << 16


def _rows_of(row_ptr):
    counts = np.diff(np.asarray(row_ptr, dtype=np.int64))
    return np.repeat(np.arange(counts.size, dtype=np.int64), counts)


def _accumulate(nout, dst, src, val, B):
    """Y(dst[t], :) += val[t] B(src[t], :) for t in order."""
    Y = np.zeros((nout, B.shape[1]))
    for s in range(0, dst.size, _CHUNK):
        e = min(dst.size, s + _CHUNK)
        np.add.at(Y, dst[s:e], val[s:e, None] * B[src[s:e]])
    return Y


def _select(out_idx, sel):
    """Entries whose output index is in sel, renumbered to positions in sel."""
    sel = np.asarray(sel, dtype=np.int64)
    keep = np.isin(out_idx, sel)
    pos = np.full(max(int(out_idx.max(initial=0)), int(sel.max(initial=0))) + 1, -1,
                  dtype=np.int64)
    pos[sel] = np.arange(sel.size)
    return keep, pos


def csr_mul(m, row_ptr, col_idx, val, X, rows=None):
    """A X for the m-row CSR (row_ptr, col_idx, val); X has n rows.  With
    ``rows``, only those rows of A X (in that order)."""
    X = np.asarray(X, dtype=np.float64)
    r = _rows_of(row_ptr)
    c = np.asarray(col_idx, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    if rows is None:
        return _accumulate(m, r, c, val, X)
    keep, pos = _select(r, rows)
    return _accumulate(len(rows), pos[r[keep]], c[keep], val[keep], X)


def csr_tmul(n, row_ptr, col_idx, val, Z, rows=None):
    """A^T Z for the same CSR of A (n columns); Z has m rows.  With
    ``rows``, only those rows of A^T Z (columns of A), in that order."""
    Z = np.asarray(Z, dtype=np.float64)
    r = _rows_of(row_ptr)
    c = np.asarray(col_idx, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    if rows is None:
        return _accumulate(n, c, r, val, Z)
    keep, pos = _select(c, rows)
    return _accumulate(len(rows), pos[c[keep]], r[keep], val[keep], Z)


class SparsePassCounter:
    """A sparse m x n A (CSR, each position stored once); every product with
    A or A^T counts as one pass over A, as in ``PassCounter``."""

    def __init__(self, m, n, row_ptr, col_idx, val):
        self.m, self.n = int(m), int(n)
        self.row_ptr = np.asarray(row_ptr, dtype=np.int64)
        self.col_idx = np.asarray(col_idx, dtype=np.int64)
        self.val = np.asarray(val, dtype=np.float64)
        self.passes = 0

    @property
    def shape(self):
        return (self.m, self.n)

    def frob2(self):            # ||A||_F^2 (positions unique)
        return float(np.sum(self.val * self.val))

    def mul(self, X):           # A X
        self.passes += 1
        return csr_mul(self.m, self.row_ptr, self.col_idx, self.val, X)

    def tmul(self, Z):          # A^T Z
        self.passes += 1
        return csr_tmul(self.n, self.row_ptr, self.col_idx, self.val, Z)
