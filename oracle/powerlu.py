"""PowerLU and its relatives, step by step as the paper states them (oracle).

Each function follows one algorithm of Zhang & Mascagni (arXiv 2002.07138)
in its order and notation.  Every product with A or A^T goes through a
``PassCounter`` so that tests can count the passes over A (Sec. 3.3: RandLU
reads A 2p+2 times, PowerLU with Alg. gpowerlu exactly v times).

Readings of silent or garbled points:
* p = floor((v - 1)/2) inside Alg. gpowerlu (its statement); the "v = 2p+2"
  of Sec. 6 only maps experiment labels and is not used here;
* the output of Alg. basicpoweriteration2 is n x l, a basis of
  (A^T A)^p Omega (its "m x l ... (A A^T)^p" header is a typo);
* Y = A V(:, 1:k) uses the first k basis columns (Alg. bpowerlu step 3);
* P A Q^T = L U with Q the row permutation of lu(B^T) (Eq. secondlu gives
  Q B^T = L2 U2, hence B = U2^T L2^T Q);
* blocked rank determination (Alg. adaptivewithoutupdating) stops at the
  first block with E <= eps^2 ||A||_F^2; the precise variant (Sec. 6.4)
  replaces the block test by a per-column loop over G(:, t1 + j - 1),
  j = 1..b, with the same "<=" test; k is the number of columns consumed;
  a partial last block is used when b does not divide l; if the tolerance
  is not met within l columns, k = l and the status says so;
* Alg. singlepasslu: Omega is m x k (its step 1), G^{dagger T} = G (G^T G)^-1,
  U = L2^T (Sec. 5, "U = L_2^T");
* Alg. rlu: "LU with column pivoting" of the k x n matrix B is lu(B^T):
  Q B^T = L' U', L_b = U'^T, U_b = L'^T;
* the restart of the Remark after Alg. adaptivewithoutupdating: when the l
  columns of a round leave E > eps^2 ||A||_F^2, the next round reruns the
  algorithm on the remainder A_r = A - A W W^T (W = every basis column so
  far) with a fresh Gaussian matrix (Philox streams shifted by 16 per round),
  the indicator E carrying over; the remainder is applied as
  A_r X = A X - G (W^T X), A_r^T Z = A^T Z - W (G^T Z) with G = A W the
  stacked G's of the earlier rounds (equal in exact arithmetic, since each
  round's basis lies in the row space of its remainder, orthogonal to W);
  k is the total number of columns consumed and Alg. powerlufp's tail runs
  on [G] and [W].
"""
import numpy as np

from .gaussian import gaussian_matrix
from .philox import STREAM_OMEGA_N, STREAM_OMEGA_M, STREAM_OMEGA_SP
from .lu import getrf, lu_permuted_L
from .qr import qr_economy
from .sparse import SparsePassCounter


class PassCounter:
    """Wraps A; every product with A or A^T counts as one pass over A."""

    def __init__(self, A):
        self.A = np.asarray(A, dtype=np.float64)
        self.passes = 0

    @property
    def shape(self):
        return self.A.shape

    def frob2(self):            # ||A||_F^2
        return float(np.sum(self.A * self.A))

    def mul(self, X):           # A X
        self.passes += 1
        return self.A @ X

    def tmul(self, X):          # A^T X
        self.passes += 1
        return self.A.T @ X


def _wrap(A):
    return A if isinstance(A, (PassCounter, Remainder, SparsePassCounter)) else PassCounter(A)


class Remainder:
    """A_r = A - A W W^T applied through G = A W (see the module notes);
    every product is one pass over A."""

    def __init__(self, Ac, W, G):
        self.base = Ac
        self.W = W
        self.G = G

    @property
    def A(self):
        return self.base.A

    @property
    def shape(self):
        return self.base.shape

    def frob2(self):            # ||A||_F^2 of the original A
        return self.base.frob2()

    @property
    def passes(self):
        return self.base.passes

    def mul(self, X):           # A_r X
        return self.base.mul(X) - self.G @ (self.W.T @ X)

    def tmul(self, Z):          # A_r^T Z
        return self.base.tmul(Z) - self.W @ (self.G.T @ Z)


RESTART_STREAM_STRIDE = 16       # Philox stream shift per restart round


def gpowerlu(A, l, v, seed, stream_shift=0):
    """Alg. gpowerlu: orthonormal basis V (n x l) of (A^T A)^p A^T Omega
    (v even, Omega m x l) or (A^T A)^p Omega (v odd, Omega n x l),
    p = floor((v-1)/2), with LU re-orthogonalisation between passes and a
    QR at the end.  Uses v - 1 passes over A."""
    Ac = _wrap(A)
    m, n = Ac.shape
    if v < 2:
        raise ValueError("v >= 2 required (Alg. gpowerlu)")
    p = (v - 1) // 2
    if v % 2 == 0:
        Omega = gaussian_matrix(m, l, seed, STREAM_OMEGA_M + stream_shift)
        if v > 2:
            V = lu_permuted_L(Ac.tmul(Omega))
        else:
            V, _ = qr_economy(Ac.tmul(Omega))
    else:
        V = gaussian_matrix(n, l, seed, STREAM_OMEGA_N + stream_shift)
    for i in range(1, p + 1):
        V = lu_permuted_L(Ac.mul(V))
        if i == p:
            V, _ = qr_economy(Ac.tmul(V))
        else:
            V = lu_permuted_L(Ac.tmul(V))
    return V


def _lu_tail(Y, Vk):
    """Alg. bpowerlu steps 4-8 (= Alg. powerlufp steps 2-6)."""
    p, L1, U1, info1 = getrf(Y)           # P Y = L1 U1
    Bt = Vk @ U1.T                        # B = U1 Vk^T
    q, L2, U2, info2 = getrf(Bt)          # Q B^T = L2 U2
    L = L1 @ U2.T
    U = L2.T
    return p, q, L, U, (info1, info2)


def powerlu(A, k, l, v, seed, return_basis=False):
    """Alg. bpowerlu with steps 1-2 replaced by Alg. gpowerlu.
    Returns (p, q, L, U): A[p][:, q] ~= L U, L m x k, U k x n."""
    Ac = _wrap(A)
    V = gpowerlu(Ac, l, v, seed)
    Vk = V[:, :k]
    Y = Ac.mul(Vk)
    p, q, L, U, info = _lu_tail(Y, Vk)
    if return_basis:
        return p, q, L, U, V, info
    return p, q, L, U


def rank_scan(G, normA2, eps, b, precise=False, E_start=None):
    """The loop of Alg. adaptivewithoutupdating (steps 4-10), or with the
    per-column refinement of Sec. 6.4, on G = A V and E = ||A||_F^2 (or the
    indicator E_start carried over from an earlier round).
    Returns (k, E, met)."""
    E = float(normA2) if E_start is None else float(E_start)
    acc = eps * eps * float(normA2)
    l = G.shape[1]
    k = 0
    met = False
    nblocks = (l + b - 1) // b
    for i in range(1, nblocks + 1):
        t1 = (i - 1) * b
        t2 = min(i * b, l)
        if precise:
            for j in range(t1, t2):
                E -= float(np.sum(G[:, j] * G[:, j]))
                k = j + 1
                if E <= acc:
                    met = True
                    break
        else:
            blk = G[:, t1:t2]
            E -= float(np.sum(blk * blk))
            k = t2
            if E <= acc:
                met = True
        if met:
            break
    return k, E, met


def adaptive_rank(A, eps, b, l, v, seed, precise=False):
    """Alg. adaptivewithoutupdating (precise=True: with the per-column loop
    of Sec. 6.4).  Returns (k, V, G, E, met): V n x l, G = A V m x l, E the
    residual indicator after k columns (Thm. errorerror), met whether
    E <= eps^2 ||A||_F^2 was reached."""
    Ac = _wrap(A)
    E0 = Ac.frob2()
    V = gpowerlu(Ac, l, v, seed)
    G = Ac.mul(V)
    k, E, met = rank_scan(G, E0, eps, b, precise)
    return k, V, G, E, met


def adaptive_rank_restart(A, eps, b, l, v, seed, precise=False, max_rounds=1):
    """Alg. adaptivewithoutupdating with the restart of its Remark: up to
    max_rounds rounds, round r on the remainder of the r earlier bases.
    Returns (k, W, G, E, met, rounds): W n x k, G = A W m x k."""
    Ac = _wrap(A)
    m, n = Ac.shape
    nA2 = Ac.frob2()
    W = np.zeros((n, 0))
    G = np.zeros((m, 0))
    E = nA2
    met = False
    rounds = 0
    for r in range(max_rounds):
        Ar = Ac if r == 0 else Remainder(Ac, W, G)
        V = gpowerlu(Ar, l, v, seed, stream_shift=RESTART_STREAM_STRIDE * r)
        Gr = Ar.mul(V)
        kr, E, met = rank_scan(Gr, nA2, eps, b, precise, E_start=E)
        W = np.hstack([W, V[:, :kr]])
        G = np.hstack([G, Gr[:, :kr]])
        rounds = r + 1
        if met:
            break
    return W.shape[1], W, G, E, met, rounds


def powerlu_fp(A, eps, b, l, v, seed, precise=False, max_rounds=1):
    """Alg. powerlufp (with max_rounds > 1: the restart of the Remark after
    Alg. adaptivewithoutupdating).  Returns (k, p, q, L, U, E, met)."""
    Ac = _wrap(A)
    k, W, G, E, met, _ = adaptive_rank_restart(Ac, eps, b, l, v, seed, precise, max_rounds)
    p, q, L, U, _ = _lu_tail(G, W)
    return k, p, q, L, U, E, met


def basic_power_iteration_lu(A, l, p, seed):
    """Alg. basicpoweriteration: returns (perm, Ly, Uy) of the last full LU,
    P (A (A^T A)^p Omega) = Ly Uy up to the re-orthogonalisation."""
    Ac = _wrap(A)
    m, n = Ac.shape
    Omega = gaussian_matrix(n, l, seed, STREAM_OMEGA_N)
    perm, L, U, _ = getrf(Ac.mul(Omega))
    if p > 0:
        Lp = np.empty_like(L)
        Lp[perm, :] = L
        L = Lp
        for i in range(1, p + 1):
            L = lu_permuted_L(Ac.tmul(L))
            if i == p:
                perm, L, U, _ = getrf(Ac.mul(L))
            else:
                L = lu_permuted_L(Ac.mul(L))
    return perm, L, U


def randlu(A, k, l, p, seed):
    """Alg. rlu with steps 1-3 replaced by Alg. basicpoweriteration.
    Returns (P, Q, L, U) as index vectors: A[P][:, Q] ~= L U.
    Pinned by: the pass count 2p + 2; Thm. acc:t (same range as PowerLU);
    the tail identity L U = (Pi P A) Q^T with Pi the orthogonal projector
    onto range(L_y(:, 1:k)) (Eq. pseudoinverse); exact reconstruction of a
    rank-k A; U unit upper with |u_ij| <= 1 and L lower trapezoidal."""
    Ac = _wrap(A)
    perm, Ly, Uy = basic_power_iteration_lu(Ac, l, p, seed)
    Ly = Ly[:, :k]
    PA = Ac.A[perm, :]
    Ac.passes += 1                                   # B = Ly^+ P A reads A
    Lpinv = np.linalg.solve(Ly.T @ Ly, Ly.T)         # Eq. pseudoinverse
    B = Lpinv @ PA
    q, L2, U2, _ = getrf(B.T)                        # Q B^T = L' U'
    Lb = U2.T
    Ub = L2.T
    L = Ly @ Lb
    return perm, q, L, Ub


def singlepass(A, k, seed):
    """Alg. singlepasslu.  Returns (p, q, L, U): A[p][:, q] ~= L U.
    Pinned by: H = A A^T Omega and the column-streaming form of Sec. 5
    (Eqs. gi, hi); the identity L U = P (A P_G) Q^T with P_G the orthogonal
    projector onto range(A^T Omega), which holds in exact arithmetic; the
    structural invariants and the Eckart-Young lower bound."""
    Ac = _wrap(A)
    m, n = Ac.shape
    Omega = gaussian_matrix(m, k, seed, STREAM_OMEGA_SP)
    A0 = Ac.A
    Ac.passes += 1                      # one column-streaming pass (Sec. 5 remark)
    G = A0.T @ Omega                    # Eq. G
    H = A0 @ G                          # Eq. H
    p, L1, U1, _ = getrf(H)             # P H = L1 U1
    W = G @ np.linalg.inv(G.T @ G)      # G^{dagger T}
    q, L2, U2, _ = getrf(W @ U1.T)      # Q G^{dagger T} U1^T = L2 U2
    L = L1 @ U2.T
    U = L2.T
    return p, q, L, U


def singlepass_streamed_GH(A, Omega):
    """Sec. 5 remark, Eqs. gi and hi: one sweep over the columns of A,
    G(i,:) = A(:,i)^T Omega and H += A(:,i) G(i,:)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    G = np.zeros((n, Omega.shape[1]))
    H = np.zeros((m, Omega.shape[1]))
    for i in range(n):
        G[i, :] = A[:, i] @ Omega
        H += np.outer(A[:, i], G[i, :])
    return G, H
