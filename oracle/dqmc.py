"""Plain FP64 CPU oracle of the stabilised DQMC Green's-function path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports or calls this
module; only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA path.

Every function follows the paper (C. Bauer, "Fast and stable determinant
quantum Monte Carlo", SciPost 2020) step by step, using NumPy/SciPy LAPACK
primitives (eigh, geqp3 through ``scipy.linalg.qr(pivoting=True)``, LU solves)
for the individual steps and nothing blocked, fused or reordered beyond what
the paper writes.

Conventions (identical to the CUDA library's):
* matrices are float64 arrays with A[i, j] = A_ij;
* V has shape (M, N); V[l-1] is the diagonal of V_l;
* the slice matrix is B_l = exp(-dtau*K) exp(V_l) (K symmetric).  The paper's
  symmetric split exp(-dtau K/2) exp(V) exp(-dtau K/2) (Eq. (Ztr)) is related
  to it by the similarity W^{-1} B_l W with W = exp(-dtau K/2), which changes
  no determinant and conjugates every Green's function by W;
* tau = l*dtau; G_l = [1 + B_{l-1}...B_1 B_M...B_l]^{-1} (Eq. (etgf_tau)), and
  G(tau_l, tau_l) denotes G_{l+1}.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


# ---------------------------------------------------------------------------
# Slice matrices (Sec. 2, Eq. (Ztr))
# ---------------------------------------------------------------------------

def hopping_exponential(K: np.ndarray, dtau: float, sign: float = -1.0) -> np.ndarray:
    """exp(sign*dtau*K) of a symmetric K from its eigendecomposition.

    Sec. 3: the non-interacting slice exp(-dtau T) is diagonal in K's
    eigenbasis."""
    eps, Q = np.linalg.eigh(K)
    return (Q * np.exp(sign * dtau * eps)[None, :]) @ Q.T


def slice_matrix(EK: np.ndarray, v: np.ndarray) -> np.ndarray:
    """B_l = exp(-dtau K) exp(V_l): column j of E_K scaled by exp(v_j)."""
    return EK * np.exp(v)[None, :]


def inverse_slice_matrix(EKinv: np.ndarray, v: np.ndarray) -> np.ndarray:
    """B_l^{-1} = exp(-V_l) exp(+dtau K): row i of E_K^{-1} scaled by exp(-v_i)."""
    return np.exp(-v)[:, None] * EKinv


# ---------------------------------------------------------------------------
# Decomposition B = U D X by pivoted QR (Sec. 4.2.2)
# ---------------------------------------------------------------------------

def udt(A: np.ndarray):
    """Column-pivoted QR of A written as U D X (Sec. 4.2.2, "QR (UDT)").

    A P = Q R (LAPACK geqp3); U = Q; D = |diag R|; X = D^{-1} R P^T, so X is
    upper triangular up to the column permutation, with unit-modulus
    diagonal.  The signs of diag R are kept in X so that D >= 0 (the paper
    leaves the sign placement open; no result depends on it)."""
    Q, R, p = sla.qr(A, pivoting=True)
    d = np.abs(np.diag(R))
    T = R / d[:, None]
    X = np.empty_like(T)
    X[:, p] = T
    return Q, d, X


def udx_chain(slices, k: int, N: int):
    """Stabilised product of a chain of slice matrices (Sec. 4.1, Eq. (stabmult)).

    ``slices`` yields B_1, B_2, ... in the order they are applied (B_1 is the
    rightmost factor).  Every k slices are multiplied naively (the mixture of
    naive and stabilised products at the end of Sec. 4.1); the chunk product
    C then enters Eq. (stabmult) with U_2 = D_2 = 1, X_2 = C:
        C U_1 D_1 X_1 = U' D' (X' X_1),   U' D' X' = udt((C U_1) D_1).
    Returns (U, D, X) with B_n ... B_1 = U diag(D) X; an empty chain gives the
    identity."""
    U = np.eye(N)
    D = np.ones(N)
    X = np.eye(N)
    chunk = []

    def fold(chunk, U, D, X):
        A = U
        for B in chunk:
            A = B @ A
        Up, Dp, Xp = udt(A * D[None, :])
        return Up, Dp, Xp @ X

    for B in slices:
        chunk.append(B)
        if len(chunk) == k:
            U, D, X = fold(chunk, U, D, X)
            chunk = []
    if chunk:
        U, D, X = fold(chunk, U, D, X)
    return U, D, X


def forward_slices(EK: np.ndarray, V: np.ndarray, order):
    """Generator of B_l for l in ``order`` (1-based slice indices)."""
    for l in order:
        yield slice_matrix(EK, V[l - 1])


def inverse_slices(EKinv: np.ndarray, V: np.ndarray, order):
    """Generator of B_l^{-1} for l in ``order`` (1-based slice indices)."""
    for l in order:
        yield inverse_slice_matrix(EKinv, V[l - 1])


# ---------------------------------------------------------------------------
# Inversion schemes for the equal-time Green's function (Sec. 5.1)
# ---------------------------------------------------------------------------

def _sign_det(A: np.ndarray) -> float:
    s, _ = np.linalg.slogdet(A)
    return float(s)


def inv_one_plus_loh(U, D, X):
    """G = [1 + U D X]^{-1} by Loh's split (Sec. 5.1, Eq. (inversion_loh)).

    D_p = max(D, 1), D_m = min(D, 1);
    1 + U D X = (X^{-1} D_p^{-1} + U D_m) D_p X;
    the bracket is decomposed (u d x), then D_p^{-1} (u d x)^{-1} is
    decomposed again (u' d' x'), and G = (X^{-1} u') d' x'.

    Also returns log|det(1 + U D X)| and its sign:
    det(1 + U D X) = det(u d x) det(D_p) det(X), with |det u| = |det x| = 1
    (pivoted-QR factors) and |det X| = 1 (product of such factors)."""
    N = D.shape[0]
    Dp = np.maximum(D, 1.0)
    Dm = np.minimum(D, 1.0)
    XinvDpinv = sla.solve(X, np.diag(1.0 / Dp))            # X^{-1} D_p^{-1}
    Mx = XinvDpinv + U * Dm[None, :]                       # X^{-1} D_p^{-1} + U D_m
    u, d, x = udt(Mx)
    inner = (1.0 / Dp)[:, None] * (sla.solve(x, np.eye(N)) / d[None, :]) @ u.T
    u2, d2, x2 = udt(inner)                                # D_p^{-1} (u d x)^{-1}
    G = (sla.solve(X, u2) * d2[None, :]) @ x2              # X^{-1} u' d' x'
    logdet = float(np.sum(np.log(Dp)) + np.sum(np.log(d)))
    sign = _sign_det(u) * _sign_det(x) * _sign_det(X)
    return G, logdet, sign


def inv_one_plus(U, D, X):
    """G = [1 + U D X]^{-1} with one intermediate decomposition (Eq. (inversion)).

    1 + U D X = U (U^T X^{-1} + D) X; the bracket is decomposed as u d x and
    G = (x X)^{-1} d^{-1} (U u)^T."""
    N = D.shape[0]
    inner = U.T @ sla.solve(X, np.eye(N)) + np.diag(D)
    u, d, x = udt(inner)
    xX = x @ X
    G = sla.solve(xX, np.diag(1.0 / d)) @ (U @ u).T
    logdet = float(np.sum(np.log(d)))
    sign = _sign_det(U) * _sign_det(u) * _sign_det(x) * _sign_det(X)
    return G, logdet, sign


# ---------------------------------------------------------------------------
# Equal-time Green's function and log det (Eqs. (etgf), (DQMC), (etgf_tau))
# ---------------------------------------------------------------------------

def cyclic_order(M: int, l: int):
    """Slices of G_l = [1 + B_{l-1}...B_1 B_M...B_l]^{-1}, first applied first:
    B_l, B_{l+1}, ..., B_M, B_1, ..., B_{l-1}  (1 <= l <= M+1; l = M+1 is l = 1)."""
    if l == M + 1:
        l = 1
    return list(range(l, M + 1)) + list(range(1, l))


def greens(K, dtau, V, k, l: int = 1, scheme: str = "loh"):
    """G_l, log|det(1 + B_{l-1}...B_1 B_M...B_l)| and its sign.

    The chain is stabilised every k slices (Sec. 4.1) and inverted with
    inv_one_plus_loh (Eq. (inversion_loh)) or inv_one_plus (Eq. (inversion)).
    l = 1 gives the equal-time G of Eq. (etgf)."""
    M, N = V.shape
    EK = hopping_exponential(K, dtau)
    U, D, X = udx_chain(forward_slices(EK, V, cyclic_order(M, l)), k, N)
    if scheme == "loh":
        return inv_one_plus_loh(U, D, X)
    return inv_one_plus(U, D, X)


def logdet(K, dtau, V, k):
    """log|det(1 + B_M...B_1)| and sign (Eq. (DQMC): Z ~ det G^{-1})."""
    _, ld, s = greens(K, dtau, V, k)
    return ld, s


# ---------------------------------------------------------------------------
# Time-displaced Green's function (Sec. 6, Eqs. (tdgf_propagate), (inversion_tdgf_loh))
# ---------------------------------------------------------------------------

def _loh_mid(UL, DL, XL, UR, DR, XR):
    """The middle matrix of Eq. (inversion_tdgf_loh) (see inv_sum_loh)."""
    N = DL.shape[0]
    DLp, DLm = np.maximum(DL, 1.0), np.minimum(DL, 1.0)
    DRp, DRm = np.maximum(DR, 1.0), np.minimum(DR, 1.0)
    XRinv = sla.solve(XR, np.eye(N))
    mid = (DLm[:, None] * (XL @ XRinv)) / DRp[None, :] \
        + ((UL.T @ UR) / DLp[:, None]) * DRm[None, :]
    return mid, XRinv, DLp, DRp


def inv_sum_loh(UL, DL, XL, UR, DR, XR):
    """[U_L D_L X_L + U_R D_R X_R]^{-1} by the split of Eq. (inversion_tdgf_loh).

    D_{L,R} = D_{L,R p} D_{L,R m} with D_p = max(D,1), D_m = min(D,1);
      U_L D_L X_L + U_R D_R X_R = U_L D_Lp [mid] D_Rp X_R,
      mid = D_Lm (X_L X_R^{-1}) D_Rp^{-1} + D_Lp^{-1} (U_L^T U_R) D_Rm
    (the printed fractions D_Lm/D_Rp and D_Rm/D_Lp read as the only side
    assignment that reconstructs the sum).  mid is decomposed (u d x), then
    D_Rp^{-1} (u d x)^{-1} D_Lp^{-1} is decomposed again (u' d' x'), and the
    result is (X_R^{-1} u') d' (x' U_L^T)."""
    N = DL.shape[0]
    mid, XRinv, DLp, DRp = _loh_mid(UL, DL, XL, UR, DR, XR)
    u, d, x = udt(mid)
    inner = (sla.solve(x, np.eye(N)) / d[None, :]) @ u.T
    inner = inner / DRp[:, None] / DLp[None, :]
    u2, d2, x2 = udt(inner)
    return ((XRinv @ u2) * d2[None, :]) @ (x2 @ UL.T)


def inv_sum(UL, DL, XL, UR, DR, XR):
    """[U_L D_L X_L + U_R D_R X_R]^{-1} by Eq. (inversion_tdgf), without the D+/D- split.

    U_L D_L X_L + U_R D_R X_R = U_L (D_L X_L X_R^{-1} + U_L^T U_R D_R) X_R; the
    bracket is decomposed (u d x) and the result is (x X_R)^{-1} d^{-1} (U_L u)^T
    (the printed d^{-1} inside the inverse read as d, as in Eq. (inversion)).
    The bracket adds the scales of D_L and D_R, which Sec. 6.2.1 shows to lose
    accuracy at tau ~ beta/2."""
    N = DL.shape[0]
    inner = DL[:, None] * (XL @ sla.solve(XR, np.eye(N))) + (UL.T @ UR) * DR[None, :]
    u, d, x = udt(inner)
    return sla.solve(x @ XR, (1.0 / d)[:, None] * (UL @ u).T)


def _displaced_chains(K, dtau, V, k, l1: int, l2: int):
    """U_L D_L X_L of B_{l2+1}^{-1}...B_{l1}^{-1} and U_R D_R X_R of
    B_{l2}...B_1 B_M...B_{l1+1} (Sec. 6), tau_1 = l1*dtau >= tau_2 = l2*dtau."""
    M, N = V.shape
    assert 0 <= l2 <= l1 <= M
    EK = hopping_exponential(K, dtau)
    EKinv = hopping_exponential(K, dtau, sign=+1.0)
    left = inverse_slices(EKinv, V, list(range(l1, l2, -1)))
    right = forward_slices(EK, V, list(range(l1 + 1, M + 1)) + list(range(1, l2 + 1)))
    return udx_chain(left, k, N) + udx_chain(right, k, N)


def displaced_condition(K, dtau, V, k, l1: int, l2: int = 0) -> float:
    """2-norm condition number of the middle matrix that inv_sum_loh inverts for
    G(tau_1, tau_2) (Eq. (inversion_tdgf_loh)).  A backward-stable FP64 inversion
    resolves G(tau_1, tau_2) to about eps * this number relative to max|G|; it is
    the accuracy bound of an ill-conditioned field, for the oracle and any other
    FP64 route alike."""
    mid = _loh_mid(*_displaced_chains(K, dtau, V, k, l1, l2))[0]
    return float(np.linalg.cond(mid))


def greens_displaced(K, dtau, V, k, l1: int, l2: int = 0, scheme: str = "loh"):
    """G(tau_1, tau_2) for tau_1 = l1*dtau > tau_2 = l2*dtau (Sec. 6).

    G(tau_1,tau_2) = [B_{l2+1}^{-1}...B_{l1}^{-1} + B_{l2}...B_1 B_M...B_{l1+1}]^{-1};
    the left chain grows by B_{l1}^{-1} first, the right chain by B_{l1+1}
    first; both are stabilised every k slices and combined by inv_sum_loh
    (scheme "loh", Eq. (inversion_tdgf_loh)) or inv_sum (scheme "sum",
    Eq. (inversion_tdgf)).  l1 == l2 gives G_{l1+1} (the tau_1 -> tau_2^+ limit)."""
    chains = _displaced_chains(K, dtau, V, k, l1, l2)
    return inv_sum(*chains) if scheme == "sum" else inv_sum_loh(*chains)


def greens_displaced_back(K, dtau, V, k, l1: int, l2: int):
    """G(tau_1, tau_2) for tau_2 = l2*dtau > tau_1 = l1*dtau (Sec. 6, second case
    of Eq. (tdgf_propagate)): -(1 - G_{l1+1}) (B_{l2}...B_{l1+1})^{-1}.

    With C = B_{l2}...B_{l1+1} and Y = B_{l1}...B_1 B_M...B_{l2+1}, so that
    G_{l1+1} = [1 + Y C]^{-1}, one has 1 - G_{l1+1} = (1 + Y C)^{-1} Y C and
    hence, as in the paper's derivation of the first case,
        G(tau_1, tau_2) = -[C + Y^{-1}]^{-1},
        Y^{-1} = B_{l2+1}^{-1}...B_M^{-1} B_1^{-1}...B_{l1}^{-1}.
    C grows by B_{l1+1} first, Y^{-1} by B_{l1}^{-1} first; both are
    stabilised every k slices and combined by inv_sum_loh.  l1 == l2 gives
    -(1 - G_{l1+1}) (the tau_2 -> tau_1^+ limit); (l1, l2) = (0, M) gives -G_1."""
    M, N = V.shape
    assert 0 <= l1 <= l2 <= M
    EK = hopping_exponential(K, dtau)
    EKinv = hopping_exponential(K, dtau, sign=+1.0)
    UL, DL, XL = udx_chain(forward_slices(EK, V, list(range(l1 + 1, l2 + 1))), k, N)
    right = inverse_slices(EKinv, V, list(range(l1, 0, -1)) + list(range(M, l2, -1)))
    UR, DR, XR = udx_chain(right, k, N)
    return -inv_sum_loh(UL, DL, XL, UR, DR, XR)


def tau_grid(M: int, k: int):
    """Slice indices l_j = min(j*k, M), j = 0..ceil(M/k), of the k-grid."""
    nc = -(-M // k)
    return [min(j * k, M) for j in range(nc + 1)]


def greens_tdisplaced(K, dtau, V, k):
    """Gtt[j] = G(tau_j, tau_j) = G_{l_j + 1} and Gt0[j] = G(tau_j, 0) on the k-grid."""
    M, N = V.shape
    grid = tau_grid(M, k)
    Gtt = np.stack([greens(K, dtau, V, k, l=l + 1)[0] for l in grid])
    Gt0 = np.stack([greens_displaced(K, dtau, V, k, l, 0) for l in grid])
    return Gtt, Gt0


def greens_tdisplaced_0t(K, dtau, V, k):
    """G0t[j] = G(0, tau_j) on the k-grid by the second case of Eq. (tdgf_propagate);
    G0t[0] is its tau -> 0^+ limit -(1 - G_1), G0t[-1] = G(0, beta) = -G_1."""
    M, N = V.shape
    return np.stack([greens_displaced_back(K, dtau, V, k, 0, l) for l in tau_grid(M, k)])


# ---------------------------------------------------------------------------
# Gradient of log|det(1 + B_M...B_1)| with respect to V
# ---------------------------------------------------------------------------

def logdet_grad(K, dtau, V, k, slices=None):
    """dV[l-1, i] = d log|det(1 + B_M...B_1)| / dV_l(i) = 1 - G_l(i, i).

    Jacobi's formula with dB_l/dV_l(i) = B_l E_ii gives
    tr[G_1 B_M...B_{l+1} B_l E_ii B_{l-1}...B_1] = [B_{l-1}...B_1 G_1 B_M...B_l]_ii
    = [1 - G_l]_ii with G_l of Eq. (etgf_tau).  Every G_l is computed from
    scratch from its own cyclically shifted chain.  ``slices`` restricts the
    computation to the given 1-based l (other rows are NaN)."""
    M, N = V.shape
    out = np.full((M, N), np.nan)
    for l in (range(1, M + 1) if slices is None else slices):
        G = greens(K, dtau, V, k, l=l)[0]
        out[l - 1] = 1.0 - np.diag(G)
    return out
