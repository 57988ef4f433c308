"""Exact references that pin the FP64 oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/dqmc.py``).

* Closed forms of the non-interacting problem (Sec. 3: eps_k of K; the
  paper's footnote in Sec. 4.1 notes that this case can be diagonalised
  exactly).  A slice-dependent but site-independent field V_l = c_l * 1
  commutes with K, so the same closed forms hold with exp(-beta*eps) replaced
  by exp(-beta*eps + sum_l c_l).
* Arbitrary-precision brute force (Sec. 4.1: the paper benchmarks against
  BigFloat): the naive product B_M...B_1, the inverse [1 + B_M...B_1]^{-1}
  and the determinant, all in mpmath at a working precision chosen from the
  condition number of the chain.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# Closed forms, K symmetric, V_l = c_l * 1
# ---------------------------------------------------------------------------

def _fermi_weights(x: np.ndarray) -> np.ndarray:
    """1 / (1 + exp(-x)) evaluated without overflow."""
    out = np.empty_like(x)
    pos = x >= 0
    out[pos] = 1.0 / (1.0 + np.exp(-x[pos]))
    e = np.exp(x[~pos])
    out[~pos] = e / (1.0 + e)
    return out


def closed_form_greens(K: np.ndarray, beta: float, shift: float = 0.0):
    """G = [1 + exp(-beta K + shift)]^{-1}, log det(1 + exp(-beta K + shift)).

    shift = sum_l c_l for the field V_l = c_l * 1."""
    eps, Q = np.linalg.eigh(K)
    x = beta * eps - shift                     # P has eigenvalues exp(-x)
    G = (Q * _fermi_weights(x)[None, :]) @ Q.T
    logdet = float(np.sum(np.logaddexp(0.0, -x)))
    return G, logdet


def closed_form_displaced(K: np.ndarray, beta: float, tau: float,
                          shift_total: float = 0.0, shift_tau: float = 0.0):
    """G(tau, 0) = B(tau, 0) G_1 = Q diag(exp(-tau eps + s_tau) / (1 + exp(-beta eps + s))) Q^T.

    s = sum of all c_l, s_tau = sum of c_l over the first tau/dtau slices;
    each weight is evaluated in the overflow-free form."""
    eps, Q = np.linalg.eigh(K)
    a = -tau * eps + shift_tau                 # log of the numerator
    b = -beta * eps + shift_total              # log of exp(...) in the denominator
    # w = exp(a) / (1 + exp(b)) = exp(a - logaddexp(0, b))
    w = np.exp(a - np.logaddexp(0.0, b))
    return (Q * w[None, :]) @ Q.T


def closed_form_displaced_back(K: np.ndarray, beta: float, tau: float,
                               shift_total: float = 0.0, shift_tau: float = 0.0):
    """G(0, tau) = -(1 - G_1) B(tau, 0)^{-1}
    = -Q diag(exp(tau eps - s_tau) / (1 + exp(beta eps - s))) Q^T.

    1 - G_1 has eigenvalues 1 / (1 + exp(beta eps - s)) and B(tau, 0)^{-1} has
    exp(tau eps - s_tau); each weight is evaluated in the overflow-free form."""
    eps, Q = np.linalg.eigh(K)
    w = np.exp(tau * eps - shift_tau - np.logaddexp(0.0, beta * eps - shift_total))
    return -(Q * w[None, :]) @ Q.T


# ---------------------------------------------------------------------------
# Arbitrary-precision brute force
# ---------------------------------------------------------------------------

def required_dps(K: np.ndarray, dtau: float, V: np.ndarray, guard: int = 30) -> int:
    """Decimal digits that resolve every scale of B_M...B_1 plus a guard.

    log kappa(B_M...B_1) <= sum_l [dtau (eps_max - eps_min) + max V_l - min V_l]."""
    eps = np.linalg.eigvalsh(K)
    spread = V.shape[0] * dtau * (eps[-1] - eps[0]) + float(np.sum(V.max(1) - V.min(1)))
    return int(math.ceil(spread / math.log(10.0))) + guard


class BruteForce:
    """Naive chain algebra in mpmath at a fixed precision (the BigFloat method)."""

    def __init__(self, K: np.ndarray, dtau: float, V: np.ndarray, dps: int | None = None):
        import mpmath as mp
        self.mp = mp
        self.M, self.N = V.shape
        self.dps = dps if dps is not None else required_dps(K, dtau, V)
        mp.mp.dps = self.dps
        Kmp = mp.matrix(K.tolist())
        # exp(-dtau K) through the symmetric eigendecomposition at full precision
        E, Q = mp.eigsy(Kmp)
        N = self.N
        self.EK = mp.matrix(N, N)
        for i in range(N):
            for j in range(N):
                self.EK[i, j] = mp.fsum(Q[i, m] * mp.exp(-dtau * E[m]) * Q[j, m]
                                        for m in range(N))
        self.expV = [[mp.exp(mp.mpf(float(V[l, i]))) for i in range(N)]
                     for l in range(self.M)]

    def slice(self, l: int):
        """B_l (1-based) at full precision."""
        mp, N = self.mp, self.N
        B = mp.matrix(N, N)
        for i in range(N):
            for j in range(N):
                B[i, j] = self.EK[i, j] * self.expV[l - 1][j]
        return B

    def chain(self, order):
        """Product of B_l for l in ``order``; the first index is applied first."""
        mp = self.mp
        P = mp.eye(self.N)
        for l in order:
            P = self.slice(l) * P
        return P

    def greens(self, l: int = 1):
        """G_l = [1 + B_{l-1}...B_1 B_M...B_l]^{-1} and log|det|, sign of the bracket."""
        mp = self.mp
        M = self.M
        l = 1 if l == M + 1 else l
        P = self.chain(list(range(l, M + 1)) + list(range(1, l)))
        A = mp.eye(self.N) + P
        det = mp.det(A)
        return mp.inverse(A), mp.log(abs(det)), (1 if det > 0 else -1)

    def displaced(self, l1: int):
        """G(tau_{l1}, 0) = B_{l1}...B_1 [1 + B_M...B_1]^{-1}."""
        G1, _, _ = self.greens(1)
        return self.chain(range(1, l1 + 1)) * G1

    def displaced_pair(self, l1: int, l2: int):
        """G(tau_{l1}, tau_{l2}), l1 >= l2: B_{l1}...B_{l2+1} G_{l2+1} (Eq. (tdgf_propagate))."""
        G, _, _ = self.greens(l2 + 1)
        return self.chain(range(l2 + 1, l1 + 1)) * G

    def displaced_back(self, l1: int, l2: int):
        """G(tau_{l1}, tau_{l2}), l2 >= l1: -(1 - G_{l1+1}) (B_{l2}...B_{l1+1})^{-1}."""
        mp = self.mp
        G, _, _ = self.greens(l1 + 1)
        C = self.chain(range(l1 + 1, l2 + 1))
        return -(mp.eye(self.N) - G) * mp.inverse(C)

    @staticmethod
    def to_numpy(A) -> np.ndarray:
        return np.array([[float(A[i, j]) for j in range(A.cols)] for i in range(A.rows)])
