"""Seeded synthetic inputs for the DQMC stabilisation path.

This module holds NO arithmetic of the stabilisation method itself.  It only
builds the model inputs that both the CPU oracle and the CUDA path consume:

* the hopping matrix K of the half-filled Hubbard model (Sec. 3, Eq. (model):
  nearest-neighbour hopping -t, t = 1, chemical potential 0), on a periodic
  L x L square lattice (site i = x + L*y) or on a 1D chain;
* the Hirsch coupling lambda = acosh(exp(U*dtau/2)) of the discrete
  Hubbard-Stratonovich decoupling (Sec. 3, footnote on the spin channel);
* Ising fields s_{i,l} = +-1 and Gaussian fields phi_{i,l} ~ N(0,1), and the
  per-slice diagonals V_l they define (V_l = lambda*s_{.,l}, or
  V_l = dtau*g*phi_{.,l} for the continuous field).

Random numbers come from one counter-based generator, SplitMix64
(G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output(seed, c) = mix64(seed + (c+1)*0x9E3779B97F4A7C15)
with the published mix64 finaliser.  Uniforms take the top 53 bits; normals use
the Box-Muller transform on two consecutive counters.

Layout conventions shared by everything that consumes these inputs:
* K is an (N, N) float64 array, row-major, K[i, j] = K_ij.
* V is an (M, N) float64 array, row-major: V[l-1, i] is the diagonal entry i
  of V_l, so slice l is contiguous.  Batches stack a leading axis: (B, M, N).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_BASE_SEED = 2003_05286 * 1000


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for the given uint64 counters under ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    z = splitmix64(seed, counters)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def ising_field(seed: int, M: int, N: int) -> np.ndarray:
    """s[l, i] = +-1 with equal probability; counter = l*N + i."""
    z = splitmix64(seed, np.arange(M * N, dtype=np.uint64))
    s = np.where((z >> np.uint64(63)) == 0, 1.0, -1.0)
    return s.reshape(M, N)


def gaussian_field(seed: int, M: int, N: int) -> np.ndarray:
    """phi[l, i] ~ N(0,1) by Box-Muller on counters 2c and 2c+1, c = l*N + i."""
    c = np.arange(M * N, dtype=np.uint64)
    u1 = 1.0 - uniform01(seed, 2 * c)           # (0, 1]
    u2 = uniform01(seed, 2 * c + 1)             # [0, 1)
    phi = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return phi.reshape(M, N)


def square_hopping(L: int, t: float = 1.0) -> np.ndarray:
    """Nearest-neighbour hopping on a periodic L x L square lattice.

    K[i, j] = -t for each bond (i, j); site i = x + L*y.  For L = 2 the two
    periodic bonds between the same pair of sites add up (K_ij = -2t)."""
    N = L * L
    K = np.zeros((N, N))
    for y in range(L):
        for x in range(L):
            i = x + L * y
            for dx, dy in ((1, 0), (0, 1)):
                j = (x + dx) % L + L * ((y + dy) % L)
                if i != j:
                    K[i, j] -= t
                    K[j, i] -= t
    return K


def chain_hopping(N: int, t: float = 1.0, periodic: bool = True) -> np.ndarray:
    """Nearest-neighbour hopping on a 1D chain of N sites (ring if periodic)."""
    K = np.zeros((N, N))
    for i in range(N - 1):
        K[i, i + 1] -= t
        K[i + 1, i] -= t
    if periodic and N > 2:
        K[0, N - 1] -= t
        K[N - 1, 0] -= t
    return K


def hirsch_lambda(U: float, dtau: float) -> float:
    """lambda = acosh(exp(U*dtau/2)) of the discrete spin-channel decoupling."""
    return math.acosh(math.exp(U * dtau / 2.0))


def instance_seed(config: int, instance: int) -> int:
    """Seed of one instance of a workload: 2003_05286*1000 + 100*config + instance."""
    return _BASE_SEED + 100 * config + instance


@dataclass
class Instance:
    """One field configuration: K (N,N), dtau, V (M,N) and the interval k."""
    K: np.ndarray
    dtau: float
    V: np.ndarray
    k: int
    L: int
    U: float
    beta: float

    @property
    def N(self) -> int:
        return self.K.shape[0]

    @property
    def M(self) -> int:
        return self.V.shape[0]


def hubbard_instance(L: int, U: float, dtau: float, beta: float, k: int,
                     seed: int) -> Instance:
    """Square-lattice Hubbard slice data with a +-1 Hirsch field."""
    M = int(round(beta / dtau))
    K = square_hopping(L)
    lam = hirsch_lambda(U, dtau)
    V = lam * ising_field(seed, M, L * L)
    return Instance(K, dtau, V, k, L, U, beta)


def gaussian_instance(L: int, g: float, dtau: float, beta: float, k: int,
                      seed: int) -> Instance:
    """Square-lattice slice data with V_l = dtau*g*phi_{.,l}, phi ~ N(0,1)."""
    M = int(round(beta / dtau))
    K = square_hopping(L)
    V = dtau * g * gaussian_field(seed, M, L * L)
    return Instance(K, dtau, V, k, L, 0.0, beta)


# ---- the five workloads: sizes and recipes -----------------------------------

def single_n16(instance: int = 0) -> Instance:
    """4x4 lattice (N=16), U=4, dtau=0.1, beta=8 (M=80), k=10, +-1 field."""
    return hubbard_instance(4, 4.0, 0.1, 8.0, 10, instance_seed(1, instance))


def batch_n64_tdisplaced(instance: int) -> Instance:
    """8x8 lattice (N=64), U=4, dtau=0.1, beta=40 (M=400), k=10; 256 instances."""
    return hubbard_instance(8, 4.0, 0.1, 40.0, 10, instance_seed(2, instance))


RAGGED_L = (6, 8, 10, 12, 16)


def ragged_params(instance: int) -> tuple[int, float, float]:
    """(L, beta, U) of one instance of the ragged batch.

    L uniform over {6,8,10,12,16}; beta uniform in [10,50] rounded to the
    dtau=0.1 grid; U uniform in [2,8].  Drawn from counters 2^40 + {0,1,2} of
    the instance's seed so they never overlap the field's counters."""
    seed = instance_seed(3, instance)
    u = uniform01(seed, np.array([1 << 40, (1 << 40) + 1, (1 << 40) + 2], dtype=np.uint64))
    L = RAGGED_L[min(int(u[0] * len(RAGGED_L)), len(RAGGED_L) - 1)]
    M = int(round((10.0 + 40.0 * u[1]) / 0.1))
    beta = M * 0.1
    U = 2.0 + 6.0 * u[2]
    return L, beta, U


def ragged_instance(instance: int, k: int) -> Instance:
    """Instance of the ragged batch (N in {36..256}, M in [100,500])."""
    L, beta, U = ragged_params(instance)
    return hubbard_instance(L, U, 0.1, beta, k, instance_seed(3, instance))


def batch_n256(instance: int) -> Instance:
    """16x16 lattice (N=256), U=4, dtau=0.1, beta=20 (M=200), k=10; 128 instances."""
    return hubbard_instance(16, 4.0, 0.1, 20.0, 10, instance_seed(4, instance))


def batch_n144_gaussian(instance: int) -> Instance:
    """12x12 lattice (N=144), g=1.5, dtau=0.1, beta=20 (M=200), k=10; 64 instances."""
    return gaussian_instance(12, 1.5, 0.1, 20.0, 10, instance_seed(5, instance))


def stack_V(instances: list[Instance]) -> np.ndarray:
    """(B, M, N) array of the fields of a uniform batch."""
    return np.stack([inst.V for inst in instances])
