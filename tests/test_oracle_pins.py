"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses a closed form,
an arbitrary-precision brute force, a naive computation in its well-conditioned
range, an exact identity of the model, or a property a correct factorisation
must have.  Sizes keep the whole file to well under a minute on CPU.
"""
import numpy as np
import pytest

import dqmc_inputs as di
from oracle import dqmc as od
from oracle import exact as ex


def _hubbard(L, U, beta, seed, dtau=0.1):
    M = int(round(beta / dtau))
    K = di.square_hopping(L)
    V = di.hirsch_lambda(U, dtau) * di.ising_field(seed, M, L * L)
    return K, V


# ---------------------------------------------------------------------------
# Decomposition (Sec. 4.2.2): properties of a column-pivoted QR written as UDX
# ---------------------------------------------------------------------------

def test_udt_properties(rng):
    A = rng.standard_normal((13, 13)) * np.exp(rng.uniform(-20, 20, 13))[None, :]
    U, D, X = od.udt(A)
    assert np.abs(U.T @ U - np.eye(13)).max() < 1e-14
    assert np.abs((U * D[None, :]) @ X - A).max() <= 1e-14 * np.abs(A).max()
    assert np.all(np.diff(D) <= 0)                   # pivoting orders the scales
    assert np.all(np.abs(X) <= 1 + 1e-14)            # |r_ij| <= |r_ii| under pivoting
    # X is a column permutation of a unit-modulus-diagonal upper triangle
    perm = np.argmax(np.abs(X) == 1.0, axis=1)
    assert sorted(perm) == list(range(13))


# ---------------------------------------------------------------------------
# P1: non-interacting closed forms, up to beta = 50
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("beta", [1.0, 10.0, 40.0, 50.0])
@pytest.mark.parametrize("lattice", ["chain8", "square4"])
def test_closed_form_equal_time(beta, lattice):
    K = di.chain_hopping(8) if lattice == "chain8" else di.square_hopping(4)
    M = int(round(beta / 0.1))
    V = np.zeros((M, K.shape[0]))
    G, ld, s = od.greens(K, 0.1, V, 10)
    Gx, ldx = ex.closed_form_greens(K, beta)
    assert np.abs(G - Gx).max() < 1e-12
    assert abs(ld - ldx) <= 1e-12 * max(1.0, abs(ldx))
    assert s == 1.0


def test_closed_form_site_independent_field(rng):
    """V_l = c_l * 1 commutes with K: exp(V) enters only through sum_l c_l."""
    K = di.square_hopping(4)
    M = 300
    c = rng.uniform(-0.5, 0.5, M)
    V = np.repeat(c[:, None], 16, axis=1)
    G, ld, _ = od.greens(K, 0.1, V, 10)
    Gx, ldx = ex.closed_form_greens(K, 30.0, shift=c.sum())
    assert np.abs(G - Gx).max() < 1e-12
    assert abs(ld - ldx) <= 1e-12 * max(1.0, abs(ldx))
    # the gradient is 1 - diag(G) at every slice
    dV = od.logdet_grad(K, 0.1, V, 10, slices=[1, 77, 300])
    for l in (1, 77, 300):
        assert np.abs(dV[l - 1] - (1 - np.diag(Gx))).max() < 1e-12


@pytest.mark.parametrize("l1", [0, 10, 100, 200, 300, 390, 400])
def test_closed_form_displaced(l1, rng):
    """G(tau,0) at beta = 40, including tau ~ beta/2 where inv_sum fails (Sec. 6.2.1)."""
    K = di.chain_hopping(8)
    M = 400
    c = rng.uniform(-0.3, 0.3, M)
    V = np.repeat(c[:, None], 8, axis=1)
    G = od.greens_displaced(K, 0.1, V, 10, l1, 0)
    Gx = ex.closed_form_displaced(K, 40.0, 0.1 * l1, shift_total=c.sum(),
                                  shift_tau=c[:l1].sum())
    assert np.abs(G - Gx).max() < 1e-12


def test_stack_scales_follow_spectrum():
    """P3: at U = 0 the pivoted-QR scales of B(beta,0) track exp(-beta*eps) (Fig. 2)."""
    K = di.chain_hopping(8)
    EK = od.hopping_exponential(K, 0.1)
    V = np.zeros((400, 8))
    _, D, _ = od.udx_chain(od.forward_slices(EK, V, range(1, 401)), 10, 8)
    sigma = np.sort(np.exp(-40.0 * np.linalg.eigvalsh(K)))[::-1]
    # |r_ii| of a pivoted QR brackets sigma_i within a modest factor of N on
    # (near-)degenerate levels; the scales themselves span e^{+-80}
    assert np.abs(np.log(D) - np.log(sigma)).max() < np.log(8.0)


# ---------------------------------------------------------------------------
# P2: naive inversion where the chain is well conditioned
# ---------------------------------------------------------------------------

def test_naive_small_beta():
    K, V = _hubbard(4, 4.0, 1.0, seed=7)
    EK = od.hopping_exponential(K, 0.1)
    P = np.eye(16)
    for l in range(V.shape[0]):
        P = (EK * np.exp(V[l])[None, :]) @ P
    Gn = np.linalg.inv(np.eye(16) + P)
    sn, ldn = np.linalg.slogdet(np.eye(16) + P)
    for k in (1, 3, 10):
        G, ld, s = od.greens(K, 0.1, V, k)
        assert np.abs(G - Gn).max() < 1e-12
        assert abs(ld - ldn) < 1e-12 * abs(ldn)
        assert s == sn


# ---------------------------------------------------------------------------
# P4: arbitrary-precision brute force on small chains (the paper's BigFloat method)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,M,k,scale,seed", [
    (2, 20, 1, 0.9, 1), (3, 40, 7, 0.7, 2), (4, 60, 10, 0.65, 3), (4, 35, 8, 1.2, 4)])
def test_brute_force_chain(N, M, k, scale, seed):
    K = di.chain_hopping(N, periodic=N > 2)
    V = scale * di.ising_field(seed, M, N)
    bf = ex.BruteForce(K, 0.1, V)
    G, ld, s = od.greens(K, 0.1, V, k)
    Gb, ldb, sb = bf.greens(1)
    assert np.abs(G - bf.to_numpy(Gb)).max() < 1e-12
    assert abs(ld - float(ldb)) <= 1e-12 * max(1.0, abs(float(ldb)))
    assert s == sb
    for l1 in (1, M // 2, M):
        Gd = od.greens_displaced(K, 0.1, V, k, l1, 0)
        assert np.abs(Gd - bf.to_numpy(bf.displaced(l1))).max() < 1e-12
    for l in (2, M // 3, M):
        g = od.logdet_grad(K, 0.1, V, k, slices=[l])[l - 1]
        Gl = bf.to_numpy(bf.greens(l)[0])
        assert np.abs(g - (1.0 - np.diag(Gl))).max() < 1e-12


def test_brute_force_sign_negative():
    """A field with det(1 + B_M...B_1) < 0 (possible for a single spin species)."""
    K = di.chain_hopping(3)
    found = False
    for seed in range(40):
        V = 2.0 * di.gaussian_field(seed, 6, 3)
        bf = ex.BruteForce(K, 0.5, V)
        _, ldb, sb = bf.greens(1)
        G, ld, s = od.greens(K, 0.5, V, 2)
        assert s == sb
        assert abs(ld - float(ldb)) < 1e-12 * max(1.0, abs(float(ldb)))
        found |= sb < 0
    assert found


def test_golden_single_n16():
    """4x4 lattice, U=4, beta=8, k=10: oracle vs the stored mpmath values."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "single_n16_mpmath.txt")
    rows = [ln.split() for ln in open(path) if not ln.startswith("#")]
    logdet_x, sign_x = float(rows[0][0]), float(rows[0][1])
    Gx = np.array([float(r[0]) for r in rows[1:]]).reshape(16, 16)
    inst = di.single_n16()
    G, ld, s = od.greens(inst.K, inst.dtau, inst.V, inst.k)
    # a single-species G of an Ising field is not bounded by 1 (here |G| ~ 7):
    # the bound is relative to its largest entry
    assert np.abs(G - Gx).max() < 1e-12 * np.abs(Gx).max()
    assert abs(ld - logdet_x) <= 1e-12 * abs(logdet_x)
    assert s == sign_x


# ---------------------------------------------------------------------------
# P5/P6: wrapping, propagation, anti-periodicity (Eqs. (etgf_tau), (tdgf_propagate))
# ---------------------------------------------------------------------------

def test_wrapping_and_propagation():
    K, V = _hubbard(4, 4.0, 6.0, seed=11)
    M = V.shape[0]
    EK = od.hopping_exponential(K, 0.1)
    for l in (1, 17, 59):
        Gl = od.greens(K, 0.1, V, 10, l=l)[0]
        Gn = od.greens(K, 0.1, V, 10, l=l + 1)[0]
        B = od.slice_matrix(EK, V[l - 1])
        assert np.abs(Gn - B @ Gl @ np.linalg.inv(B)).max() < 1e-10
    G1 = od.greens(K, 0.1, V, 10)[0]
    assert np.abs(od.greens_displaced(K, 0.1, V, 10, 0, 0) - G1).max() < 1e-12
    assert np.abs(od.greens_displaced(K, 0.1, V, 10, M, 0) - (np.eye(16) - G1)).max() < 1e-12
    for l1 in (0, 23, 44):
        Ga = od.greens_displaced(K, 0.1, V, 10, l1, 0)
        Gb = od.greens_displaced(K, 0.1, V, 10, l1 + 1, 0)
        assert np.abs(Gb - od.slice_matrix(EK, V[l1]) @ Ga).max() < 1e-10


# ---------------------------------------------------------------------------
# P7: particle-hole symmetry of the half-filled bipartite lattice
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("beta", [4.0, 20.0])
def test_particle_hole(beta):
    """Lambda K Lambda = -K gives G(-V) = 1 - Lambda G(V)^T Lambda and
    log det(-V) = log det(V) - sum V (det exp(-dtau K) = 1 as tr K = 0)."""
    L = 4
    K, V = _hubbard(L, 4.0, beta, seed=5)
    lam = np.array([(-1.0) ** (x + y) for y in range(L) for x in range(L)])
    Gp, ldp, sp = od.greens(K, 0.1, V, 10)
    Gm, ldm, sm = od.greens(K, 0.1, -V, 10)
    assert np.abs(Gm - (np.eye(16) - lam[:, None] * Gp.T * lam[None, :])).max() < 1e-10
    assert abs(ldm - (ldp - V.sum())) < 1e-9 * abs(ldp)
    assert sm == sp


# ---------------------------------------------------------------------------
# P8: the symmetric Trotter split differs by a similarity
# ---------------------------------------------------------------------------

def test_trotter_similarity():
    K, V = _hubbard(4, 4.0, 5.0, seed=9)
    W = od.hopping_exponential(K, 0.05)           # exp(-dtau K / 2)
    Winv = od.hopping_exponential(K, 0.05, +1.0)
    sym = (W @ (np.exp(V[l])[:, None] * W) for l in range(V.shape[0]))
    U, D, X = od.udx_chain(sym, 10, 16)
    Gs, lds, _ = od.inv_one_plus_loh(U, D, X)
    G, ld, _ = od.greens(K, 0.1, V, 10)
    assert np.abs(Gs - Winv @ G @ W).max() < 1e-10
    assert abs(lds - ld) < 1e-10 * abs(ld)


# ---------------------------------------------------------------------------
# P9: the gradient against central finite differences of the stable log det
# ---------------------------------------------------------------------------

def test_gradient_finite_difference():
    L = 4
    M = 40
    phi = di.gaussian_field(21, M, L * L)
    K = di.square_hopping(L)
    g, dtau, h = 1.5, 0.1, 1e-6
    V = dtau * g * phi
    dV = od.logdet_grad(K, dtau, V, 10, slices=[1, 13, 40])
    for (l, i) in [(1, 0), (13, 5), (40, 15)]:
        Vp, Vm = V.copy(), V.copy()
        Vp[l - 1, i] += dtau * g * h
        Vm[l - 1, i] -= dtau * g * h
        fd = (od.logdet(K, dtau, Vp, 10)[0] - od.logdet(K, dtau, Vm, 10)[0]) / (2 * h)
        assert abs(fd - dtau * g * dV[l - 1, i]) < 1e-5


# ---------------------------------------------------------------------------
# P10: the two equal-time inversion schemes agree for QR (Fig. 4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("beta", [2.0, 20.0, 40.0])
def test_inv_one_plus_vs_loh(beta):
    K, V = _hubbard(4, 1.0, beta, seed=3)
    Gl, ldl, sl = od.greens(K, 0.1, V, 10, scheme="loh")
    Go, ldo, so = od.greens(K, 0.1, V, 10, scheme="plain")
    assert np.abs(Gl - Go).max() < 1e-11
    assert abs(ldl - ldo) < 1e-11 * abs(ldl)
    assert sl == so


# ---------------------------------------------------------------------------
# Index conventions of the k-grid
# ---------------------------------------------------------------------------

def test_tau_grid():
    assert od.tau_grid(80, 10) == [0, 10, 20, 30, 40, 50, 60, 70, 80]
    assert od.tau_grid(25, 10) == [0, 10, 20, 25]
    assert od.tau_grid(5, 10) == [0, 5]


# ---------------------------------------------------------------------------
# G(tau_1, tau_2) for tau_2 > tau_1 (second case of Eq. (tdgf_propagate))
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("l2", [0, 1, 10, 200, 390, 400])
def test_closed_form_displaced_back(l2, rng):
    """P1 for G(0, tau) at beta = 40: -(1 - G_1) B(tau,0)^{-1} in the eigenbasis of K."""
    K = di.chain_hopping(8)
    M = 400
    c = rng.uniform(-0.3, 0.3, M)
    V = np.repeat(c[:, None], 8, axis=1)
    G = od.greens_displaced_back(K, 0.1, V, 10, 0, l2)
    Gx = ex.closed_form_displaced_back(K, 40.0, 0.1 * l2, shift_total=c.sum(),
                                       shift_tau=c[:l2].sum())
    assert np.abs(G - Gx).max() < 1e-12


@pytest.mark.parametrize("N,M,k,scale,seed", [(3, 40, 7, 0.7, 2), (4, 35, 8, 1.2, 4)])
def test_brute_force_displaced_back(N, M, k, scale, seed):
    """P4 for tau_2 > tau_1: mpmath -(1 - G_{l1+1}) (B_{l2}...B_{l1+1})^{-1}."""
    K = di.chain_hopping(N, periodic=N > 2)
    V = scale * di.ising_field(seed, M, N)
    bf = ex.BruteForce(K, 0.1, V)
    for l1, l2 in ((0, 0), (0, 1), (0, M // 2), (0, M), (M // 3, 2 * M // 3), (5, 5)):
        G = od.greens_displaced_back(K, 0.1, V, k, l1, l2)
        assert np.abs(G - bf.to_numpy(bf.displaced_back(l1, l2))).max() < 1e-12


def test_displaced_back_propagation_and_ends():
    """P6: G(0, tau + dtau) = G(0, tau) B_{l+1}^{-1}; G(0, 0^+) = -(1 - G_1); G(0, beta) = -G_1."""
    K, V = _hubbard(4, 4.0, 6.0, seed=11)
    M = V.shape[0]
    EKinv = od.hopping_exponential(K, 0.1, +1.0)
    G1 = od.greens(K, 0.1, V, 10)[0]
    assert np.abs(od.greens_displaced_back(K, 0.1, V, 10, 0, 0) + (np.eye(16) - G1)).max() < 1e-12
    assert np.abs(od.greens_displaced_back(K, 0.1, V, 10, 0, M) + G1).max() < 1e-12
    for l in (0, 23, 44):
        Ga = od.greens_displaced_back(K, 0.1, V, 10, 0, l)
        Gb = od.greens_displaced_back(K, 0.1, V, 10, 0, l + 1)
        assert np.abs(Gb - Ga @ od.inverse_slice_matrix(EKinv, V[l])).max() < 1e-10


@pytest.mark.parametrize("beta", [4.0, 20.0])
def test_particle_hole_displaced(beta):
    """P7 links the two cases: B_{-V}(tau,0) = Lambda B_V(tau,0)^{-T} Lambda gives
    G_{-V}(tau, 0) = -Lambda G_V(0, tau)^T Lambda at every tau."""
    L = 4
    K, V = _hubbard(L, 4.0, beta, seed=5)
    M = V.shape[0]
    lam = np.array([(-1.0) ** (x + y) for y in range(L) for x in range(L)])
    for l in (0, 7, M // 2, M):
        Gm = od.greens_displaced(K, 0.1, -V, 10, l, 0)
        Gp = od.greens_displaced_back(K, 0.1, V, 10, 0, l)
        assert np.abs(Gm + lam[:, None] * Gp.T * lam[None, :]).max() < 1e-10


# ---------------------------------------------------------------------------
# inv_sum (Eq. (inversion_tdgf)): right where the chain is well conditioned,
# inaccurate at tau ~ beta/2 (the paper's Fig. 6 finding for QR)
# ---------------------------------------------------------------------------

def test_inv_sum_naive_small_beta():
    K, V = _hubbard(4, 4.0, 1.0, seed=17)
    M = V.shape[0]
    EK = od.hopping_exponential(K, 0.1)
    Bs = [od.slice_matrix(EK, V[l]) for l in range(M)]
    P = np.eye(16)
    for B in Bs:
        P = B @ P
    G1 = np.linalg.inv(np.eye(16) + P)
    for l in (0, 3, 5, 9, 10):
        Bt = np.eye(16)
        for B in Bs[:l]:
            Bt = B @ Bt
        for scheme in ("sum", "loh"):
            G = od.greens_displaced(K, 0.1, V, 3, l, 0, scheme=scheme)
            assert np.abs(G - Bt @ G1).max() < 1e-12, (l, scheme)


@pytest.mark.parametrize("l1,sum_ok", [(0, True), (120, False), (400, True)])
def test_inv_sum_degrades_mid_tau(l1, sum_ok):
    """beta = 40, U = 0: Loh's split stays at rounding level for every tau; the
    plain sum loses many digits in between (1e-6 at tau = 12)."""
    K = di.chain_hopping(8)
    M = 400
    c = np.random.default_rng(1).uniform(-0.3, 0.3, M)
    V = np.repeat(c[:, None], 8, axis=1)
    Gx = ex.closed_form_displaced(K, 40.0, 0.1 * l1, c.sum(), c[:l1].sum())
    e_loh = np.abs(od.greens_displaced(K, 0.1, V, 10, l1, 0) - Gx).max()
    e_sum = np.abs(od.greens_displaced(K, 0.1, V, 10, l1, 0, scheme="sum") - Gx).max()
    assert e_loh < 1e-12
    assert (e_sum < 1e-12) if sum_ok else (e_sum > 1e-9)


# ---------------------------------------------------------------------------
# G(tau_1, tau_2) for pairs away from tau = 0, and time translation
# ---------------------------------------------------------------------------

def test_brute_force_general_pairs():
    """P4 for both cases of Eq. (tdgf_propagate) with neither time at 0."""
    K = di.chain_hopping(4)
    V = 1.1 * di.ising_field(12, 36, 4)
    bf = ex.BruteForce(K, 0.1, V)
    for l1, l2 in ((20, 7), (36, 12), (15, 15), (33, 1)):
        # single-species G reaches |G| ~ 1e2 here: the bound is relative to its largest entry
        R = bf.to_numpy(bf.displaced_pair(l1, l2))
        G = od.greens_displaced(K, 0.1, V, 6, l1, l2)
        assert np.abs(G - R).max() < 1e-12 * max(1.0, np.abs(R).max()), (l1, l2)
        Rb = bf.to_numpy(bf.displaced_back(l2, l1))
        Gb = od.greens_displaced_back(K, 0.1, V, 6, l2, l1)
        assert np.abs(Gb - Rb).max() < 1e-12 * max(1.0, np.abs(Rb).max()), (l2, l1)


def test_time_translation():
    """The products of Eqs. (etgf_tau) and (tdgf_propagate) depend only on the cyclic
    order of the slices: G(tau_{l0+d}, tau_{l0}) of V is G(tau_d, 0) of V shifted by l0,
    and past beta the shifted result is the anti-periodic continuation."""
    K, V = _hubbard(3, 4.0, 3.0, seed=9)
    M = V.shape[0]
    for l0 in (4, 13, 29):
        Vs = np.roll(V, -l0, axis=0)
        for d in (0, 6, M - l0, M):
            l1 = l0 + d
            G = od.greens_displaced(K, 0.1, Vs, 10, d, 0)
            G0 = od.greens_displaced_back(K, 0.1, Vs, 10, 0, d)
            if l1 <= M:
                R = od.greens_displaced(K, 0.1, V, 10, l1, l0)
                R0 = od.greens_displaced_back(K, 0.1, V, 10, l0, l1)
            else:
                R = -od.greens_displaced_back(K, 0.1, V, 10, l1 - M, l0)
                R0 = -od.greens_displaced(K, 0.1, V, 10, l0, l1 - M)
            assert np.abs(G - R).max() < 1e-12 * max(1.0, np.abs(R).max()), (l0, d)
            assert np.abs(G0 - R0).max() < 1e-12 * max(1.0, np.abs(R0).max()), (l0, d)


def _golden_displaced(name="single_n16_displaced_mpmath.txt", N=16):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    blocks, cur = {}, None
    for ln in open(path):
        if ln.startswith("#"):
            continue
        parts = ln.split()
        if len(parts) == 2:
            cur = (parts[0], int(parts[1]))
            blocks[cur] = []
        else:
            blocks[cur].append(float(parts[0]))
    return {key: np.array(v).reshape(N, N) for key, v in blocks.items()}


def test_golden_displaced_n16():
    """4x4 lattice, U=4, beta=8, k=10: G(tau,0) and G(0,tau) of the oracle against the
    stored mpmath values (tests/golden/make_golden.py, Eq. (tdgf_propagate))."""
    inst = di.single_n16()
    gold = _golden_displaced()
    for (name, l), Gx in gold.items():
        if name == "t0":
            G = od.greens_displaced(inst.K, inst.dtau, inst.V, inst.k, l, 0)
        else:
            G = od.greens_displaced_back(inst.K, inst.dtau, inst.V, inst.k, 0, l)
        assert np.abs(G - Gx).max() < 1e-12 * max(1.0, np.abs(Gx).max()), (name, l)


def test_golden_displaced_n64_ill_conditioned():
    """Instance 229 of the 8x8, U=4, beta=40 batch, the ill-conditioned field
    (|G(tau,0)| up to ~1e4): the oracle's G(tau,0) (Eq. (inversion_tdgf_loh))
    against the stored mpmath values at tau = 1, 5, 8 (397 digits,
    tests/golden/make_golden.py n64).  A backward-stable FP64 inversion of the
    middle matrix resolves G only to about eps * cond(mid) of max|G|; the
    oracle must stay within 16 times that, and the middle matrix must be as
    ill-conditioned as the field suggests (cond > 1e5), so the pin exercises
    that regime."""
    x = di.batch_n64_tdisplaced(229)
    gold = _golden_displaced("batch_n64_229_displaced_mpmath.txt", 64)
    assert sorted(gold) == [("t0", 10), ("t0", 50), ("t0", 80)]
    eps = np.finfo(np.float64).eps
    for (_, l), Gx in gold.items():
        G = od.greens_displaced(x.K, x.dtau, x.V, x.k, l, 0)
        kappa = od.displaced_condition(x.K, x.dtau, x.V, x.k, l, 0)
        scale = max(1.0, np.abs(Gx).max())
        assert kappa > 1e5 and scale > 1e3, (l, kappa, scale)
        assert np.abs(G - Gx).max() / scale <= 16.0 * eps * kappa, l
