"""GPU parity of the equal-time path (dqmc_greens / dqmc_logdet) against the oracle.

Tolerances (FP64 mode): max|dG| <= 1e-10 * max(1, max|G|) and relative
|d logdet| <= 1e-9, the sign exactly.  The oracle and the CUDA path round in
different orders (LAPACK blocking vs one-thread-per-column kernels) and pick
pivots with different arithmetic, so agreement is to the accumulated rounding
of the stabilised chain (~1e-13 here), not bitwise.
"""
import numpy as np
import pytest

import dqmc_inputs as di
from oracle import dqmc as od
from oracle import exact as ex

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GTOL = 1e-10
LTOL = 1e-9


@pytest.fixture(scope="module")
def dq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_05286_gb300 as m
    m.lib()
    return m


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _check(G, ld, sg, st, K, dtau, V, k):
    Go, ldo, so = od.greens(K, dtau, V, k)
    err = np.abs(G - Go).max()
    assert err <= GTOL * max(1.0, np.abs(Go).max()), err
    assert abs(ld - ldo) <= LTOL * max(1.0, abs(ldo)), (ld, ldo)
    assert sg == so
    assert st == 0


# k = M means no intermediate stabilisation: only well conditioned when beta is
# small (here kappa(B(beta,0)) ~ e^{8 beta} e^{2 lambda M} at beta = 1).
@pytest.mark.parametrize("L,beta,k,seed", [(2, 2.0, 3, 1), (3, 4.0, 10, 2), (4, 8.0, 10, 3),
                                            (4, 8.0, 1, 4), (4, 1.0, 10, 5), (6, 10.0, 7, 6),
                                            (8, 20.0, 10, 7)])
def test_greens_square_lattices(dq, L, beta, k, seed):
    inst = di.hubbard_instance(L, 4.0, 0.1, beta, k, seed)
    G, ld, sg, st = dq.greens(_dev(inst.K), inst.dtau, _dev(inst.V), k)
    _check(G.cpu().numpy(), float(ld), int(sg), int(st), inst.K, inst.dtau, inst.V, k)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 17, 33, 37, 65, 97, 100])
def test_greens_ragged_sizes(dq, N):
    """Sizes that are not multiples of any tile: boundary handling of every kernel."""
    K = di.chain_hopping(N) if N > 1 else np.zeros((1, 1))
    M = 23
    V = 0.7 * di.ising_field(100 + N, M, N)
    G, ld, sg, st = dq.greens(_dev(K), 0.1, _dev(V), 5)
    _check(G.cpu().numpy(), float(ld), int(sg), int(st), K, 0.1, V, 5)


def test_greens_batch_matches_solo(dq):
    """Each instance of a batch equals its own single-instance run, bitwise."""
    insts = [di.batch_n64_tdisplaced(i) for i in range(3)]
    K = _dev(insts[0].K)
    Vb = _dev(np.stack([i.V[:120] for i in insts]))
    Gb, ldb, sgb, stb = dq.greens(K, 0.1, Vb, 10)
    for b in range(3):
        G1, ld1, sg1, st1 = dq.greens(K, 0.1, Vb[b], 10)
        assert torch.equal(Gb[b], G1)
        assert float(ldb[b]) == float(ld1)


def test_greens_single_n16_against_mpmath(dq):
    """The 4x4, U=4, beta=8, k=10 workload against the stored mpmath values."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "single_n16_mpmath.txt")
    rows = [ln.split() for ln in open(path) if not ln.startswith("#")]
    ldx, sx = float(rows[0][0]), int(float(rows[0][1]))
    Gx = np.array([float(r[0]) for r in rows[1:]]).reshape(16, 16)
    inst = di.single_n16()
    G, ld, sg, st = dq.greens(_dev(inst.K), inst.dtau, _dev(inst.V), inst.k)
    assert np.abs(G.cpu().numpy() - Gx).max() <= GTOL * np.abs(Gx).max()
    assert abs(float(ld) - ldx) <= LTOL * abs(ldx)
    assert int(sg) == sx and int(st) == 0


@pytest.mark.parametrize("beta", [10.0, 50.0])
def test_greens_closed_form_large_beta(dq, beta):
    """U = 0 with a site-independent field: the exact closed form at beta up to 50."""
    K = di.square_hopping(6)
    M = int(round(beta / 0.1))
    c = np.random.default_rng(int(beta)).uniform(-0.3, 0.3, M)
    V = np.repeat(c[:, None], 36, axis=1)
    G, ld, sg, st = dq.greens(_dev(K), 0.1, _dev(V), 10)
    Gx, ldx = ex.closed_form_greens(K, beta, shift=c.sum())
    assert np.abs(G.cpu().numpy() - Gx).max() <= GTOL
    assert abs(float(ld) - ldx) <= LTOL * max(1.0, abs(ldx))


def test_greens_brute_force_small(dq):
    K = di.chain_hopping(4)
    V = 0.9 * di.ising_field(77, 50, 4)
    bf = ex.BruteForce(K, 0.1, V)
    Gb, ldb, sb = bf.greens(1)
    G, ld, sg, st = dq.greens(_dev(K), 0.1, _dev(V), 7)
    Gx = bf.to_numpy(Gb)     # single-species G of a strong Ising field: |G| ~ 30 here
    assert np.abs(G.cpu().numpy() - Gx).max() <= GTOL * max(1.0, np.abs(Gx).max())
    assert abs(float(ld) - float(ldb)) <= LTOL * abs(float(ldb))
    assert int(sg) == sb


def test_negative_sign(dq):
    """Fields with det(1 + B_M...B_1) < 0 give the same sign as the oracle."""
    K = di.chain_hopping(3)
    signs = []
    for seed in range(40):
        V = 2.0 * di.gaussian_field(seed, 6, 3)
        _, ld, sg, st = dq.greens(_dev(K), 0.5, _dev(V), 2)
        _, ldo, so = od.greens(K, 0.5, V, 2)
        assert int(sg) == so
        assert abs(float(ld) - ldo) <= LTOL * max(1.0, abs(ldo))
        signs.append(int(sg))
    assert -1 in signs


def test_logdet_only_matches_greens(dq):
    inst = di.hubbard_instance(6, 4.0, 0.1, 12.0, 10, 9)
    K, V = _dev(inst.K), _dev(np.stack([inst.V, -inst.V]))
    _, ld, sg, _ = dq.greens(K, 0.1, V, 10)
    ld2, sg2, st2 = dq.logdet(K, 0.1, V, 10)
    assert torch.equal(ld, ld2) and torch.equal(sg, sg2)
    # particle-hole: logdet(-V) = logdet(V) - sum V
    assert abs(float(ld[1]) - (float(ld[0]) - inst.V.sum())) <= 1e-9 * abs(float(ld[0]))


def test_deterministic(dq):
    inst = di.hubbard_instance(8, 4.0, 0.1, 10.0, 10, 3)
    K, V = _dev(inst.K), _dev(inst.V)
    a = dq.greens(K, 0.1, V, 10)[0].clone()
    b = dq.greens(K, 0.1, V, 10)[0]
    assert torch.equal(a, b)


def test_status_flags(dq):
    inst = di.hubbard_instance(4, 4.0, 0.1, 2.0, 5, 3)
    V = inst.V.copy()
    V[3, 2] = np.nan
    _, _, _, st = dq.greens(_dev(inst.K), 0.1, _dev(np.stack([inst.V, V])), 5)
    st = st.cpu().numpy()
    assert st[0] == 0 and (st[1] & 1)
    Kbad = inst.K.copy()
    Kbad[0, 1] += 0.5
    _, _, _, st = dq.greens(_dev(Kbad), 0.1, _dev(inst.V), 5)
    assert int(st) & (1 << 4)


def test_empty_batch_and_bad_args(dq):
    K = _dev(di.square_hopping(4))
    V = torch.zeros((0, 10, 16), dtype=torch.float64, device="cuda")
    G, ld, sg, st = dq.greens(K, 0.1, V, 5)
    assert G.shape == (0, 16, 16)
    with pytest.raises(RuntimeError):
        dq.greens(K, 0.1, torch.zeros((1, 10, 16), dtype=torch.float64, device="cuda"), 11)


def test_host_pointer_mode(dq):
    import ctypes as C
    inst = di.hubbard_instance(4, 4.0, 0.1, 6.0, 10, 12)
    h = dq.Handle()
    h.set_pointer_mode(True)
    Kh = np.ascontiguousarray(inst.K)
    Vh = np.ascontiguousarray(inst.V)
    G = np.empty((16, 16))
    ld = np.empty(1)
    sg = np.empty(1, dtype=np.int32)
    st = np.empty(1, dtype=np.int32)
    p = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    rc = h._lib.dqmc_greens(h.h, 1, 16, inst.M, p(Kh), 0.1, p(Vh), 10, p(G), p(ld), p(sg), p(st))
    assert rc == 0
    Gd, ldd, sgd, _ = dq.greens(_dev(inst.K), 0.1, _dev(inst.V), 10)
    assert np.array_equal(G, Gd.cpu().numpy())
    assert ld[0] == float(ldd) and sg[0] == int(sgd) and st[0] == 0


def test_greens_full_size_sampled(dq):
    """16x16 lattice, U=4, beta=20 (M=200), k=10, 128 instances in one call (the
    benchmark's launch configuration); instances 0, 64 and 127 against the oracle."""
    insts = [di.batch_n256(i) for i in range(128)]
    K = _dev(insts[0].K)
    V = _dev(np.stack([x.V for x in insts]))
    G, ld, sg, st = dq.greens(K, 0.1, V, 10)
    assert int((st != 0).sum()) == 0
    for b in (0, 64, 127):
        x = insts[b]
        _check(G[b].cpu().numpy(), float(ld[b]), int(sg[b]), int(st[b]), x.K, 0.1, x.V, 10)
