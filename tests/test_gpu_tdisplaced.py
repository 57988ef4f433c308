"""GPU parity of the time-displaced path (dqmc_greens_tdisplaced) against the oracle.

The oracle computes G(tau_j, tau_j) from scratch on the cyclically shifted
chain and G(tau_j, 0) from two independent chains (the inverse chain
B_1^{-1}...B_l^{-1} and the remainder B_M...B_{l+1}) through inv_sum_loh;
the GPU takes both from one forward and one backward stack.  Same tolerance
as the equal-time path: max|dG| <= 1e-10 * max(1, max|G|).
"""
import numpy as np
import pytest

import dqmc_inputs as di
from oracle import dqmc as od
from oracle import exact as ex

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GTOL = 1e-10


@pytest.fixture(scope="module")
def dq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_05286_gb300 as m
    m.lib()
    return m


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _cmp(A, B):
    scale = max(1.0, np.abs(B).max())
    return np.abs(A - B).max() / scale


@pytest.mark.parametrize("L,beta,k,seed", [(2, 3.0, 10, 1), (3, 2.5, 10, 2), (4, 4.0, 10, 3),
                                            (4, 4.0, 7, 4), (6, 6.0, 10, 5)])
def test_tdisplaced_vs_oracle(dq, L, beta, k, seed):
    inst = di.hubbard_instance(L, 4.0, 0.1, beta, k, seed)
    Gtt, Gt0, st = dq.greens_tdisplaced(_dev(inst.K), 0.1, _dev(inst.V), k)
    Gtt, Gt0 = Gtt.cpu().numpy(), Gt0.cpu().numpy()
    Ott, Ot0 = od.greens_tdisplaced(inst.K, 0.1, inst.V, k)
    assert int(st) == 0
    for j in range(Ott.shape[0]):
        assert _cmp(Gtt[j], Ott[j]) <= GTOL, j
        assert _cmp(Gt0[j], Ot0[j]) <= GTOL, j


def test_tdisplaced_identities(dq):
    """G(0,0) = G(beta,beta) = G_1, G(beta,0) = 1 - G_1 (Eq. (etgf_tau), anti-periodicity)."""
    inst = di.hubbard_instance(4, 4.0, 0.1, 6.0, 10, 8)
    K, V = _dev(inst.K), _dev(inst.V)
    Gtt, Gt0, _ = dq.greens_tdisplaced(K, 0.1, V, 10)
    G1 = dq.greens(K, 0.1, V, 10)[0]
    I = torch.eye(16, dtype=torch.float64, device="cuda")
    assert (Gtt[0] - G1).abs().max() <= GTOL
    assert (Gtt[-1] - G1).abs().max() <= GTOL
    assert (Gt0[0] - G1).abs().max() <= GTOL
    assert (Gt0[-1] - (I - G1)).abs().max() <= GTOL


def test_tdisplaced_closed_form_beta40(dq):
    """U = 0, site-independent field, beta = 40: flat accuracy over all tau (Fig. 6)."""
    K = di.chain_hopping(8)
    M = 400
    c = np.random.default_rng(40).uniform(-0.3, 0.3, M)
    V = np.repeat(c[:, None], 8, axis=1)
    Gtt, Gt0, st = dq.greens_tdisplaced(_dev(K), 0.1, _dev(V), 10)
    Gt0 = Gt0.cpu().numpy()
    Gtt = Gtt.cpu().numpy()
    for j, l in enumerate(od.tau_grid(M, 10)):
        Gx = ex.closed_form_displaced(K, 40.0, 0.1 * l, c.sum(), c[:l].sum())
        assert np.abs(Gt0[j] - Gx).max() <= GTOL, (j, np.abs(Gt0[j] - Gx).max())
        Gxx, _ = ex.closed_form_greens(K, 40.0, c.sum())
        assert np.abs(Gtt[j] - Gxx).max() <= GTOL


def test_tdisplaced_brute_force(dq):
    K = di.chain_hopping(4)
    V = 0.8 * di.ising_field(5, 60, 4)
    bf = ex.BruteForce(K, 0.1, V)
    _, Gt0, _ = dq.greens_tdisplaced(_dev(K), 0.1, _dev(V), 10)
    Gt0 = Gt0.cpu().numpy()
    for j, l in enumerate(od.tau_grid(60, 10)):
        assert np.abs(Gt0[j] - bf.to_numpy(bf.displaced(l))).max() <= GTOL


def test_tdisplaced_only_one_output(dq):
    inst = di.hubbard_instance(4, 4.0, 0.1, 3.0, 10, 2)
    K, V = _dev(inst.K), _dev(inst.V)
    Gtt, Gt0, _ = dq.greens_tdisplaced(K, 0.1, V, 10)
    a, _, _ = dq.greens_tdisplaced(K, 0.1, V, 10, want_t0=False)
    _, b, _ = dq.greens_tdisplaced(K, 0.1, V, 10, want_tt=False)
    assert (a - Gtt).abs().max() <= 1e-12 and (b - Gt0).abs().max() <= 1e-12


def test_tdisplaced_full_size_sampled(dq):
    """8x8 lattice, U=4, beta=40 (M=400), k=10, 256 instances in one call;
    instances 0 and 255 checked against the oracle at tau_j for j in {0,10,20,30,40}."""
    insts = [di.batch_n64_tdisplaced(i) for i in range(256)]
    K = _dev(insts[0].K)
    V = _dev(np.stack([x.V for x in insts]))
    Gtt, Gt0, st = dq.greens_tdisplaced(K, 0.1, V, 10)
    assert int((st != 0).sum()) == 0
    assert Gtt.shape == (256, 41, 64, 64)
    for b in (0, 255):
        x = insts[b]
        for j in (0, 10, 20, 30, 40):
            l = min(10 * j, 400)
            Ot0 = od.greens_displaced(x.K, 0.1, x.V, 10, l, 0)
            Ott = od.greens(x.K, 0.1, x.V, 10, l=l + 1)[0]
            assert _cmp(Gt0[b, j].cpu().numpy(), Ot0) <= GTOL, (b, j)
            assert _cmp(Gtt[b, j].cpu().numpy(), Ott) <= GTOL, (b, j)
