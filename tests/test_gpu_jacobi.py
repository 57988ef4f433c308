"""One-sided Jacobi SVD as the chain stabiliser (dqmc_set_decomposition).

The decomposition differs from the pivoted QR (U D V^T with X = V^T
orthogonal), the results do not: G, log det, sign, G(tau,0) and the gradient
must match the oracle (whose chains use pivoted QR, pinned by closed forms
and mpmath) to the same tolerances (Sec. 4.2: both decompositions are
accurate).  Sizes stay small: a Jacobi decomposition costs ~10 sweeps of N^2/2
rotations.
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


def _h(dq):
    return dq.Handle(decomposition=1)


@pytest.mark.parametrize("L,beta,k,batch", [(2, 3.0, 10, 2), (3, 4.1, 7, 3), (4, 8.0, 10, 2),
                                            (6, 6.0, 10, 1), (5, 5.0, 5, 2)])
def test_jacobi_greens_vs_oracle(dq, L, beta, k, batch):
    insts = [di.hubbard_instance(L, 4.0, 0.1, beta, k, 60 + i) for i in range(batch)]
    G, ld, sg, st = dq.greens(_dev(insts[0].K), 0.1, _dev(np.stack([x.V for x in insts])), k,
                              handle=_h(dq))
    assert int((st != 0).sum()) == 0
    for b, x in enumerate(insts):
        Go, ldo, so = od.greens(x.K, 0.1, x.V, k)
        assert np.abs(G[b].cpu().numpy() - Go).max() <= GTOL * max(1.0, np.abs(Go).max()), b
        assert abs(float(ld[b]) - ldo) <= 1e-9 * max(1.0, abs(ldo)) and int(sg[b]) == so


def test_jacobi_closed_form_beta50(dq):
    """U = 0, site-independent field, beta = 50: scales e^{+-200} in D."""
    K = di.chain_hopping(8)
    M = 500
    c = np.random.default_rng(51).uniform(-0.3, 0.3, M)
    V = np.repeat(c[:, None], 8, axis=1)
    G, ld, _, st = dq.greens(_dev(K), 0.1, _dev(V), 10, handle=_h(dq))
    Gx, ldx = ex.closed_form_greens(K, 50.0, c.sum())
    assert int(st) == 0
    assert np.abs(G.cpu().numpy() - Gx).max() <= GTOL
    assert abs(float(ld) - ldx) <= 1e-9 * abs(ldx)


def test_jacobi_brute_force(dq):
    K = di.chain_hopping(4)
    V = 1.2 * di.ising_field(4, 35, 4)
    bf = ex.BruteForce(K, 0.1, V)
    G, ld, sg, st = dq.greens(_dev(K), 0.1, _dev(V), 8, handle=_h(dq))
    Gb, ldb, sb = bf.greens(1)
    assert np.abs(G.cpu().numpy() - bf.to_numpy(Gb)).max() <= GTOL
    assert abs(float(ld) - float(ldb)) <= 1e-9 * max(1.0, abs(float(ldb))) and int(sg) == sb


def test_jacobi_tdisplaced_and_grad(dq):
    """Both stacks stabilised by Jacobi: G(tau,tau), G(tau,0), G(0,tau) and the gradient."""
    inst = di.hubbard_instance(3, 4.0, 0.1, 3.0, 10, 71)
    K, V = _dev(inst.K), _dev(inst.V)
    h = _h(dq)
    Gtt, Gt0, G0t, st = dq.greens_tdisplaced(K, 0.1, V, 10, handle=h, want_0t=True)
    assert int(st) == 0
    Ott, Ot0 = od.greens_tdisplaced(inst.K, 0.1, inst.V, 10)
    O0t = od.greens_tdisplaced_0t(inst.K, 0.1, inst.V, 10)
    for A, O in ((Gtt, Ott), (Gt0, Ot0), (G0t, O0t)):
        A = A.cpu().numpy()
        for j in range(O.shape[0]):
            assert np.abs(A[j] - O[j]).max() <= GTOL * max(1.0, np.abs(O[j]).max()), j
    ld, sg, dV, st = dq.logdet_grad(K, 0.1, V, 10, handle=h)
    assert int(st) == 0
    assert np.abs(dV.cpu().numpy() - od.logdet_grad(inst.K, 0.1, inst.V, 10)).max() <= 1e-9


def test_jacobi_rejects_mixed_precision(dq):
    h = dq.Handle(chain_precision=8, decomposition=1)
    inst = di.hubbard_instance(2, 4.0, 0.1, 2.0, 10, 1)
    with pytest.raises(RuntimeError, match="unsupported"):
        dq.greens(_dev(inst.K), 0.1, _dev(inst.V), 10, handle=h)
