"""GPU parity of the log-det gradient (dqmc_logdet_grad) and its autograd wrapper.

dV_l(i) = d log|det(1 + B_M...B_1)| / dV_l(i) = 1 - G_l(i,i).  The oracle
computes every G_l from scratch; the GPU takes G at the k-grid from the two
stacks and wraps G_{l+1} = B_l G_l B_l^{-1} in between (at most k-1 wraps),
which costs a few digits: tolerance 1e-9 absolute.  Against central finite
differences (h = 1e-6 on phi) the round-off floor is ~1e-7, tolerance 1e-5.
"""
import numpy as np
import pytest

import dqmc_inputs as di
from oracle import dqmc as od

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DTOL = 1e-9


@pytest.fixture(scope="module")
def dq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_05286_gb300 as m
    m.lib()
    return m


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("L,beta,k,seed", [(2, 2.0, 5, 1), (3, 3.3, 10, 2), (4, 4.0, 10, 3),
                                            (4, 4.0, 1, 4), (6, 5.0, 8, 5)])
def test_grad_vs_oracle(dq, L, beta, k, seed):
    inst = di.gaussian_instance(L, 1.5, 0.1, beta, k, seed)
    ld, sg, dV, st = dq.logdet_grad(_dev(inst.K), 0.1, _dev(inst.V), k)
    dVo = od.logdet_grad(inst.K, 0.1, inst.V, k)
    ldo, so = od.logdet(inst.K, 0.1, inst.V, k)
    assert int(st) == 0
    assert np.abs(dV.cpu().numpy() - dVo).max() <= DTOL
    assert abs(float(ld) - ldo) <= 1e-9 * max(1.0, abs(ldo))
    assert int(sg) == so


def test_grad_finite_difference(dq):
    inst = di.gaussian_instance(4, 1.5, 0.1, 4.0, 10, 7)
    K = _dev(inst.K)
    g, dtau, h = 1.5, 0.1, 1e-6
    phi = inst.V / (dtau * g)
    ld, _, dV, _ = dq.logdet_grad(K, dtau, _dev(inst.V), 10)
    dphi = dtau * g * dV.cpu().numpy()
    for (l, i) in [(0, 0), (13, 5), (39, 15), (20, 7)]:
        pp, pm = phi.copy(), phi.copy()
        pp[l, i] += h
        pm[l, i] -= h
        lp = float(dq.logdet(K, dtau, _dev(dtau * g * pp), 10)[0])
        lm = float(dq.logdet(K, dtau, _dev(dtau * g * pm), 10)[0])
        assert abs((lp - lm) / (2 * h) - dphi[l, i]) <= 1e-5


def test_logdet_autograd(dq):
    inst = di.gaussian_instance(4, 1.5, 0.1, 3.0, 10, 9)
    K = _dev(inst.K)
    V = _dev(np.stack([inst.V, 0.5 * inst.V])).requires_grad_(True)
    ld = dq.LogDet.apply(V, K, 0.1, 10)
    (ld * torch.tensor([1.0, -2.0], dtype=torch.float64, device="cuda")).sum().backward()
    _, _, dV, _ = dq.logdet_grad(K, 0.1, V.detach(), 10)
    assert torch.allclose(V.grad[0], dV[0], atol=0, rtol=0)
    assert torch.allclose(V.grad[1], -2.0 * dV[1], atol=0, rtol=0)


def test_logdet_forward_paths(dq):
    """LogDet.forward: the log det alone when no gradient is wanted, log det +
    gradient otherwise; both against the oracle, and the forward-only call
    launches fewer kernels (one chain and one inversion, no stacks or wraps)."""
    inst = di.gaussian_instance(4, 1.5, 0.1, 3.0, 10, 11)
    K = _dev(inst.K)
    ldo, _ = od.logdet(inst.K, 0.1, inst.V, 10)
    dVo = od.logdet_grad(inst.K, 0.1, inst.V, 10)
    h = dq.Handle()
    V0 = _dev(inst.V)                                   # no grad wanted
    ld0 = dq.LogDet.apply(V0, K, 0.1, 10, h)
    n_fwd = h.last_launch_count
    assert not ld0.requires_grad
    assert abs(float(ld0) - ldo) <= 1e-9 * max(1.0, abs(ldo))
    V1 = _dev(inst.V).requires_grad_(True)
    with torch.no_grad():
        ld1 = dq.LogDet.apply(V1, K, 0.1, 10, h)
    assert h.last_launch_count == n_fwd
    assert float(ld1) == float(ld0)
    ld2 = dq.LogDet.apply(V1, K, 0.1, 10, h)
    assert h.last_launch_count > n_fwd
    assert abs(float(ld2.detach()) - ldo) <= 1e-9 * max(1.0, abs(ldo))
    ld2.backward()
    assert np.abs(V1.grad.cpu().numpy() - dVo).max() <= DTOL
    h.close()


def test_grad_full_size_sampled(dq):
    """12x12 lattice, phi ~ N(0,1), g=1.5, dtau=0.1, beta=20 (M=200), k=10, 64
    instances in one call; instance 0 and 63 checked at sampled slices."""
    insts = [di.batch_n144_gaussian(i) for i in range(64)]
    K = _dev(insts[0].K)
    V = _dev(np.stack([x.V for x in insts]))
    ld, sg, dV, st = dq.logdet_grad(K, 0.1, V, 10)
    assert int((st != 0).sum()) == 0
    for b in (0, 63):
        x = insts[b]
        ls = [1, 2, 10, 11, 105, 199, 200]
        dVo = od.logdet_grad(x.K, 0.1, x.V, 10, slices=ls)
        for l in ls:
            assert np.abs(dV[b, l - 1].cpu().numpy() - dVo[l - 1]).max() <= DTOL, (b, l)
        ldo, so = od.logdet(x.K, 0.1, x.V, 10)
        assert abs(float(ld[b]) - ldo) <= 1e-9 * abs(ldo) and int(sg[b]) == so
