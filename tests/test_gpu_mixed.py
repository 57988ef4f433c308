"""Mixed-precision chain products (BF16 slices on the tensor cores).

Only the k-slice products change precision; QR, D splits and inversions stay
FP64.  The error of G against the FP64 oracle is a property of the slicing
(about N 2^{-7s} per product, amplified by the chain) and is reported rather
than pinned by the paper; these tests check that it shrinks with the slice
count and that eight slices reach 1e-8 in G and 1e-9 relative in log det.
"""
import numpy as np
import pytest

import dqmc_inputs as di
from oracle import dqmc as od

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_05286_gb300 as m
    m.lib()
    return m


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _errors(dq, insts, s):
    K = _dev(insts[0].K)
    V = _dev(np.stack([x.V for x in insts]))
    h = dq.Handle(chain_precision=s)
    G, ld, sg, st = dq.greens(K, insts[0].dtau, V, insts[0].k, handle=h)
    assert int((st != 0).sum()) == 0
    eg = el = 0.0
    for b, x in enumerate(insts):
        Go, ldo, so = od.greens(x.K, x.dtau, x.V, x.k)
        eg = max(eg, float(np.abs(G[b].cpu().numpy() - Go).max()) / max(1.0, np.abs(Go).max()))
        el = max(el, abs(float(ld[b]) - ldo) / abs(ldo))
        assert int(sg[b]) == so
    h.close()
    return eg, el


@pytest.mark.parametrize("L,beta", [(4, 8.0), (8, 10.0), (10, 6.0)])
def test_mixed_error_decreases_with_slices(dq, L, beta):
    insts = [di.hubbard_instance(L, 4.0, 0.1, beta, 10, 500 + i) for i in range(3)]
    errs = {s: _errors(dq, insts, s) for s in (4, 6, 8)}
    print({s: f"dG {e[0]:.2e} dlogdet {e[1]:.2e}" for s, e in errs.items()})
    assert errs[8][0] <= 1e-8 and errs[8][1] <= 1e-9
    assert errs[8][0] < errs[6][0] < errs[4][0]


def test_mixed_full_size_sampled(dq):
    """16x16 lattice, beta = 20, 128 instances, eight slices: instances 0 and 127."""
    insts = [di.batch_n256(i) for i in range(128)]
    K = _dev(insts[0].K)
    V = _dev(np.stack([x.V for x in insts]))
    h = dq.Handle(chain_precision=8)
    G, ld, sg, st = dq.greens(K, 0.1, V, 10, handle=h)
    assert int((st != 0).sum()) == 0
    for b in (0, 127):
        x = insts[b]
        Go, ldo, so = od.greens(x.K, 0.1, x.V, 10)
        assert np.abs(G[b].cpu().numpy() - Go).max() <= 1e-8 * max(1.0, np.abs(Go).max())
        assert abs(float(ld[b]) - ldo) <= 1e-9 * abs(ldo)
        assert int(sg[b]) == so


@pytest.mark.parametrize("L,beta,k,seed", [(4, 4.0, 10, 3), (6, 6.0, 7, 5)])
def test_mixed_tdisplaced(dq, L, beta, k, seed):
    """Both stacks of the time-displaced path on the tensor cores (eight slices)."""
    inst = di.hubbard_instance(L, 4.0, 0.1, beta, k, seed)
    h = dq.Handle(chain_precision=8)
    Gtt, Gt0, st = dq.greens_tdisplaced(_dev(inst.K), 0.1, _dev(inst.V), k, handle=h)
    assert int(st) == 0
    Ott, Ot0 = od.greens_tdisplaced(inst.K, 0.1, inst.V, k)
    Gtt, Gt0 = Gtt.cpu().numpy(), Gt0.cpu().numpy()
    for j in range(Ott.shape[0]):
        sc = max(1.0, np.abs(Ott[j]).max())
        assert np.abs(Gtt[j] - Ott[j]).max() <= 1e-8 * sc, j
        assert np.abs(Gt0[j] - Ot0[j]).max() <= 1e-8 * max(1.0, np.abs(Ot0[j]).max()), j
    h.close()


def test_mixed_grad(dq):
    inst = di.hubbard_instance(6, 4.0, 0.1, 8.0, 10, 11)
    h = dq.Handle(chain_precision=8)
    ld, sg, dV, st = dq.logdet_grad(_dev(inst.K), 0.1, _dev(inst.V), 10, handle=h)
    assert int(st) == 0
    dVo = od.logdet_grad(inst.K, 0.1, inst.V, 10)
    ldo, so = od.logdet(inst.K, 0.1, inst.V, 10)
    assert np.abs(dV.cpu().numpy() - dVo).max() <= 1e-8
    assert abs(float(ld) - ldo) <= 1e-9 * abs(ldo)
    assert int(sg) == so
    h.close()


def test_mixed_rejected_where_not_built(dq):
    """N above 256 has no tensor-core chain, also inside a ragged batch."""
    h = dq.Handle(chain_precision=5)
    big = torch.zeros((1, 20, 324), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        dq.greens(_dev(di.square_hopping(18)), 0.1, big, 10, handle=h)
    with pytest.raises(RuntimeError):
        dq.greens_tdisplaced(_dev(di.square_hopping(18)), 0.1, big, 10, handle=h)
    inst = di.hubbard_instance(4, 4.0, 0.1, 2.0, 10, 1)
    with pytest.raises(RuntimeError):
        dq.greens_ragged([(_dev(inst.K), 0.1, _dev(inst.V), 10),
                          (_dev(di.square_hopping(18)), 0.1, big[0], 10)], handle=h)
