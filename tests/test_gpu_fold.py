"""Tree-parallel fold of the equal-time chain (dqmc_set_chain_fold).

The pairwise product of Eq. (stabmult) is associative, so the chunk products
can be decomposed independently and folded in log2 levels.  Both folds must
give the oracle's G, log det and sign; the automatic choice must equal the
explicit one it picks.  Cases cover a short last chunk, chunk counts that are
not powers of two (identity padding), N = 256, and beta = 50 at U = 0, where
the scales span e^{+-200}.
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


def _run(dq, fold, K, dtau, V, k):
    h = dq.Handle(fold=fold)
    out = dq.greens(_dev(K), dtau, _dev(V), k, handle=h)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in out], h.last_launch_count


@pytest.mark.parametrize("L,beta,k,batch,seed", [
    (4, 8.0, 10, 1, 1),     # 8 chunks
    (2, 3.1, 10, 3, 2),     # 4 chunks, the last one short
    (6, 5.0, 7, 2, 3),      # M = 50: 8 chunks, the last one short
    (8, 13.0, 10, 1, 4),    # 13 chunks: padded to 16
    (3, 2.0, 10, 5, 5),     # 2 chunks (tree by setting only)
])
def test_tree_and_sequential_vs_oracle(dq, L, beta, k, batch, seed):
    insts = [di.hubbard_instance(L, 4.0, 0.1, beta, k, seed * 10 + i) for i in range(batch)]
    K = insts[0].K
    V = np.stack([x.V for x in insts])
    (Gt, ldt, sgt, stt), nt = _run(dq, 1, K, 0.1, V, k)
    (Gs, lds, sgs, sts), ns = _run(dq, 0, K, 0.1, V, k)
    assert (stt == 0).all() and (sts == 0).all()
    for b, x in enumerate(insts):
        G, ld, sg = od.greens(x.K, 0.1, x.V, k)
        sc = max(1.0, np.abs(G).max())
        assert np.abs(Gt[b] - G).max() <= GTOL * sc, b
        assert np.abs(Gs[b] - G).max() <= GTOL * sc, b
        assert abs(ldt[b] - ld) <= 1e-9 * max(1.0, abs(ld)) and sgt[b] == sg
        assert abs(lds[b] - ld) <= 1e-9 * max(1.0, abs(ld)) and sgs[b] == sg
    if -(-V.shape[1] // k) >= 8:
        # fewer launches: ceil(log2(chunks)) + 1 dependent QRs instead of one per
        # chunk (the k slice products of a chunk are one launch for N <= 128)
        assert nt < ns


def test_tree_n256(dq):
    """16x16 lattice, U=4, beta=20, k=10 (20 chunks, padded to 32), two instances."""
    insts = [di.hubbard_instance(16, 4.0, 0.1, 20.0, 10, 700 + i) for i in range(2)]
    V = np.stack([x.V for x in insts])
    (Gt, ldt, sgt, stt), _ = _run(dq, 1, insts[0].K, 0.1, V, 10)
    assert (stt == 0).all()
    G, ld, sg = od.greens(insts[1].K, 0.1, insts[1].V, 10)
    assert np.abs(Gt[1] - G).max() <= GTOL * max(1.0, np.abs(G).max())
    assert abs(ldt[1] - ld) <= 1e-9 * abs(ld) and sgt[1] == sg


def test_tree_closed_form_beta50(dq):
    """U = 0 with a site-independent field at beta = 50 (scales e^{+-200})."""
    K = di.square_hopping(4)
    M = 500
    c = np.random.default_rng(50).uniform(-0.3, 0.3, M)
    V = np.repeat(c[:, None], 16, axis=1)
    (Gt, ldt, _, stt), _ = _run(dq, 1, K, 0.1, V[None], 10)
    Gx, ldx = ex.closed_form_greens(K, 50.0, c.sum())
    assert int(stt[0]) == 0
    assert np.abs(Gt[0] - Gx).max() <= GTOL
    assert abs(ldt[0] - ldx) <= 1e-9 * abs(ldx)


def test_auto_picks_by_batch(dq):
    """Auto equals the tree bitwise for one instance and the sequential chain for 64."""
    for batch, want in ((1, 1), (64, 0)):
        insts = [di.hubbard_instance(4, 4.0, 0.1, 8.0, 10, 900 + i) for i in range(batch)]
        V = np.stack([x.V for x in insts])
        (Ga, lda, _, _), _ = _run(dq, 2, insts[0].K, 0.1, V, 10)
        (Gw, ldw, _, _), _ = _run(dq, want, insts[0].K, 0.1, V, 10)
        assert np.array_equal(Ga, Gw) and np.array_equal(lda, ldw), batch


def test_fold_setting_rejects_bad_mode(dq):
    h = dq.Handle()
    with pytest.raises(RuntimeError):
        h.set_chain_fold(7)
