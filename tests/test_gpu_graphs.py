"""CUDA-graph mode (dqmc_set_graph_mode): recorded calls replayed for identical arguments.

Graph mode must change nothing but launch cost: every result is compared
bitwise with the same call on a handle without graphs, for the first
(captured) call and for replays, after the inputs were overwritten in place,
and after a change of arguments forced a new capture.
"""
import numpy as np
import pytest

import dqmc_inputs as di

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_05286_gb300 as m
    m.lib()
    return m


def _fields(L, beta, n, seed):
    insts = [di.hubbard_instance(L, 4.0, 0.1, beta, 10, seed + i) for i in range(n)]
    K = torch.tensor(insts[0].K, device="cuda")
    V = torch.tensor(np.stack([x.V for x in insts]), device="cuda")
    return K, V


@pytest.mark.parametrize("prec,batch", [(0, 1), (0, 16), (8, 1), (8, 16)])
def test_graph_greens_bitwise_and_inplace_update(dq, prec, batch):
    K, V = _fields(4, 4.0, batch, 300)
    _, V2 = _fields(4, 4.0, batch, 400)
    hg = dq.Handle(chain_precision=prec, graphs=True)
    he = dq.Handle(chain_precision=prec)
    G = torch.empty((batch, 16, 16), dtype=torch.float64, device="cuda")
    ld = torch.empty(batch, dtype=torch.float64, device="cuda")
    sg = torch.empty(batch, dtype=torch.int32, device="cuda")
    st = torch.empty(batch, dtype=torch.int32, device="cuda")
    p = lambda t: t.data_ptr()  # noqa: E731

    def call(h, Vx):
        rc = h._lib.dqmc_greens(h.h, batch, 16, 40, p(K), 0.1, p(Vx), 10, p(G), p(ld), p(sg), p(st))
        assert rc == 0
        torch.cuda.synchronize()
        return G.clone(), ld.clone(), sg.clone(), st.clone()

    he.bind_stream(); hg.bind_stream()
    ref1 = call(he, V)
    ref2 = call(he, V2)
    Vbuf = V.clone()
    for rep in range(3):                       # capture, then replays
        out = call(hg, Vbuf)
        assert all(torch.equal(a, b) for a, b in zip(out, ref1)), rep
    Vbuf.copy_(V2)                             # new field in the same buffer: replay, new result
    out = call(hg, Vbuf)
    assert all(torch.equal(a, b) for a, b in zip(out, ref2))
    assert int((out[3] != 0).sum()) == 0
    hg.close(); he.close()


def test_graph_recapture_on_new_arguments(dq):
    K, V = _fields(4, 6.0, 2, 500)
    hg = dq.Handle(graphs=True)
    he = dq.Handle()
    for k in (10, 5, 10):                      # k changes the captured sequence
        Gg, ldg, _, _ = dq.greens(K, 0.1, V, k, handle=hg)
        Ge, lde, _, _ = dq.greens(K, 0.1, V, k, handle=he)
        assert torch.equal(Gg, Ge) and torch.equal(ldg, lde), k
    hg.close(); he.close()


def test_graph_tdisplaced_grad_logdet(dq):
    K, V = _fields(4, 4.0, 3, 600)
    hg = dq.Handle(graphs=True)
    he = dq.Handle()
    for _ in range(2):
        a = dq.greens_tdisplaced(K, 0.1, V, 10, handle=hg)
        b = dq.greens_tdisplaced(K, 0.1, V, 10, handle=he)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
        a = dq.logdet_grad(K, 0.1, V, 10, handle=hg)
        b = dq.logdet_grad(K, 0.1, V, 10, handle=he)
        assert all(torch.equal(x, y) for x, y in zip(a, b))
        a = dq.logdet(K, 0.1, V, 10, handle=hg)
        b = dq.logdet(K, 0.1, V, 10, handle=he)
        assert all(torch.equal(x, y) for x, y in zip(a, b))
    hg.close(); he.close()
