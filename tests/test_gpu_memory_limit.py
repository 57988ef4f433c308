"""Allocation-failure paths under a handle memory cap (dqmc_set_memory_limit).

A cap below what a call needs makes its buffer growth fail with
DQMC_ERR_NOMEM instead of exhausting the device; the handle keeps the buffers
it had and still runs problems that fit, with results bitwise equal to a
handle without a cap."""
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


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _inst(L, beta, batch, seed):
    inst = di.hubbard_instance(L, 4.0, 0.1, beta, 10, seed)
    V = np.stack([inst.V] + [di.hubbard_instance(L, 4.0, 0.1, beta, 10, seed + 1 + b).V
                             for b in range(batch - 1)])
    return _dev(inst.K), inst.dtau, _dev(V), inst.k


def _nomem(fn):
    with pytest.raises(RuntimeError, match="allocation failed"):
        fn()


@pytest.mark.parametrize("graphs", [False, True])
def test_limit_fails_then_recovers(dq, graphs):
    K, dtau, V, k = _inst(4, 4.0, 3, 7100)
    free = dq.Handle(graphs=graphs)
    G0, ld0, s0, st0 = dq.greens(K, dtau, V, k, handle=free)

    h = dq.Handle(graphs=graphs)
    h.set_memory_limit(4096)
    _nomem(lambda: dq.greens(K, dtau, V, k, handle=h))
    torch.cuda.synchronize()
    assert h.device_bytes <= 4096
    h.set_memory_limit(0)
    G1, ld1, s1, st1 = dq.greens(K, dtau, V, k, handle=h)
    assert torch.equal(G0, G1) and torch.equal(ld0, ld1) and torch.equal(s0, s1)
    assert int((st1 != 0).sum()) == 0

    # cap at what the handle now holds: a larger problem fails, the same one still runs
    held = h.device_bytes
    h.set_memory_limit(held)
    K2, dtau2, V2, k2 = _inst(6, 4.0, 8, 7200)
    _nomem(lambda: dq.greens(K2, dtau2, V2, k2, handle=h))
    assert h.device_bytes == held
    G2, ld2, s2, _ = dq.greens(K, dtau, V, k, handle=h)
    assert torch.equal(G0, G2) and torch.equal(ld0, ld2) and torch.equal(s0, s2)


def test_limit_on_other_calls(dq):
    K, dtau, V, k = _inst(4, 4.0, 2, 7300)
    h = dq.Handle()
    h.set_memory_limit(4096)
    _nomem(lambda: dq.greens_tdisplaced(K, dtau, V, k, handle=h))
    _nomem(lambda: dq.logdet_grad(K, dtau, V, k, handle=h))
    _nomem(lambda: h.register_K(K, dtau))
    _nomem(lambda: dq.greens_ragged([(K, dtau, V[0], k), (K, dtau, V[1], k)], handle=h))
    torch.cuda.synchronize()
    assert h.device_bytes <= 4096
    h.set_memory_limit(0)
    ref = dq.greens_ragged([(K, dtau, V[0], k), (K, dtau, V[1], k)], handle=dq.Handle())
    out = dq.greens_ragged([(K, dtau, V[0], k), (K, dtau, V[1], k)], handle=h)
    for a, b in zip(ref[0], out[0]):
        assert torch.equal(a, b)
    kid = h.register_K(K, dtau)
    assert kid >= 0


def test_limit_argument_check(dq):
    h = dq.Handle()
    with pytest.raises(RuntimeError, match="invalid argument"):
        h.set_memory_limit(-1)
