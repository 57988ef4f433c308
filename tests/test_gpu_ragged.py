"""GPU parity of the ragged batch (dqmc_greens_ragged): instances of different N,
M, U and k in one call, each against the oracle and against its own uniform
single-instance call (same kernels, so bitwise equal)."""
import numpy as np
import pytest

import dqmc_inputs as di
from oracle import dqmc as od

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


def test_ragged_small_mixed(dq):
    rng = np.random.default_rng(5)
    insts = []
    for i in range(14):
        L = int(rng.choice([2, 3, 4, 5]))
        beta = round(float(rng.uniform(1.0, 6.0)), 1)
        k = int(rng.choice([5, 10]))
        insts.append(di.hubbard_instance(L, float(rng.uniform(2, 8)), 0.1, beta, min(k, int(beta * 10)),
                                         1000 + i))
    Gs, ld, sg, st = dq.greens_ragged([(_dev(x.K), x.dtau, _dev(x.V), x.k) for x in insts])
    assert int((st != 0).sum()) == 0
    seq = dq.Handle(fold=0)     # the ragged chains fold sequentially
    for i, x in enumerate(insts):
        Go, ldo, so = od.greens(x.K, x.dtau, x.V, x.k)
        assert np.abs(Gs[i].cpu().numpy() - Go).max() <= GTOL * max(1.0, np.abs(Go).max()), i
        assert abs(float(ld[i]) - ldo) <= 1e-9 * max(1.0, abs(ldo))
        assert int(sg[i]) == so
        G1, ld1, _, _ = dq.greens(_dev(x.K), x.dtau, _dev(x.V), x.k, handle=seq)
        assert torch.equal(G1, Gs[i]) and float(ld1) == float(ld[i])


def test_ragged_shared_K_batches(dq):
    """Instances that share a K tensor run as one batched chain per (N, k, dtau), with
    different M inside a batch; each result still equals its own single-instance call."""
    insts = []
    for i in range(24):
        L = (3, 4)[i % 2]
        beta = 1.0 + 0.5 * (i % 7)
        insts.append(di.hubbard_instance(L, 4.0, 0.1, beta, 5, 2000 + i))
    Ks = {L: _dev(di.square_hopping(L)) for L in (3, 4)}
    items = [(Ks[int(round(x.N ** 0.5))], x.dtau, _dev(x.V), x.k) for x in insts]
    Gs, ld, sg, st = dq.greens_ragged(items)
    assert int((st != 0).sum()) == 0
    seq = dq.Handle(fold=0)     # the ragged chains fold sequentially
    for i, x in enumerate(insts):
        Go, ldo, so = od.greens(x.K, x.dtau, x.V, x.k)
        assert np.abs(Gs[i].cpu().numpy() - Go).max() <= GTOL * max(1.0, np.abs(Go).max()), i
        G1, ld1, _, _ = dq.greens(_dev(x.K), x.dtau, _dev(x.V), x.k, handle=seq)
        assert torch.equal(G1, Gs[i]) and float(ld1) == float(ld[i]), i


def test_ragged_full_size_sampled(dq):
    """1024 instances, N in {36,64,100,144,256}, beta in [10,50] (M in [100,500]),
    U in [2,8], k = 10, one K per lattice size; the smallest and largest instances of
    each N against the oracle."""
    insts = [di.ragged_instance(i, 10) for i in range(1024)]
    Ks = {}
    for x in insts:
        Ks.setdefault(x.N, _dev(x.K))
    Gs, ld, sg, st = dq.greens_ragged([(Ks[x.N], x.dtau, _dev(x.V), x.k) for x in insts])
    assert int((st != 0).sum()) == 0
    byN = {}
    for i, x in enumerate(insts):
        byN.setdefault(x.N, []).append(i)
    assert sorted(byN) == [36, 64, 100, 144, 256]
    for N, idx in byN.items():
        picks = {min(idx, key=lambda i: insts[i].M), max(idx, key=lambda i: insts[i].M)}
        for i in picks:
            x = insts[i]
            Go, ldo, so = od.greens(x.K, x.dtau, x.V, x.k)
            assert np.abs(Gs[i].cpu().numpy() - Go).max() <= GTOL * max(1.0, np.abs(Go).max()), (N, i)
            assert abs(float(ld[i]) - ldo) <= 1e-9 * abs(ldo)
            assert int(sg[i]) == so


def _mixed_sizes(n, seed):
    rng = np.random.default_rng(seed)
    insts = []
    for i in range(n):
        L = int(rng.choice([2, 3, 4]))
        beta = float(rng.choice([1.0, 1.5, 2.0]))
        insts.append(di.hubbard_instance(L, float(rng.uniform(2, 6)), 0.1, beta, int(rng.choice([5, 10])),
                                         seed * 100 + i))
    Ks = {L: _dev(di.square_hopping(L)) for L in (2, 3, 4)}
    items = [(Ks[int(round(x.N ** 0.5))], x.dtau, _dev(x.V), x.k) for x in insts]
    return insts, items


def test_ragged_tdisplaced(dq):
    """Groups of equal (N, M, k, K): every instance equals its own uniform call bitwise
    and matches the oracle."""
    insts, items = _mixed_sizes(18, 31)
    Gtt, Gt0, st = dq.greens_tdisplaced_ragged(items)
    assert int((st != 0).sum()) == 0
    for i, x in enumerate(insts):
        a, b, s1 = dq.greens_tdisplaced(_dev(x.K), x.dtau, _dev(x.V), x.k)
        assert torch.equal(Gtt[i], a) and torch.equal(Gt0[i], b), i
        if i < 6:
            Ott, Ot0 = od.greens_tdisplaced(x.K, x.dtau, x.V, x.k)
            sc = max(1.0, np.abs(Ott).max())
            assert np.abs(Gtt[i].cpu().numpy() - Ott).max() <= GTOL * sc
            assert np.abs(Gt0[i].cpu().numpy() - Ot0).max() <= GTOL * max(1.0, np.abs(Ot0).max())


def test_ragged_tdisplaced_g0t(dq):
    """dqmc_greens_tdisplaced_ragged_ex: G(0, tau_j) per instance equals the uniform call."""
    insts, items = _mixed_sizes(9, 33)
    Gtt, Gt0, G0t, st = dq.greens_tdisplaced_ragged(items, want_t0=False, want_0t=True)
    assert Gt0 is None and int((st != 0).sum()) == 0
    for i, x in enumerate(insts):
        a, _, c, _ = dq.greens_tdisplaced(_dev(x.K), x.dtau, _dev(x.V), x.k, want_t0=False,
                                          want_0t=True)
        assert torch.equal(Gtt[i], a) and torch.equal(G0t[i], c), i
        if i < 3:
            O = od.greens_tdisplaced_0t(x.K, x.dtau, x.V, x.k)
            assert np.abs(G0t[i].cpu().numpy() - O).max() <= GTOL * max(1.0, np.abs(O).max())


def test_ragged_grad(dq):
    insts, items = _mixed_sizes(14, 47)
    ld, sg, dVs, st = dq.logdet_grad_ragged(items)
    assert int((st != 0).sum()) == 0
    for i, x in enumerate(insts):
        l1, s1, d1, t1 = dq.logdet_grad(_dev(x.K), x.dtau, _dev(x.V), x.k)
        assert torch.equal(dVs[i], d1) and float(l1) == float(ld[i]) and int(s1) == int(sg[i]), i
        if i < 4:
            dVo = od.logdet_grad(x.K, x.dtau, x.V, x.k)
            assert np.abs(dVs[i].cpu().numpy() - dVo).max() <= 1e-9


def _uneven_M_items(seed, n=12):
    """Instances of N = 9, 16 and 36 sharing one K per size, with M = 10 .. 33
    (last chunks of several lengths inside one batched chain of k = 10)."""
    rng = np.random.default_rng(seed)
    insts = []
    for i in range(n):
        L = (3, 4, 6)[i % 3]
        beta = round(float(rng.uniform(1.0, 3.3)), 1)
        insts.append(di.hubbard_instance(L, float(rng.uniform(2, 6)), 0.1, beta, 10, seed * 100 + i))
    Ks = {L: _dev(di.square_hopping(L)) for L in (3, 4, 6)}
    items = [(Ks[int(round(x.N ** 0.5))], x.dtau, _dev(x.V), x.k) for x in insts]
    return insts, items


def test_ragged_mixed_precision(dq):
    """The tensor-core chain (8 BF16 digit slices) in a ragged batch: instances of
    one group end at different chunks, so ended instances copy their product and X
    through.  Against the oracle to 1e-8 of max(1, max|G|) and 1e-9 relative in log det."""
    insts, items = _uneven_M_items(31)
    h = dq.Handle(chain_precision=8)
    Gs, ld, sg, st = dq.greens_ragged(items, handle=h)
    assert int((st != 0).sum()) == 0
    for i, x in enumerate(insts):
        Go, ldo, so = od.greens(x.K, x.dtau, x.V, x.k)
        err = np.abs(Gs[i].cpu().numpy() - Go).max() / max(1.0, np.abs(Go).max())
        assert err <= 1e-8, (i, x.N, x.M, err)
        assert abs(float(ld[i]) - ldo) <= 1e-9 * max(1.0, abs(ldo))
        assert int(sg[i]) == so
    h.close()


@pytest.mark.parametrize("prec", [0, 8])
def test_ragged_graph_replay(dq, prec):
    """In CUDA-graph mode a repeated ragged call replays its graph: bitwise the
    eager result, and new fields written into the same V pool give the eager
    result for those fields."""
    insts, items = _uneven_M_items(47)
    batch = dq.RaggedBatch(items)
    eager = dq.Handle(chain_precision=prec)
    G0 = [g.clone() for g in batch.run(handle=eager)[0]]
    ld0 = batch.ld.clone()
    hg = dq.Handle(chain_precision=prec, graphs=True)
    for _ in range(3):                      # capture, then replays
        Gs, ld, sg, st = batch.run(handle=hg)
        torch.cuda.synchronize()
        assert int((st != 0).sum()) == 0
        assert all(torch.equal(a, b) for a, b in zip(Gs, G0))
        assert torch.equal(ld, ld0)
    n_graph = hg.last_launch_count
    # new fields in place: the replayed graph reads them
    batch.set_fields([0.5 * _dev(x.V) for x in insts])
    G1 = [g.clone() for g in batch.run(handle=eager)[0]]
    ld1 = batch.ld.clone()
    Gs, ld, _, st = batch.run(handle=hg)
    torch.cuda.synchronize()
    assert hg.last_launch_count == n_graph
    assert all(torch.equal(a, b) for a, b in zip(Gs, G1))
    assert torch.equal(ld, ld1)
    assert not all(torch.equal(a, b) for a, b in zip(G1, G0))
    # a different descriptor set on the same handle is recorded anew
    insts2, items2 = _uneven_M_items(48, n=7)
    b2 = dq.RaggedBatch(items2)
    Gs2, ld2, _, st2 = b2.run(handle=hg)
    torch.cuda.synchronize()
    for i, x in enumerate(insts2):
        Go, ldo, so = od.greens(x.K, x.dtau, x.V, x.k)
        tol = 1e-10 if prec == 0 else 1e-8
        assert np.abs(Gs2[i].cpu().numpy() - Go).max() <= tol * max(1.0, np.abs(Go).max())
    eager.close()
    hg.close()


def test_registered_K_batched(dq):
    """dqmc_register_K + dqmc_greens_batched with a device-resident descriptor
    array: against the oracle, bitwise equal to the ragged call on the same
    instances (same exponentials, same kernels), replayed as a graph."""
    insts, items = _uneven_M_items(53)
    for graphs in (False, True):
        h = dq.Handle(graphs=graphs)
        ids = {}
        for x in insts:
            L = int(round(x.N ** 0.5))
            if L not in ids:
                ids[L] = h.register_K(_dev(di.square_hopping(L)), 0.1)
        bt = dq.Batched(h, [(ids[int(round(x.N ** 0.5))], _dev(x.V), x.k) for x in insts])
        for _ in range(2):
            Gs, ld, sg, st = bt.run()
            torch.cuda.synchronize()
            assert int((st != 0).sum()) == 0
        Gr, ldr, sgr, _ = dq.greens_ragged(items, handle=dq.Handle())
        for i, x in enumerate(insts):
            assert torch.equal(Gs[i], Gr[i]), i
            assert float(ld[i]) == float(ldr[i]) and int(sg[i]) == int(sgr[i])
            Go, ldo, so = od.greens(x.K, x.dtau, x.V, x.k)
            assert np.abs(Gs[i].cpu().numpy() - Go).max() <= GTOL * max(1.0, np.abs(Go).max())
        h.close()


def test_registered_K_errors(dq):
    h = dq.Handle()
    K = di.square_hopping(3)
    K[0, 1] += 0.5                                   # not symmetric
    with pytest.raises(RuntimeError):
        h.register_K(_dev(K), 0.1)
    kid = h.register_K(_dev(di.square_hopping(3)), 0.1)
    assert kid == 0
    inst = di.hubbard_instance(3, 4.0, 0.1, 1.0, 5, 3)
    bt = dq.Batched(h, [(kid, _dev(inst.V), 5)])
    bt.desc.view(torch.int32)[3] = 7                 # K_id of instance 0 -> not registered
    with pytest.raises(RuntimeError):
        bt.run()
    h.close()
