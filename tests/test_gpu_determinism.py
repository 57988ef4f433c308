"""Determinism: repeated calls and different stream schedules give bitwise equal results.

Every instance's arithmetic is fixed by its own inputs; neither the sub-batch
pipeline (how instances are split over streams), nor a second call on the same
handle, nor the precision's kernel mix may change a bit of the output.  This
stands in for a race detector (compute-sanitizer is not available here): a
data race between streams or CTAs would show up as run-to-run differences.
"""
import os

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


def _run(dq, fn, prec, pipeline):
    old = os.environ.get("DQMC_PIPELINE")
    os.environ["DQMC_PIPELINE"] = pipeline
    try:
        h = dq.Handle(chain_precision=prec)
        out = [tuple(t.clone() for t in fn(h)) for _ in range(2)]
        h.close()
    finally:
        if old is None:
            del os.environ["DQMC_PIPELINE"]
        else:
            os.environ["DQMC_PIPELINE"] = old
    return out


@pytest.mark.parametrize("prec", [0, 8])
def test_greens_bitwise_across_runs_and_schedules(dq, prec):
    insts = [di.hubbard_instance(6, 4.0, 0.1, 6.0, 10, 900 + i) for i in range(32)]
    K = torch.tensor(insts[0].K, device="cuda")
    V = torch.tensor(np.stack([x.V for x in insts]), device="cuda")
    fn = lambda h: dq.greens(K, 0.1, V, 10, handle=h)  # noqa: E731
    runs = _run(dq, fn, prec, "0") + _run(dq, fn, prec, "2") + _run(dq, fn, prec, "4")
    for r in runs[1:]:
        assert all(torch.equal(a, b) for a, b in zip(runs[0], r))


def test_stacks_bitwise_across_runs_and_schedules(dq):
    insts = [di.hubbard_instance(4, 4.0, 0.1, 4.0, 10, 950 + i) for i in range(8)]
    K = torch.tensor(insts[0].K, device="cuda")
    V = torch.tensor(np.stack([x.V for x in insts]), device="cuda")
    for fn in (lambda h: dq.greens_tdisplaced(K, 0.1, V, 10, handle=h),
               lambda h: dq.logdet_grad(K, 0.1, V, 10, handle=h)):
        runs = _run(dq, fn, 0, "0") + _run(dq, fn, 0, "1")
        for r in runs[1:]:
            assert all(torch.equal(a, b) for a, b in zip(runs[0], r) if a is not None)


@pytest.mark.parametrize("prec", [0, 8])
def test_ragged_bitwise_across_runs_and_schedules(dq, prec):
    """Ragged groups large enough to run as staggered sub-batches (with the
    per-instance chain lengths of uneven M): bitwise equal to the unpipelined
    schedule and to a second call."""
    rng = np.random.default_rng(61)
    insts = []
    for i in range(40):
        L = 4 if i < 20 else 6
        beta = round(float(rng.uniform(2.0, 6.0)), 1)
        insts.append(di.hubbard_instance(L, 4.0, 0.1, beta, 10, 6100 + i))
    Ks = {4: torch.tensor(di.square_hopping(4), device="cuda"),
          6: torch.tensor(di.square_hopping(6), device="cuda")}
    items = [(Ks[int(round(x.N ** 0.5))], x.dtau, torch.tensor(x.V, device="cuda"), x.k)
             for x in insts]
    batch = dq.RaggedBatch(items)

    def fn(h):
        Gs, ld, sg, st = batch.run(handle=h)
        assert int((st != 0).sum()) == 0
        return tuple(g.clone() for g in Gs) + (ld.clone(), sg.clone())

    runs = _run(dq, fn, prec, "0") + _run(dq, fn, prec, "2") + _run(dq, fn, prec, "4")
    for r in runs[1:]:
        assert all(torch.equal(a, b) for a, b in zip(runs[0], r))
