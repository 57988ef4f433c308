"""Autotuner of k and the FP64 product tile (paper_2003_05286_gb300.tune)."""
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


def test_tune_picks_accurate_fast_k(dq, tmp_path):
    from paper_2003_05286_gb300 import tune
    insts = [di.hubbard_instance(6, 4.0, 0.1, 15.0, 10, 700 + i) for i in range(4)]
    K = torch.tensor(insts[0].K, device="cuda")
    V = torch.tensor(np.stack([x.V for x in insts]), device="cuda")
    cache = str(tmp_path / "tune.json")
    best, table = tune.tune(K, 0.1, V, candidates=(4, 8, 12, 20), tiles=(0, 32), tol=1e-10,
                            cache_file=cache)
    assert table and best["err"] <= 1e-10
    assert best["k"] in (4, 8, 12, 20)
    # every accepted candidate is within tolerance; the pick is the fastest of them
    ok = [r for r in table if r["err"] <= 1e-10]
    assert best["ms"] == min(r["ms"] for r in ok)
    # cached on the second call
    again, t2 = tune.tune(K, 0.1, V, candidates=(4, 8, 12, 20), tiles=(0, 32), tol=1e-10,
                          cache_file=cache)
    assert t2 is None and again == best
