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


def test_tune_modes(dq, tmp_path, monkeypatch):
    """DQMC_TUNE=off returns the default k without timing, force re-tunes past the cache."""
    from paper_2003_05286_gb300 import tune
    insts = [di.hubbard_instance(4, 4.0, 0.1, 4.0, 10, 710 + i) for i in range(2)]
    K = torch.tensor(insts[0].K, device="cuda")
    V = torch.tensor(np.stack([x.V for x in insts]), device="cuda")
    cache = str(tmp_path / "tune.json")
    kw = dict(candidates=(4, 8), tiles=(0,), tol=1e-10, cache_file=cache, tag="modes")
    monkeypatch.setenv("DQMC_TUNE", "off")
    best, table = tune.tune(K, 0.1, V, default_k=7, **kw)
    assert table is None and best["k"] == 7 and best["ms"] is None
    monkeypatch.setenv("DQMC_TUNE", "on")
    best, table = tune.tune(K, 0.1, V, **kw)
    assert table and best["k"] in (4, 8)
    again, t2 = tune.tune(K, 0.1, V, **kw)
    assert t2 is None and again == best
    monkeypatch.setenv("DQMC_TUNE", "force")
    forced, t3 = tune.tune(K, 0.1, V, **kw)
    assert t3 and forced["k"] in (4, 8)
    monkeypatch.setenv("DQMC_TUNE", "sometimes")
    with pytest.raises(ValueError):
        tune.tune(K, 0.1, V, **kw)
