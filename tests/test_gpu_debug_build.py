"""The debug library (sources compiled with -DDQMC_DEBUG): device-side checks
of the kernels' index invariants that record a failure instead of trapping.

A child process with DQMC_DEBUG=1 loads the debug library and runs a set of
calls that reaches every checked kernel (FP64 chain at N = 16, 64, 144, 256
and 324, the fused small-N chunk products, both pivoted QR kernels, the LU
solves of every inversion, the Jacobi SVD, the BF16 splitter and tensor-core
product, ragged batches, graph replay, the allocation-free call).  No check may
fail, and every result must be bitwise equal to the release library's on the
same inputs: the checks change no arithmetic.  The check mechanism itself is
exercised by dqmc_selftest_check, whose failing check guards an access that
stays inside its array either way."""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

import dqmc_inputs as di

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_05286_gb300 as m
    from paper_2003_05286_gb300 import build as b
    b.build(debug=True)
    m.lib()
    return m


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _batch(L, beta, k, batch, seed):
    xs = [di.hubbard_instance(L, 4.0, 0.1, beta, k, seed + b) for b in range(batch)]
    return _dev(xs[0].K), 0.1, _dev(np.stack([x.V for x in xs])), k


def _workload(dq):
    """Named results of one pass over the checked kernels (CPU tensors)."""
    out = {}

    def put(name, res):
        for i, t in enumerate(res):
            if isinstance(t, torch.Tensor):
                out[f"{name}.{i}"] = t.detach().cpu()
            elif isinstance(t, (list, tuple)):
                for j, u in enumerate(t):
                    out[f"{name}.{i}.{j}"] = u.detach().cpu()

    for L, beta, k, nb in ((4, 4.0, 10, 3), (8, 2.0, 10, 2), (12, 1.0, 10, 1), (16, 1.0, 10, 1),
                           (18, 0.5, 5, 1)):
        K, dtau, V, k = _batch(L, beta, k, nb, 9000 + L)
        put(f"greens_n{L * L}", dq.greens(K, dtau, V, k, handle=dq.Handle()))
        put(f"greens_seq_n{L * L}", dq.greens(K, dtau, V, k, handle=dq.Handle(fold=0)))
    K, dtau, V, k = _batch(4, 2.0, 5, 2, 9100)
    put("tdisp", dq.greens_tdisplaced(K, dtau, V, k, want_0t=True, handle=dq.Handle()))
    put("tdisp_plain", dq.greens_tdisplaced(K, dtau, V, k, handle=dq.Handle(inversion=1)))
    put("grad", dq.logdet_grad(K, dtau, V, k, handle=dq.Handle()))
    put("jacobi", dq.greens(K, dtau, V, k, handle=dq.Handle(decomposition=1)))
    hg = dq.Handle(graphs=True)
    put("graph0", dq.greens(K, dtau, V, k, handle=hg))
    put("graph1", dq.greens(K, dtau, V, k, handle=hg))
    K8, dtau8, V8, k8 = _batch(8, 2.0, 10, 2, 9200)
    put("mixed", dq.greens(K8, dtau8, V8, k8, handle=dq.Handle(chain_precision=8)))
    put("mixed_tdisp", dq.greens_tdisplaced(K8, dtau8, V8, k8, handle=dq.Handle(chain_precision=8)))
    insts = [di.hubbard_instance(L, 4.0, 0.1, beta, 10, 9300 + i)
             for i, (L, beta) in enumerate(((4, 2.0), (6, 1.5), (4, 3.0)))]
    put("ragged", dq.greens_ragged([(_dev(x.K), x.dtau, _dev(x.V), x.k) for x in insts],
                                   handle=dq.Handle()))
    B, M, N = V.shape
    G = torch.empty((B, N, N), dtype=torch.float64, device="cuda")
    ld = torch.empty(B, dtype=torch.float64, device="cuda")
    sg = torch.empty(B, dtype=torch.int32, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    rc = dq.lib().dqmc_greens_noalloc(C.c_void_p(torch.cuda.current_stream().cuda_stream), B, N,
                                      M, p(K), float(dtau), p(V), int(k), p(G), p(ld), p(sg),
                                      p(st))
    assert rc == 0, rc
    put("noalloc", (G, ld, sg, st))
    torch.cuda.synchronize()
    return out


def _child(path):
    import paper_2003_05286_gb300 as dq
    assert dq.is_debug_build()
    fired, value = dq.selftest_check()
    try:
        out = _workload(dq)
    except RuntimeError:
        print("recorded check failure:", dq.debug_read())
        raise
    torch.save({"out": out, "fired": fired, "value": value, "failure": dq.debug_read(clear=True)},
               path)


def test_debug_build_checks_pass_and_match_release(dq, tmp_path):
    assert not dq.is_debug_build()
    path = str(tmp_path / "debug_out.pt")
    env = dict(os.environ, DQMC_DEBUG="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    code = ("import sys; sys.path.insert(0, %r); import test_gpu_debug_build as t; t._child(%r)"
            % (os.path.dirname(os.path.abspath(__file__)), path))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    res = torch.load(path)
    assert res["fired"] and res["value"] == 63, (res["fired"], res["value"])
    assert res["failure"] is None, res["failure"]
    ref = _workload(dq)
    assert set(ref) == set(res["out"])
    diff = [n for n in ref if not torch.equal(ref[n], res["out"][n])]
    assert not diff, diff


def test_release_library_has_no_checks(dq):
    with pytest.raises(RuntimeError, match="unsupported"):
        dq.debug_read()
    with pytest.raises(RuntimeError, match="unsupported"):
        dq.selftest_check()
