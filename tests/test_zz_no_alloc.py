"""dqmc_greens_noalloc: the allocation-free entry point, called through the C ABI.

It is meant for callers that cannot allocate device memory themselves (a pool
or application that owns the device budget, a plugin bound to its host's
allocator).  Checked here against the regular dqmc_greens entry point on the
same inputs, twice in a row (the fixed scratch array keeps the previous
call's contents), and for the clear rejection of a problem larger than the
scratch.  This file is collected last so that a failure here cannot hide
another test's result; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import dqmc_inputs as di

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GTOL = 1e-10
DQMC_ERR_SCRATCH = 8


@pytest.fixture(scope="module")
def dq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_05286_gb300 as m
    m.lib()
    return m


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _noalloc(lib, K, dtau, V, k):
    B, M, N = V.shape
    G = torch.empty((B, N, N), dtype=torch.float64, device="cuda")
    ld = torch.empty(B, dtype=torch.float64, device="cuda")
    sg = torch.empty(B, dtype=torch.int32, device="cuda")
    st = torch.full((B,), 12345, dtype=torch.int32, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.dqmc_greens_noalloc(stream, B, N, M, p(K), float(dtau), p(V), int(k), p(G), p(ld),
                                 p(sg), p(st))
    torch.cuda.synchronize()
    return rc, G, ld, sg, st


def test_noalloc_matches_greens_twice(dq):
    lib = dq.lib()
    insts = [di.hubbard_instance(8, 4.0, 0.1, 12.0, 10, 300 + i) for i in range(4)]
    K = _dev(insts[0].K)
    V = _dev(np.stack([x.V for x in insts]))
    Gr, ldr, sgr, str_ = dq.greens(K, 0.1, V, 10)
    for _ in range(2):
        rc, G, ld, sg, st = _noalloc(lib, K, 0.1, V, 10)
        assert rc == 0
        assert (G - Gr).abs().max().item() <= GTOL * max(1.0, Gr.abs().max().item())
        assert torch.allclose(ld, ldr, rtol=1e-9, atol=0)
        assert torch.equal(sg, sgr)
        assert int((st != 0).sum()) == 0          # status cleared by the call itself
    # a different problem in the same scratch right after
    inst = di.hubbard_instance(4, 4.0, 0.1, 5.0, 7, 99)
    K2, V2 = _dev(inst.K), _dev(inst.V[None])
    rc, G, ld, sg, st = _noalloc(lib, K2, 0.1, V2, 7)
    Gr2, ldr2, _, _ = dq.greens(K2, 0.1, V2, 7)
    assert rc == 0
    assert (G - Gr2).abs().max().item() <= GTOL * max(1.0, Gr2.abs().max().item())
    assert abs(float(ld[0]) - float(ldr2[0])) <= 1e-9 * abs(float(ldr2[0]))


def test_noalloc_rejects_oversize(dq):
    lib = dq.lib()
    N, M, B = 256, 200, 8                  # ~50 MB of intermediates > 32 MiB
    K = _dev(di.square_hopping(16))
    V = torch.zeros((B, M, N), dtype=torch.float64, device="cuda")
    rc, _, _, _, _ = _noalloc(lib, K, 0.1, V, 10)
    assert rc == DQMC_ERR_SCRATCH
    msg = lib.dqmc_status_string(rc)
    assert b"scratch" in msg
