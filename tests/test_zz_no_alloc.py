"""dqmc_greens_noalloc: the allocation-free entry point, called through the C ABI.

It is meant for callers that cannot allocate device memory themselves (a pool
or application that owns the device budget, a plugin bound to its host's
allocator).  Checked here against the regular dqmc_greens entry point on the
same inputs, twice in a row (the fixed scratch array keeps the previous
call's contents), against the CPU oracle on one instance, at the documented
size limit (the largest batch that fits runs, one more is rejected with
DQMC_ERR_SCRATCH), and for the rejection of host buffers with DQMC_ERR_ARG
before anything is launched.  This file is collected last so that a failure
here cannot hide another test's result; it also passes on its own in a fresh
process.
"""
import ctypes as C

import numpy as np
import pytest

import dqmc_inputs as di
from oracle import dqmc as od

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GTOL = 1e-10
LTOL = 1e-9
DQMC_ERR_ARG = 1
DQMC_ERR_SCRATCH = 8
SCRATCH_BYTES = 32 << 20


def _r(x):
    return (x + 255) // 256 * 256


def scratch_bytes(b, N, M, k):
    """Bytes of intermediates of one call, as the header states them."""
    Mp = (-(-M // k) + 1) * k
    return (2 * _r(8 * N * N) + 768 + _r(8 * Mp * N * b) + 9 * _r(8 * N * N * b)
            + _r(16 * N * N * b) + 2 * _r(8 * N * b) + _r(4 * N * b) + _r(8 * b) + 3 * _r(4 * b))


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


def test_noalloc_matches_oracle(dq):
    """The allocation-free call pinned directly against the CPU oracle."""
    lib = dq.lib()
    inst = di.hubbard_instance(6, 4.0, 0.1, 10.0, 10, 4242)
    K, V = _dev(inst.K), _dev(inst.V[None])
    rc, G, ld, sg, st = _noalloc(lib, K, inst.dtau, V, inst.k)
    assert rc == 0 and int(st[0]) == 0
    Go, ldo, so = od.greens(inst.K, inst.dtau, inst.V, inst.k)
    err = np.abs(G[0].cpu().numpy() - Go).max()
    assert err <= GTOL * max(1.0, np.abs(Go).max()), err
    assert abs(float(ld[0]) - ldo) <= LTOL * abs(ldo)
    assert int(sg[0]) == so


@pytest.mark.parametrize("N,M,k,bmax", [(256, 200, 10, 5), (64, 400, 10, 58)])
def test_noalloc_size_limit_boundary(dq, N, M, k, bmax):
    """The batch limits quoted in the header are exact: bmax runs, bmax + 1 is rejected."""
    assert scratch_bytes(bmax, N, M, k) <= SCRATCH_BYTES < scratch_bytes(bmax + 1, N, M, k)
    lib = dq.lib()
    L = int(round(N ** 0.5))
    K = _dev(di.square_hopping(L))
    V = _dev(np.stack([di.hubbard_instance(L, 4.0, 0.1, M * 0.1, k, 77 + i).V
                       for i in range(bmax + 1)]))
    rc, _, _, _, _ = _noalloc(lib, K, 0.1, V[:bmax + 1].contiguous(), k)
    assert rc == DQMC_ERR_SCRATCH
    rc, G, ld, sg, st = _noalloc(lib, K, 0.1, V[:bmax].contiguous(), k)
    assert rc == 0
    assert int((st != 0).sum()) == 0
    Gr, ldr, sgr, _ = dq.greens(K, 0.1, V[:bmax].contiguous(), k)
    assert (G - Gr).abs().max().item() <= GTOL * max(1.0, Gr.abs().max().item())
    assert torch.allclose(ld, ldr, rtol=LTOL, atol=0)


def test_noalloc_rejects_host_pointers(dq):
    """A host buffer for any array argument is an argument error, not a device fault."""
    lib = dq.lib()
    inst = di.hubbard_instance(4, 4.0, 0.1, 2.0, 10, 5)
    N, M = inst.N, inst.M
    Kd, Vd = _dev(inst.K), _dev(inst.V[None])
    Gd = torch.empty((1, N, N), dtype=torch.float64, device="cuda")
    ldd = torch.empty(1, dtype=torch.float64, device="cuda")
    sgd = torch.empty(1, dtype=torch.int32, device="cuda")
    std = torch.empty(1, dtype=torch.int32, device="cuda")
    Kh = np.ascontiguousarray(inst.K)
    Vh = np.ascontiguousarray(inst.V)
    Gh = np.zeros((N, N))
    ldh = np.zeros(1)
    ih = np.zeros(1, dtype=np.int32)
    dp = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    hp = lambda a: C.c_void_p(a.ctypes.data)  # noqa: E731
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    good = [dp(Kd), dp(Vd), dp(Gd), dp(ldd), dp(sgd), dp(std)]
    host = [hp(Kh), hp(Vh), hp(Gh), hp(ldh), hp(ih), hp(ih)]
    for i in range(6):
        args = list(good)
        args[i] = host[i]
        K_, V_, G_, ld_, sg_, st_ = args
        rc = lib.dqmc_greens_noalloc(stream, 1, N, M, K_, 0.1, V_, 10, G_, ld_, sg_, st_)
        assert rc == DQMC_ERR_ARG, (i, rc)
    torch.cuda.synchronize()
    K_, V_, G_, ld_, sg_, st_ = good
    assert lib.dqmc_greens_noalloc(stream, 1, N, M, K_, 0.1, V_, 10, G_, ld_, sg_, st_) == 0
    torch.cuda.synchronize()
    assert int(std[0]) == 0


def test_noalloc_rejects_oversize(dq):
    lib = dq.lib()
    N, M, B = 256, 200, 8                  # ~50 MB of intermediates > 32 MiB
    K = _dev(di.square_hopping(16))
    V = torch.zeros((B, M, N), dtype=torch.float64, device="cuda")
    rc, _, _, _, _ = _noalloc(lib, K, 0.1, V, 10)
    assert rc == DQMC_ERR_SCRATCH
    msg = lib.dqmc_status_string(rc)
    assert b"scratch" in msg
