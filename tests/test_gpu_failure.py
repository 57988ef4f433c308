"""Bounded device-side waits: a wait that runs out reports a status, the context survives.

The only device-side waits are the mbarrier waits of the tensor-core slice
product.  dqmc_selftest_wait_timeout launches one CTA of it with its operand
loads switched off, so nothing ever arrives on the first stage: the wait must
give up (about 2 s), set DQMC_STATUS_TIMEOUT, drain and free its tensor memory.
No fault, trap or unbounded wait is involved.  Afterwards the same process
must still compute a correct Green's function on the tensor cores.
"""
import numpy as np
import pytest

import dqmc_inputs as di
from oracle import dqmc as od

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_05286_gb300 as m
    m.lib()
    return m


def test_bounded_wait_reports_timeout_and_context_survives(dq):
    from paper_2003_05286_gb300 import _abi
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    dq.selftest_wait_timeout(st)
    torch.cuda.synchronize()
    assert int(st.item()) & _abi.STATUS_BITS["TIMEOUT"]
    # the context is still usable: a mixed-precision G afterwards matches the oracle
    inst = di.hubbard_instance(4, 4.0, 0.1, 4.0, 10, 21)
    h = dq.Handle(chain_precision=8)
    G, ld, sg, s2 = dq.greens(torch.tensor(inst.K, device="cuda"), 0.1,
                              torch.tensor(inst.V, device="cuda"), 10, handle=h)
    Go, ldo, so = od.greens(inst.K, 0.1, inst.V, 10)
    assert int(s2) == 0
    assert np.abs(G.cpu().numpy() - Go).max() <= 1e-8 * max(1.0, np.abs(Go).max())
    h.close()


def test_selftest_rejects_null_status(dq):
    rc = dq.lib().dqmc_selftest_wait_timeout(None, None)
    assert rc == 1   # DQMC_ERR_ARG
