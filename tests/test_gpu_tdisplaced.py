"""GPU parity of the time-displaced path (dqmc_greens_tdisplaced) against the oracle.

The oracle computes G(tau_j, tau_j) from scratch on the cyclically shifted
chain and G(tau_j, 0) from two independent chains (the inverse chain
B_1^{-1}...B_l^{-1} and the remainder B_M...B_{l+1}) through inv_sum_loh;
the GPU takes both from one forward and one backward stack.  Same tolerance
as the equal-time path: max|dG| <= 1e-10 * max(1, max|G|).
"""
import os

import numpy as np
import pytest

import dqmc_inputs as di
from oracle import dqmc as od
from oracle import exact as ex

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


def _cmp(A, B):
    scale = max(1.0, np.abs(B).max())
    return np.abs(A - B).max() / scale


@pytest.mark.parametrize("L,beta,k,seed", [(2, 3.0, 10, 1), (3, 2.5, 10, 2), (4, 4.0, 10, 3),
                                            (4, 4.0, 7, 4), (6, 6.0, 10, 5)])
def test_tdisplaced_vs_oracle(dq, L, beta, k, seed):
    inst = di.hubbard_instance(L, 4.0, 0.1, beta, k, seed)
    Gtt, Gt0, st = dq.greens_tdisplaced(_dev(inst.K), 0.1, _dev(inst.V), k)
    Gtt, Gt0 = Gtt.cpu().numpy(), Gt0.cpu().numpy()
    Ott, Ot0 = od.greens_tdisplaced(inst.K, 0.1, inst.V, k)
    assert int(st) == 0
    for j in range(Ott.shape[0]):
        assert _cmp(Gtt[j], Ott[j]) <= GTOL, j
        assert _cmp(Gt0[j], Ot0[j]) <= GTOL, j


def test_tdisplaced_identities(dq):
    """G(0,0) = G(beta,beta) = G_1, G(beta,0) = 1 - G_1 (Eq. (etgf_tau), anti-periodicity)."""
    inst = di.hubbard_instance(4, 4.0, 0.1, 6.0, 10, 8)
    K, V = _dev(inst.K), _dev(inst.V)
    Gtt, Gt0, _ = dq.greens_tdisplaced(K, 0.1, V, 10)
    G1 = dq.greens(K, 0.1, V, 10)[0]
    I = torch.eye(16, dtype=torch.float64, device="cuda")
    assert (Gtt[0] - G1).abs().max() <= GTOL
    assert (Gtt[-1] - G1).abs().max() <= GTOL
    assert (Gt0[0] - G1).abs().max() <= GTOL
    assert (Gt0[-1] - (I - G1)).abs().max() <= GTOL


def test_tdisplaced_closed_form_beta40(dq):
    """U = 0, site-independent field, beta = 40: flat accuracy over all tau (Fig. 6)."""
    K = di.chain_hopping(8)
    M = 400
    c = np.random.default_rng(40).uniform(-0.3, 0.3, M)
    V = np.repeat(c[:, None], 8, axis=1)
    Gtt, Gt0, st = dq.greens_tdisplaced(_dev(K), 0.1, _dev(V), 10)
    Gt0 = Gt0.cpu().numpy()
    Gtt = Gtt.cpu().numpy()
    for j, l in enumerate(od.tau_grid(M, 10)):
        Gx = ex.closed_form_displaced(K, 40.0, 0.1 * l, c.sum(), c[:l].sum())
        assert np.abs(Gt0[j] - Gx).max() <= GTOL, (j, np.abs(Gt0[j] - Gx).max())
        Gxx, _ = ex.closed_form_greens(K, 40.0, c.sum())
        assert np.abs(Gtt[j] - Gxx).max() <= GTOL


def test_tdisplaced_brute_force(dq):
    K = di.chain_hopping(4)
    V = 0.8 * di.ising_field(5, 60, 4)
    bf = ex.BruteForce(K, 0.1, V)
    _, Gt0, _ = dq.greens_tdisplaced(_dev(K), 0.1, _dev(V), 10)
    Gt0 = Gt0.cpu().numpy()
    for j, l in enumerate(od.tau_grid(60, 10)):
        assert np.abs(Gt0[j] - bf.to_numpy(bf.displaced(l))).max() <= GTOL


def test_tdisplaced_only_one_output(dq):
    inst = di.hubbard_instance(4, 4.0, 0.1, 3.0, 10, 2)
    K, V = _dev(inst.K), _dev(inst.V)
    Gtt, Gt0, _ = dq.greens_tdisplaced(K, 0.1, V, 10)
    a, _, _ = dq.greens_tdisplaced(K, 0.1, V, 10, want_t0=False)
    _, b, _ = dq.greens_tdisplaced(K, 0.1, V, 10, want_tt=False)
    assert (a - Gtt).abs().max() <= 1e-12 and (b - Gt0).abs().max() <= 1e-12


def test_tdisplaced_full_size_sampled(dq):
    """8x8 lattice, U=4, beta=40 (M=400), k=10, 256 instances in one call;
    instances 0 and 255 checked against the oracle at tau_j for j in {0,10,20,30,40}."""
    insts = [di.batch_n64_tdisplaced(i) for i in range(256)]
    K = _dev(insts[0].K)
    V = _dev(np.stack([x.V for x in insts]))
    Gtt, Gt0, st = dq.greens_tdisplaced(K, 0.1, V, 10)
    assert int((st != 0).sum()) == 0
    assert Gtt.shape == (256, 41, 64, 64)
    for b in (0, 255):
        x = insts[b]
        for j in (0, 10, 20, 30, 40):
            l = min(10 * j, 400)
            Ot0 = od.greens_displaced(x.K, 0.1, x.V, 10, l, 0)
            Ott = od.greens(x.K, 0.1, x.V, 10, l=l + 1)[0]
            assert _cmp(Gt0[b, j].cpu().numpy(), Ot0) <= GTOL, (b, j)
            assert _cmp(Gtt[b, j].cpu().numpy(), Ott) <= GTOL, (b, j)


# ---------------------------------------------------------------------------
# G(0, tau_j): the second case of Eq. (tdgf_propagate) (dqmc_greens_tdisplaced_ex)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,beta,k,seed", [(2, 3.0, 10, 1), (3, 2.5, 10, 2), (4, 4.0, 7, 4),
                                            (6, 6.3, 10, 5)])
def test_g0t_vs_oracle(dq, L, beta, k, seed):
    """G(0, tau_j) on every grid point, incl. a short last chunk (M = 63, k = 10 or 7)."""
    inst = di.hubbard_instance(L, 4.0, 0.1, beta, k, seed)
    K, V = _dev(inst.K), _dev(inst.V)
    Gtt, Gt0, G0t, st = dq.greens_tdisplaced(K, 0.1, V, k, want_0t=True)
    assert int(st) == 0
    # the two existing outputs are the same numbers as without G0t
    a, b, _ = dq.greens_tdisplaced(K, 0.1, V, k)
    assert torch.equal(a, Gtt) and torch.equal(b, Gt0)
    O0t = od.greens_tdisplaced_0t(inst.K, 0.1, inst.V, k)
    G0t = G0t.cpu().numpy()
    assert G0t.shape == O0t.shape
    for j in range(O0t.shape[0]):
        assert _cmp(G0t[j], O0t[j]) <= GTOL, j


def test_g0t_alone_and_ends(dq):
    """G0t without the other outputs (one right-hand side block); G(0,0^+) = -(1 - G_1),
    G(0, beta) = -G_1."""
    inst = di.hubbard_instance(4, 4.0, 0.1, 6.0, 10, 8)
    K, V = _dev(inst.K), _dev(inst.V)
    _, _, G0t, st = dq.greens_tdisplaced(K, 0.1, V, 10, want_tt=False, want_t0=False,
                                         want_0t=True)
    _, _, full, _ = dq.greens_tdisplaced(K, 0.1, V, 10, want_0t=True)
    assert int(st) == 0
    assert (G0t - full).abs().max() <= 1e-12
    G1 = dq.greens(K, 0.1, V, 10)[0]
    I = torch.eye(16, dtype=torch.float64, device="cuda")
    assert (G0t[0] + (I - G1)).abs().max() <= GTOL
    assert (G0t[-1] + G1).abs().max() <= GTOL


def test_g0t_closed_form_beta40(dq):
    """U = 0, site-independent field, beta = 40: -(1 - G_1) B(tau,0)^{-1} at every tau."""
    K = di.chain_hopping(8)
    M = 400
    c = np.random.default_rng(41).uniform(-0.3, 0.3, M)
    V = np.repeat(c[:, None], 8, axis=1)
    _, _, G0t, st = dq.greens_tdisplaced(_dev(K), 0.1, _dev(V), 10, want_tt=False,
                                         want_t0=False, want_0t=True)
    G0t = G0t.cpu().numpy()
    for j, l in enumerate(od.tau_grid(M, 10)):
        Gx = ex.closed_form_displaced_back(K, 40.0, 0.1 * l, c.sum(), c[:l].sum())
        assert np.abs(G0t[j] - Gx).max() <= GTOL, (j, np.abs(G0t[j] - Gx).max())


def test_g0t_brute_force(dq):
    K = di.chain_hopping(4)
    V = 0.8 * di.ising_field(6, 60, 4)
    bf = ex.BruteForce(K, 0.1, V)
    _, _, G0t, _ = dq.greens_tdisplaced(_dev(K), 0.1, _dev(V), 10, want_0t=True)
    G0t = G0t.cpu().numpy()
    for j, l in enumerate(od.tau_grid(60, 10)):
        assert np.abs(G0t[j] - bf.to_numpy(bf.displaced_back(0, l))).max() <= GTOL


def test_g0t_full_size(dq):
    """8x8 lattice, U=4, beta=40, k=10, 256 instances in one call.  Every tau_j of
    every instance: the particle-hole link G_{-V}(tau,0) = -Lambda G_V(0,tau)^T Lambda
    between two calls; instances 0 and 255 against the oracle at four tau_j.

    The link holds to 1e-10 * max(1, max|G|) except on ill-conditioned fields
    (|G(tau,0)| up to ~1e4), where any FP64 route, the oracle's included, resolves
    G only to about eps * cond(mid) (mid: the middle matrix of Eq.
    (inversion_tdgf_loh), cond ~ 1e6 there).  At those points the link, a sum of
    two such errors, must stay below 16 * eps * cond(mid)."""
    insts = [di.batch_n64_tdisplaced(i) for i in range(256)]
    K = _dev(insts[0].K)
    V = _dev(np.stack([x.V for x in insts]))
    _, _, G0t, st = dq.greens_tdisplaced(K, 0.1, V, 10, want_tt=False, want_t0=False,
                                         want_0t=True)
    assert int((st != 0).sum()) == 0 and G0t.shape == (256, 41, 64, 64)
    _, Gt0m, st2 = dq.greens_tdisplaced(K, 0.1, -V, 10, want_tt=False)
    assert int((st2 != 0).sum()) == 0
    lam = torch.tensor([(-1.0) ** (x + y) for y in range(8) for x in range(8)],
                       dtype=torch.float64, device="cuda")
    link = Gt0m + lam[:, None] * G0t.transpose(-1, -2) * lam[None, :]
    scale = torch.clamp(Gt0m.abs().amax(dim=(-1, -2)), min=1.0)
    r = (link.abs().amax(dim=(-1, -2)) / scale).cpu().numpy()
    over = np.argwhere(r > GTOL)
    assert len(over) <= 64, len(over)
    eps = np.finfo(np.float64).eps
    for b, j in over:
        x = insts[b]
        l = min(10 * int(j), 400)
        kappa = od.displaced_condition(x.K, 0.1, -x.V, 10, l, 0)
        assert r[b, j] <= 16.0 * eps * kappa, (int(b), int(j), r[b, j], kappa)
    for b in (0, 255):
        x = insts[b]
        for j in (0, 13, 20, 40):
            l = min(10 * j, 400)
            O = od.greens_displaced_back(x.K, 0.1, x.V, 10, 0, l)
            assert _cmp(G0t[b, j].cpu().numpy(), O) <= GTOL, (b, j)


def test_g_tau0_ill_conditioned_vs_mpmath(dq):
    """Instance 229 of the same batch, the ill-conditioned field: the library's
    G(tau,0) at tau = 1, 5, 8 against stored mpmath values at 397 digits
    (tests/golden/make_golden.py n64), within 16 * eps * cond(mid) of max|G|
    (cond(mid) from the oracle, 7e5 to 4e6 here), the accuracy any FP64 route
    of Eq. (inversion_tdgf_loh) has on this field.  The bf16x8 chain is held to
    four times that factor: its slice products are accurate to N 2^-57 of
    (row max x column max), i.e. 2 eps normwise at N = 64, where an FP64
    product has eps / 2 per operation elementwise."""
    path = os.path.join(os.path.dirname(__file__), "golden", "batch_n64_229_displaced_mpmath.txt")
    gold, cur = {}, None
    for ln in open(path):
        if ln.startswith("#"):
            continue
        parts = ln.split()
        if len(parts) == 2:
            cur = int(parts[1])
            gold[cur] = []
        else:
            gold[cur].append(float(parts[0]))
    assert sorted(gold) == [10, 50, 80]
    x = di.batch_n64_tdisplaced(229)
    eps = np.finfo(np.float64).eps
    for prec, factor in ((0, 16.0), (8, 64.0)):
        h = dq.Handle(chain_precision=prec)
        _, Gt0, st = dq.greens_tdisplaced(_dev(x.K), x.dtau, _dev(x.V), x.k, want_tt=False,
                                          handle=h)
        assert int(st) == 0
        for l, vals in gold.items():
            Gx = np.array(vals).reshape(64, 64)
            kappa = od.displaced_condition(x.K, x.dtau, x.V, x.k, l, 0)
            err = _cmp(Gt0[l // x.k].cpu().numpy(), Gx)
            assert err <= factor * eps * kappa, (prec, l, err, kappa)


# ---------------------------------------------------------------------------
# every tau_l = l dtau (dqmc_greens_tdisplaced_all)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L,beta,k,seed", [(3, 2.3, 5, 1), (4, 4.0, 10, 2), (2, 3.7, 7, 3)])
def test_all_tau_vs_oracle(dq, L, beta, k, seed):
    """All three functions at every l (short last chunks included); grid values
    bitwise equal to the k-grid call."""
    inst = di.hubbard_instance(L, 4.0, 0.1, beta, k, seed)
    K, V = _dev(inst.K), _dev(inst.V)
    Att, At0, A0t, st = dq.greens_tdisplaced_all(K, 0.1, V, k)
    assert int(st) == 0 and Att.shape == (inst.M + 1, inst.N, inst.N)
    Gtt, Gt0, G0t, _ = dq.greens_tdisplaced(K, 0.1, V, k, want_0t=True)
    for j, l in enumerate(od.tau_grid(inst.M, k)):
        assert torch.equal(Att[l], Gtt[j]) and torch.equal(At0[l], Gt0[j]) and torch.equal(A0t[l], G0t[j])
    Att, At0, A0t = (x.cpu().numpy() for x in (Att, At0, A0t))
    for l in range(inst.M + 1):
        Ott = od.greens(inst.K, 0.1, inst.V, k, l=l + 1)[0]
        Ot0 = od.greens_displaced(inst.K, 0.1, inst.V, k, l, 0)
        O0t = od.greens_displaced_back(inst.K, 0.1, inst.V, k, 0, l)
        assert _cmp(Att[l], Ott) <= GTOL, ("tt", l)
        assert _cmp(At0[l], Ot0) <= GTOL, ("t0", l)
        assert _cmp(A0t[l], O0t) <= GTOL, ("0t", l)


def test_all_tau_full_size_sampled(dq):
    """8x8, U=4, beta=40, k=10, 256 instances: G(tau_l, 0) and G(0, tau_l) at every
    l = 0..400; instances 0 and 255 against the oracle at off-grid l."""
    insts = [di.batch_n64_tdisplaced(i) for i in range(256)]
    K = _dev(insts[0].K)
    V = _dev(np.stack([x.V for x in insts]))
    _, At0, A0t, st = dq.greens_tdisplaced_all(K, 0.1, V, 10, want_tt=False)
    assert int((st != 0).sum()) == 0 and At0.shape == (256, 401, 64, 64)
    for b in (0, 255):
        x = insts[b]
        for l in (1, 9, 137, 255, 399):
            assert _cmp(At0[b, l].cpu().numpy(), od.greens_displaced(x.K, 0.1, x.V, 10, l, 0)) <= GTOL
            assert _cmp(A0t[b, l].cpu().numpy(), od.greens_displaced_back(x.K, 0.1, x.V, 10, 0, l)) <= GTOL


# ---------------------------------------------------------------------------
# G(tau_1, tau_2) for every pair of grid times (dqmc_greens_tdisplaced_from)
# ---------------------------------------------------------------------------

def _pair_refs(inst, k, l0, l1):
    """Oracle G(tau_1,tau_1), G(tau_1,tau_0), G(tau_0,tau_1) for tau_1 = l1 dtau >= tau_0,
    continued anti-periodically past beta (G(tau + beta, tau') = -G(tau, tau'))."""
    M = inst.M
    Gtt = od.greens(inst.K, 0.1, inst.V, k, l=l1 % M + 1)[0]
    if l1 <= M:
        return (Gtt, od.greens_displaced(inst.K, 0.1, inst.V, k, l1, l0),
                od.greens_displaced_back(inst.K, 0.1, inst.V, k, l0, l1))
    return (Gtt, -od.greens_displaced_back(inst.K, 0.1, inst.V, k, l1 - M, l0),
            -od.greens_displaced(inst.K, 0.1, inst.V, k, l0, l1 - M))


@pytest.mark.parametrize("every_tau", [False, True])
def test_from_every_grid_pair(dq, every_tau):
    """3x3 lattice, beta = 3 (M = 30), k = 10: origins on the grid and off it (7);
    one call for all origins; origin 0 equals dqmc_greens_tdisplaced_ex bitwise."""
    inst = di.hubbard_instance(3, 4.0, 0.1, 3.0, 10, 9)
    M = inst.M
    origins = [0, 7, 10, 20]
    K = _dev(inst.K)
    V = _dev(np.stack([inst.V] * len(origins)))
    Att, At0, A0t, st = dq.greens_tdisplaced_from(K, 0.1, V, 10, origins, every_tau=every_tau)
    assert int((st != 0).sum()) == 0
    offs = list(range(M + 1)) if every_tau else od.tau_grid(M, 10)
    for b, l0 in enumerate(origins):
        for j, d in enumerate(offs):
            if every_tau and d % 3:
                continue
            rtt, rt0, r0t = _pair_refs(inst, 10, l0, l0 + d)
            assert _cmp(Att[b, j].cpu().numpy(), rtt) <= GTOL, ("tt", l0, d)
            assert _cmp(At0[b, j].cpu().numpy(), rt0) <= GTOL, ("t0", l0, d)
            assert _cmp(A0t[b, j].cpu().numpy(), r0t) <= GTOL, ("0t", l0, d)
    if not every_tau:
        a, b_, c, _ = dq.greens_tdisplaced(K, 0.1, V[0], 10, want_0t=True)
        assert torch.equal(Att[0], a) and torch.equal(At0[0], b_) and torch.equal(A0t[0], c)


def test_from_rejects_missing_origins(dq):
    inst = di.hubbard_instance(2, 4.0, 0.1, 2.0, 10, 1)
    with pytest.raises(ValueError):
        dq.greens_tdisplaced_from(_dev(inst.K), 0.1, _dev(inst.V[None]), 10, [0, 1])


def test_displaced_n16_against_mpmath(dq):
    """The 4x4, U=4, beta=8, k=10 workload: G(tau_l, 0) and G(0, tau_l) at l = 10, 40, 70
    (grid points j = 1, 4, 7) against the stored mpmath values."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "single_n16_displaced_mpmath.txt")
    gold, cur = {}, None
    for ln in open(path):
        if ln.startswith("#"):
            continue
        parts = ln.split()
        if len(parts) == 2:
            cur = (parts[0], int(parts[1]))
            gold[cur] = []
        else:
            gold[cur].append(float(parts[0]))
    inst = di.single_n16()
    _, Gt0, G0t, st = dq.greens_tdisplaced(_dev(inst.K), inst.dtau, _dev(inst.V), inst.k,
                                           want_tt=False, want_0t=True)
    assert int(st) == 0
    for (name, l), vals in gold.items():
        Gx = np.array(vals).reshape(16, 16)
        A = (Gt0 if name == "t0" else G0t)[l // inst.k].cpu().numpy()
        assert _cmp(A, Gx) <= GTOL, (name, l)
