"""GB300 library for stabilised DQMC Green's functions (Bauer, SciPost 2020).

A thin PyTorch binding over the C ABI of ``include/dqmc.h``: torch supplies
device memory and the current CUDA stream; every step of the computation runs
in the library's CUDA kernels.  There is no CPU fallback: if the shared
library is missing or no GPU is present the calls raise.

Shapes (row-major, float64):
    K  (N, N)         symmetric hopping matrix, B_l = exp(-dtau K) exp(V_l)
    V  (B, M, N)      V[b, l-1] = diagonal of V_l  (a 2-D (M, N) V means B = 1)
    G  (B, N, N)      G[b, i, j] = G_ij
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _abi

__all__ = ["Handle", "greens", "logdet", "greens_tdisplaced", "greens_tdisplaced_all",
           "greens_tdisplaced_from",
           "logdet_grad", "greens_ragged", "RaggedBatch", "Batched",
           "greens_tdisplaced_ragged", "logdet_grad_ragged", "selftest_wait_timeout",
           "selftest_fp64_rate", "LogDet", "is_debug_build", "debug_read", "selftest_check",
           "n_tau", "lib"]


def lib():
    return _abi.load()


def n_tau(M: int, k: int) -> int:
    """Number of points tau_j = min(j k, M) dtau of the k-grid."""
    return -(-M // k) + 1


class Handle:
    """Owns a dqmc_handle (workspace + settings) bound to the current device."""

    def __init__(self, chain_precision: int = _abi.CHAIN_FP64, graphs: bool = False,
                 fold: int = _abi.FOLD_AUTO, inversion: int = _abi.INV_LOH,
                 decomposition: int = _abi.DECOMP_QR):
        self._lib = lib()
        h = C.c_void_p()
        _abi.check(self._lib.dqmc_create(C.byref(h)), "dqmc_create")
        self.h = h
        if chain_precision != _abi.CHAIN_FP64:
            _abi.check(self._lib.dqmc_set_chain_precision(self.h, chain_precision),
                       "dqmc_set_chain_precision")
        if graphs:
            self.set_graph_mode(True)
        if fold != _abi.FOLD_AUTO:
            self.set_chain_fold(fold)
        if inversion != _abi.INV_LOH:
            self.set_inversion_scheme(inversion)
        if decomposition != _abi.DECOMP_QR:
            self.set_decomposition(decomposition)

    def register_K(self, K: torch.Tensor, dtau: float) -> int:
        """Registers a hopping matrix (dqmc_register_K): exp(-dtau K) is computed
        once and kept in the handle; returns the id for dqmc_desc.K_id."""
        if not (K.is_cuda and K.dtype == torch.float64 and K.dim() == 2 and K.shape[0] == K.shape[1]):
            raise ValueError("K must be a square CUDA float64 tensor")
        K = K.contiguous()
        kid = C.c_int(-1)
        self.bind_stream()
        _abi.check(self._lib.dqmc_register_K(self.h, K.shape[0], _ptr(K), float(dtau), C.byref(kid)),
                   "dqmc_register_K")
        self._kN = getattr(self, "_kN", [])
        self._kN.append(int(K.shape[0]))
        return kid.value

    def set_decomposition(self, decomposition: int):
        """Chain stabiliser: DECOMP_QR (pivoted QR, default) or DECOMP_JACOBI (one-sided SVD)."""
        _abi.check(self._lib.dqmc_set_decomposition(self.h, int(decomposition)),
                   "dqmc_set_decomposition")

    def set_inversion_scheme(self, scheme: int):
        """INV_LOH (D+/D- split, default) or INV_PLAIN (Eq. (inversion) / Eq. (inversion_tdgf))."""
        _abi.check(self._lib.dqmc_set_inversion_scheme(self.h, int(scheme)),
                   "dqmc_set_inversion_scheme")

    def set_chain_fold(self, mode: int):
        """Equal-time chain: FOLD_SEQUENTIAL, FOLD_TREE (pairwise Eq. (stabmult)) or FOLD_AUTO."""
        _abi.check(self._lib.dqmc_set_chain_fold(self.h, int(mode)), "dqmc_set_chain_fold")

    def set_graph_mode(self, enable: bool):
        """Record calls as CUDA graphs and replay them for identical arguments."""
        _abi.check(self._lib.dqmc_set_graph_mode(self.h, int(enable)), "dqmc_set_graph_mode")

    def close(self):
        if getattr(self, "h", None):
            self._lib.dqmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bind_stream(self, stream: torch.cuda.Stream | None = None):
        s = stream if stream is not None else torch.cuda.current_stream()
        _abi.check(self._lib.dqmc_set_stream(self.h, C.c_void_p(s.cuda_stream)), "dqmc_set_stream")

    def set_gemm_tile(self, tile: int):
        _abi.check(self._lib.dqmc_set_gemm_tile(self.h, int(tile)), "dqmc_set_gemm_tile")

    def set_pointer_mode(self, host: bool):
        _abi.check(self._lib.dqmc_set_pointer_mode(self.h, _abi.PTR_HOST if host else _abi.PTR_DEVICE),
                   "dqmc_set_pointer_mode")

    # kernel classes of the event profiler
    PROF_CHAIN, PROF_QRP, PROF_XUPD, PROF_LU, PROF_OTHER = range(5)

    def profile(self, enable: bool = True):
        _abi.check(self._lib.dqmc_profile_enable(self.h, int(enable)), "dqmc_profile_enable")

    def profile_reset(self):
        _abi.check(self._lib.dqmc_profile_reset(self.h), "dqmc_profile_reset")

    def profile_read(self, cls: int):
        """(event ms, launches, algorithmic FP64 flops) of one kernel class since the reset."""
        ms = C.c_double()
        n = C.c_longlong()
        fl = C.c_double()
        _abi.check(self._lib.dqmc_profile_read(self.h, cls, C.byref(ms), C.byref(n), C.byref(fl)),
                   "dqmc_profile_read")
        return ms.value, n.value, fl.value

    @property
    def last_launch_count(self) -> int:
        return int(self._lib.dqmc_last_launch_count(self.h))

    @property
    def workspace_bytes(self) -> int:
        return int(self._lib.dqmc_workspace_bytes(self.h))

    @property
    def device_bytes(self) -> int:
        """Device bytes held by all grow-only buffers of the handle."""
        return int(self._lib.dqmc_device_bytes(self.h))

    def set_memory_limit(self, nbytes: int):
        """Caps device_bytes (0: no cap); growth past it raises RuntimeError (NOMEM)."""
        _abi.check(self._lib.dqmc_set_memory_limit(self.h, int(nbytes)), "dqmc_set_memory_limit")


_default: dict[int, Handle] = {}


def _handle(h: Handle | None) -> Handle:
    if h is not None:
        h.bind_stream()
        return h
    dev = torch.cuda.current_device()
    if dev not in _default:
        _default[dev] = Handle()
    _default[dev].bind_stream()
    return _default[dev]


def _ptr(t: torch.Tensor | None):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _prep(K: torch.Tensor, V: torch.Tensor):
    if not (K.is_cuda and V.is_cuda):
        raise ValueError("K and V must be CUDA tensors (the library has no CPU path)")
    if K.dtype != torch.float64 or V.dtype != torch.float64:
        raise ValueError("K and V must be float64")
    K = K.contiguous()
    squeeze = V.dim() == 2
    V = (V.unsqueeze(0) if squeeze else V).contiguous()
    if V.dim() != 3 or K.dim() != 2 or K.shape[0] != K.shape[1] or V.shape[2] != K.shape[0]:
        raise ValueError(f"bad shapes K {tuple(K.shape)} V {tuple(V.shape)}")
    return K, V, squeeze


def greens(K, dtau: float, V, k: int, *, handle: Handle | None = None, want_G: bool = True):
    """Equal-time G = [1 + B_M...B_1]^{-1}, log|det(1 + B_M...B_1)|, sign, status."""
    K, V, sq = _prep(K, V)
    B, M, N = V.shape
    h = _handle(handle)
    G = torch.empty((B, N, N), dtype=torch.float64, device=V.device) if want_G else None
    ld = torch.empty(B, dtype=torch.float64, device=V.device)
    sg = torch.empty(B, dtype=torch.int32, device=V.device)
    st = torch.empty(B, dtype=torch.int32, device=V.device)
    rc = h._lib.dqmc_greens(h.h, B, N, M, _ptr(K), float(dtau), _ptr(V), int(k), _ptr(G),
                            _ptr(ld), _ptr(sg), _ptr(st))
    _abi.check(rc, "dqmc_greens")
    if sq:
        return (G[0] if G is not None else None), ld[0], sg[0], st[0]
    return G, ld, sg, st


def logdet(K, dtau: float, V, k: int, *, handle: Handle | None = None):
    """log|det(1 + B_M...B_1)|, sign, status."""
    K, V, sq = _prep(K, V)
    B, M, N = V.shape
    h = _handle(handle)
    ld = torch.empty(B, dtype=torch.float64, device=V.device)
    sg = torch.empty(B, dtype=torch.int32, device=V.device)
    st = torch.empty(B, dtype=torch.int32, device=V.device)
    _abi.check(h._lib.dqmc_logdet(h.h, B, N, M, _ptr(K), float(dtau), _ptr(V), int(k), _ptr(ld),
                                  _ptr(sg), _ptr(st)), "dqmc_logdet")
    if sq:
        return ld[0], sg[0], st[0]
    return ld, sg, st


def greens_tdisplaced(K, dtau: float, V, k: int, *, handle: Handle | None = None,
                      want_tt: bool = True, want_t0: bool = True, want_0t: bool = False):
    """G(tau_j, tau_j) and G(tau_j, 0) on the k-grid: tensors (B, n_tau, N, N) and status.

    With ``want_0t`` also G(0, tau_j) (dqmc_greens_tdisplaced_ex), returned
    after Gt0: (Gtt, Gt0, G0t, status)."""
    K, V, sq = _prep(K, V)
    B, M, N = V.shape
    nt = n_tau(M, k)
    h = _handle(handle)

    def out(want):
        return torch.empty((B, nt, N, N), dtype=torch.float64, device=V.device) if want else None
    Gtt, Gt0, G0t = out(want_tt), out(want_t0), out(want_0t)
    st = torch.empty(B, dtype=torch.int32, device=V.device)
    if want_0t:
        _abi.check(h._lib.dqmc_greens_tdisplaced_ex(h.h, B, N, M, _ptr(K), float(dtau), _ptr(V),
                                                    int(k), _ptr(Gtt), _ptr(Gt0), _ptr(G0t),
                                                    _ptr(st)), "dqmc_greens_tdisplaced_ex")
        res = (Gtt, Gt0, G0t)
    else:
        _abi.check(h._lib.dqmc_greens_tdisplaced(h.h, B, N, M, _ptr(K), float(dtau), _ptr(V),
                                                 int(k), _ptr(Gtt), _ptr(Gt0), _ptr(st)),
                   "dqmc_greens_tdisplaced")
        res = (Gtt, Gt0)
    if sq:
        return tuple(x[0] if x is not None else None for x in res) + (st[0],)
    return res + (st,)


def greens_tdisplaced_all(K, dtau: float, V, k: int, *, handle: Handle | None = None,
                          want_tt: bool = True, want_t0: bool = True, want_0t: bool = True):
    """G(tau_l, tau_l), G(tau_l, 0), G(0, tau_l) for every l = 0..M (dqmc_greens_tdisplaced_all):
    tensors (B, M+1, N, N) (None where not wanted) and status."""
    K, V, sq = _prep(K, V)
    B, M, N = V.shape
    h = _handle(handle)

    def out(want):
        return torch.empty((B, M + 1, N, N), dtype=torch.float64, device=V.device) if want else None
    Gtt, Gt0, G0t = out(want_tt), out(want_t0), out(want_0t)
    st = torch.empty(B, dtype=torch.int32, device=V.device)
    _abi.check(h._lib.dqmc_greens_tdisplaced_all(h.h, B, N, M, _ptr(K), float(dtau), _ptr(V),
                                                 int(k), _ptr(Gtt), _ptr(Gt0), _ptr(G0t),
                                                 _ptr(st)), "dqmc_greens_tdisplaced_all")
    res = (Gtt, Gt0, G0t)
    if sq:
        return tuple(x[0] if x is not None else None for x in res) + (st[0],)
    return res + (st,)


def greens_tdisplaced_from(K, dtau: float, V, k: int, l0, *, every_tau: bool = False,
                           handle: Handle | None = None, want_tt: bool = True,
                           want_t0: bool = True, want_0t: bool = True):
    """G(tau_l0 + d, tau_l0 + d), G(tau_l0 + d, tau_l0) and G(tau_l0, tau_l0 + d) from the
    origin tau_l0 of each instance (dqmc_greens_tdisplaced_from), d on the k-grid or at
    every slice; l0 an int sequence or tensor of length B.  Times past beta continue
    anti-periodically.  Returns tensors (B, n_tau or M+1, N, N) (None where not wanted)
    and status."""
    K, V, sq = _prep(K, V)
    B, M, N = V.shape
    h = _handle(handle)
    l0 = torch.as_tensor(l0, dtype=torch.int32, device=V.device).reshape(-1).contiguous()
    if l0.numel() != B:
        raise ValueError(f"l0 has {l0.numel()} entries for {B} instances")
    nt = M + 1 if every_tau else n_tau(M, k)

    def out(want):
        return torch.empty((B, nt, N, N), dtype=torch.float64, device=V.device) if want else None
    Gtt, Gt0, G0t = out(want_tt), out(want_t0), out(want_0t)
    st = torch.empty(B, dtype=torch.int32, device=V.device)
    _abi.check(h._lib.dqmc_greens_tdisplaced_from(h.h, B, N, M, _ptr(K), float(dtau), _ptr(V),
                                                  int(k), _ptr(l0), int(every_tau), _ptr(Gtt),
                                                  _ptr(Gt0), _ptr(G0t), _ptr(st)),
               "dqmc_greens_tdisplaced_from")
    res = (Gtt, Gt0, G0t)
    if sq:
        return tuple(x[0] if x is not None else None for x in res) + (st[0],)
    return res + (st,)


def logdet_grad(K, dtau: float, V, k: int, *, handle: Handle | None = None):
    """log|det(1 + B_M...B_1)|, sign, dV = d logdet / dV (same shape as V), status."""
    K, V, sq = _prep(K, V)
    B, M, N = V.shape
    h = _handle(handle)
    ld = torch.empty(B, dtype=torch.float64, device=V.device)
    sg = torch.empty(B, dtype=torch.int32, device=V.device)
    dV = torch.empty((B, M, N), dtype=torch.float64, device=V.device)
    st = torch.empty(B, dtype=torch.int32, device=V.device)
    _abi.check(h._lib.dqmc_logdet_grad(h.h, B, N, M, _ptr(K), float(dtau), _ptr(V), int(k),
                                       _ptr(ld), _ptr(sg), _ptr(dV), _ptr(st)), "dqmc_logdet_grad")
    if sq:
        return ld[0], sg[0], dV[0], st[0]
    return ld, sg, dV, st


class RaggedBatch:
    """A ragged batch packed once into device pools (dqmc_greens_ragged).

    ``instances``: list of (K, dtau, V, k) with CUDA float64 K (N,N), V (M,N).
    Instances that pass the same K tensor share one copy of it in the K pool,
    which lets the library batch them (groups are keyed by N, k, dtau, K).
    ``run`` calls the library on the same pools and outputs every time, so in
    CUDA-graph mode a second ``run`` is a single graph launch; ``set_fields``
    writes new fields into the V pool in place."""

    def __init__(self, instances, device=None):
        device = device or instances[0][0].device
        self.descs = (_abi.DqmcInstance * len(instances))()
        offK = offV = offG = 0
        Ks, Vs = [], []
        seenK = {}
        for i, (K, dtau, V, k) in enumerate(instances):
            N = K.shape[0]
            M = V.shape[0]
            key = (K.data_ptr(), tuple(K.shape), tuple(K.stride()))
            if key not in seenK:
                seenK[key] = offK
                Ks.append(K.reshape(-1))
                offK += N * N
            self.descs[i] = _abi.DqmcInstance(N, M, int(k), 0, float(dtau), seenK[key], offV, offG)
            Vs.append(V.reshape(-1))
            offV += M * N
            offG += N * N
        self.K = torch.cat(Ks).to(device=device, dtype=torch.float64).contiguous()
        self.V = torch.cat(Vs).to(device=device, dtype=torch.float64).contiguous()
        self.Gp = torch.empty(offG, dtype=torch.float64, device=device)
        B = len(instances)
        self.ld = torch.empty(B, dtype=torch.float64, device=device)
        self.sg = torch.empty(B, dtype=torch.int32, device=device)
        self.st = torch.empty(B, dtype=torch.int32, device=device)
        self.Gs = [self.Gp[d.off_G: d.off_G + d.N * d.N].view(d.N, d.N) for d in self.descs]

    def __len__(self):
        return len(self.descs)

    def set_fields(self, fields):
        """Copy new fields (list of (M, N) tensors, same shapes) into the V pool."""
        for d, V in zip(self.descs, fields):
            self.V[d.off_V: d.off_V + d.M * d.N].copy_(V.reshape(-1))

    def run(self, handle: Handle | None = None):
        """(list of G views into the output pool, logdet, sign, status)."""
        h = _handle(handle)
        _abi.check(h._lib.dqmc_greens_ragged(h.h, len(self.descs), self.descs, _ptr(self.K),
                                             _ptr(self.V), _ptr(self.Gp), _ptr(self.ld),
                                             _ptr(self.sg), _ptr(self.st)), "dqmc_greens_ragged")
        return self.Gs, self.ld, self.sg, self.st


class Batched:
    """Instances over hopping matrices registered on ``handle`` (dqmc_greens_batched).

    ``items``: list of (K_id, V (M, N) CUDA float64, k).  The dqmc_desc array is
    built once and kept on the device together with the V pool and the
    outputs; ``run`` calls the library on them (a single graph launch on a
    repeated call in graph mode)."""

    def __init__(self, handle: Handle, items):
        kN = getattr(handle, "_kN", [])
        descs = (_abi.DqmcDesc * len(items))()
        offV = offG = 0
        Vs = []
        for i, (kid, V, k) in enumerate(items):
            if not 0 <= kid < len(kN):
                raise ValueError(f"K_id {kid} is not registered on this handle")
            N = kN[kid]
            M = V.shape[0]
            if V.dim() != 2 or V.shape[1] != N:
                raise ValueError(f"field of instance {i} has shape {tuple(V.shape)}, N = {N}")
            descs[i] = _abi.DqmcDesc(N, M, int(k), int(kid), offV, offG)
            Vs.append(V.reshape(-1))
            offV += M * N
            offG += N * N
        dev = Vs[0].device
        raw = bytes(C.string_at(C.addressof(descs), C.sizeof(descs)))
        self.desc = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(dev)
        self.handle = handle
        self.V = torch.cat(Vs).to(dtype=torch.float64).contiguous()
        self.Gp = torch.empty(offG, dtype=torch.float64, device=dev)
        B = len(items)
        self.ld = torch.empty(B, dtype=torch.float64, device=dev)
        self.sg = torch.empty(B, dtype=torch.int32, device=dev)
        self.st = torch.empty(B, dtype=torch.int32, device=dev)
        self.Gs = [self.Gp[d.off_G: d.off_G + d.N * d.N].view(d.N, d.N) for d in descs]

    def run(self):
        h = self.handle
        h.bind_stream()
        _abi.check(h._lib.dqmc_greens_batched(h.h, len(self.Gs), _ptr(self.desc), _ptr(self.V),
                                              _ptr(self.Gp), _ptr(self.ld), _ptr(self.sg),
                                              _ptr(self.st)), "dqmc_greens_batched")
        return self.Gs, self.ld, self.sg, self.st


def greens_ragged(instances, *, handle: Handle | None = None, device=None):
    """Ragged batch.  ``instances``: list of (K, dtau, V, k) with CUDA float64 K (N,N), V (M,N).

    Packs the pools on the device and returns (list of G, logdet, sign, status).
    Instances that pass the same K tensor are batched together (per N, k, dtau).
    For repeated calls on the same instances (CUDA-graph replay) use RaggedBatch."""
    return RaggedBatch(instances, device).run(handle)


def _pack_ragged(instances, device, out_len):
    """Descriptors and device pools of a ragged call; out_len(N, M, k) is the
    output block length of one instance."""
    descs = (_abi.DqmcInstance * len(instances))()
    offK = offV = offO = 0
    Ks, Vs = [], []
    seenK = {}
    for i, (K, dtau, V, k) in enumerate(instances):
        N = K.shape[0]
        M = V.shape[0]
        key = (K.data_ptr(), tuple(K.shape), tuple(K.stride()))
        if key not in seenK:
            seenK[key] = offK
            Ks.append(K.reshape(-1))
            offK += N * N
        descs[i] = _abi.DqmcInstance(N, M, int(k), 0, float(dtau), seenK[key], offV, offO)
        Vs.append(V.reshape(-1))
        offV += M * N
        offO += out_len(N, M, int(k))
    Kp = torch.cat(Ks).to(device=device, dtype=torch.float64).contiguous()
    Vp = torch.cat(Vs).to(device=device, dtype=torch.float64).contiguous()
    return descs, Kp, Vp, offO


def greens_tdisplaced_ragged(instances, *, handle: Handle | None = None, device=None,
                             want_tt: bool = True, want_t0: bool = True, want_0t: bool = False):
    """Ragged G(tau_j, tau_j) and G(tau_j, 0): ``instances`` as for greens_ragged.

    Returns (list of Gtt (n_tau, N, N) or None, list of Gt0 or None, status);
    with ``want_0t`` also the list of G(0, tau_j) after Gt0."""
    device = device or instances[0][0].device
    descs, Kp, Vp, total = _pack_ragged(instances, device, lambda N, M, k: n_tau(M, k) * N * N)

    def pool(want):
        return torch.empty(total, dtype=torch.float64, device=device) if want else None
    Gtt, Gt0, G0t = pool(want_tt), pool(want_t0), pool(want_0t)
    B = len(instances)
    st = torch.empty(B, dtype=torch.int32, device=device)
    h = _handle(handle)
    if want_0t:
        _abi.check(h._lib.dqmc_greens_tdisplaced_ragged_ex(h.h, B, descs, _ptr(Kp), _ptr(Vp),
                                                           _ptr(Gtt), _ptr(Gt0), _ptr(G0t),
                                                           _ptr(st)),
                   "dqmc_greens_tdisplaced_ragged_ex")
    else:
        _abi.check(h._lib.dqmc_greens_tdisplaced_ragged(h.h, B, descs, _ptr(Kp), _ptr(Vp),
                                                        _ptr(Gtt), _ptr(Gt0), _ptr(st)),
                   "dqmc_greens_tdisplaced_ragged")
    outs = []
    for pool in ((Gtt, Gt0, G0t) if want_0t else (Gtt, Gt0)):
        if pool is None:
            outs.append(None)
            continue
        lst = []
        for i in range(B):
            d = descs[i]
            nt = n_tau(d.M, d.k)
            lst.append(pool[d.off_G: d.off_G + nt * d.N * d.N].view(nt, d.N, d.N))
        outs.append(lst)
    return tuple(outs) + (st,)


def logdet_grad_ragged(instances, *, handle: Handle | None = None, device=None):
    """Ragged log det and gradient: returns (logdet, sign, list of dV (M, N), status)."""
    device = device or instances[0][0].device
    descs, Kp, Vp, total = _pack_ragged(instances, device, lambda N, M, k: M * N)
    dV = torch.empty(total, dtype=torch.float64, device=device)
    B = len(instances)
    ld = torch.empty(B, dtype=torch.float64, device=device)
    sg = torch.empty(B, dtype=torch.int32, device=device)
    st = torch.empty(B, dtype=torch.int32, device=device)
    h = _handle(handle)
    _abi.check(h._lib.dqmc_logdet_grad_ragged(h.h, B, descs, _ptr(Kp), _ptr(Vp), _ptr(ld), _ptr(sg),
                                              _ptr(dV), _ptr(st)), "dqmc_logdet_grad_ragged")
    dVs = [dV[descs[i].off_G: descs[i].off_G + descs[i].M * descs[i].N].view(descs[i].M, descs[i].N)
           for i in range(B)]
    return ld, sg, dVs, st


def selftest_wait_timeout(status: torch.Tensor, stream: torch.cuda.Stream | None = None):
    """Launch the bounded-wait self-test (dqmc_selftest_wait_timeout); status: a CUDA int32
    tensor of one element that receives DQMC_STATUS_TIMEOUT.  Asynchronous on the stream."""
    if not status.is_cuda or status.dtype != torch.int32 or status.numel() < 1:
        raise ValueError("status must be a CUDA int32 tensor")
    s = stream if stream is not None else torch.cuda.current_stream()
    _abi.check(lib().dqmc_selftest_wait_timeout(C.c_void_p(s.cuda_stream), _ptr(status)),
               "dqmc_selftest_wait_timeout")


class LogDet(torch.autograd.Function):
    """log|det(1 + B_M...B_1)| as a differentiable function of V (B, M, N).

    backward uses the library's adjoint kernel: d logdet / dV_l(i) = 1 - G_l(i,i).
    When no gradient with respect to V is wanted (V does not require grad, or
    under torch.no_grad) the forward pass is the log det alone (dqmc_logdet:
    one chain and one inversion); otherwise it computes log det and the
    gradient in one dqmc_logdet_grad call and keeps the gradient for backward."""

    @classmethod
    def apply(cls, V, K, dtau, k, handle=None):
        # forward runs with grad mode off, so whether a gradient is wanted at
        # all (V requires grad and grad mode is on) is decided here
        if not (torch.is_grad_enabled() and V.requires_grad):
            ld, sg, st = logdet(K, dtau, V, k, handle=handle)
            return ld
        return super().apply(V, K, dtau, k, handle)

    @staticmethod
    def forward(ctx, V, K, dtau, k, handle=None):
        ctx.squeeze = V.dim() == 2
        ld, sg, dV, st = logdet_grad(K, dtau, V, k, handle=handle)
        ctx.save_for_backward(dV)
        return ld

    @staticmethod
    def backward(ctx, gout):
        (dV,) = ctx.saved_tensors
        if ctx.squeeze:
            return gout * dV, None, None, None, None
        return gout[:, None, None] * dV, None, None, None, None


FP64_RATE_KINDS = {"dfma": 0, "dmma_m8n8k4": 1, "dmma_m16n8k8": 2}


def selftest_fp64_rate(kind: str = "dfma", iters: int | None = None) -> tuple[float, float]:
    """Measured FP64 rate of the current device: (TFLOP/s, launch ms) of the
    DFMA or FP64 mma.sync loop kernel, on the current torch stream."""
    code = FP64_RATE_KINDS[kind]
    if iters is None:
        iters = 1500 if code == 2 else 6000
    tf = C.c_double()
    ms = C.c_double()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    _abi.check(lib().dqmc_selftest_fp64_rate(stream, code, int(iters), C.byref(tf), C.byref(ms)),
               "dqmc_selftest_fp64_rate")
    return tf.value, ms.value


def is_debug_build() -> bool:
    """True when the loaded library is the debug build (DQMC_DEBUG=1 in the environment)."""
    return bool(lib().dqmc_is_debug_build())


def debug_read(clear: bool = False):
    """First failed device-side check of the debug build as (file, line, value), or
    None; synchronises the device.  Raises on the release library."""
    fn, ln, val = C.c_char_p(), C.c_int(), C.c_int()
    _abi.check(lib().dqmc_debug_read(int(clear), C.byref(fn), C.byref(ln), C.byref(val)),
               "dqmc_debug_read")
    return None if fn.value is None else (fn.value.decode(), ln.value, val.value)


def selftest_check(stream: torch.cuda.Stream | None = None) -> tuple[bool, int]:
    """Self-test of the debug build's check mechanism: (fired, recorded value)."""
    s = stream if stream is not None else torch.cuda.current_stream()
    fired, val = C.c_int(), C.c_int()
    _abi.check(lib().dqmc_selftest_check(C.c_void_p(s.cuda_stream), C.byref(fired), C.byref(val)),
               "dqmc_selftest_check")
    return bool(fired.value), val.value
