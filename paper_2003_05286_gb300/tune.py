"""Autotuner for the stabilisation interval k and the FP64 product tile.

The paper leaves the interval between stabilised products open (Sec. 4.1:
a mixture of naive and stabilised products "for the sake of speed while
retaining accuracy").  Larger k means fewer pivoted QRs (faster) but a wider
dynamic range inside each naive chunk (less accurate).  ``tune`` measures both
on a sample of the caller's own fields: for every candidate (k, tile) it runs
the library, compares G with a reference computed at a small k, times it with
CUDA events, and returns the fastest candidate whose deviation stays within
``tol``.  Results are cached per (N, M, dtau, precision, SM count).

The environment variable DQMC_TUNE selects the mode: ``on`` (default) uses a
cached result when there is one, ``force`` tunes again and overwrites the
cache, ``off`` times nothing and returns ``default_k`` with the library's
tile choice.

All computation runs through the library's C ABI; this module only chooses
parameters.
"""
from __future__ import annotations

import json
import os

import torch

from . import Handle, greens

_CACHE: dict[str, dict] = {}


def _key(N, M, dtau, prec, tag):
    sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return f"N{N}-M{M}-dt{dtau:g}-p{prec}-sm{sm}-{tag}"


def tune_mode() -> str:
    """DQMC_TUNE: 'on' (default), 'force' or 'off'; anything else is an error."""
    mode = os.environ.get("DQMC_TUNE", "on").strip().lower() or "on"
    if mode not in ("on", "force", "off"):
        raise ValueError(f"DQMC_TUNE must be on, force or off (got {mode!r})")
    return mode


def _time_ms(fn, reps):
    fn()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        out = fn()
    ev[1].record()
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / reps, out


def tune(K: torch.Tensor, dtau: float, V: torch.Tensor, *, candidates=(5, 8, 10, 12, 15, 20),
         tiles=(0, 32, 48, 64), ref_k: int = 2, tol: float = 1e-10, chain_precision: int = 0,
         reps: int = 2, cache_file: str | None = None, tag: str = "", fold: int | None = None,
         default_k: int = 10):
    """Pick (k, tile) for fields shaped like V (B, M, N).

    Returns (best, table): best = dict(k, tile, err, ms); table = every
    candidate tried.  tile 0 lets the library choose by size.  ``fold`` is the
    chain fold the timed candidates use (dqmc_set_chain_fold; None: the
    library's choice for the sample's own size): a small sample of a large
    batch should be timed with the fold the large batch will run."""
    V3 = V if V.dim() == 3 else V.unsqueeze(0)
    B, M, N = V3.shape
    mode = tune_mode()
    if mode == "off":
        return dict(k=min(default_k, M), tile=0, err=None, ms=None), None
    key = _key(N, M, dtau, chain_precision, tag + ("" if fold is None else f"-f{fold}"))
    if cache_file and not _CACHE and os.path.exists(cache_file):
        with open(cache_file) as f:
            _CACHE.update(json.load(f))
    if key in _CACHE and mode == "on":
        return _CACHE[key], None
    href = Handle()
    Gref = greens(K, dtau, V3, min(ref_k, M), handle=href)[0]
    scale = float(Gref.abs().max().clamp(min=1.0))
    table = []
    for tile in tiles:
        h = Handle(chain_precision=chain_precision) if fold is None else \
            Handle(chain_precision=chain_precision, fold=fold)
        h.set_gemm_tile(tile)
        for k in candidates:
            if k > M:
                continue
            ms, out = _time_ms(lambda: greens(K, dtau, V3, k, handle=h), reps)
            err = float((out[0] - Gref).abs().max()) / scale
            table.append(dict(k=k, tile=tile, err=err, ms=ms))
        h.close()
    href.close()
    ok = [r for r in table if r["err"] <= tol]
    best = min(ok, key=lambda r: r["ms"]) if ok else dict(k=min(ref_k, M), tile=0, err=0.0, ms=None)
    _CACHE[key] = best
    if cache_file:
        with open(cache_file, "w") as f:
            json.dump(_CACHE, f, indent=1)
    return best, table
