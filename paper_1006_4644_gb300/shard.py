"""Bank sharding across GPUs, one process per GPU.

Templates are independent (Sec. "Matched filtering": every template of the
bank is correlated with the same data chunk), so a bank splits into shards that
separate ranks filter against the same segment.  The only exchanges are the
segment itself, broadcast from rank 0, and the results, gathered to rank 0.
Nothing crosses between GPUs inside the filter.

Shards are contiguous chirp-mass ranges (neighbouring templates have similar
bands) balanced by estimated cost.  A template's cost is a fixed part (the
inverse-FFT row pass, which runs over all N samples whatever the band) plus a
part proportional to its band k_hi - k_low (template generation and the pruned
column pass).  Host-side bookkeeping only: every rank filters its shard with
its own :class:`Bank` on its own GPU.
"""

from __future__ import annotations

import numpy as np

from .regions import chirp_mass


def band_bins(m1, m2, *, n: int, fs: float, f_low: float):
    """k_hi - k_low per template, by the library's own band rule
    (cui_template_bands, host code; no GPU needed)."""
    from . import template_bands

    k_lo, k_hi = template_bands(m1, m2, n=n, fs=fs, f_low=f_low)
    return np.maximum(k_hi.astype(np.float64) - k_lo, 0.0)


def template_cost(m1, m2, *, n: int, fs: float, f_low: float, band_weight: float = 0.5):
    """Relative cost per template: 1 for the fixed part plus `band_weight` for
    a band spanning the whole one-sided spectrum.  The default weight matches
    the measured split at N = 2^20 (row pass about 2.6 us per template for any
    band, column pass about 2.1 us at the full band)."""
    return 1.0 + band_weight * band_bins(m1, m2, n=n, fs=fs, f_low=f_low) / (n // 2)


def partition(m1, m2, world: int, *, n: int, fs: float, f_low: float, band_weight: float = 0.5):
    """Template-index arrays, one per rank: contiguous ranges of the bank sorted
    by chirp mass, cut where the running cost crosses k/world of the total."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(chirp_mass(m1, m2), kind="stable")
    cost = template_cost(m1, m2, n=n, fs=fs, f_low=f_low, band_weight=band_weight)[order]
    if len(order) == 0:
        return [order.copy() for _ in range(world)]
    cum = np.cumsum(cost)
    # shard r ends at the first template whose running cost reaches (r+1)/world of the total
    cuts = np.searchsorted(cum, cum[-1] * np.arange(1, world) / world, side="left") + 1
    cuts = np.minimum(cuts, len(order))
    return np.split(order, cuts)


def merge(n_templates: int, parts):
    """Bank-wide (peaks, triggers, n_total) from per-shard results.

    parts: iterable of (global template ids, peaks, triggers, n_total) with the
    shard's peaks in its own template order and its trigger records numbered by
    shard-local template.  Triggers come back sorted by (template, sample), as
    ``cui_triggers`` orders them."""
    from ._lib import PEAK_DTYPE, TRIGGER_DTYPE

    peaks = np.zeros(n_templates, dtype=PEAK_DTYPE)
    trig = []
    total = 0
    for idx, pk, tr, n_tot in parts:
        idx = np.asarray(idx)
        if len(idx):
            peaks[idx] = pk
        tr = np.array(tr, dtype=TRIGGER_DTYPE, copy=True)
        if len(tr):
            tr["tmpl"] = idx[tr["tmpl"]]
        trig.append(tr)
        total += int(n_tot)
    trig = np.concatenate(trig) if trig else np.zeros(0, dtype=TRIGGER_DTYPE)
    trig = trig[np.lexsort((trig["sample"], trig["tmpl"]))]
    return peaks, trig, total


class ShardedSearch:
    """This rank's share of a bank search.

    Every rank constructs it with the whole bank; it keeps the shard
    ``partition`` assigns to its rank and builds a :class:`Bank` for it
    (``bank_factory`` replaces that constructor, e.g. in host-only tests).
    Without an initialised process group it is a single shard."""

    def __init__(self, m1, m2, *, n: int, fs: float, f_low: float, group=None, bank_factory=None,
                 band_weight: float = 0.5, **bank_kw):
        import torch.distributed as dist

        self.group = group
        self.dist = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank(group) if self.dist else 0
        self.world = dist.get_world_size(group) if self.dist else 1
        m1 = np.ascontiguousarray(m1, dtype=np.float64)
        m2 = np.ascontiguousarray(m2, dtype=np.float64)
        self.n, self.fs, self.n_templates = int(n), float(fs), len(m1)
        self.shards = partition(m1, m2, self.world, n=n, fs=fs, f_low=f_low, band_weight=band_weight)
        self.index = self.shards[self.rank]
        if bank_factory is None:
            from . import Bank as bank_factory
        self.bank = (bank_factory(m1[self.index], m2[self.index], n=n, fs=fs, f_low=f_low, **bank_kw)
                     if len(self.index) else None)

    def _device(self):
        import torch
        import torch.distributed as dist

        if self.dist and dist.get_backend(self.group) == "nccl":
            return torch.device("cuda", torch.cuda.current_device())
        return torch.device("cpu")

    def broadcast_segment(self, strain=None, psd=None):
        """Rank 0's (strain, psd) on every rank, as float64 tensors (on the GPU
        for NCCL groups, on the host for gloo)."""
        import torch
        import torch.distributed as dist

        dev = self._device()
        if self.rank == 0:
            s = torch.as_tensor(np.ascontiguousarray(strain, dtype=np.float64)).to(dev)
            p = torch.as_tensor(np.ascontiguousarray(psd, dtype=np.float64)).to(dev)
        else:
            s = torch.empty(self.n, dtype=torch.float64, device=dev)
            p = torch.empty(self.n // 2 + 1, dtype=torch.float64, device=dev)
        if self.dist:
            src = dist.get_global_rank(self.group, 0) if self.group is not None else 0
            dist.broadcast(s, src=src, group=self.group)
            dist.broadcast(p, src=src, group=self.group)
        return s, p

    def search(self, strain=None, psd=None, capacity: int = 1 << 20):
        """Filter this rank's shard against rank 0's segment.  Returns
        (peaks, triggers, n_total) for the whole bank on rank 0, None on the
        other ranks."""
        import torch.distributed as dist

        from ._lib import PEAK_DTYPE, TRIGGER_DTYPE

        s, p = self.broadcast_segment(strain, psd)
        if self.bank is not None:
            if s.is_cuda:
                self.bank.upload(s, p)
            else:
                self.bank.upload(s.numpy(), p.numpy())
            self.bank.filter()
            part = (self.index, self.bank.peaks(), *self.bank.triggers(capacity, allow_overflow=True))
        else:
            part = (self.index, np.zeros(0, dtype=PEAK_DTYPE), np.zeros(0, dtype=TRIGGER_DTYPE), 0)
        if not self.dist:
            return merge(self.n_templates, [part])
        dst = dist.get_global_rank(self.group, 0) if self.group is not None else 0
        parts = [None] * self.world if self.rank == 0 else None
        dist.gather_object(part, parts, dst=dst, group=self.group)
        return merge(self.n_templates, parts) if self.rank == 0 else None

    def close(self):
        if self.bank is not None:
            self.bank.close()
            self.bank = None
