"""Helpers for the sharding tests: a host-only stand-in for Bank and the
per-rank body of a world-size-2 gloo run (spawned processes import this
module, so it holds no tests)."""

import numpy as np

N, FS, F_LOW = 1 << 12, 4096.0, 30.0


def bank_masses(seed=7, count=37):
    rng = np.random.default_rng(seed)
    return rng.uniform(1.0, 10.0, count), rng.uniform(1.0, 10.0, count)


def segment(seed=11):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(N), 1.0 + rng.random(N // 2 + 1)


class FakeBank:
    """Deterministic results from the masses and the uploaded segment, with the
    Bank methods ShardedSearch calls; checks that the segment arrived."""

    def __init__(self, m1, m2, *, n, fs, f_low, **kw):
        self.m1, self.m2, self.n = np.asarray(m1), np.asarray(m2), n
        self.key = None

    def upload(self, strain, psd):
        strain, psd = np.asarray(strain), np.asarray(psd)
        assert strain.shape == (self.n,) and psd.shape == (self.n // 2 + 1,)
        self.key = float(strain[:64].sum() + psd[1])

    def filter(self):
        assert self.key is not None

    def peaks(self):
        from paper_1006_4644_gb300 import PEAK_DTYPE

        pk = np.zeros(len(self.m1), dtype=PEAK_DTYPE)
        pk["sample"] = (self.m1 * 1000).astype(np.int64) % self.n
        pk["snr"] = self.m1 + self.m2 + self.key
        pk["phase"] = self.m2
        return pk

    def triggers(self, capacity=1 << 20, allow_overflow=False):
        from paper_1006_4644_gb300 import TRIGGER_DTYPE

        sel = np.nonzero(self.m1 > 4.0)[0]
        tr = np.zeros(2 * len(sel), dtype=TRIGGER_DTYPE)
        tr["tmpl"] = np.repeat(sel, 2)
        tr["sample"] = np.repeat((self.m2[sel] * 100).astype(np.int64), 2) + np.tile([0, 4096], len(sel))
        tr["snr"] = self.key
        order = np.lexsort((tr["sample"], tr["tmpl"]))
        return tr[order], len(tr)

    def close(self):
        pass


def run_rank(rank, world, port, out_path):
    import torch.distributed as dist

    from paper_1006_4644_gb300.shard import ShardedSearch

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        m1, m2 = bank_masses()
        strain, psd = segment() if rank == 0 else (None, None)
        ss = ShardedSearch(m1, m2, n=N, fs=FS, f_low=F_LOW, bank_factory=FakeBank, pn_x2=7)
        res = ss.search(strain, psd)
        shard = ss.index
        all_idx = [None] * world
        dist.all_gather_object(all_idx, shard)
        if rank == 0:
            peaks, trig, total = res
            np.savez(out_path, peaks=peaks, trig=trig, total=total,
                     **{f"shard{r}": np.asarray(s) for r, s in enumerate(all_idx)})
        else:
            assert res is None
    finally:
        dist.destroy_process_group()
