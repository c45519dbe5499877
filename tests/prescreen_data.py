"""Prescreen training / evaluation data (test infrastructure): segments with
one injection each, built by the oracle, labelled with the bank region of the
injected chirp mass (soft labels on the neighbours)."""

from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle
import synth
from oracle import prescreen as ops


def injection_params(seed: int, idx: int, mass_lo: float, mass_hi: float, snr_lo: float, snr_hi: float, n: int):
    u = synth.uniform(seed, 20_000_000 + idx, 4)
    m1 = math.exp(math.log(mass_lo) + u[0] * (math.log(mass_hi) - math.log(mass_lo)))
    m2 = math.exp(math.log(mass_lo) + u[1] * (math.log(mass_hi) - math.log(mass_lo)))
    snr = snr_lo + u[2] * (snr_hi - snr_lo)
    j0 = min(int(u[3] * n), n - 1)
    return m1, m2, snr, j0


def make_segments(seed: int, start: int, count: int, n: int, fs: float, f_low: float, psd, bounds, regions: int,
                  pn_x2: int = 7, mass=(1.0, 25.0), snr=(6.0, 20.0), threads: int | None = None):
    """(d~ [count, n/2+1] complex128, targets [count, regions] float32,
    meta list of dicts)."""
    oracle.build()

    def one(i):
        idx = start + i
        d = synth.noise_spectrum(seed, 10_000_000 + idx, n, fs, psd, f_low)
        m1, m2, s, j0 = injection_params(seed, idx, mass[0], mass[1], snr[0], snr[1], n)
        h, lo, hi = oracle.spa_template(m1, m2, pn_x2, f_low, fs, n)
        s2 = oracle.sigma2(h, psd, fs, n, lo, hi)
        if s2 > 0:
            synth.add_signal(d, h, s / math.sqrt(s2), j0, n)
        mc = float(ops.chirp_mass(m1, m2))
        r = ops.region_of(mc, bounds)
        return d, ops.soft_labels(r, regions).astype(np.float32), dict(m1=m1, m2=m2, snr=s, j0=j0, mc=mc, region=r)

    with ThreadPoolExecutor(max_workers=threads or len(os.sched_getaffinity(0))) as ex:
        out = list(ex.map(one, range(count)))
    return (np.stack([o[0] for o in out]), np.stack([o[1] for o in out]), [o[2] for o in out])


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest even) and back to float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _worker(args):
    (shm_name, shape, seed, start, lo, hi, n, fs, f_low, psd, bounds, regions, pn_x2, mass, snr) = args
    from multiprocessing import shared_memory

    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        buf = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
        d, y, meta = make_segments(seed, start + lo, hi - lo, n, fs, f_low, psd, bounds, regions, pn_x2, mass, snr,
                                   threads=1)
        buf[lo:hi] = d
        return lo, y, meta
    finally:
        shm.close()


def make_segments_mp(seed: int, start: int, count: int, n: int, fs: float, f_low: float, psd, bounds, regions: int,
                     pn_x2: int = 7, mass=(1.0, 25.0), snr=(6.0, 20.0), procs: int | None = None, pool=None):
    """make_segments spread over a process pool (spawn), the spectra written
    into shared memory.  Pass a pool created with the spawn context to reuse it."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    shape = (count, n // 2 + 1)
    shm = shared_memory.SharedMemory(create=True, size=int(np.prod(shape)) * 16)
    try:
        procs = procs or len(os.sched_getaffinity(0))
        step = max(1, -(-count // (4 * procs)))
        jobs = [(shm.name, shape, seed, start, lo, min(count, lo + step), n, fs, f_low, psd, bounds, regions, pn_x2,
                 mass, snr) for lo in range(0, count, step)]
        own = pool is None
        if own:
            pool = mp.get_context("spawn").Pool(procs)
        try:
            res = pool.map(_worker, jobs)
        finally:
            if own:
                pool.close()
                pool.join()
        d = np.array(np.ndarray(shape, dtype=np.complex128, buffer=shm.buf))
    finally:
        shm.close()
        shm.unlink()
    res.sort(key=lambda r: r[0])
    y = np.concatenate([r[1] for r in res])
    meta = [m for r in res for m in r[2]]
    return d, y, meta
