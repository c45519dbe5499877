"""Oracle filter-output labels for the prescreen (test infrastructure; calls
only oracle/ and synth/, no GPU):

    python tests/prescreen_labels/make_oracle_labels.py [--count 512] [--start 0]

The first `count` training segments of the prescreen workload (the seeded
segments tests/prescreen_config4.py trains on: N = 2^16 at 4096 Hz, one
oracle-made injection each, SNR U[6, 20], masses log-U[1, 25] Msun, 3.5PN,
f_low 20 Hz) are filtered by the FP64 oracle against every template of the
10^4-template bank, with the same trigger rule the held-out segments are
judged by (windows of 4096 samples, threshold 6).  For each segment and each
of the 100 equal-count chirp-mass regions the file keeps the region's
response: the largest trigger rho of its templates within 4096 samples
(circularly) of the injection, 0 where none.  A region whose response
reaches 8 detects the injection.  Written to oracle_response_seed4.npz here.
"""

from __future__ import annotations

import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import prescreen as ops  # noqa: E402
from prescreen_data import make_segments  # noqa: E402

N, FS, F_LOW, REGIONS, WINDOW, SEED = 1 << 16, 4096.0, 20.0, 100, 4096, 4


def region_response(trig_by_tmpl, region_of_tmpl, j0, n=N, window=WINDOW, regions=REGIONS):
    """Largest trigger rho per region within `window` samples of j0 (circular)."""
    out = np.zeros(regions)
    for t, (tj, tr) in enumerate(trig_by_tmpl):
        if len(tj) == 0:
            continue
        dist = np.abs(tj - j0)
        dist = np.minimum(dist, n - dist)
        near = tr[dist <= window]
        if len(near):
            out[region_of_tmpl[t]] = max(out[region_of_tmpl[t]], float(near.max()))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--start", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(HERE, "oracle_response_seed4.npz"))
    args = ap.parse_args()
    oracle.build()
    psd = synth.psd_onesided(N, FS)
    bankw = synth.WORKLOADS["seg256s_bank10k_pn35"]
    m1, m2 = bankw.masses()
    groups, bounds = ops.regions_of_bank(m1, m2, REGIONS)
    region_of_tmpl = np.empty(len(m1), dtype=np.int64)
    for r, g in enumerate(groups):
        region_of_tmpl[g] = r
    resp = np.zeros((args.count, REGIONS), dtype=np.float32)
    j0s, snrs, regs = [], [], []
    t0 = time.time()
    for i in range(args.count):
        d, _, meta = make_segments(SEED, args.start + i, 1, N, FS, F_LOW, psd, bounds, REGIONS)
        strain = synth.strain_from_spectrum(d[0], N, FS)
        dt = oracle.segment_spectrum(strain, FS)
        res = oracle.filter_bank(dt, psd, m1, m2, 7, F_LOW, FS, N, window=WINDOW, thr=6.0)
        mt = meta[0]
        resp[i] = region_response([(r["trig_j"], r["trig_rho"]) for r in res], region_of_tmpl, mt["j0"])
        j0s.append(mt["j0"])
        snrs.append(mt["snr"])
        regs.append(mt["region"])
        if i % 16 == 15:
            print(f"{i + 1}/{args.count} segments, {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(args.out, response=resp, start=args.start, j0=np.array(j0s), snr=np.array(snrs),
                        region=np.array(regs), seed=SEED, n=N, window=WINDOW)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
