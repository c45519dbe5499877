"""Multi-band hierarchical search (Sec. "Online analysis considerations"): the
frequency range is split at f_split; the upper band, where a chirp is short
and carries most of its SNR, is searched first on short segments cut from the
band-passed data; every detection is then completed by the lower band, summed
directly at the detection's time on the whole segment (or on a decimated copy
of its lower band), and the two bands are added coherently.

Every step is a library call (cui_segment_band_series, cui_bank_set_band,
cui_filter_bank, cui_triggers, cui_band_combine); this module only cuts the
device series into segments and gathers the candidates.  The combination
rho = |z_high + z_low| / sqrt(sigma_high^2 + sigma_low^2) runs in the library.
"""

from __future__ import annotations

import numpy as np

CANDIDATE_DTYPE = np.dtype([("tmpl", np.int32), ("t", np.float64), ("rho_high", np.float32), ("rho", np.float64),
                            ("phase", np.float64)])


def chunk_plan(n: int, n_short: int, lo: int, hi: int):
    """Short segments over a segment of n samples: (start, first, end) with
    [first, end) the absolute samples a segment reports, inside its valid range
    [start + lo, start + hi); together they tile [lo, n - n_short + hi) with no
    gap or overlap (the last segment is moved back to end at n)."""
    if not (0 <= lo < hi <= n_short <= n):
        raise ValueError("need 0 <= lo < hi <= n_short <= n")
    plan, s = [], 0
    while True:
        plan.append((s, s + lo, s + hi))
        nxt = s + (hi - lo)
        if nxt + n_short <= n:
            s = nxt
            continue
        last = n - n_short
        if last + hi > s + hi:
            plan.append((last, s + hi, last + hi))
        return plan


def hierarchical_search(segment, detect, f_split: float, psd_short, low=None):
    """Candidates of a multi-band hierarchical search.

    segment: Bank holding the whole segment (N samples at fs, uploaded).
    detect:  Bank over the same templates at the same fs with a short length;
             its valid range and SNR threshold select detections in the band
             [f_split, ...), which is set on it here.
    psd_short: one-sided PSD at the detect bank's bins (float64 device tensor).
    low:     optional Bank holding the lower band of the same data at a lower
             rate (uploaded from segment.band_series(..., 0, f_split, decim));
             without it the lower band is summed on ``segment``.
    Returns CANDIDATE_DTYPE records in time order: template, time t (s), the
    upper band's SNR, the combined SNR and phase."""
    import torch

    n, ns = segment.n, detect.n
    lo, hi = int(detect.desc.valid_lo), int(detect.desc.valid_hi)
    fs = segment.fs
    if detect.fs != fs:
        raise ValueError("the detect bank runs at the segment's sample rate")
    hp = torch.empty(n, dtype=torch.float64, device="cuda")
    segment.band_series(hp, f_split, 0.0, 1)
    detect.set_band(f_split, 0.0)
    parts = []
    for s0, first, end in chunk_plan(n, ns, lo, hi):
        detect.upload(hp[s0:s0 + ns].contiguous(), psd_short)
        detect.filter()
        trig, _ = detect.triggers()
        trig = trig[(trig["sample"] + s0 >= first) & (trig["sample"] + s0 < end)]
        if len(trig) == 0:
            continue
        rec = np.zeros(len(trig), dtype=CANDIDATE_DTYPE)
        rec["tmpl"] = trig["tmpl"]
        rec["t"] = (s0 + trig["sample"]) / fs
        rec["rho_high"] = trig["snr"]
        # completed while this short segment is still the detect bank's
        rec["rho"], rec["phase"], _ = detect.band_combine(trig["sample"] / fs, segment if low is None else low,
                                                          rec["t"], rec["tmpl"], f_split)
        parts.append(rec)
    if not parts:
        return np.zeros(0, dtype=CANDIDATE_DTYPE)
    rec = np.concatenate(parts)
    return rec[np.argsort(rec["t"], kind="stable")]
