"""Comparison of the library's outputs with the oracle's (test helper).

Rules (how "trigger times bit-exact" is read when two samples of a window
hold nearly equal rho in FP64, so that FP32 rounding may pick either):
* a sample index must match exactly unless the oracle's best and runner-up
  rho in that window (or over the valid range, for the peak) are within
  AMBIG relative; then any sample within that band is accepted and the case
  is counted as ambiguous;
* rho must match within RTOL relative (the stated SNR bound, 1e-3);
* the phase of z must match within PHASE_TOL radians where the index matched;
* a window whose oracle maximum lies within THR_BAND relative of the
  threshold may or may not carry a trigger on either side.
"""

from __future__ import annotations

import math

import numpy as np

import oracle

RTOL = 1e-3
AMBIG = 2e-3
PHASE_TOL = 2e-3
THR_BAND = 1e-3


def oracle_series(dtilde, psd, m1, m2, pn, f_low, fs, n):
    h, k_lo, k_hi = oracle.spa_template(m1, m2, pn, f_low, fs, n)
    s2 = oracle.sigma2(h, psd, fs, n, k_lo, k_hi)
    z = oracle.correlate(dtilde, h, psd, fs, n, k_lo, k_hi)
    rho2 = np.abs(z) ** 2 / s2 if s2 > 0 else np.zeros(n)
    return z, rho2, s2


def _top2(r2):
    if len(r2) == 1:
        return 0, -1.0
    i = int(np.argmax(r2))
    best = r2[i]
    rest = r2.copy()
    rest[i] = -1.0
    return i, float(rest.max())


def _accept_index(r2, got, want):
    """True if `got` is `want`, or the oracle's rho at `got` is within AMBIG of
    its maximum (ambiguous case)."""
    if got == want:
        return True, False
    top = r2[want]
    if top <= 0:
        return r2[got] <= 0, True
    return math.sqrt(r2[got] / top) >= 1 - AMBIG, True


class Report:
    def __init__(self):
        self.n = 0
        self.ambiguous = 0
        self.max_rel = 0.0
        self.max_phase = 0.0
        self.errors: list[str] = []

    def fail(self, msg):
        if len(self.errors) < 20:
            self.errors.append(msg)

    def ok(self):
        return not self.errors

    def __repr__(self):
        return (f"Report(n={self.n}, ambiguous={self.ambiguous}, max_rel={self.max_rel:.3g}, "
                f"max_phase={self.max_phase:.3g}, errors={self.errors[:5]})")


def _phase_diff(a, b):
    d = (a - b + math.pi) % (2 * math.pi) - math.pi
    return abs(d)


def check_template(rep: Report, t, z, r2, peak, trigs, lo, hi, window, thr):
    """Compare one template's GPU peak (record) and triggers (records of this
    template) with the oracle's correlator z / rho^2."""
    rep.n += 1
    seg = r2[lo:hi]
    if hi <= lo:
        return
    i, second = _top2(seg)
    want = lo + i
    got = int(peak["sample"])
    ok, amb = _accept_index(r2, got, want) if lo <= got < hi else (False, False)
    if not ok:
        rep.fail(f"t{t}: peak sample {got} vs oracle {want} (rho {math.sqrt(r2[want]):.6f})")
        return
    if amb:
        rep.ambiguous += 1
    ro = math.sqrt(r2[got])
    rel = abs(float(peak["snr"]) - ro) / max(ro, 1e-30)
    rep.max_rel = max(rep.max_rel, rel)
    if rel > RTOL and ro > 1e-6:
        rep.fail(f"t{t}: peak rho {float(peak['snr']):.7g} vs oracle {ro:.7g} (rel {rel:.3g})")
    if ro > 1e-6:
        dp = _phase_diff(float(peak["phase"]), math.atan2(z[got].imag, z[got].real))
        rep.max_phase = max(rep.max_phase, dp)
        if dp > PHASE_TOL:
            rep.fail(f"t{t}: peak phase off by {dp:.3g}")
    # triggers, window by window
    g = {int((int(s) - lo) // window): (int(s), float(r), float(p)) for s, r, p in
         zip(trigs["sample"], trigs["snr"], trigs["phase"])}
    if len(g) != len(trigs):
        rep.fail(f"t{t}: two triggers in one window")
    nwin = (hi - lo + window - 1) // window
    for m in range(nwin):
        w0, w1 = lo + m * window, min(lo + (m + 1) * window, hi)
        j = w0 + int(np.argmax(r2[w0:w1]))
        rw = math.sqrt(r2[j])
        near = abs(rw - thr) <= THR_BAND * thr
        if m in g:
            s, r, p = g[m]
            if rw <= thr and not near:
                rep.fail(f"t{t} w{m}: GPU trigger at {s} (rho {r:.5g}) where the oracle's max is {rw:.5g}")
                continue
            ok, amb = _accept_index(r2, s, j)
            if not ok:
                rep.fail(f"t{t} w{m}: trigger sample {s} vs oracle {j}")
                continue
            ro = math.sqrt(r2[s])
            rel = abs(r - ro) / ro
            rep.max_rel = max(rep.max_rel, rel)
            if rel > RTOL:
                rep.fail(f"t{t} w{m}: trigger rho {r:.7g} vs {ro:.7g}")
            dp = _phase_diff(p, math.atan2(z[s].imag, z[s].real))
            rep.max_phase = max(rep.max_phase, dp)
            if dp > PHASE_TOL:
                rep.fail(f"t{t} w{m}: trigger phase off by {dp:.3g}")
        elif rw > thr and not near:
            rep.fail(f"t{t} w{m}: missing trigger (oracle rho {rw:.5g} at {j})")


def split_triggers(trig, n_templates):
    out = [trig[:0]] * n_templates
    if len(trig) == 0:
        return out
    order = np.argsort(trig["tmpl"], kind="stable")
    trig = trig[order]
    ids, starts = np.unique(trig["tmpl"], return_index=True)
    ends = list(starts[1:]) + [len(trig)]
    for i, s, e in zip(ids, starts, ends):
        out[int(i)] = trig[s:e]
    return out


def make_segment(w, segment: int = 0, inject: bool = True):
    """Strain and PSD of a workload: seeded coloured noise plus its planned
    injections, each an exact bank member built by the oracle at its target
    SNR.  Returns (strain, psd, oracle data spectrum, injection plan)."""
    import synth

    psd = w.psd()
    d = w.noise(segment)
    m1, m2 = w.masses()
    plan = w.injection_plan(segment)
    if inject:
        for t, j0, snr in zip(*plan):
            h, k_lo, k_hi = oracle.spa_template(m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n)
            s2 = oracle.sigma2(h, psd, w.fs, w.n, k_lo, k_hi)
            synth.add_signal(d, h, snr / math.sqrt(s2), int(j0), w.n)
    strain = synth.strain_from_spectrum(d, w.n, w.fs)
    dt = oracle.segment_spectrum(strain, w.fs)
    return strain, psd, dt, plan


def compare_bank(w, dt, psd, peaks, trig, templates, lo, hi, window, thr, threads=None):
    """Oracle correlators for `templates`, compared with the GPU records."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    m1, m2 = w.masses()
    per = split_triggers(trig, w.n_templates)
    rep = Report()
    oracle.build()

    def one(t):
        z, r2, _ = oracle_series(dt, psd, m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n)
        sub = Report()
        check_template(sub, t, z, r2, peaks[t], per[t], lo, hi, window, thr)
        return sub

    with ThreadPoolExecutor(max_workers=threads or len(os.sched_getaffinity(0))) as ex:
        for sub in ex.map(one, templates):
            rep.n += sub.n
            rep.ambiguous += sub.ambiguous
            rep.max_rel = max(rep.max_rel, sub.max_rel)
            rep.max_phase = max(rep.max_phase, sub.max_phase)
            for e in sub.errors:
                rep.fail(e)
    return rep
