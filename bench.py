#!/usr/bin/env python3
"""Bank matched-filter benchmark: templates/s on one 2^20-sample segment.

One step = one pass of the whole hot path over one segment: upload and
transform the segment (FP64 FFT, noise weighting, every template's sigma),
then filter the whole bank (fused generate x correlate -> two-pass FFT ->
|z|^2 peak / threshold reduction) with peaks and triggers left on the device.
Workload (default): N = 2^20 at 4096 Hz (256 s), 1024 3.5PN templates with
m1, m2 uniform in [1, 10] Msun, f_low = 30 Hz, 5 injections at SNR 8-15,
synthetic coloured Gaussian noise.  Prints one JSON line (rank 0).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "templates/s on 2^20-sample segments, mixed vs plain, at SNR rel err <=1e-3"
UNIT = "templates/s"
DEFAULT_WORKLOAD = "seg256s_bank1024_pn35"
FALLBACK_HBM_GBS = 6800.0


def measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def source_digest() -> str:
    """Digest of the fused kernels' source, to tell whether a stored ncu
    capture still describes them."""
    h = hashlib.sha256()
    for f in ("fused.cu", "common.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_1006_4644_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(kernel: str, workload: str):
    """DRAM bytes per template of `kernel` from a committed ncu summary, or None
    when absent or taken on other source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_template:\s*([0-9.eE+]+)", text)
    d = re.search(r"source_digest:\s*([0-9a-f]+)", text)
    if not m or not d or d.group(1) != source_digest():
        return None
    return float(m.group(1))


class Clocks:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)  # sampling is running before the timed region starts
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if getattr(self, "_summary", None) is not None:
            return self._summary
        if not self.proc or not self.file:
            return None
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.file.name)
        if not sm:
            return None
        self._summary = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                         "samples": len(sm)}
        return self._summary


def build_segment(w, bank, psd):
    """Noise plus the workload's injections.  The injected waveforms are the
    library's own templates (cui_bank_template) scaled by its sigma."""
    import numpy as np
    import torch

    import synth

    d = w.noise()
    strain0 = synth.strain_from_spectrum(d, w.n, w.fs)
    bank.upload(strain0, psd)
    sig = bank.sigma()
    out = torch.zeros(w.n // 2 + 1, dtype=torch.complex64, device="cuda")
    for t, j0, snr in zip(*w.injection_plan()):
        bank.template(int(t), out)
        h = out.cpu().numpy().astype(np.complex128)
        synth.add_signal(d, h, float(snr) / sig[t], int(j0), w.n)
    return synth.strain_from_spectrum(d, w.n, w.fs)


def cpu_baseline(w, budget_s: float = 15.0, per_step: int | None = None, strain=None):
    """The FP64 oracle as it stands, on this host's cores, on a bounded sample
    of the same workload: the given strain, else noise plus oracle-built
    injections.  Also returns the oracle's per-template results and indices."""
    import numpy as np

    import oracle
    import synth

    oracle.build()
    cores = len(os.sched_getaffinity(0))
    psd = w.psd()
    m1, m2 = w.masses()
    if strain is None:
        d = w.noise()
        for t, j0, snr in zip(*w.injection_plan()):
            h, lo, hi = oracle.spa_template(m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n)
            synth.add_signal(d, h, float(snr) / math.sqrt(oracle.sigma2(h, psd, w.fs, w.n, lo, hi)), int(j0), w.n)
        strain = synth.strain_from_spectrum(d, w.n, w.fs)
    dt = oracle.segment_spectrum(strain, w.fs)
    t0 = time.perf_counter()
    oracle.filter_template(dt, psd, m1[0], m2[0], w.pn_x2, w.f_low, w.fs, w.n)
    one = time.perf_counter() - t0
    if per_step is None:
        per_step = int(max(cores, min(w.n_templates, budget_s * cores / max(one, 1e-3))))
    sel = np.arange(per_step) % w.n_templates
    t0 = time.perf_counter()
    res = oracle.filter_bank(dt, psd, m1[sel], m2[sel], w.pn_x2, w.f_low, w.fs, w.n, threads=cores)
    el = time.perf_counter() - t0
    return {"value": per_step / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{per_step} templates of {w.name} (segment FFT excluded, one template per thread)",
            "seconds": el, "results": res, "templates": sel}


def accuracy(gpu_peaks, cpu, only=None):
    """The GPU peaks against the oracle's on the templates the CPU baseline
    filtered (same strain and PSD), or on those of them in `only`: peak
    sample, SNR and phase."""
    import numpy as np

    seen, rel, dphi, mism = set(), [], [], 0
    for t, r in zip(cpu["templates"], cpu["results"]):
        t = int(t)
        if t in seen or (only is not None and t not in only):
            continue
        seen.add(t)
        g = gpu_peaks[t]
        rel.append(abs(float(g["snr"]) - r["peak_rho"]) / max(r["peak_rho"], 1e-30))
        if int(g["sample"]) != int(r["peak_j"]):
            mism += 1
        else:
            d = (float(g["phase"]) - r["peak_phase"] + math.pi) % (2 * math.pi) - math.pi
            dphi.append(abs(d))
    return {"reference": "the FP64 oracle on the same strain and PSD", "templates": len(seen),
            "max_rel_err_snr": max(rel), "rms_rel_err_snr": float(np.sqrt(np.mean(np.square(rel)))),
            "peak_sample_mismatches": mism, "max_phase_err_rad": max(dphi) if dphi else None}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0))
    # size each step to ~5 s of oracle work so the whole run stays short
    probe = cpu_baseline(w, per_step=cores)
    per_step = int(max(cores, probe["value"] * 5.0))
    for _ in range(args.warmup):
        cpu_baseline(w, per_step=cores)
    tot, n = 0.0, 0
    for _ in range(args.steps):
        r = cpu_baseline(w, per_step=per_step)
        tot += r["seconds"]
        n += per_step
    value = n / tot
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "templates": w.n_templates, "sample_per_step": per_step},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} templates per step of {w.name}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_stream(args, w):
    """A stream of consecutive segments with 50 % overlap (each keeps triggers in
    its middle half, [N/4, 3N/4)), every segment scored by the region prescreen
    and then filtered against the whole bank; reports the sustained rate.  The
    segments are drawn independently in the frequency domain (continuity across
    the overlap does not change the work).  The tiling is autotuned on a
    4096-template sample of the bank."""
    import numpy as np
    import torch

    import synth
    from paper_1006_4644_gb300 import Bank, Prescreen
    from paper_1006_4644_gb300._lib import CUI_NO_GRAPH

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    m1, m2 = w.masses()
    psd = w.psd()
    psd_fin = psd.copy()
    psd_fin[0] = 1.0
    n = w.n
    kw = dict(n=n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    if args.tuning:
        tuning = dict(zip(("n1", "ccols", "rpc", "batch"), (int(x) for x in args.tuning.split(","))))
    else:
        with Bank(m1[:4096], m2[:4096], **kw) as small:
            small.upload(synth.strain_from_spectrum(w.noise(0), n, w.fs), psd_fin)
            tuning, _ = small.autotune(reps=1)
    # direct launches: a bank this size is thousands of batches, more than a
    # graph is worth capturing for a handful of segments
    bank = Bank(m1, m2, valid=(n // 4, 3 * n // 4), flags=CUI_NO_GRAPH, **kw)
    bank.set_tuning(**tuning)
    ps = Prescreen(n=n, fs=w.fs, f_low=w.f_low, bands=16, frame=n // 256, regions=100, max_batch=1,
                   stream=stream.cuda_stream)
    setup_s = time.perf_counter() - t0
    feat = torch.empty((1, ps.bands, ps.frames), dtype=torch.float32, device="cuda")
    scores = torch.empty((1, ps.regions), dtype=torch.float32, device="cuda")
    psd_h = torch.from_numpy(psd_fin).pin_memory()
    segs = []
    for s in range(args.stream):  # host-side synthesis, outside the timed region
        d = w.noise(s)
        strain = torch.from_numpy(synth.strain_from_spectrum(d, n, w.fs)).pin_memory()
        segs.append(strain)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in segs]
    n_trig = 0
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for strain, (a, b, c) in zip(segs, ev):
        a.record(stream)
        bank.upload(strain.numpy(), psd_h.numpy())
        ps.bank_features(bank, feat)
        ps.scores(feat, scores)
        b.record(stream)
        bank.filter()
        _, nt = bank.triggers(allow_overflow=True)
        c.record(stream)
        n_trig += nt
    torch.cuda.synchronize()
    wall = time.perf_counter() - t1
    pre_ms = sum(a.elapsed_time(b) for a, b, _ in ev)
    filt_ms = sum(b.elapsed_time(c) for _, b, c in ev)
    bank.close()
    line = {"metric": "templates/s sustained over a 50 %-overlap segment stream", "value": w.n_templates * len(segs) / wall,
            "unit": "templates/s", "n_gpus": 1, "segments": len(segs), "data": "synthetic",
            "config": {"workload": w.name, "n": n, "templates": w.n_templates, "f_low": w.f_low,
                       "psd_scale": w.psd_scale, "valid": [n // 4, 3 * n // 4], "tiling": tuning},
            "seconds": wall, "setup_s": setup_s, "upload_plus_prescreen_ms_per_segment": pre_ms / len(segs),
            "filter_ms_per_segment": filt_ms / len(segs), "triggers": n_trig,
            "prescreen": "untrained network (inference cost only; every region is filtered)"}
    print(json.dumps(line), flush=True)
    return 0


def run_extras(args, w):
    """Rates of the steps that follow the filter: cross-template clustering,
    the chi^2 test, the time-domain generator, the band sums and series of the
    multi-band search (all on --workload), then the multi-band hierarchical
    search over one 1024 s segment from 10 Hz (the long-template workload),
    against the exhaustive full-band filter of the same templates."""
    import numpy as np
    import torch

    import synth
    from paper_1006_4644_gb300 import Bank
    from paper_1006_4644_gb300.multiband import hierarchical_search

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()

    def cuda_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, 1e3 * (time.perf_counter() - t0) / reps

    def dev(x):
        x = np.array(x, dtype=np.float64)
        x[0] = 1.0  # bin 0 is never read
        return torch.from_numpy(x).cuda()

    out = {"metric": "rates of the post-filter steps and the multi-band search", "n_gpus": 1, "data": "synthetic"}
    m1, m2 = w.masses()
    psd = w.psd()
    with Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=5.0,
              stream=stream.cuda_stream) as bank:
        strain = torch.from_numpy(build_segment(w, bank, psd)).cuda()
        bank.upload(strain, dev(psd))
        bank.filter()
        trig, total = bank.triggers()
        _, ms = cuda_ms(lambda: bank.clustered_triggers(), 20)
        out["cluster"] = {"ms_per_readout": ms, "triggers": int(total)}
        pick = trig[np.arange(256) % len(trig)]
        ms, _ = cuda_ms(lambda: bank.trigger_chisq(pick, 16), 5)
        out["chisq"] = {"triggers_per_s": 256 / (ms / 1e3), "bands": 16, "triggers_per_call": 256}
        pk = bank.peaks()
        times = pk["sample"] / w.fs
        tm = np.arange(w.n_templates)
        ms, _ = cuda_ms(lambda: bank.band_correlate(tm, times), 5)
        out["band_correlate"] = {"queries_per_s": w.n_templates / (ms / 1e3), "band": "full"}
        series = torch.empty(w.n, dtype=torch.float64, device="cuda")
        ms1, _ = cuda_ms(lambda: bank.band_series(series, 40.0, 0.0, 1), 10)
        ms8, _ = cuda_ms(lambda: bank.band_series(series[: w.n // 8], 0.0, 40.0, 8), 10)
        out["band_series_ms"] = {"decim_1": ms1, "decim_8": ms8}
        hp = torch.empty(w.n, dtype=torch.float64, device="cuda")
        hx = torch.empty(w.n, dtype=torch.float64, device="cuda")
        ms, _ = cuda_ms(lambda: [bank.td_template(t, hp, hx) for t in range(64)], 3)
        out["td_template"] = {"templates_per_s": 64 / (ms / 1e3), "n": w.n, "pn_order": 2.5}

    # multi-band hierarchical search: 256 templates of the long-template
    # workload (f_low 10 Hz, chirps up to ~30 min) over one 1024 s segment
    wl = synth.WORKLOADS["seg1024s_bank1m_et"]
    l1, l2 = wl.masses()
    l1, l2 = l1[:256], l2[:256]
    f_split, ns, valid = 40.0, 1 << 19, (48 * 4096, 1 << 19)
    kw = dict(fs=wl.fs, f_low=wl.f_low, pn_x2=wl.pn_x2, stream=stream.cuda_stream)
    psd_l = wl.psd()
    with Bank(l1, l2, n=wl.n, **kw) as seg, \
            Bank(l1, l2, n=ns, snr_threshold=8.0, valid=valid, **kw) as det:
        d = wl.noise(0)
        seg.upload(torch.from_numpy(synth.strain_from_spectrum(d, wl.n, wl.fs)).cuda(), dev(psd_l))
        sig = seg.sigma()
        h = torch.zeros(wl.n // 2 + 1, dtype=torch.complex64, device="cuda")
        seg.template(0, h)
        j0 = 700 * 4096
        synth.add_signal(d, h.cpu().numpy().astype(np.complex128), 15.0 / sig[0], j0, wl.n)
        strain_l = torch.from_numpy(synth.strain_from_spectrum(d, wl.n, wl.fs)).cuda()
        psd_d, psd_s = dev(psd_l), dev(synth.psd_onesided(ns, wl.fs, wl.psd_scale))
        seg.upload(strain_l, psd_d)
        cand = hierarchical_search(seg, det, f_split, psd_s)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cand = hierarchical_search(seg, det, f_split, psd_s)
        torch.cuda.synchronize()
        t_hier = time.perf_counter() - t0
        ms_full, _ = cuda_ms(lambda: seg.filter(), 2)
        hit = cand[(cand["tmpl"] == 0) & (np.abs(cand["t"] * wl.fs - j0) <= 2)]
        best = hit[np.argmax(hit["rho"])] if len(hit) else None
        zf, sf = seg.band_correlate([0], [best["t"]]) if best is not None else (np.zeros(1), np.ones(1))
        out["hierarchical"] = {
            "workload": f"256 templates of {wl.name}, one {wl.n} sample segment, split at {f_split} Hz, "
                        f"upper band on {ns}-sample segments valid on [{valid[0]}, {valid[1]})",
            "seconds": t_hier, "templates_per_s": 256 / t_hier, "candidates": int(len(cand)),
            "injection_rho": float(best["rho"]) if best is not None else None, "injected_snr": 15.0,
            "injection_rho_full_band_whole_segment": float(abs(zf[0]) / np.sqrt(sf[0])) if best is not None else None,
            "exhaustive_full_band_seconds": ms_full / 1e3,
            "note": "the full-band filter of the 2^22-sample segment wraps every chirp longer than 1024 s"}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--flags", type=int, default=0, help="extra CUI_* flags for the fused path")
    ap.add_argument("--plain-templates", type=int, default=64)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false",
                    help="skip the end-to-end leg (a smaller process for profiler captures)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--tuning", default=None, help="fixed tiling n1,ccols,rpc,batch (skips the autotuner)")
    ap.add_argument("--extras", action="store_true",
                    help="instead of the step benchmark, time clustering, chi^2, the time-domain generator and "
                         "the multi-band search")
    ap.add_argument("--stream", type=int, default=0,
                    help="instead of the step benchmark, stream this many overlapping segments of --workload")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    import synth

    w = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    if args.stream > 0:
        return run_stream(args, w)
    if args.extras:
        return run_extras(args, w)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1006_4644_gb300 import CUI_PLAIN, Bank

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # weak scaling: every rank filters its own bank of the workload's size
    m1, m2 = synth.sample_masses(w.seed, 1 + 7919 * rank, w.n_templates, w.mass_lo, w.mass_hi, w.mass_log)
    psd = w.psd()
    stream = torch.cuda.current_stream()
    bank = Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, flags=args.flags, stream=stream.cuda_stream)
    strain = build_segment(w, bank, psd)
    strain_d = torch.from_numpy(strain).cuda()
    psd_fin = psd.copy()
    psd_fin[0] = 1.0  # bin 0 is never read
    psd_d = torch.from_numpy(psd_fin).cuda()
    peaks_d = torch.empty(w.n_templates * 16, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def step():
        bank.upload(strain_d, psd_d)
        bank.filter(peaks_dev=peaks_d)

    # pick the tiling on this GPU (outside the timed region)
    bank.upload(strain_d, psd_d)
    if args.tuning:
        n1, cc, rpc, bt = (int(x) for x in args.tuning.split(","))
        bank.set_tuning(n1=n1, ccols=cc, rpc=rpc, batch=bt)
        tuning = bank.tuning()
    else:
        tuning, _ = bank.autotune(reps=2) if args.autotune else (bank.tuning(), None)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    lib = bank._l

    def timed(steps, level):
        """Time `steps` steps (L2 flushed between them, outside the intervals)
        with library tracing at `level`: 1 keeps the captured-graph path and
        counts its kernels, 2 launches directly and times every kernel group."""
        bank.trace_read()
        lib.cui_trace_enable(bank._h, level)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        lib.cui_trace_enable(bank._h, 0)
        return sum(a.elapsed_time(b) for a, b in ev), bank.trace_read()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_ms, calls = timed(args.steps, 1)
        # the same steps once more with per-kernel events, for the roofline
        _, trace = timed(args.steps, 2)
    if world > 1:
        dist.barrier()
    launches = sum(v[0] for v in calls.values())
    if world > 1:
        tt = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    value = w.n_templates * args.steps * world / (t_ms / 1e3)

    # roofline of the dominant kernel: algorithmic bytes = one write (pass 1)
    # or one read (pass 2) of the N-point complex64 spectrum per template
    per_tmpl = w.n * (4 if args.flags & 2 else 8)
    p1 = trace.get("pass1", (0, 0, 0.0))
    p2 = trace.get("pass2", (0, 0, 0.0))
    dom, dv = ("pass2", p2) if p2[2] >= p1[2] else ("pass1", p1)
    n_units = w.n_templates * args.steps
    peak, peak_src = measured_hbm()
    achieved = n_units * per_tmpl / (dv[2] / 1e3) / 1e9
    traffic = stored_traffic(dom, w.name)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic * n_units / max(1, dv[1]) if traffic is not None else None,
            "kernel": dom, "peak_source": peak_src,
            "avg_launch_ms": dv[2] / max(1, dv[1]), "templates_per_launch": n_units / max(1, dv[1]),
            "both_passes": {"achieved": n_units * 2 * per_tmpl / ((p1[2] + p2[2]) / 1e3) / 1e9,
                            "frac": n_units * 2 * per_tmpl / ((p1[2] + p2[2]) / 1e3) / 1e9 / peak},
            "kernel_ms": {k: v[2] for k, v in trace.items()}}
    # secondary roof: the transform's 5 N log2 N flops per template (mostly adds
    # that cannot fuse) against one FP32 operation per lane per clock
    flop = 5.0 * w.n * math.log2(w.n) * n_units
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clk_sum = clk.summary()
    mhz = clk_sum["sm_mhz"] if clk_sum else 2070.0  # the median SM clock sampled during the timed steps
    alu_peak = sms * 128 * mhz * 1e6 / 1e12
    roof["alu_secondary"] = {"flop_per_template": 5.0 * w.n * math.log2(w.n),
                             "achieved_tflops": flop / ((p1[2] + p2[2]) / 1e3) / 1e12, "peak_tflops": alu_peak,
                             "frac": flop / ((p1[2] + p2[2]) / 1e3) / 1e12 / alu_peak,
                             "peak_basis": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz "
                                           f"({'median sampled' if clk_sum else 'maximum'} SM clock), "
                                           "one add per lane per clock"}

    # end to end through the public API with pinned host buffers
    e2e = None
    if args.e2e:
        e2e = e2e_leg(w, m1, m2, strain, psd_fin, tuning, args, stream)

    plain, plain_peaks = None, None
    if args.plain_templates > 0:
        plain, plain_peaks = plain_leg(w, m1, m2, strain_d, psd_d, args, stream, value)

    cpu, acc = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        bank.upload(strain_d, psd_d)
        bank.filter()
        gpu_peaks = bank.peaks()
        cpu = cpu_baseline(w, strain=strain)
        acc = accuracy(gpu_peaks, cpu)
        if plain is not None:  # the plain path at equal accuracy: its peaks against the same oracle results
            plain["accuracy"] = accuracy(plain_peaks, cpu, only=set(range(plain["templates"])))
        for k in ("seconds", "results", "templates"):
            cpu.pop(k, None)

    bank.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "n": w.n, "fs": w.fs, "templates_per_gpu": w.n_templates,
                           "pn_order": w.pn_x2 / 2, "f_low": w.f_low, "mass_range": [w.mass_lo, w.mass_hi],
                           "injections": w.n_inj, "l2": "flushed between steps (256 MiB write)",
                           "phase": "fp64 anchors + fp32 cubic" if args.flags & 1 else "double-float anchors + fp32 cubic",
                           "storage": "bf16x2" if args.flags & 2 else "complex64",
                           "parallelism": f"bank replicas x{world}", "tiling": tuning},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "plain": plain, "accuracy": acc, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def e2e_leg(w, m1, m2, strain, psd_fin, tuning, args, stream):
    """The same metric end to end through the public API: every step uploads
    the strain and PSD from pinned host memory and reads peaks and triggers
    back (cui_results)."""
    import torch

    from paper_1006_4644_gb300 import Bank

    strain_h = torch.from_numpy(strain).pin_memory()
    psd_h = torch.from_numpy(psd_fin).pin_memory()
    e2e_steps = max(3, args.steps // 2)
    bank2 = Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, flags=args.flags, stream=stream.cuda_stream)
    bank2.set_tuning(**tuning)
    n_trig = 0

    def e2e_step():
        nonlocal n_trig
        bank2.upload(strain_h.numpy(), psd_h.numpy())
        bank2.filter()
        _, tr, n_trig = bank2.results()

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": w.n_templates * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": w.n * 8 + (w.n // 2 + 1) * 8,
           # peaks, the count, and the trigger prefix the read-out stages (at least 1024 records,
           # twice the previous count; the count is the same every step here)
           "d2h_bytes_per_step": w.n_templates * 16 + 8 + min(1 << 20, max(1024, 2 * n_trig)) * 24}
    bank2.close()
    return e2e


def plain_leg(w, m1, m2, strain_d, psd_d, args, stream, value):
    """The plain per-template FP32 path on a subset of the bank, same segment."""
    import numpy as np
    import torch

    from paper_1006_4644_gb300 import CUI_PLAIN, Bank

    npl = min(args.plain_templates, w.n_templates)
    pb = Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, flags=CUI_PLAIN, stream=stream.cuda_stream)
    pb.upload(strain_d, psd_d)
    order = np.arange(npl)
    pb.filter(order)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    reps = 3
    for _ in range(reps):
        pb.upload(strain_d, psd_d)
        pb.filter(order)
    b.record(stream)
    torch.cuda.synchronize()
    pv = npl * reps / (a.elapsed_time(b) / 1e3)
    peaks = pb.peaks()
    pb.close()
    return {"value": pv, "unit": UNIT, "templates": npl, "mixed_over_plain": value / pv}, peaks


if __name__ == "__main__":
    sys.exit(main())
