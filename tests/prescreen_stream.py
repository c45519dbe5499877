"""The learned prescreen on the third-generation stream workload (run on a GPU
box; not collected by pytest):

    python tests/prescreen_stream.py [--train 8192] [--test 16] [--stream 3] [--epochs 20] [--out FILE]

Workload seg1024s_bank1m_et: 10^6 3.5PN templates (masses log-uniform in
[1, 50] Msun, f_low 10 Hz), 1024 s segments (N = 2^22 at 4096 Hz), the
analytic PSD scaled by 1e-4.  A three-network ensemble is trained on the GPU
with oracle-made segments at N = 2^22 (one injection each, SNR uniform in
[6, 20], masses from the bank's range), labelled with the injected chirp
mass's region (1 of 100 equal-count regions of the 10^6-template bank, 0.5
on its neighbours).  Held-out segments are judged by the exhaustive bank: K*
is the fewest top-scored regions that miss none of the injections it detects
at rho >= 8 within 1 s.  Then a stream of overlapping segments (each keeping
triggers in its middle half) is filtered twice, exhaustively and by
prescreen + top-K*, and both sustained rates are reported in one JSON line.
Every step runs through the library: features, standardisation, training,
ensemble scores, region plan, filter.
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import prescreen as ops  # noqa: E402
from prescreen_data import make_segments_mp  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=8192)
    ap.add_argument("--test", type=int, default=16)
    ap.add_argument("--stream", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--ensemble", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()

    import multiprocessing as mp

    procs = len(os.sched_getaffinity(0))
    pool = mp.get_context("spawn").Pool(procs)  # started before the first GPU call

    import torch

    from paper_1006_4644_gb300 import Bank, Prescreen, Regions, build, ensemble_scores
    from paper_1006_4644_gb300._lib import CUI_NO_GRAPH

    build.build()
    w = synth.WORKLOADS["seg1024s_bank1m_et"]
    n, fs, f_low, R, W = w.n, w.fs, w.f_low, 100, int(w.fs)
    psd = w.psd()
    psd_fin = psd.copy()
    psd_fin[0] = 1.0
    psd_d = torch.from_numpy(psd_fin).cuda()
    m1, m2 = w.masses()
    groups, bounds = ops.regions_of_bank(m1, m2, R)
    region_of_tmpl = np.empty(len(m1), dtype=np.int64)
    for r, g in enumerate(groups):
        region_of_tmpl[g] = r
    rep = {"workload": w.name, "n": n, "templates": len(m1), "regions": R, "train": args.train, "test": args.test,
           "epochs": args.epochs, "ensemble": args.ensemble, "seed": args.seed, "host_procs": procs}
    nets = [Prescreen(n=n, fs=fs, f_low=f_low, bands=16, frame=n // 256, regions=R, max_batch=args.batch,
                      lr=args.lr, seed=args.seed + e) for e in range(args.ensemble)]
    p = nets[0]

    def segments(start, count, keep=False):
        X, Y, D, M = [], [], [], []
        for s0 in range(start, start + count, 64):
            d, y, meta = make_segments_mp(11, s0, min(64, start + count - s0), n, fs, f_low, psd, bounds, R,
                                          mass=(1.0, 50.0), pool=pool)
            out = torch.zeros((len(d), p.bands, p.frames), dtype=torch.float32, device="cuda")
            p.features(torch.from_numpy(d).cuda(), psd_d, out)
            X.append(out)
            Y.append(torch.from_numpy(y).cuda())
            M += meta
            if keep:
                D.append(d)
        return torch.cat(X), torch.cat(Y), (np.concatenate(D) if keep else None), M

    t0 = time.perf_counter()
    xtr, ytr, _, _ = segments(0, args.train)
    rep["data_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    for net in nets:
        net.fit_norm(xtr)
        g = torch.Generator(device="cpu").manual_seed(0)
        for epoch in range(args.epochs):
            perm = torch.randperm(len(xtr), generator=g).cuda()
            for i in range(0, len(xtr) - args.batch + 1, args.batch):
                idx = perm[i:i + args.batch]
                net.train_step(xtr[idx].contiguous(), ytr[idx].contiguous(), want_loss=False)
    torch.cuda.synchronize()
    rep["train_s"] = time.perf_counter() - t0
    del xtr, ytr

    xte, yte, dte, meta = segments(50_000_000, args.test, keep=True)
    probs = torch.zeros((len(xte), R), dtype=torch.float32, device="cuda")
    ensemble_scores(nets, xte, probs)
    sc = probs.cpu().numpy()
    true = yte.argmax(dim=1).cpu().numpy()
    rep["recall_at"] = {k: float(np.mean([t in np.argsort(-s)[:k] for t, s in zip(true, sc)])) for k in (1, 5, 10, 20)}

    stream = torch.cuda.current_stream()
    kw = dict(n=n, fs=fs, f_low=f_low, pn_x2=w.pn_x2, stream=stream.cuda_stream)
    with Bank(m1[:4096], m2[:4096], **kw) as small:  # the tiling, tuned on a sample of the bank
        small.upload(synth.strain_from_spectrum(w.noise(0), n, fs), psd_fin)
        tuning, _ = small.autotune(reps=1)
    rep["tiling"] = tuning
    plan = Regions(m1, m2, R)
    rng = np.random.default_rng(0)
    k_net, k_rand = [], []
    cap = 1 << 23  # room for every trigger of a loud injection across the bank
    with Bank(m1, m2, snr_threshold=6.0, window=W, flags=CUI_NO_GRAPH, trigger_capacity=cap, **kw) as bank:
        bank.set_tuning(**tuning)
        t0 = time.perf_counter()
        for i, mt in enumerate(meta):
            bank.upload(synth.strain_from_spectrum(dte[i], n, fs), psd_fin)
            bank.filter()
            tr, total = bank.triggers(capacity=cap, allow_overflow=True)
            assert total <= cap, total
            dist = np.abs(tr["sample"] - mt["j0"])
            near = tr[np.minimum(dist, n - dist) <= W]
            reg = np.zeros(R)
            if len(near):
                np.maximum.at(reg, region_of_tmpl[near["tmpl"]], near["snr"])
            if reg.max() < 8.0:
                continue
            hit = reg >= 8.0
            k_net.append(int(np.argmax(hit[np.argsort(-sc[i], kind="stable")])) + 1)
            k_rand.append(int(np.argmax(hit[rng.permutation(R)])) + 1)
        rep["judge_s"] = time.perf_counter() - t0
        rep["detectable"] = len(k_net)
        rep["K_per_detectable"] = k_net
        k_star = int(max(k_net)) if k_net else R
        rep["K_star"] = k_star
        rep["K_star_random_order"] = int(max(k_rand)) if k_rand else R

    # the stream: overlapping segments keeping triggers in [N/4, 3N/4), filtered
    # exhaustively and by prescreen + top-K* (segments drawn independently)
    segs = [torch.from_numpy(synth.strain_from_spectrum(w.noise(s), n, fs)).pin_memory()
            for s in range(args.stream)]
    psd_h = torch.from_numpy(psd_fin).pin_memory()
    feat1 = torch.zeros((1, p.bands, p.frames), dtype=torch.float32, device="cuda")
    prob1 = torch.zeros((1, R), dtype=torch.float32, device="cuda")
    rates = {}
    with Bank(m1, m2, valid=(n // 4, 3 * n // 4), flags=CUI_NO_GRAPH, **kw) as bank:
        bank.set_tuning(**tuning)
        for mode in ("exhaustive", "prescreen"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for strain in segs:
                bank.upload(strain.numpy(), psd_h.numpy())
                if mode == "exhaustive":
                    bank.filter()
                else:
                    p.bank_features(bank, feat1)
                    ensemble_scores(nets, feat1, prob1)
                    bank.filter(plan.order(prob1.cpu().numpy()[0], k_star))
                bank.triggers(allow_overflow=True)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            rates[mode] = {"seconds": el, "segments": len(segs),
                           "templates_per_s": len(m1) * len(segs) / el}
    rep["stream"] = rates
    rep["speedup"] = rates["exhaustive"]["seconds"] / rates["prescreen"]["seconds"]
    for q in nets:
        q.close()
    pool.close()
    pool.join()
    line = json.dumps(rep)
    print(line)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(line + "\n")


if __name__ == "__main__":
    main()
