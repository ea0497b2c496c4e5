#!/usr/bin/env python
"""Benchmark of the FB-LISA hot path on GB300: prints ONE JSON line.

The contract line's step is the metric's own quantity, "GUPS fwd+back at
512^3 / 720 views": one forward projection A x of all 720 views (K1, 768x768
detector, N samples per ray) and one backprojection A^T y of all 720 views
(K2, N^3 voxel-views per view), both through the C ABI on buffers resident in
HBM.  value = (720 nu nv N + 720 N^3) / step time.  Beside it:

  fblisa_iteration   one FB-LISA iteration (Algorithm 1, Steps 2a-2d: the
                     mini-batch, the residual projection and f_N(x), the
                     gradient backprojection, the backtracking loop of prox +
                     trial objective until (2.3) holds) on 40-view
                     mini-batches, with the rooflines of K1, K2 and K3;
  time_to_objective  the metric's second part: wall time to the plain FP32
                     method's objective within 1e-3, for learned proposal +
                     BF16 + graph and for each of the three alone;
  c2                 the 256^3 Poisson configuration run for its 20 epochs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the method does not shard here; each rank runs an independent
replica (replicas only), value = all ranks' units / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GUPS fwd+back at 512^3/720 views; FB-LISA time-to-1e-3 rel-err vs plain FP32"
UNIT = "GUPS"
# Algorithmic FP32 operations.  A Joseph sample of K1 (one ray, one plane):
# 3 linear interpolations of 2 operations, 1 accumulation and the 2
# coordinate steps along the ray, plus the 2 fractions of the crossing (10).
# Each in-volume sample is 4 nonzeros of A; the transpose costs, per nonzero,
# its vertical weight (1 - f or f of the row's crossing), its product with
# the in-plane weight, the accumulation and the step to the next row (4), so
# 16 per in-volume sample, whatever order K2 visits them in.
K1_OPS_PER_SAMPLE = 10
K2_OPS_PER_SAMPLE = 16
K3_BYTES_PER_VOXEL = 12  # read x and g, write x_bar (FP32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c3_512")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--iter-steps", type=int, default=10, help="timed FB-LISA iterations (fblisa_iteration)")
    ap.add_argument("--c2", type=int, default=1, help="also run the 256^3 Poisson configuration (20 epochs)")
    ap.add_argument("--tto-decompose", type=int, default=1,
                    help="time-to-objective also for the learned proposal, BF16 and graph alone")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", type=int, default=1, help="also time BF16/FP16 storage")
    ap.add_argument("--variant-steps", type=int, default=5)
    ap.add_argument("--tto-epochs", type=int, default=10,
                    help="epochs of plain FP32 that define F* (0: skip time-to-objective)")
    ap.add_argument("--tto-check", type=int, default=3, help="iterations between F evaluations")
    ap.add_argument("--batched", type=int, default=1, help="also time the 16-volume batched launch")
    ap.add_argument("--launch", default=None,
                    help="k1_cols,k1_split,k2_vpl for the timed FP32 run instead of the autotuned ones")
    ap.add_argument("--comparators", type=int, default=0,
                    help="also run the paper's comparison: FB, full-batch and mini-batch FB-LISA (2+ min)")
    ap.add_argument("--paper-cases", type=int, default=0,
                    help="also run the paper-shaped 560^3 cases with RE / PSNR over time (several minutes)")
    ap.add_argument("--paper-mu-sweep", type=int, default=0,
                    help="also sweep mu = c * max(A^T b) on the paper-shaped case 2 (about two minutes)")
    ap.add_argument("--paper-mu-fraction", type=float, default=None,
                    help="with --paper-cases: mu = (2c, c, c) * max(A^T b) instead of the paper's 2 / 1 / 1")
    ap.add_argument("--c5b", type=int, default=0,
                    help="also time the 1024^3 / 1440-view FP16 configuration (a few minutes more)")
    ap.add_argument("--tv-only", type=int, default=0,
                    help="time only prox_tv (20 FGP iterations) on the phantom of --workload (--steps calls)")
    ap.add_argument("--kernels-only", type=int, default=0,
                    help="run only the hot kernels of one mini-batch of --workload (profiler captures)")
    ap.add_argument("--fdk-only", type=int, default=0,
                    help="time only FDK over all views of --workload (--steps reconstructions after one warm-up)")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def batched_record(fbl, device, wls, label, proposal=False, steps=5, warmup=3):
    """Uneven volumes in one batch: one fblisa_batch_step per iteration of all
    volumes (persistent launches, one graph) against the same iterations run
    volume after volume by graph-mode single-volume solvers, FP32.  Every
    geometry is tuned once; the batch takes the largest volume's columns per
    block and each volume's own plane-loop form and voxels per lane, and the
    single-volume solvers run on exactly the same configurations."""
    import torch
    stream = torch.cuda.current_stream(device)
    data = [make_data(fbl, wl, device) for wl in wls]
    Gs = [d[0] for d in data]
    bs = [d[2] for d in data]
    big = max(range(len(wls)), key=lambda q: wls[q].geom.n_vox)
    tunes = [fbl.geometry_autotune(G, fbl.F32, wl.N0) for G, wl in zip(Gs, wls)]
    cols = tunes[big]["k1_cols"]
    for G, t in zip(Gs, tunes):
        fbl.geometry_set_launch(G, cols, t["k1_split"], t["k2_vpl"])
    net = None
    if proposal:
        from paper_2605_12085_gb300 import proposal as prop
        net, _ = prop.load()

    def params(wl, **kw):
        return fbl.params_default(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0, seed=wl.seed_batches, **kw)

    def timed(step_fn):
        for _ in range(warmup):
            step_fn()
        torch.cuda.synchronize(device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        recs = [step_fn() for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize(device)
        return e0.elapsed_time(e1) / steps, recs

    B = fbl.fblisa_batch_create(Gs, [params(wl) for wl in wls])
    if net is not None:
        B.set_proposal(net)
    xs = [torch.zeros(wl.geom.vol_shape, dtype=torch.float32, device=device) for wl in wls]
    launches0 = B.info()["launches"]
    b_ms, b_recs = timed(lambda: B.step(xs, bs))
    b_launches = (B.info()["launches"] - launches0) / (warmup + steps)
    units = sum(step_units(st, wl.geom) for rec in b_recs for st, wl in zip(rec, wls)) / steps
    del B, xs
    Ss = [fbl.fblisa_create(G, params(wl, use_graph=1)) for G, wl in zip(Gs, wls)]
    if net is not None:
        for S in Ss:
            S.set_proposal(net)
    xs = [torch.zeros(wl.geom.vol_shape, dtype=torch.float32, device=device) for wl in wls]
    s_ms, s_recs = timed(lambda: [S.step(x, b) for S, x, b in zip(Ss, xs, bs)])
    s_units = sum(step_units(st, wl.geom) for rec in s_recs for st, wl in zip(rec, wls)) / steps
    del Ss, xs, data, Gs, bs
    return {"workload": label, "step_rule": "learned proposal" if proposal else "plain (alpha_0 reset)",
            "batched_ms_per_iteration": b_ms, "batched_gups": units / (b_ms * 1e-3) / 1e9,
            "batched_launches_per_iteration": b_launches,
            "sequential_ms_per_iteration": s_ms, "sequential_gups": s_units / (s_ms * 1e-3) / 1e9,
            "speedup": s_ms / b_ms, "steps": steps, "warmup": warmup,
            "launch_config": {"k1_cols": cols, "k1_split": [t["k1_split"] for t in tunes],
                              "k2_vpl": [t["k2_vpl"] for t in tunes]},
            "backtracks_per_volume_iteration":
                statistics.mean(st["backtracks"] for rec in b_recs for st in rec)}


def c5b_record(fbl, device, steps=5, warmup=2):
    """The large configuration: 1024^3 volume, 1440 views, 1536^2 detector,
    60-view mini-batches; FP16 storage (FP32 accumulation, FP64 line-search
    sums) with the learned step proposal and graph-captured iterations, next
    to plain FP16 and plain FP32 iterations of the same problem."""
    import torch
    import synth
    from paper_2605_12085_gb300 import proposal as prop
    wl = synth.WORKLOADS["c5b_1024"]
    g = wl.geom
    G, xt, b = make_data(fbl, wl, device)
    del xt
    tune = fbl.geometry_autotune(G, fbl.F16, wl.N0)
    net, _ = prop.load()
    stream = torch.cuda.current_stream(device)
    out = {"workload": "c5b_1024: 1024^3 volume, 1440 views, 1536x1536 detector, mini-batch 60 views",
           "autotune_f16": tune}
    for name, code, td, learned, graph in (("f16_learned_graph", fbl.F16, torch.float16, True, 1),
                                           ("f16_plain", fbl.F16, torch.float16, False, 0),
                                           ("f32_plain", fbl.F32, torch.float32, False, 0)):
        bv = b if code == fbl.F32 else b.to(td)
        p = fbl.params_default(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0, seed=wl.seed_batches,
                               x_dtype=code, b_dtype=code, use_graph=graph)
        S = fbl.fblisa_create(G, p)
        if learned:
            S.set_proposal(net)
        x = torch.zeros(g.vol_shape, dtype=td, device=device)
        for _ in range(warmup):
            S.step(x, bv)
        torch.cuda.synchronize(device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = [S.step(x, bv) for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize(device)
        ms = e0.elapsed_time(e1) / steps
        units = sum(step_units(r, g) for r in st) / steps
        out[name] = {"ms_per_iteration": ms, "gups": units / (ms * 1e-3) / 1e9,
                     "trials_per_iteration": statistics.mean(r["backtracks"] + 1 for r in st),
                     "steps": steps, "warmup": warmup}
        del S, x
        if bv is not b:
            del bv
        torch.cuda.empty_cache()
    del b, G
    torch.cuda.empty_cache()
    return out


def comparators_record(fbl, device, budget_s=30.0):
    """The paper's comparison (Sec. 3) on the 512^3 workload, each method for a
    fixed budget of GPU time (sum of CUDA-event step times; F and RE are
    evaluated off the clock): deterministic forward-backward (full batch,
    constant step 0.9/L, L = ||A||^2 by power iteration), FB-LISA with the full
    batch, FB-LISA with 40-view mini-batches (plain FP32), and the fast
    configuration (learned proposal + BF16 + graph)."""
    import torch
    import synth
    from paper_2605_12085_gb300 import proposal as prop
    wl = synth.WORKLOADS["c3_512"]
    g = wl.geom
    G, xt, b = make_data(fbl, wl, device)
    fbl.geometry_autotune(G, fbl.F32, wl.N0)
    xt_d = torch.from_numpy(xt).to(device)
    stream = torch.cuda.current_stream(device)
    views = list(range(g.n_views))
    # L by power iteration on A^T A over all views
    v = torch.ones(g.vol_shape, dtype=torch.float32, device=device)
    y = torch.empty((g.n_views, g.nv, g.nu), dtype=torch.float32, device=device)
    lam = 0.0
    for _ in range(12):
        fbl.project(G, v, views, y=y)
        w = fbl.backproject(G, y, views)
        lam = float(torch.linalg.vector_norm(w) / torch.linalg.vector_norm(v))
        v = w / torch.linalg.vector_norm(w)
    del y, v, w
    L = lam * 1.02
    net, _ = prop.load()
    b16 = b.to(torch.bfloat16)

    def run(params, fast=False, check_every=1):
        S = fbl.fblisa_create(G, params)
        if fast:
            S.set_proposal(net, margin=0.25)
        x = torch.zeros(g.vol_shape, dtype=torch.bfloat16 if fast else torch.float32, device=device)
        bb = b16 if fast else b
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        el, k, hist = 0.0, 0, []
        F0, _, re0 = fbl.evaluate(G, x.float(), b, wl.mu, x_true=xt_d)
        hist.append((0.0, 0, F0, re0))
        while el < budget_s and k < 2000:
            e0.record(stream)
            S.step(x, bb)
            e1.record(stream)
            torch.cuda.synchronize(device)
            el += e0.elapsed_time(e1) * 1e-3
            k += 1
            if k % check_every == 0:
                F, _, re = fbl.evaluate(G, x.float(), b, wl.mu, x_true=xt_d)
                hist.append((el, k, F, re))
        return hist

    base = dict(beta=0.5, mu=wl.mu, seed=wl.seed_batches)
    runs = {
        "fb_fixed_full_batch": run(fbl.params_default(alpha0=0.9 / L, N0=g.n_views, fixed_step=1, **base)),
        "fblisa_full_batch": run(fbl.params_default(alpha0=1e-3, N0=g.n_views, **base)),
        "fblisa_minibatch_fp32": run(fbl.params_default(alpha0=1e-3, N0=wl.N0, **base), check_every=5),
        "fblisa_fast": run(fbl.params_default(alpha0=1e-3, N0=wl.N0, x_dtype=fbl.BF16, b_dtype=fbl.BF16,
                                              use_graph=1, proposal=1, **base), fast=True, check_every=5),
    }
    # target: the mini-batch FP32 method's objective after 10 epochs (180 iterations)
    mb = runs["fblisa_minibatch_fp32"]
    F_star = next((h[2] for h in mb if h[1] >= 180), mb[-1][2])
    out = {"workload": "c3_512", "budget_s_per_method": budget_s, "L_estimate": L,
           "fb_step": 0.9 / L, "F_star_minibatch_10_epochs": F_star}
    for name, h in runs.items():
        at = {}
        for t in (5.0, 10.0, 20.0, budget_s):
            last = [r for r in h if r[0] <= t]
            at["%gs" % t] = {"F": last[-1][2], "rel_error": last[-1][3], "iterations": last[-1][1]}
        hit = next((r for r in h if r[2] <= F_star * (1 + 1e-3)), None)
        out[name] = {"at": at, "time_to_F_star_1e-3_s": hit[0] if hit else None,
                     "iterations_run": h[-1][1], "final_F": h[-1][2], "final_rel_error": h[-1][3]}
    del G, b, b16, xt_d
    torch.cuda.empty_cache()
    return out


def mu_max(fbl, G, g, b):
    """max_j (A^T b)_j over all views: for R = mu ||x||_1 + indicator{x >= 0},
    x = 0 minimises (2.1) exactly when mu >= this value, so mu is read as a
    fraction of it (the paper's mu values belong to its own data scaling)."""
    return float(fbl.backproject(G, b, list(range(g.n_views))).max())


def paper_mu_sweep_record(fbl, device, budget_s=15.0, fractions=(1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2)):
    """Case 2 in shape (560^3, 36 views, 2% noise): plain FP32 FB-LISA for
    budget_s of GPU time at mu = c * max(A^T b) for each fraction c; the final
    and the best relative error to the phantom, the final F, and the share of
    zero voxels.  The fraction whose final error is smallest is the reading
    used for the paper-shaped cases."""
    import torch
    import synth
    wl = synth.WORKLOADS["case2_560"]
    g = wl.geom
    G, xt, b = make_data(fbl, wl, device)
    fbl.geometry_autotune(G, fbl.F32, wl.N0)
    xt_d = torch.from_numpy(xt).to(device)
    mmax = mu_max(fbl, G, g, b)
    stream = torch.cuda.current_stream(device)
    out = {"workload": "case2_560", "budget_s": budget_s, "mu_max": mmax, "runs": []}
    for c in fractions:
        mu = c * mmax
        S = fbl.fblisa_create(G, fbl.params_default(alpha0=1e-3, beta=0.5, mu=mu, N0=wl.N0, seed=wl.seed_batches))
        x = torch.zeros(g.vol_shape, dtype=torch.float32, device=device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        el, k, best = 0.0, 0, (float("inf"), 0)
        while el < budget_s and k < 5000:
            e0.record(stream)
            S.step(x, b)
            e1.record(stream)
            torch.cuda.synchronize(device)
            el += e0.elapsed_time(e1) * 1e-3
            k += 1
            if k % 10 == 0:
                re = float(torch.linalg.vector_norm(x - xt_d) / torch.linalg.vector_norm(xt_d))
                best = min(best, (re, k))
        F, _, re = fbl.evaluate(G, x, b, mu, x_true=xt_d)
        out["runs"].append({"fraction": c, "mu": mu, "iterations": k, "final_rel_error": re, "F": F,
                            "best_rel_error": min(best[0], re), "best_at_iteration": best[1],
                            "zero_share": float((x == 0).float().mean())})
        del S, x
    out["chosen_fraction"] = min(out["runs"], key=lambda r: r["final_rel_error"])["fraction"]
    del G, b, xt_d
    torch.cuda.empty_cache()
    return out


def paper_cases_record(fbl, device, budget_s=30.0, mu_fraction=None):
    """The paper's three cases (Sec. 3) in shape on seeded phantoms (the walnut
    data are not available): 560^3, 36 / 36 / 72 views, 840^2 detector,
    N_0 = 8, alpha_0 = 1e-3, mu = 2 / 1 / 1 -- or, with mu_fraction c, the
    data-scaled reading mu = (2c, c, c) * max(A^T b) of the case's data, so that
    the three cases keep the paper's ratio.  Each method runs for budget_s of
    GPU time: plain FB-LISA (FP32), the fast configuration, and constant-step
    FB on the full batch (step 0.9/L).  Reported: RE = ||x - x_true|| /
    ||x_true|| and PSNR = 10 log10(max(x_true)^2 / MSE) at fixed times and at
    iterations 120 and 240 (the paper's 120 s / 240 s budgets ran at about one
    iteration per second), and the best RE seen.  Also FDK on the case's
    views (time, RE, PSNR) and plain FB-LISA started from that FDK volume."""
    import math
    import torch
    import synth
    from paper_2605_12085_gb300 import proposal as prop
    net, _ = prop.load()
    stream = torch.cuda.current_stream(device)
    out = {"budget_s_per_method": budget_s, "mu_fraction": mu_fraction}
    for case in ("case1_560", "case2_560", "case3_560"):
        wl = synth.WORKLOADS[case]
        g = wl.geom
        G, xt, b = make_data(fbl, wl, device)
        fbl.geometry_autotune(G, fbl.F32, wl.N0)
        mu = wl.mu
        if mu_fraction is not None:
            mmax = mu_max(fbl, G, g, b)
            mu = (2.0 if case == "case1_560" else 1.0) * mu_fraction * mmax
        xt_d = torch.from_numpy(xt).to(device)
        peak2 = float(xt.max()) ** 2
        xt_n2 = float((xt.astype("float64") ** 2).sum())
        views = list(range(g.n_views))
        v = torch.ones(g.vol_shape, dtype=torch.float32, device=device)
        lam = 0.0
        for _ in range(12):
            w = fbl.backproject(G, fbl.project(G, v, views), views)
            lam = float(torch.linalg.vector_norm(w) / torch.linalg.vector_norm(v))
            v = w / torch.linalg.vector_norm(w)
        del v, w
        L = lam * 1.02
        b16 = b.to(torch.bfloat16)

        def psnr(re):
            mse = re * re * xt_n2 / g.n_vox
            return 10.0 * math.log10(peak2 / mse) if mse > 0 else float("inf")

        # FDK on the case's (undersampled) views: the paper's analytic baseline,
        # and a warm start for FB-LISA
        x_fdk = fbl.fdk(G, b, views)
        torch.cuda.synchronize(device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fbl.fdk(G, b, views, x=x_fdk)
        e1.record(stream)
        torch.cuda.synchronize(device)
        re_fdk = float(torch.linalg.vector_norm(x_fdk - xt_d) / torch.linalg.vector_norm(xt_d))
        fdk_rec = {"ms": e0.elapsed_time(e1), "rel_error": re_fdk, "psnr_db": None}

        def run(params, fast=False, x0=None):
            S = fbl.fblisa_create(G, params)
            if fast:
                S.set_proposal(net, margin=0.25)
            x = torch.zeros(g.vol_shape, dtype=torch.bfloat16 if fast else torch.float32, device=device)
            if x0 is not None:
                x.copy_(x0)
            bb = b16 if fast else b
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            el, k, hist, stopped = 0.0, 0, [], None
            while el < budget_s and k < 5000:
                e0.record(stream)
                try:
                    S.step(x, bb)
                except fbl.FblError as ex:
                    # e.g. no trial passes (2.3) within the backtrack cap: the
                    # solver keeps x; the method stops here
                    torch.cuda.synchronize(device)
                    stopped = {"iteration": k + 1, "seconds": el, "error": str(ex)}
                    F, _, re = fbl.evaluate(G, x.float(), b, mu, x_true=xt_d)
                    hist.append((el, k, F, re))
                    break
                e1.record(stream)
                torch.cuda.synchronize(device)
                el += e0.elapsed_time(e1) * 1e-3
                k += 1
                if k % 10 == 0 or k in (120, 240):
                    F, _, re = fbl.evaluate(G, x.float(), b, mu, x_true=xt_d)
                    hist.append((el, k, F, re))
            rec = {"iterations": k, "ms_per_iteration": 1e3 * el / max(k, 1)}
            if stopped:
                rec["stopped"] = stopped
            for t in (budget_s / 4, budget_s / 2, budget_s):
                last = [h for h in hist if h[0] <= t]
                if last:
                    rec["at_%gs" % t] = {"rel_error": last[-1][3], "psnr_db": psnr(last[-1][3]),
                                         "F": last[-1][2], "iterations": last[-1][1]}
            for it in (120, 240):
                h = next((h for h in hist if h[1] == it), None)
                if h:
                    rec["at_iteration_%d" % it] = {"rel_error": h[3], "psnr_db": psnr(h[3]), "F": h[2],
                                                   "seconds": h[0]}
            if hist:
                best = min(hist, key=lambda h: h[3])
                rec["best"] = {"rel_error": best[3], "psnr_db": psnr(best[3]), "iterations": best[1],
                               "seconds": best[0]}
            return rec

        base = dict(beta=0.5, mu=mu, seed=wl.seed_batches)
        out[case] = {
            "views": g.n_views, "mu": mu, "noise_rel": wl.noise_rel, "L_estimate": L,
            "fblisa_fp32": run(fbl.params_default(alpha0=1e-3, N0=wl.N0, **base)),
            "fblisa_fast": run(fbl.params_default(alpha0=1e-3, N0=wl.N0, x_dtype=fbl.BF16, b_dtype=fbl.BF16,
                                                  use_graph=1, proposal=1, **base), fast=True),
            "fb_fixed_full_batch": run(fbl.params_default(alpha0=0.9 / L, N0=g.n_views, fixed_step=1, **base)),
            "fdk": dict(fdk_rec, psnr_db=psnr(re_fdk)),
            "fblisa_fp32_from_fdk": run(fbl.params_default(alpha0=1e-3, N0=wl.N0, **base), x0=x_fdk),
        }
        del G, b, b16, xt_d, x_fdk
        torch.cuda.empty_cache()
    return out


def batched_records(fbl, device):
    import synth
    c5a = ("c5a: 16 volumes N_i = round(96 + 224 i/15) (96^3..320^3), 120 + 24 i views, "
           "detector ceil(1.5 N_i)^2, N_0 = ceil(views/12)")
    small = ("c5s: 16 volumes N_i = round(24 + 56 i/15) (24^3..80^3), 30 + 6 i views, "
             "detector ceil(1.5 N_i)^2, N_0 = ceil(views/12)")
    return {"c5a_plain": batched_record(fbl, device, synth.batched_workloads(), c5a),
            "c5a_learned": batched_record(fbl, device, synth.batched_workloads(), c5a, proposal=True),
            "c5s_plain": batched_record(fbl, device, synth.batched_small_workloads(), small)}


def fdk_record(fbl, G, g, b, xt, device, reps=2):
    """FDK over all views of the workload (the paper's analytic baseline):
    time per reconstruction (CUDA events, one warm-up), voxel-views per second,
    and its relative error against the phantom."""
    import torch
    stream = torch.cuda.current_stream(device)
    views = list(range(g.n_views))
    x = torch.empty(g.vol_shape, dtype=torch.float32, device=device)
    fbl.fdk(G, b, views, x=x)
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fbl.fdk(G, b, views, x=x)
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms = e0.elapsed_time(e1) / reps
    xt_d = torch.from_numpy(xt).to(device)
    re = float(torch.linalg.vector_norm(x - xt_d) / torch.linalg.vector_norm(xt_d))
    del x, xt_d
    return {"views": g.n_views, "ms": ms, "gups_voxel_views": float(g.n_views) * g.n_vox / (ms * 1e-3) / 1e9,
            "rel_error_vs_phantom": re}


def regularisers_record(fbl, G, g, b, xt, device, peaks, iters=4):
    """The other regularisers at the workload's size: prox_tv alone (20 FGP
    iterations on a volume, its algorithmic HBM bytes: 24 B/voxel to start the
    dual, 72 B/voxel per iteration (20 for y = P_C(b - lam K^T r), 52 for the
    dual step), 20 B/voxel for the result) against the measured copy
    bandwidth; and FB-LISA iterations with R = mu||x||_1 + box and with
    R = mu TV + box (10 FGP iterations per prox), ms per iteration from CUDA
    events, beside the paper's R."""
    import torch
    stream = torch.cuda.current_stream(device)
    n = g.n_vox
    v = torch.from_numpy(xt).to(device)
    q = torch.zeros((3,) + tuple(v.shape), dtype=torch.float32, device=device)
    xo = torch.empty_like(v)
    fgp = 20
    for _ in range(2):
        fbl.prox_tv(v, 0.01, fgp, q=q, x=xo)
    torch.cuda.synchronize(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        fbl.prox_tv(v, 0.01, fgp, q=q, x=xo)
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms = e0.elapsed_time(e1) / reps
    byt = float(n) * (24 + 72 * fgp + 20)
    gbs = byt / (ms * 1e-3) / 1e9
    tv_x = fbl.tv_norm(v)
    del q, xo
    out = {"prox_tv": {"voxels": n, "fgp_iterations": fgp, "ms": ms, "algorithmic_bytes": byt,
                       "achieved_gbs": gbs, "peak_gbs": peaks.get("hbm_gbs"),
                       "frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None},
           "tv_of_phantom": tv_x}
    x_max = 1.0
    runs = {"l1": {}, "l1_box": {"x_max": x_max}, "tv_box": {"reg": fbl.REG_TV, "tv_iters": 10, "x_max": x_max}}
    wl_mu = 0.02
    for name, kw in runs.items():
        S = fbl.fblisa_create(G, fbl.params_default(alpha0=1e-3, beta=0.5, mu=wl_mu, N0=40, seed=3003, **kw))
        x = torch.zeros(g.vol_shape, dtype=torch.float32, device=device)
        S.step(x, b)
        torch.cuda.synchronize(device)
        e0.record(stream)
        st = [S.step(x, b) for _ in range(iters)]
        e1.record(stream)
        torch.cuda.synchronize(device)
        out[name] = {"ms_per_iteration": e0.elapsed_time(e1) / iters,
                     "backtracks_per_iteration": sum(t["backtracks"] for t in st) / iters,
                     "max_x": float(x.max()), "tv_x": fbl.tv_norm(x)}
        del S, x
    out["mu"] = wl_mu
    return out


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200",
                                          "-i", str(gpu_index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_data(fbl, wl, device):
    import numpy as np
    import torch
    import synth
    g = wl.geom
    xt = synth.phantom(g, wl.n_ellipsoids, wl.seed_phantom, inclusions=wl.inclusions,
                       texture_std=wl.texture_std)
    G = fbl.geometry_create(g)
    xt_d = torch.from_numpy(xt).to(device)
    b = torch.empty((g.n_views, g.nv, g.nu), dtype=torch.float32, device=device)
    chunk = 90
    for v0 in range(0, g.n_views, chunk):
        vs = list(range(v0, min(g.n_views, v0 + chunk)))
        fbl.project(G, xt_d, vs, y=b[v0:v0 + len(vs)])
    torch.cuda.synchronize(device)
    if wl.noise == "poisson":
        bh = synth.poisson_log_data(b.cpu().numpy(), wl.I0, wl.seed_noise)
        b.copy_(torch.from_numpy(bh))
    else:
        sigma = wl.noise_rel * float(b.max())
        n = synth.gaussian_noise(tuple(b.shape), sigma, wl.seed_noise)
        b += torch.from_numpy(n).to(device)
    del xt_d
    return G, xt, b


def step_units(st, g):
    N_t = st["N_t"]
    n_proj = st["backtracks"] + 2
    samples = n_proj * N_t * g.nu * g.nv * g.nx
    voxel_views = N_t * g.nx * g.ny * g.nz
    return samples + voxel_views


def active_samples(g, views):
    """Ray-plane samples K1 actually takes for these views (planes where the
    crossing lies inside (-1, Nb) x (-1, nz)), from the geometry in float64.
    For every view of a square volume on a uniform orbit whose view count is a
    multiple of 4, the counts of views a quarter turn apart are equal (the
    setup maps onto itself), so the first quarter is counted four times."""
    import math
    import numpy as np
    views = list(views)
    if (g.angles is None and g.nx == g.ny and g.vx == g.vy and g.n_views % 4 == 0
            and views == list(range(g.n_views))):
        return 4 * active_samples(g, range(g.n_views // 4))
    cu, cv = 0.5 * (g.nu - 1), 0.5 * (g.nv - 1)
    V = (g.vx, g.vy, g.vz)
    Nn = (g.nx, g.ny, g.nz)
    total = 0
    for v in views:
        th = 2.0 * math.pi * v / g.n_views if g.angles is None else g.angles[v]
        c, s_ = math.cos(th), math.sin(th)
        src = (g.sod * c, g.sod * s_)
        u = (np.arange(g.nu) - cu) * g.du
        off = g.sdd - g.sod
        dx = -off * c - u * s_ - src[0]
        dy = -off * s_ + u * c - src[1]
        fam = (np.abs(dy) > np.abs(dx)).astype(int)
        for f in (0, 1):
            sel = fam == f
            if not sel.any():
                continue
            a, b = f, 1 - f
            da = (dx, dy)[a][sel]
            db = (dx, dy)[b][sel]
            ca, cb = 0.5 * (Nn[a] - 1), 0.5 * (Nn[b] - 1)
            p0 = -ca * V[a] - src[a]
            qb1 = V[a] * db / (da * V[b])
            qb0 = (src[b] + p0 * db / da) / V[b] + cb
            zc1 = V[a] / (da * V[2])
            zc0 = p0 / (da * V[2])
            w = (np.arange(g.nv) - cv) * g.dv
            m = np.arange(Nn[a])[:, None]
            inb = ((qb0[None] + m * qb1[None]) > -1) & ((qb0[None] + m * qb1[None]) < Nn[b])
            # q_z per (m, column, row): count inside per column via the row range
            Z = zc0[None] + m * zc1[None]                       # [m, col]
            qz_lo = (-1 - 0.5 * (g.nz - 1)) / np.where(Z == 0, 1e-30, Z)
            qz_hi = (g.nz - 0.5 * (g.nz - 1)) / np.where(Z == 0, 1e-30, Z)
            # rows with -1 < w*Z + cz < nz  <=>  qz_lo < w < qz_hi (Z > 0)
            lo = np.searchsorted(w, qz_lo, side="right")
            hi = np.searchsorted(w, qz_hi, side="left")
            rows = np.clip(hi - lo, 0, None)
            total += int((rows * inb).sum())
    return total


def time_to_objective(fbl, G, g, wl, b, device, epochs, check_every, xt=None, decompose=True):
    """Wall time (sum of CUDA-event step times; objective evaluations off the
    clock) to reach F(x) <= F* (1 + 1e-3), where F* is the plain FP32 method's
    full objective after `epochs` epochs: for learned proposal + BF16 storage
    + graph capture and (decompose) for each of the three alone, on FP32
    host-loop iterations otherwise."""
    import torch
    from paper_2605_12085_gb300 import proposal
    params, meta = proposal.load()
    stream = torch.cuda.current_stream(device)
    b16 = b.to(torch.bfloat16)
    xt_d = torch.from_numpy(xt).to(device) if xt is not None else None

    def run(learned, bf16, graph, max_epochs, target=None):
        p = fbl.params_default(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0, seed=wl.seed_batches,
                               x_dtype=fbl.BF16 if bf16 else fbl.F32,
                               b_dtype=fbl.BF16 if bf16 else fbl.F32,
                               use_graph=1 if graph else 0, proposal=1 if learned else 0,
                               autotune=1)
        S = fbl.fblisa_create(G, p)
        if learned:
            S.set_proposal(params, margin=0.25)
        x = torch.zeros(g.vol_shape, dtype=torch.bfloat16 if bf16 else torch.float32, device=device)
        bb = b16 if bf16 else b
        elapsed, hist, k, trials = 0.0, [], 0, 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n_iter = sum(it for _, it in fbl.fbl_schedule(g.n_views, wl.N0, g.n_views, 1.0, 0.99, max_epochs))
        stopped = None
        while k < n_iter:
            e0.record(stream)
            try:
                st = S.step(x, bb)
            except fbl.FblError as ex:
                # e.g. no trial passes (2.3) within the backtrack cap: the solver
                # keeps x, and this configuration stops here
                torch.cuda.synchronize(device)
                stopped = {"iteration": k + 1, "seconds": elapsed, "error": str(ex)}
                F, _, re = fbl.evaluate(G, x.float() if bf16 else x, b, wl.mu, x_true=xt_d)
                hist.append((k, elapsed, F, re))
                break
            e1.record(stream)
            torch.cuda.synchronize(device)
            elapsed += e0.elapsed_time(e1) * 1e-3
            k += 1
            trials += st["backtracks"] + 1
            if k % check_every == 0 or k == n_iter:
                # BF16 -> FP32 widening is exact, so F is that of the stored iterate
                F, _, re = fbl.evaluate(G, x.float() if bf16 else x, b, wl.mu, x_true=xt_d)
                hist.append((k, elapsed, F, re))
                if target is not None and F <= target:
                    break
        del S, x
        return hist, trials / max(k, 1), stopped

    plain, plain_trials, plain_stop = run(False, False, False, epochs)
    F_star = plain[-1][2]
    target = F_star * (1.0 + 1e-3)
    plain_hit = next(h for h in plain if h[2] <= target)
    out = {"F_star": F_star, "rel_tol": 1e-3, "epochs_for_F_star": epochs,
           "plain_fp32_s": plain_hit[1], "plain_iterations": plain_hit[0],
           "plain_rel_error_vs_x_true": plain_hit[3] if xt is not None else None,
           "plain_trials_per_iteration": plain_trials,
           "check_every_iterations": check_every, "proposal_margin": 0.25,
           "proposal_traces": meta.get("traces")}
    if plain_stop:
        out["plain_stopped"] = plain_stop
    configs = [("fast", True, True, True)]
    if decompose:
        configs += [("learned_only", True, False, False), ("bf16_only", False, True, False),
                    ("graph_only", False, False, True)]
    for name, learned, bf16, graph in configs:
        h, tr, stop = run(learned, bf16, graph, 2 * epochs, target)
        hit = next((r for r in h if r[2] <= target), None)
        rec = {"learned_proposal": learned, "bf16_storage": bf16, "graph_captured": graph,
               "s": hit[1] if hit else None, "iterations": hit[0] if hit else None,
               "trials_per_iteration": tr, "rel_error_vs_x_true": hit[3] if hit and xt is not None else None,
               "speedup": (plain_hit[1] / hit[1]) if hit else None}
        if stop:
            rec["stopped"] = stop
        if name == "fast":
            out["fast"] = "learned proposal + BF16 storage + graph-captured iteration"
            out["fast_s"] = rec["s"]
            out["fast_iterations"] = rec["iterations"]
            out["fast_trials_per_iteration"] = tr
            out["fast_rel_error_vs_x_true"] = rec["rel_error_vs_x_true"]
            out["speedup"] = rec["speedup"]
            if stop:
                out["fast_stopped"] = stop
        else:
            out[name] = rec
    del b16
    return out


def aggregate_ranks(ms, units, dist=None):
    """Replicas: the job's time is the slowest rank's, its work the sum of all
    ranks' units (host-side reduction over the process group, gloo)."""
    if dist is None:
        return float(ms), float(units)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def run_fdk_only(args):
    """FDK alone on the workload's data (one GPU): a side measurement, not the
    contract line."""
    import torch
    import paper_2605_12085_gb300 as fbl
    import synth
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    wl = synth.WORKLOADS[args.workload]
    G, xt, b = make_data(fbl, wl, device)
    rec = fdk_record(fbl, G, wl.geom, b, xt, device, reps=max(1, args.steps))
    return {"workload": args.workload, "fdk": rec}


def run_tv_only(args):
    """prox_tv alone on the workload's phantom (one GPU): a side measurement,
    not the contract line."""
    import torch
    import paper_2605_12085_gb300 as fbl
    import synth
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    wl = synth.WORKLOADS[args.workload]
    g = wl.geom
    xt = synth.phantom(g, wl.n_ellipsoids, wl.seed_phantom, inclusions=wl.inclusions, texture_std=wl.texture_std)
    v = torch.from_numpy(xt).to(device)
    q = torch.zeros((3,) + tuple(v.shape), dtype=torch.float32, device=device)
    x = torch.empty_like(v)
    fgp = 20
    fbl.prox_tv(v, 0.01, fgp, q=q, x=x)
    torch.cuda.synchronize(device)
    stream = torch.cuda.current_stream(device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = max(1, args.steps)
    e0.record(stream)
    for _ in range(reps):
        fbl.prox_tv(v, 0.01, fgp, q=q, x=x)
    e1.record(stream)
    torch.cuda.synchronize(device)
    ms = e0.elapsed_time(e1) / reps
    byt = float(g.n_vox) * (24 + 72 * fgp + 20)
    return {"workload": args.workload, "prox_tv": {"voxels": g.n_vox, "fgp_iterations": fgp, "ms": ms,
                                                  "achieved_gbs": byt / (ms * 1e-3) / 1e9}}


def alu_peak_tops(clk, peaks):
    """FP32 issue peak: 152 SMs x 128 lanes x the max SM clock seen (Tops/s)."""
    sm_clock = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    return 152 * 128 * sm_clock * 1e6 / 1e12, sm_clock


def alu_roofline(kernel, ops_per_sample, samples, avg_ms, algorithmic_bytes, clk, peaks, **extra):
    peak, sm_clock = alu_peak_tops(clk, peaks)
    achieved = ops_per_sample * samples / (avg_ms * 1e-3) / 1e12 if avg_ms else None
    out = {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": (achieved / peak) if achieved else None, "traffic": None,
           "traffic_note": "null: DRAM bytes are not measured inside this run",
           "algorithmic_bytes": algorithmic_bytes,
           "peak_source": "derived: 152 SMs x 128 FP32 lanes x %.0f MHz (max SM clock seen)" % sm_clock,
           "ops_per_sample": ops_per_sample, "in_volume_samples_per_launch": samples,
           "avg_launch_ms": avg_ms}
    out.update(extra)
    return out


def fblisa_iteration_record(fbl, G, g, wl, b, device, steps, warmup, peaks):
    """One FB-LISA iteration (Steps 2a-2d, host loop, FP32) on the workload's
    40-view mini-batches: GUPS over the work an iteration does (every forward
    projection N_t nu nv N samples, the backprojection N_t N^3 voxel-views),
    per-kernel CUDA-event times recorded by the library on the launching
    stream, and the rooflines of the trial-objective projection (K1), the
    gradient backprojection (K2) and the prox (K3)."""
    import numpy as np
    import torch
    params = fbl.params_default(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0, seed=wl.seed_batches,
                                max_backtracks=60)
    S = fbl.fblisa_create(G, params)
    x = torch.zeros(g.vol_shape, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream(device)
    for _ in range(warmup):
        S.step(x, b)
    S.profile(True)
    torch.cuda.synchronize(device)
    clocks = ClockSampler(device.index or 0)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    stats, batches = [], []
    for _ in range(steps):
        stats.append(S.step(x, b))
        batches.append(S.last_batch())
    t1.record(stream)
    torch.cuda.synchronize(device)
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    prof = S.profile(False)
    units = sum(step_units(st, g) for st in stats)
    samples = float(np.mean([active_samples(g, vs) for vs in batches[:3]]))
    N_t = stats[0]["N_t"]
    k1_ms, k1_n = prof["objective_projection"]
    k2_ms, k2_n = prof["gradient_backprojection"]
    k3_ms, k3_n = prof["prox_reduce"]
    k3_avg = k3_ms / max(k3_n, 1)
    k3_gbs = K3_BYTES_PER_VOXEL * g.n_vox / (k3_avg * 1e-3) / 1e9 if k3_n else None
    return {
        "what": "one FB-LISA iteration (Steps 2a-2d, host-loop line search), FP32 storage, "
                "mini-batch %d views" % N_t,
        "gups": units / (ms * 1e-3) / 1e9, "ms_per_iteration": ms / steps, "steps": steps, "warmup": warmup,
        "backtracks_per_iteration": statistics.mean(st["backtracks"] for st in stats),
        "in_volume_samples_per_projection": samples,
        "roofline_k1": alu_roofline("k1_project, trial objective (Step 2c, eq. (2.3))", K1_OPS_PER_SAMPLE,
                                    samples, k1_ms / max(k1_n, 1), g.n_vox * 4 + N_t * g.nu * g.nv * 4, clk,
                                    peaks),
        "roofline_k2": alu_roofline("k2_backproject, gradient (Step 2b, eq. (2.5))", K2_OPS_PER_SAMPLE,
                                    samples, k2_ms / max(k2_n, 1),
                                    N_t * g.nu * (g.nv + 16) * 4 + g.n_vox * 4, clk, peaks,
                                    voxel_views_per_launch=float(N_t) * g.n_vox),
        "roofline_k3": {"kernel": "k_prox_zi", "bound": "hbm", "achieved": k3_gbs,
                        "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                        "frac": (k3_gbs / peaks["hbm_gbs"]) if k3_gbs else None,
                        "bytes_per_voxel": K3_BYTES_PER_VOXEL, "avg_launch_ms": k3_avg},
        "kernels": {name: {"ms": round(v[0], 3), "launches": v[1]} for name, v in prof.items()},
        "clocks": clk,
    }


def sweep_units(g):
    return float(g.n_views) * g.nu * g.nv * g.nx, float(g.n_views) * g.n_vox


def c2_record(fbl, device, peaks):
    """The 256^3 Poisson configuration as stated: 40-ellipsoid phantom with
    small high-contrast inclusions, 360 views, 384x384 detector, log-Poisson
    data (I_0 = 1e4), 20-view mini-batches growing by Step 1's schedule, 20
    epochs, FP32; F, RE and backtracks at every epoch end (F and RE off the
    clock), and the operators' full sweep at this size."""
    import numpy as np
    import torch
    import synth
    wl = synth.WORKLOADS["c2_256"]
    g = wl.geom
    G, xt, b = make_data(fbl, wl, device)
    tune = fbl.geometry_autotune(G, fbl.F32, wl.N0)
    xt_d = torch.from_numpy(xt).to(device)
    stream = torch.cuda.current_stream(device)
    S = fbl.fblisa_create(G, fbl.params_default(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0,
                                                seed=wl.seed_batches))
    x = torch.zeros(g.vol_shape, dtype=torch.float32, device=device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    epochs, el, per_epoch = [], 0.0, {}
    sched = fbl.fbl_schedule(g.n_views, wl.N0, g.n_views, 1.0, 0.99, wl.epochs)
    for t, (N_t, iters) in enumerate(sched, start=1):
        bts = []
        for _ in range(iters):
            e0.record(stream)
            st = S.step(x, b)
            e1.record(stream)
            torch.cuda.synchronize(device)
            el += e0.elapsed_time(e1) * 1e-3
            bts.append(st["backtracks"])
            assert st["N_t"] == N_t
        F, _, re = fbl.evaluate(G, x, b, wl.mu, x_true=xt_d)
        epochs.append({"epoch": t, "N_t": N_t, "iterations": iters, "F": F, "rel_error": re,
                       "backtracks_per_iteration": float(np.mean(bts)), "seconds": el})
    fwd_u, bp_u = sweep_units(g)
    y = torch.empty((g.n_views, g.nv, g.nu), dtype=torch.float32, device=device)
    gr = torch.empty(g.vol_shape, dtype=torch.float32, device=device)
    views = list(range(g.n_views))
    fbl.project(G, x, views, y=y)
    fbl.backproject(G, y, views, x=gr)
    torch.cuda.synchronize(device)
    t = {}
    for name, call in (("forward", lambda: fbl.project(G, x, views, y=y)),
                       ("back", lambda: fbl.backproject(G, y, views, x=gr))):
        e0.record(stream)
        for _ in range(3):
            call()
        e1.record(stream)
        torch.cuda.synchronize(device)
        t[name] = e0.elapsed_time(e1) / 3
    del y, gr, S, x, b, G, xt_d
    torch.cuda.empty_cache()
    return {"workload": "c2_256: 256^3 volume (40 ellipsoids + 8 inclusions), 360 views, 384x384 detector, "
                        "log-Poisson data I0=1e4, mini-batch 20 views by the schedule, 20 epochs, FP32",
            "autotune": tune, "epochs": epochs, "seconds_total": el,
            "full_sweep": {"forward_ms": t["forward"], "back_ms": t["back"],
                           "gups_fwd_back": (fwd_u + bp_u) / ((t["forward"] + t["back"]) * 1e-3) / 1e9}}


def run_kernels_only(args):
    """The hot kernels alone, for profiler captures (one GPU; a side mode, not
    the contract line): the workload's data (ceil(n_views/90) store-mode
    projector launches), then --steps trial-objective projections of one
    mini-batch (residual_norm: k_pack, k1_project, k_reduce) and --steps
    backprojections of it (k_weight, k2_backproject, k_zi_to_natural), in the
    launch configuration --launch (else the autotuner's, whose timing
    launches come first).  Prints the CUDA-event time of each."""
    import torch
    import paper_2605_12085_gb300 as fbl
    import synth
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    wl = synth.WORKLOADS[args.workload]
    g = wl.geom
    G, xt, b = make_data(fbl, wl, device)
    if args.launch:
        cols, split, vpl = (int(v) for v in args.launch.split(","))
        fbl.geometry_set_launch(G, cols, split, vpl)
        tune = {"k1_cols": cols, "k1_split": split, "k2_vpl": vpl}
    else:
        tune = fbl.geometry_autotune(G, fbl.F32, wl.N0)
    views = fbl.fbl_epoch_batches(wl.seed_batches, 1, g.n_views, wl.N0)[0]
    x = torch.from_numpy(xt).to(device)
    y = torch.randn((len(views), g.nv, g.nu), dtype=torch.float32, device=device)
    gr = torch.empty(g.vol_shape, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream(device)
    out = {"workload": args.workload, "views": len(views), "launch": tune}
    for name, call in (("residual_norm_ms", lambda: fbl.residual_norm(G, x, views, b)),
                       ("backproject_ms", lambda: fbl.backproject(G, y, views, x=gr))):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(max(1, args.steps)):
            e0.record(stream)
            call()
            e1.record(stream)
            torch.cuda.synchronize(device)
            ts.append(e0.elapsed_time(e1))
        out[name] = ts
    return out


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2605_12085_gb300 as fbl
    import synth

    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    wl = synth.WORKLOADS[args.workload]
    g = wl.geom
    G, xt, b = make_data(fbl, wl, device)
    tune = fbl.geometry_autotune(G, fbl.F32, wl.N0)
    if args.launch:
        cols, split, vpl = (int(v) for v in args.launch.split(","))
        fbl.geometry_set_launch(G, cols, split, vpl)
        tune = dict(tune, forced={"k1_cols": cols, "k1_split": split, "k2_vpl": vpl})
    peaks, peak_src = load_peaks()
    stream = torch.cuda.current_stream(device)

    # --- the contract's timed region: K full sweeps, forward then back ------
    views = list(range(g.n_views))
    xd = torch.from_numpy(xt).to(device)
    y = torch.empty((g.n_views, g.nv, g.nu), dtype=torch.float32, device=device)
    gr = torch.empty(g.vol_shape, dtype=torch.float32, device=device)
    for _ in range(args.warmup):
        fbl.project(G, xd, views, y=y)
        fbl.backproject(G, y, views, x=gr)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(device)
    clocks = ClockSampler(local_rank)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, m, c in ev:
        a.record(stream)
        fbl.project(G, xd, views, y=y)
        m.record(stream)
        fbl.backproject(G, y, views, x=gr)
        c.record(stream)
    t1.record(stream)
    torch.cuda.synchronize(device)
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    fwd_ms = statistics.mean(a.elapsed_time(m) for a, m, _ in ev)
    bp_ms = statistics.mean(m.elapsed_time(c) for _, m, c in ev)
    fwd_u, bp_u = sweep_units(g)
    units = args.steps * (fwd_u + bp_u)
    ms_max, units_all = aggregate_ranks(ms, units, dist)
    value = units_all / (ms_max * 1e-3) / 1e9
    in_vol = float(active_samples(g, views))
    sweep = {"forward_ms": fwd_ms, "back_ms": bp_ms,
             "gups_forward": fwd_u / (fwd_ms * 1e-3) / 1e9, "gups_back": bp_u / (bp_ms * 1e-3) / 1e9,
             "gups_fwd_back": (fwd_u + bp_u) / ((fwd_ms + bp_ms) * 1e-3) / 1e9,
             "in_volume_samples": in_vol, "nominal_samples": fwd_u,
             "gsamples_in_volume_forward": in_vol / (fwd_ms * 1e-3) / 1e9,
             "units": "forward: n_views*nu*nv*N ray samples (nominal; in-volume ones beside); "
                      "back: n_views*N^3 voxel-views"}
    # dominant kernel of the step: the backprojection of all views (one K2 launch;
    # the call's events also hold its short weighting and reordering kernels)
    bp_bytes = g.n_views * g.nu * (g.nv + 16) * 4 + g.n_vox * 4
    k2 = alu_roofline("k2_backproject over all %d views (one launch; the timed call also holds "
                      "k_weight and k_zi_to_natural)" % g.n_views, K2_OPS_PER_SAMPLE, in_vol, bp_ms,
                      bp_bytes, clk, peaks, voxel_views_per_launch=bp_u)
    k1 = alu_roofline("k1_project, store mode, all %d views (one launch; the timed call also "
                      "holds k_pack)" % g.n_views, K1_OPS_PER_SAMPLE, in_vol, fwd_ms,
                      g.n_vox * 4 + g.n_views * g.nu * g.nv * 4, clk, peaks)
    dominant, other = (k2, k1) if bp_ms >= fwd_ms else (k1, k2)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "%s: %d^3 volume, %d views, %dx%d detector; step = forward projection "
                                  "of all %d views + backprojection of all %d views (FP32 storage and "
                                  "accumulation)" % (wl.name, g.nx, g.n_views, g.nu, g.nv, g.n_views,
                                                     g.n_views),
                      "l2": "inputs larger than L2 (volume %.0f MB, projections %.0f MB)"
                            % (g.n_vox * 4 / 1e6, g.n_views * g.nu * g.nv * 4 / 1e6),
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "full_sweep": sweep, "roofline": dominant, "roofline_other": other,
           "gpu_launches": 5 * args.steps,
           "gpu_launches_note": "per step: k_pack + k1_project (project call), k_weight + k2_backproject "
                                "+ k_zi_to_natural (backproject call)",
           "clocks": clk, "autotune": tune, "peak_source": peak_src}
    del y, gr

    # --- the whole hot path: one FB-LISA iteration ---------------------------
    out["fblisa_iteration"] = fblisa_iteration_record(fbl, G, g, wl, b, device, args.iter_steps, 3, peaks)

    if rank == 0:
        out["fdk"] = fdk_record(fbl, G, g, b, xt, device)
        out["regularisers"] = regularisers_record(fbl, G, g, b, xt, device, peaks)

    # storage-precision variants (BF16 / FP16 iterates and data, FP32 arithmetic)
    if args.variants:
        variants = {}
        for name, code, td, graph in (("f32_graph", fbl.F32, torch.float32, 1),
                                      ("bf16", fbl.BF16, torch.bfloat16, 0),
                                      ("f16", fbl.F16, torch.float16, 0),
                                      ("bf16_graph", fbl.BF16, torch.bfloat16, 1)):
            bv = b.to(td)
            pv = fbl.params_default(alpha0=1e-3, beta=0.5, mu=wl.mu, N0=wl.N0,
                                    seed=wl.seed_batches, max_backtracks=60, x_dtype=code,
                                    b_dtype=code, autotune=1, use_graph=graph)
            Sv = fbl.fblisa_create(G, pv)
            xv = torch.zeros(g.vol_shape, dtype=td, device=device)
            for _ in range(2):
                Sv.step(xv, bv)
            torch.cuda.synchronize(device)
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            stv = [Sv.step(xv, bv) for _ in range(args.variant_steps)]
            v1.record(stream)
            torch.cuda.synchronize(device)
            vms = v0.elapsed_time(v1)
            uv = sum(step_units(st, g) for st in stv)
            variants[name] = {"gups": uv / (vms * 1e-3) / 1e9, "ms_per_iteration": vms / len(stv),
                              "steps": len(stv),
                              "backtracks_per_iteration": statistics.mean(st["backtracks"] for st in stv)}
            del Sv, xv, bv
        out["fblisa_iteration_variants"] = variants

    if args.c2 and rank == 0:
        out["c2"] = c2_record(fbl, device, peaks)

    if args.batched and rank == 0:
        out["batched"] = batched_records(fbl, device)

    if args.c5b and rank == 0:
        out["c5b"] = c5b_record(fbl, device)

    if args.comparators and rank == 0:
        out["comparators"] = comparators_record(fbl, device)

    if args.paper_mu_sweep and rank == 0:
        out["paper_mu_sweep"] = paper_mu_sweep_record(fbl, device)

    if args.paper_cases and rank == 0:
        out["paper_cases"] = paper_cases_record(fbl, device, mu_fraction=args.paper_mu_fraction)

    if args.tto_epochs > 0 and rank == 0:
        out["time_to_objective"] = time_to_objective(fbl, G, g, wl, b, device, args.tto_epochs,
                                                     args.tto_check, xt=xt, decompose=bool(args.tto_decompose))

    # end to end: the same step through the same C-ABI calls with host (pinned)
    # buffers, host<->device copies inside the timed region
    if args.e2e_steps > 0:
        xh = torch.from_numpy(xt).pin_memory()
        yh = torch.empty((g.n_views, g.nv, g.nu), dtype=torch.float32).pin_memory()
        gh = torch.empty(g.vol_shape, dtype=torch.float32).pin_memory()
        fbl.project(G, xh, views, y=yh)
        fbl.backproject(G, yh, views, x=gh)
        torch.cuda.synchronize(device)
        e0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            fbl.project(G, xh, views, y=yh)
            fbl.backproject(G, yh, views, x=gh)
        torch.cuda.synchronize(device)
        e_ms = (time.perf_counter() - e0) * 1e3
        h2d = g.n_vox * 4 + g.n_views * g.nu * g.nv * 4 + 2 * g.n_views * 4
        d2h = g.n_views * g.nu * g.nv * 4 + g.n_vox * 4
        out["e2e"] = {"value": args.e2e_steps * (fwd_u + bp_u) / (e_ms * 1e-3) / 1e9 * (units_all / units),
                      "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                      "ms_per_step": e_ms / args.e2e_steps,
                      "what": "project(x host -> y host) + backproject(y host -> g host) of all views"}
        del xh, yh, gh

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, xt)
    return out


def cpu_baseline(wl, xt=None):
    """The FP64 oracle on the host cores, on a bounded sample of the workload."""
    import numpy as np
    import oracle
    import synth
    g = wl.geom
    if xt is None:
        xt = synth.phantom(g, wl.n_ellipsoids, wl.seed_phantom, inclusions=wl.inclusions,
                           texture_std=wl.texture_std)
    x64 = np.asarray(xt, dtype=np.float64)
    rng = np.random.default_rng(1)
    y = rng.standard_normal((1, g.nv, g.nu))
    t0 = time.perf_counter()
    oracle.project(g, x64, [0])
    t1 = time.perf_counter()
    oracle.backproject(g, y, [1])
    t2 = time.perf_counter()
    units = g.nu * g.nv * g.nx + g.n_vox
    return {"value": units / (t2 - t0) / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "FP64 oracle: forward projection of 1 view + scatter adjoint of 1 view "
                      "at the full %d^3 / %dx%d geometry (fwd %.2f s, adjoint %.2f s)"
                      % (g.nx, g.nu, g.nv, t1 - t0, t2 - t1)}


def run_reference(args):
    """Reference arm: the FP64 oracle, each step one bounded sample of the workload."""
    import numpy as np
    import oracle
    import synth
    wl = synth.WORKLOADS[args.workload]
    g = wl.geom
    xt = synth.phantom(g, wl.n_ellipsoids, wl.seed_phantom, inclusions=wl.inclusions,
                       texture_std=wl.texture_std).astype(np.float64)
    rng = np.random.default_rng(2)
    y = rng.standard_normal((1, g.nv, g.nu))

    def one(v):
        oracle.project(g, xt, [v % g.n_views])
        oracle.backproject(g, y, [(v + 1) % g.n_views])

    for w in range(args.warmup):
        one(w)
    t0 = time.perf_counter()
    for s in range(args.steps):
        one(args.warmup + s)
    sec = time.perf_counter() - t0
    units = args.steps * (g.nu * g.nv * g.nx + g.n_vox)
    value = units / sec / 1e9
    sample = ("each step: FP64 oracle forward projection of 1 view + scatter adjoint of 1 view "
              "at the full %d^3 / %dx%d geometry" % (g.nx, g.nu, g.nv))
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "%s: %d^3 volume, %d views, %dx%d detector (oracle sample)"
                                   % (wl.name, g.nx, g.n_views, g.nu, g.nv)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local_rank = env_rank()
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)), flush=True)
        return 0
    if args.fdk_only:
        if rank == 0:
            print(json.dumps(run_fdk_only(args)), flush=True)
        return 0
    if args.tv_only:
        if rank == 0:
            print(json.dumps(run_tv_only(args)), flush=True)
        return 0
    if args.kernels_only:
        if rank == 0:
            print(json.dumps(run_kernels_only(args)), flush=True)
        return 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
