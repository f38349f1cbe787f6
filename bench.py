"""Throughput of the free-energy hot path on one GB300 (or N, one process per GPU).

Workload (default): the FFLO scan at N = 1024 -- 64 q along x in [0, 0.2 pi],
32 h in [0, 0.15], T = 0.002, 256 Delta in [0, 0.2], U = 2 -- in FP32 with
pairwise/FP64 accumulation and FP64 re-evaluation of near ties.  One step = one
full pass of the path: trig tables, normal-state sums, the k-sum of every
(q, h, Delta), argmin, FP64 re-evaluation, phase labels.

value : k-point evaluations per second (one k-point x one Delta x one (q,h,T),
        both bands), whole job, plan inputs resident in HBM.
e2e   : the same through the host-buffer C-ABI call ffe_phase_scan.
Multi-GPU: the q list is split across ranks (no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("parameter points/sec and k-evals/sec at N=1024 (FP32+comp vs FP64 vs surrogate), "
          "% FP32/MUFU peak")
# Special-function unit results per clock per SM: ex2 32 (GB300), lg2 / rsqrt /
# rcp 16 (4 per SM sub-partition); ffe_probe_peaks measures both on the device.
SFU_EX2_PER_CLK = 32
SFU_OTHER_PER_CLK = 16
SM_MAX_MHZ = 2070.0


def sfu_clk_per_band_eval(per_row: int, outs_per_item: int):
    """SFU time (SM clocks) per band evaluation (one k-point, one band, one output) in the
    shared-T scan layout: (near with two exponentials, near with one, far in the closed
    form, far in the moments).  Every far band takes one rcp per k-set for y = Delta_max^2
    eta^2 / s^2, shared by the item's outputs; one outside the series range (y > 0.1) also
    needs R and a: 1 rsqrt + 1 rcp per (k, Delta, band), shared by the per_row (h, T)
    outputs of one Delta row of a tile.  A near band is evaluated in full, packed with another
    near band in a float2 slot: per output 2 ex2 -- 1 where c (R + |d|) >= 27 makes the second
    factor exactly 1 -- and an eighth of one lg2 (one lg2 per output over a lane's four
    slots), and its R and a."""
    ra = 2.0 / (SFU_OTHER_PER_CLK * per_row)
    y = 1.0 / (SFU_OTHER_PER_CLK * outs_per_item)
    rest = 0.125 / SFU_OTHER_PER_CLK + ra + y
    return 2.0 / SFU_EX2_PER_CLK + rest, 1.0 / SFU_EX2_PER_CLK + rest, ra + y, y


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons; only the samples taken inside the
    timed region (host wall clock, marked by begin()/end()) are summarised."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.t0 = self.t1 = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # let the sampler start before the timed region
        except OSError:
            self.p = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def _when(stamp: str):
        import datetime

        try:
            return datetime.datetime.strptime(stamp, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        lines = open(self.f.name).read().splitlines()
        os.unlink(self.f.name)
        return summarize_clocks(lines, self.t0, self.t1)


def summarize_clocks(lines, t0=None, t1=None):
    """Median SM clock, maximum clock and throttle reasons of the nvidia-smi CSV rows
    (timestamp, index, clocks.sm, clocks.max.sm, power, active, hw_slowdown, hw_thermal_slowdown,
    sw_thermal_slowdown, sw_power_cap) taken inside [t0, t1] (host wall clock, 50 ms slack)."""
    rows = [[x.strip() for x in line.split(",")] for line in lines]
    rows = [r for r in rows if len(r) >= 10]
    inside = rows
    if t0 is not None and t1 is not None:
        inside = [r for r in rows if (w := Clocks._when(r[0])) is not None and t0 - 0.05 <= w <= t1 + 0.05]
    if not inside:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples in the timed region"],
                "samples": 0, "samples_total": len(rows)}
    sm = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
    mx = [float(r[3]) for r in inside if r[3].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in inside for i in range(4) if r[6 + i].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(inside), "interval_ms": 100}


def cpu_baseline(cfg, lines, diagram_lines=None, tol=2e-7):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the workload:
    the whole 256-point Delta grid of a few (q, h) lines at N = 1024, parallel over Delta with
    OpenMP (timed).  The same oracle values give the per-result error of the GPU scan on those
    lines (every grid value per site, and the argmin index), and, for the phase diagram, the
    oracle at the GPU's Delta* and at Delta = 0 of a few golden-section lines."""
    import numpy as np

    import oracle
    from oracle import search

    m = oracle.make_model(U=cfg["U"])
    N = cfg["N"]
    grid = np.linspace(cfg["lo"], cfg["hi"], cfg["n"])
    oracle.omega_batch(m, N, lines[0]["qx"], 0.0, lines[0]["h"], cfg["T"][0], grid[:threads_hint()])  # warm-up
    t0 = time.perf_counter()
    refs = []
    for ln in lines:
        ref, _, threads = oracle.omega_batch(m, N, ln["qx"], 0.0, ln["h"], cfg["T"][0], grid)
        refs.append(ref)
    dt = time.perf_counter() - t0
    kev = float(N * N) * len(grid) * len(lines)
    err = max(float(np.max(np.abs(ln["omega"] - r)) / N**2) for ln, r in zip(lines, refs))
    same = all(int(ln["idx_star"]) == search.grid_argmin(r) for ln, r in zip(lines, refs))
    out = {"value": kev / dt, "unit": "k-evals/s", "cores": threads, "kind": "oracle",
           "sample": (f"the {len(grid)}-point Delta grids of {len(lines)} (q, h) lines at N={N} (FP64, OpenMP "
                      f"over Delta), {dt:.1f} s"),
           "per_result_error": {"fflo_scan": {
               "lines": [f"q={ln['qx']:.4f}, h={ln['h']:.4f}" for ln in lines], "values": len(lines) * len(grid),
               "max_err_per_site_vs_oracle": err, "tolerance_per_site": tol, "argmin_identical": same}}}
    if diagram_lines:
        d = diagram_lines
        Nd = d["N"]
        md = oracle.make_model(U=cfg["U"])
        at, _, _ = oracle.omega_batch(md, Nd, d["qx"], 0.0, d["h"], d["T"], d["delta_star"])
        at0, _, _ = oracle.omega_batch(md, Nd, d["qx"], 0.0, d["h"], d["T"], 0.0)
        e = np.concatenate([np.abs(at - d["omega_star"]), np.abs(at0 - d["omega_lo"])]) / Nd**2
        out["per_result_error"]["phase_diagram"] = {
            "lines": int(len(d["qx"])), "values": int(e.size), "max_err_per_site_vs_oracle": float(e.max()),
            "tolerance_per_site": tol, "at": "the GPU's golden-section Delta* and Delta = 0"}
    return out


# DRAM bytes (read + write) of one k-sum launch of the default workload, from
# ncu (dram__bytes_read.sum + dram__bytes_write.sum, one launch of the full-size
# plan): 3.12 GB read (mostly the FP32 k-state table, 1.34 GB, about 2.3 times)
# + 0.42 GB written (the FP64 k-chunk partial sums).
DRAM_TRAFFIC_PER_LAUNCH = 3.542e9
# From the committed one-kernel ncu capture of the same kernel on 8 of the 64 q
# (profiles/ksum_fflo_scan_N1024_q8.md): issue slots busy and the SFU (XU)
# pipe's share of its peak.
NCU_HEADLINE = {"issue_active_pct": 61.2, "sfu_pct_of_peak": 31.9,
                "source": "profiles/ksum_fflo_scan_N1024_q8.md"}


def run_extras(ffe, np, torch, stream, workloads):
    """The other workload shapes, timed once each after a warm-up (not the headline)."""
    out = {}
    # 512 uneven jobs in one persistent, graph-captured launch (FP32+comp)
    w = workloads.uneven_jobs(512, seed=1234)
    ps = ffe.params(w["N"], w["qx"], w["qy"], w["h"], w["T"], w["lo"], w["hi"], w["n"])
    with ffe.Context(prec=ffe.FFE_FP32C, U=2.0) as ctx:
        plan = ctx.plan_minimize(ps)
        shape = plan.autotune(stream)
        plan.execute(stream)
        plan.fetch_minimize()
        plan.kernel_ms()
        reps = 3
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            plan.execute(stream)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        kms, _ = plan.kernel_ms()
        k = plan.stats()["k_evals"]
        plan.destroy()
    # the three-band model of App. B (band tables by FP64 Jacobi, two band pairs per k-point)
    w3 = workloads.threeband_scan()
    with ffe.Context(prec=ffe.FFE_FP32C, U=w3["U"], model="daghofer3") as ctx3:
        plan3 = ctx3.plan_phase_scan(w3["N"], w3["qx"], w3["qy"], w3["h"], w3["T"], n=w3["n"], lo=w3["lo"],
                                     hi=w3["hi"])
        plan3.execute(stream)
        plan3.fetch()
        plan3.kernel_ms()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            plan3.execute(stream)
        _, lab3, _ = plan3.fetch()
        dt3 = (time.perf_counter() - t0) / 3
        kms3, _ = plan3.kernel_ms()
        st3 = plan3.stats()
        plan3.destroy()
    out["threeband_scan"] = {
        "k_evals_per_s": st3["k_evals"] / dt3, "ms_per_step": 1e3 * dt3, "kernel_ms": kms3,
        "kernel_k_evals_per_s": st3["k_evals"] / (kms3 / 1e3) if kms3 else None,
        "labels": [int((lab3 == i).sum()) for i in range(3)],
        "workload": (f"three-band model (App. B, eV), N={w3['N']}: {len(w3['qx'])} q x {len(w3['h'])} h x "
                     f"{w3['n']} Delta, T={w3['T'][0]}, U={w3['U']}, FP32+comp")}
    out["uneven_batch"] = {"jobs": 512, "k_evals_per_s": k / dt, "jobs_per_s": 512 / dt, "ms_per_step": 1e3 * dt,
                           "kernel_ms": kms, "autotuned": shape,
                           "workload": "512 jobs, N in {256,512,1024,2048}, 32..256 Delta, seed 1234"}

    def timed(fn, reps=3):
        fn()  # warm-up (plans, tables)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            r = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps, r

    # App. C pair susceptibility (FP64), two-band model
    qs = np.linspace(0.0, 0.2 * math.pi, 32)
    with ffe.Context(prec=ffe.FFE_FP64, U=2.0) as ctxc:
        dtc, _ = timed(lambda: ctxc.pair_susceptibility(1024, qs, 0.0, 0.05, 0.002))
    out["pair_susceptibility"] = {
        "ms": 1e3 * dtc, "k_points_per_s": len(qs) * 1024 ** 2 / dtc,
        "workload": "chi_ee'(q) of App. C, two-band model, N=1024, 32 q along x, h=0.05, T=0.002, FP64 "
                    "(4 band pairs per k-point)"}
    # full-Brillouin-zone Q scan: an 8 x 8 Q grid through its irreducible wedge
    from paper_1412_8754_gb300 import qgrid
    hs, Ts = np.linspace(0.0, 0.15, 32), np.array([0.002])
    with ffe.Context(prec=ffe.FFE_FP32C, U=2.0) as ctxf:
        dtf, rf = timed(lambda: qgrid.fbz_phase_scan(ctxf, 1024, 8, hs, Ts, n=64))
    out["fbz_scan"] = {
        "ms": 1e3 * dtf, "wedge_points": int(len(rf[3])), "grid_points": 64,
        "labels": [int((rf[1] == i).sum()) for i in range(3)],
        "workload": "Q over the 8 x 8 grid of the Brillouin zone (its 15-point wedge), N=1024, 32 h, T=0.002, "
                    "64 Delta on [0, 0.2], FP32+comp"}
    # per-band independent minimisation of the two-band model
    pb = ffe.params(512, np.linspace(0.0, 0.2 * math.pi, 16).repeat(16), 0.0,
                    np.tile(np.linspace(0.0, 0.15, 16), 16), 0.004, 0.0, 0.2, 64)
    with ffe.Context(prec=ffe.FFE_FP32C, U=2.0) as ctxb:
        dtb, _ = timed(lambda: ctxb.minimize_bands(pb))
    out["per_band_minimize"] = {
        "ms": 1e3 * dtb, "params_per_s": len(pb) / dtb,
        "workload": "256 (q, h) points, each band minimised on its own: 64-point Delta grid, N=512, T=0.004, "
                    "FP32+comp"}
    return out


def run_surrogate(ffe, np, torch, workloads, cfg, ref, full_s, fp64_rate, epochs=40, diagram=True):
    """The learned surrogate: ~2M samples at N=512, training, the guided scan of
    the headline workload against its full FP32 scan, and the N=2048 phase
    diagram (golden-section) in its full FP32, guided and sampled FP64 forms."""
    from paper_1412_8754_gb300 import surrogate as sg

    ref_res, ref_labels, ref_best = ref
    with ffe.Context(prec=ffe.FFE_FP32C, U=cfg["U"]) as ctx:
        sset = workloads.surrogate_set(n_groups=8192, n_ht=16, n_delta=16, seed=1235, T_hi=0.03)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, y = sg.training_data(ctx, 512, sset)
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        sur, losses = sg.fit(ctx, x, y, epochs=epochs, batch=4096, lr=2e-3, seed=1)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        args = (ctx.handle, sur, cfg["N"], cfg["qx"], np.zeros_like(cfg["qx"]), cfg["h"], cfg["T"])
        kw = dict(n=cfg["n"], lo=cfg["lo"], hi=cfg["hi"], window=16, q_keep=3)
        ffe.ffe_surrogate_scan(*args, **kw)
        times = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res, labels, best, st = ffe.ffe_surrogate_scan(*args, **kw)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        rms_train = sg.rms_error(sur, x, y)
        pd_check, pd_out = run_phase_diagram(ffe, np, torch, workloads, ctx, sur, 3.0 * rms_train, fp64_rate,
                                             cfg["U"]) if diagram else (None, None)
        sur.close()
    dt = statistics.median(times)
    kept = (res["flags"] & ffe.FFE_FLAG_PRUNED) == 0
    full64_s = st["k_evals_full"] / fp64_rate if fp64_rate else None
    n_pts = len(labels)
    # the MLP's arithmetic: per sample and epoch a forward (2 x (4x128 + 2x128^2 + 128) flops) and a
    # backward of twice that, against the measured BF16 dense peak
    train_flops = 3.0 * 2.0 * (4 * 128 + 2 * 128 * 128 + 128) * len(x) * epochs
    peak_bf16 = measured_peak("bf16_tflops", 1900.0) * 1e12
    return pd_check, pd_out, {
        "train_tflops": train_flops / t_train / 1e12,
        "train_frac_of_bf16_peak": train_flops / t_train / peak_bf16,
        "train_note": ("tcgen05.mma (BF16 x BF16 -> FP32 in TMEM), 128 samples per CTA; batches of 4096 keep "
                       "32 CTAs busy, so the run is latency-bound, not tensor-bound"),
        "workload": (f"train: {len(x)} samples (q,h,T,Delta) at N=512 from the FP32+comp k-sum, {epochs} epochs, "
                     f"batch 4096; guide: fflo_scan N={cfg['N']}, window 16 + Delta=0, q=0 and 3 q kept per h"),
        "datagen_s": t_data, "train_s": t_train, "train_loss_first_last": [float(losses[0]), float(losses[-1])],
        "rms_train_per_site": rms_train,
        "guided_s": dt, "points_per_s": len(cfg["qx"]) * n_pts / dt,
        "full_fp32_s": full_s, "speedup_vs_full_fp32": full_s / dt,
        "full_fp64_s_extrapolated": full64_s, "speedup_vs_full_fp64": full64_s / dt if full64_s else None,
        "k_evals": st["k_evals"], "k_evals_full": st["k_evals_full"], "mlp_flops": st["mlp_flops"],
        "rms_error_per_site": st["rms_error"], "rms_unit": "|t1| per lattice site (condensation energy)",
        "lines_kept": st["lines_kept"], "lines_pruned": st["lines_pruned"], "fallbacks": st["fallbacks"],
        "fallback_rate": st["fallbacks"] / max(1, st["lines_kept"]),
        "label_agreement": float(np.mean(labels == ref_labels)),
        "best_q_agreement": float(np.mean(best == ref_best)),
        "idx_agreement_kept_lines": float(np.mean(res["idx_star"][kept] == ref_res["idx_star"][kept])),
    }


def run_phase_diagram(ffe, np, torch, workloads, ctx, sur, margin, fp64_rate, U):
    """N=2048, 64 q x 64 h x 64 T, golden-section (24 reductions): the full FP32+comp scan, the
    surrogate-guided scan, and the FP64 kernel on a sub-grid, with their labels compared."""
    pd = workloads.phase_diagram()
    a = (pd["N"], pd["qx"], pd["qy"], pd["h"], pd["T"])
    kw = dict(search=ffe.FFE_SEARCH_GOLDEN, n=pd["n"], lo=pd["lo"], hi=pd["hi"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    full, flab, fbest = ctx.phase_scan(*a, **kw)
    torch.cuda.synchronize()
    t_full = time.perf_counter() - t0
    n_pts = len(pd["h"]) * len(pd["T"])
    k_full = float(pd["N"]) ** 2 * len(pd["qx"]) * n_pts * (3 + pd["n"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gres, glab, gbest, gst = ffe.ffe_surrogate_scan(ctx.handle, sur, *a, window=16, q_keep=3, margin=margin, **kw)
    torch.cuda.synchronize()
    t_guided = time.perf_counter() - t0
    # FP64 on a 2 h x 4 T sub-grid with every q (labels need all q of a point)
    hs, ts = pd["h"][:2], pd["T"][:4]
    with ffe.Context(prec=ffe.FFE_FP64, U=U) as c64:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, lab64, best64 = c64.phase_scan(pd["N"], pd["qx"], pd["qy"], hs, ts, **kw)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
    sub = (np.arange(2)[:, None] * len(pd["T"]) + np.arange(4)[None, :]).ravel()
    k64 = float(pd["N"]) ** 2 * len(pd["qx"]) * len(sub) * (3 + pd["n"])
    # a few golden-section lines for the oracle check of the CPU leg: (q, point) pairs spread over
    # the diagram, BCS points included where there are any
    rng = np.random.default_rng(7)
    picks = [(int(q), int(p)) for q, p in zip(rng.integers(0, len(pd["qx"]), 6), rng.integers(0, n_pts, 6))]
    picks += [(int(fbest[p]), int(p)) for p in np.flatnonzero(fbest >= 0)[:2]]
    check = {"N": pd["N"], "qx": np.array([pd["qx"][q] for q, _ in picks]),
             "h": np.array([pd["h"][p // len(pd["T"])] for _, p in picks]),
             "T": np.array([pd["T"][p % len(pd["T"])] for _, p in picks]),
             "delta_star": np.array([full["delta_star"][q, p] for q, p in picks]),
             "omega_star": np.array([full["omega_star"][q, p] for q, p in picks]),
             "omega_lo": np.array([full["omega_lo"][q, p] for q, p in picks])}
    return check, {
        "workload": (f"N={pd['N']}, {len(pd['qx'])} q x {len(pd['h'])} h x {len(pd['T'])} T, golden "
                     f"{pd['n']} reductions on [0, 0.2], U={U}"),
        "fp32c_full": {"seconds": t_full, "points_per_s": len(pd["qx"]) * n_pts / t_full,
                       "k_evals_per_s": k_full / t_full,
                       "labels": [int((flab == i).sum()) for i in range(3)]},
        "guided": {"seconds": t_guided, "speedup_vs_fp32c_full": t_full / t_guided,
                   "speedup_vs_fp64_full_extrapolated": (k_full / fp64_rate) / t_guided if fp64_rate else None,
                   "label_agreement_vs_fp32c_full": float(np.mean(glab == flab)),
                   "best_q_agreement": float(np.mean(gbest == fbest)),
                   "k_evals": gst["k_evals"], "k_evals_full": gst["k_evals_full"],
                   "lines_kept": gst["lines_kept"], "fallbacks": gst["fallbacks"],
                   "rms_error_per_site": gst["rms_error"], "margin": margin,
                   "window": 16, "q_keep": 3},
        "fp64_subgrid": {"points": len(sub), "seconds": t64, "k_evals_per_s": k64 / t64,
                         "label_agreement_vs_fp32c": float(np.mean(lab64 == flab[sub])),
                         "best_q_agreement_vs_fp32c": float(np.mean(best64 == fbest[sub])),
                         "full_seconds_extrapolated": k_full / (k64 / t64)},
    }


def measured_peak(key, fallback):
    """A peak from the measured-peaks file next to this script (HBM copy bandwidth, BF16 GEMM rate),
    else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return fallback


def threads_hint():
    import oracle

    return max(1, oracle.max_threads())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ffe", choices=["ffe", "reference"])
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--n-q", type=int, default=64, help="q values of the scan (64 = the full workload)")
    ap.add_argument("--fp64-sample-q", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-diagram", action="store_true", help="skip the N=2048 phase diagram (~70 s)")
    ap.add_argument("--U", type=float, default=2.0, help="pairing U of every workload (2 = the stated one)")
    args = ap.parse_args()

    from paper_1412_8754_gb300 import workloads

    cfg = workloads.fflo_scan(N=args.N, n_q=args.n_q)
    cfg["U"] = args.U
    ws, rank, local = dist_env()

    if args.impl == "reference":
        run_reference(args, cfg, ws, rank)
        return

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1412_8754_gb300 import ffe, shard

    # shard the q list across ranks, round robin (q = 0, the label reference, on rank 0 only)
    q_all = cfg["qx"]
    mine = shard.shard_q(len(q_all), rank, ws)
    has_q0 = 0 in mine
    qx = q_all[mine]
    qy = np.zeros_like(qx)
    n_pts = len(cfg["h"]) * len(cfg["T"])
    stream = torch.cuda.current_stream()
    ctx = ffe.Context(prec=ffe.FFE_FP32C, U=cfg["U"])
    plan = ctx.plan_phase_scan(cfg["N"], qx, qy, cfg["h"], cfg["T"], n=cfg["n"], lo=cfg["lo"], hi=cfg["hi"])
    info = plan.stats()
    k_evals, launches = info["k_evals"], info["launches"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        plan.execute(stream)
    plan.fetch(stream, labels=has_q0)
    plan.kernel_ms()  # discard warm-up kernel timings
    clocks = Clocks(local)
    barrier()
    clocks.begin()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush between timed steps (outside the event pair)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.execute(stream)
        e1.record(stream)
        evs.append((e0, e1))
    barrier()
    clocks.end()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_total = sum(step_ms) / 1e3
    kern_ms, kern_n = plan.kernel_ms()
    res, labels, best = plan.fetch(stream, labels=has_q0)
    if ws > 1:  # labels over the union of the ranks' q lists (outer argmin of Alg. 1)
        omega_n = shard.broadcast_normal_state(res["omega_lo"][0] if has_q0 else np.zeros(n_pts), src=0)
        bv, bq = shard.local_candidates(res, mine, omega_n)
        labels, best = shard.gather_labels(bv, bq, omega_n)
        t = torch.tensor([t_total], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_total = float(t.item())
        kt = torch.tensor([k_evals], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(kt)
        k_job = float(kt.item())
        pts = torch.tensor([float(len(mine) * n_pts)], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(pts)
        points_job = float(pts.item())
    else:
        k_job = k_evals
        points_job = float(len(mine) * n_pts)
    value = k_job * args.steps / t_total
    points_per_s = points_job * args.steps / t_total

    # end to end through the host-buffer C ABI (inputs copied in, results copied out, every step;
    # on several ranks each times its own part, the job's time is the slowest rank's)
    e2e_times = []
    for i in range(max(2, min(args.steps, 5))):
        barrier()
        t0 = time.perf_counter()
        full = ctx.phase_scan(cfg["N"], qx, qy, cfg["h"], cfg["T"], n=cfg["n"], lo=cfg["lo"], hi=cfg["hi"],
                              stream=stream, labels=has_q0)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_t = statistics.median(e2e_times[1:])
    h2d = len(q_all) * (cfg["n"] * 8 + n_pts * 24 + len(cfg["h"]) * 8 + 128)
    d2h = len(q_all) * n_pts * 40 + n_pts * 5
    if ws > 1:
        t = torch.tensor([e2e_t], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_t = float(t.item())

    # FP64 plain kernel on a sample of the q list (it is ~60x slower)
    fp64 = None
    if args.fp64_sample_q > 0 and rank == 0:
        ctx64 = ffe.Context(prec=ffe.FFE_FP64, U=cfg["U"])
        qs = q_all[: args.fp64_sample_q]
        p64 = ctx64.plan_phase_scan(cfg["N"], qs, np.zeros_like(qs), cfg["h"], cfg["T"], n=cfg["n"],
                                    lo=cfg["lo"], hi=cfg["hi"])
        k64 = p64.stats()["k_evals"]
        p64.execute(stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p64.execute(stream)
        torch.cuda.synchronize()
        dt64 = time.perf_counter() - t0
        fp64 = {"k_evals_per_s": k64 / dt64, "points_per_s": len(qs) * n_pts / dt64,
                "sample": f"{len(qs)} q x {n_pts} (h,T) x {cfg['n']} Delta at N={cfg['N']}"}
        p64.destroy()
        ctx64.close()

    # the Omega grids of two lines of the timed plan, for the oracle check of the CPU leg
    check_lines = []
    if rank == 0 and ws == 1 and not args.no_cpu:
        og = plan.fetch_grid(cfg["n"], stream)
        for q, ih in ((5, 3), (0, 11)):
            check_lines.append({"qx": float(qx[q]), "h": float(cfg["h"][ih]), "omega": og[q, ih],
                                "idx_star": int(res["idx_star"][q, ih])})
    extras, pd_check = {}, None
    if rank == 0 and not args.no_extras:
        extras = run_extras(ffe, np, torch, stream, workloads)
        if ws == 1:
            pd_check, pd_out, extras["surrogate"] = run_surrogate(ffe, np, torch, workloads, cfg, full, e2e_t,
                                                                  fp64["k_evals_per_s"] if fp64 else None,
                                                                  diagram=not args.no_diagram)
            if pd_out:
                extras["phase_diagram"] = pd_out

    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    pst = plan.stats()
    # a work item of the shared-T layout: tiles of 8 (h, T) entries x 4 Delta rows, 24 tiles
    # (96 Delta rows); R and a per (k-point, band, Delta row) serve the row's 8 outputs
    per_row = min(8, n_pts)
    outs_item = min(96, cfg["n"]) * per_row
    c_near, c_single, c_far, c_mom = sfu_clk_per_band_eval(per_row, outs_item)
    band_evals = 2.0 * k_evals  # two bands per k-evaluation
    b_near, b_single = pst["k_evals_near"], pst["k_evals_single"]  # full-term band evaluations
    b_fc = pst["k_evals_far_closed"]  # far band evaluations in the closed form
    near_frac = b_near / band_evals if band_evals else 0.0
    single_frac = b_single / band_evals if band_evals else 0.0
    fc_frac = b_fc / band_evals if band_evals else 0.0
    clk_per_keval = 2.0 * ((near_frac - single_frac) * c_near + single_frac * c_single + fc_frac * c_far
                           + (1.0 - near_frac - fc_frac) * c_mom)
    peak = n_sm * SM_MAX_MHZ * 1e6 / clk_per_keval  # k-evals/s with the SFU saturated, at the maximum clock
    achieved = k_evals / (kern_ms / 1e3) if kern_ms > 0 else 0.0
    # the algorithmic bound: every k-eval with its 10 transcendentals (2 sqrt + 4 exp + 4 log, both
    # bands) at the SFU rates ffe_probe_peaks measures, or the FP32 pipe at ~50 operations
    pk = ffe.ffe_probe_peaks()
    sfu_bound = 1.0 / (4.0 / pk["ex2"] + 4.0 / pk["lg2"] + 2.0 / pk["rsqrt"])
    fp32_bound = pk["fma32"] / 50.0
    alg_peak = min(sfu_bound, fp32_bound)

    out = {
        "metric": METRIC, "value": value, "unit": "k-evals/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": arm_config(cfg, ws),
        "points_per_s": points_per_s,
        "e2e": {"value": k_job / e2e_t, "unit": "k-evals/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "points_per_s": points_job / e2e_t},
        "gpu_launches": launches * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "k-evals/s (SFU-bound)",
                     "frac": achieved / peak if peak else None, "traffic": DRAM_TRAFFIC_PER_LAUNCH,
                     "kernel": f"ksum_kernel<float,{info['kpt']},shared-Delta>", "kernel_ms": kern_ms,
                     "kernel_launches": kern_n,
                     "near_band_fraction": near_frac, "near_one_exp_fraction": single_frac,
                     "far_closed_fraction": fc_frac,
                     "peak_basis": (f"{n_sm} SM x {SM_MAX_MHZ:.0f} MHz / {clk_per_keval:.4f} SFU clocks per "
                                    f"k-eval = 2 bands x ({near_frac - single_frac:.4f} x {c_near:.4f} (full "
                                    f"term, two ex2) + {single_frac:.4f} x {c_single:.4f} (full term, one ex2) "
                                    f"+ {fc_frac:.4f} x {c_far:.4f} (far, R and a) + "
                                    f"{1 - near_frac - fc_frac:.4f} x {c_mom:.5f} (far, moments)); ex2 "
                                    f"{SFU_EX2_PER_CLK}/clk, lg2 rsqrt rcp {SFU_OTHER_PER_CLK}/clk per SM; unit "
                                    f"counts checked by ffe_probe_peaks"),
                     "frac_algorithmic": achieved / alg_peak,
                     "peak_algorithmic": alg_peak,
                     "peak_algorithmic_basis": (
                         f"every k-eval with its 10 transcendentals (2 sqrt + 4 exp + 4 log) at the measured "
                         f"SFU rates (ex2 {pk['ex2']:.3g}/s, lg2 {pk['lg2']:.3g}/s, rsqrt {pk['rsqrt']:.3g}/s: "
                         f"{sfu_bound:.3g} k-evals/s), or the FP32 pipe at 50 operations ({fp32_bound:.3g}); "
                         f"work-reduced: far bands skip the transcendentals (their log factors are exactly 1 in "
                         f"FP32), so the kernel exceeds this bound"),
                     "ncu": NCU_HEADLINE},
        "fp64_reevals_per_step": {"search": pst["rescored_search"], "labels": pst["rescored_labels"]},
        "fp64": fp64,
        **extras,
        "clocks": clk,
        "labels": {"normal": int((labels == 0).sum()), "bcs": int((labels == 1).sum()),
                   "fflo": int((labels == 2).sum())},
    }
    if rank == 0 and ws == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(cfg, check_lines, pd_check)
    if rank == 0:
        print(json.dumps(out), flush=True)
    plan.destroy()
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def arm_config(cfg, ws):
    """The workload named in both arms' JSON lines."""
    return {"workload": f"fflo_scan N={cfg['N']}: {len(cfg['qx'])} q x {len(cfg['h'])} h x "
                        f"{len(cfg['T'])} T x {cfg['n']} Delta, U={cfg['U']}, FP32 + FP64 ties",
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"q sharded over {ws} rank(s)" if ws > 1 else "1 GPU"}


def run_reference(args, cfg, ws, rank):
    """The oracle (FP64, OpenMP on the host cores) on the same metric, bounded sample per step."""
    if rank != 0:
        return
    import numpy as np

    import oracle

    m = oracle.make_model(U=cfg["U"])
    N = cfg["N"]
    grid = np.linspace(cfg["lo"], cfg["hi"], cfg["n"])
    th = threads_hint()
    sample = grid[: max(th, 16)]
    for _ in range(args.warmup):
        oracle.omega_batch(m, N, cfg["qx"][5], 0.0, cfg["h"][3], cfg["T"][0], sample[:th])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, _, used = oracle.omega_batch(m, N, cfg["qx"][5], 0.0, cfg["h"][3], cfg["T"][0], sample)
    dt = time.perf_counter() - t0
    kev = float(N * N) * len(sample) * args.steps
    v = kev / dt
    desc = f"{len(sample)} Delta values of one (q, h) at N={N} per step (FP64 oracle, OpenMP)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "k-evals/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(cfg, ws),
        "cpu_baseline": {"value": v, "unit": "k-evals/s", "cores": used, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "k-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


if __name__ == "__main__":
    main()
