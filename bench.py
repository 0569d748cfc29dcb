"""Benchmark of the GRMHD Runge-Kutta stage on GB300: zone-updates/s per RK stage.

One "step" is one Runge-Kutta stage (reconstruction, Riemann fluxes, CT, divergence + sources, RK
combination, con2prim + floors, CFL reduction) over one meshblock. Default workload: the 256^3 Kerr-Schild
(a = 0.9) block of seeded random primitives (rho log-uniform in [1e-6, 1], P = 0.01 rho^5/3, W to 10,
sigma to 50; fixed ghosts), WENO5-Z-AOAH + HLL, in the mixed form (float reconstruction / fluxes / EMFs /
sources, double accumulation and con2prim); the all-FP64 form of the same workload and the L1 distance
between the two are reported beside it.

  python bench.py [--gpus N --steps K --warmup W] [--n 256] [--impl reference]

Multi-GPU (torchrun): every rank advances its own independent block (seed + rank); there is no data-path
collective, so the scaling is weak and the value is the sum of all ranks' zone updates over the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "zone-updates/s per RK stage at 1 GB300 (mixed vs all-FP64, at stated L1 err)"
UNIT = "zone-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-guess", action="store_true")
    ap.add_argument("--no-face-ct", action="store_true")
    ap.add_argument("--no-two-level", action="store_true")
    ap.add_argument("--no-scalar", action="store_true")
    ap.add_argument("--no-spherical", action="store_true")
    ap.add_argument("--guess-states", type=int, default=100_000_000)
    ap.add_argument("--guess-only", action="store_true",
                    help="run only the learned-guess con2prim section and print its JSON (profiling aid)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def workload(n, precision, rank=0):
    from paper_2410_09146_gb300 import inputs as I
    s = I.kerr_schild_setup(n, recon="weno5z_aoah", riemann="hll", precision=precision)
    return s, 2 + rank


def stage_coeffs(k):
    return (0.0, 1.0, 1.0) if k % 2 == 0 else (0.5, 0.5, 0.5)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (the JSON line carries their summary): BENCH_CLOCKS_DIR, else the temporary directory
        import tempfile
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        load = [r[0] for r in rows if r[2] > 200.0] or [r[0] for r in rows]
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def l1_rel(a, b):
    """Per-variable L1 distance sum |a - b| / sum |b| over the leading axis."""
    return np.array([np.abs(a[v] - b[v]).sum() / max(np.abs(b[v]).sum(), 1e-300) for v in range(a.shape[0])])


def measured_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


# ----------------------------------------------------------------------------- aggregation across ranks
def aggregate(ms_local, zones_local, steps, dist=None, device=None):
    """Whole-job throughput: the slowest rank's time (max over ranks) and the sum of all ranks' zone
    updates. Returns (value in zone-updates/s, max ms, world size)."""
    if dist is None or not dist.is_initialized():
        return zones_local * steps / (ms_local / 1e3), ms_local, 1
    import torch
    t = torch.tensor([ms_local, float(zones_local)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    ms = float(mx[0])
    return float(sm[1]) * steps / (ms / 1e3), ms, dist.get_world_size()


# ----------------------------------------------------------------------------- our arm
def time_stages(ctx, k0, n_stages):
    import torch
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for k in range(n_stages):
        g0, g1, b = stage_coeffs(k0 + k)
        ctx.stage(g0, g1, b, 0.0)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2410_09146_gb300 import build as B
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2410_09146_gb300 import grmhd as G
    from paper_2410_09146_gb300 import inputs as I

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    n = args.n
    fp_peaks = live_fp_peaks(G)
    s_mix, seed = workload(n, "mixed", rank)
    P, Bf = I.kerr_schild_random_prims(s_mix, seed=seed, faces=True)
    cells = n ** 3
    # ---- mixed form: warm-up, timed region (device events, clocks sampled)
    ctx = G.Context(s_mix)
    ctx.set_prims(P)
    for k in range(args.warmup):
        ctx.stage(*stage_coeffs(k), 0.0)
    k0 = args.warmup + (args.warmup % 2)
    if args.warmup % 2:
        ctx.stage(*stage_coeffs(args.warmup), 0.0)
    barrier()
    with ClockSampler(local) as clk:
        ms = time_stages(ctx, k0, args.steps)
        barrier()
    ms = max_over_ranks(ms)
    clocks = clk.summary()
    stats = ctx.stats()
    # ---- per-kernel timing pass (events around each kernel group, same stream)
    ctx.set_timing(True)
    time_stages(ctx, k0, min(args.steps, 8))
    kt, kst = ctx.timing()
    ctx.set_timing(False)
    del ctx
    torch.cuda.empty_cache()
    # ---- end to end through the C ABI with pinned host buffers: H2D of P, stage, D2H of P
    ctx = G.Context(s_mix)
    # the mixed form stores its primitives in float: the user's host buffers are float too
    Ph = torch.from_numpy(P.astype(np.float32)).pin_memory()
    Po = torch.empty_like(Ph).pin_memory()
    # one call per step: the load (its copies beside the prim->cons), the stage, and the read-back of the
    # stage's primitives beside the update (grmhd_stage_host_f32). One untimed step first (the first
    # device-to-host read into fresh pinned pages is slower).
    G.grmhd_stage_host_f32(ctx.ctx, Ph, Po, 0.0, 1.0, 1.0, 0.0)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(2, min(args.steps, 6))
    for k in range(e2e_steps):
        G.grmhd_stage_host_f32(ctx.ctx, Ph, Po, 0.0, 1.0, 1.0, 0.0)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    del ctx
    torch.cuda.empty_cache()
    # ---- all-FP64 form of the same workload, and the L1 distance after one RK2 step
    s64, _ = workload(n, "fp64", rank)
    c64 = G.Context(s64)
    c64.set_prims(P)
    c64.rk2_step(0.0)
    U64 = c64.cons()
    P64 = c64.prims()
    for k in range(2):
        c64.stage(*stage_coeffs(k), 0.0)
    barrier()
    ms64 = time_stages(c64, 0, args.fp64_steps)
    barrier()
    ms64 = max_over_ranks(ms64)
    del c64
    torch.cuda.empty_cache()
    cm = G.Context(s_mix)
    cm.set_prims(P)
    cm.rk2_step(0.0)
    ng = s_mix.ng
    inner = (slice(None),) + (slice(ng, -ng),) * 3
    l1u = l1_rel(cm.cons(), U64)
    l1p = l1_rel(cm.prims()[inner], P64[inner])
    del cm
    torch.cuda.empty_cache()
    face_ct = None if args.no_face_ct else run_face_ct(G, s_mix, P, Bf, args.steps, args.warmup)
    two_level = None if args.no_two_level else run_two_level(G, I, s_mix.recon, args.steps, args.warmup)
    scalar = None if args.no_scalar else run_scalar(G, s_mix, P, args.steps, args.warmup, ms / args.steps)
    spherical = None if args.no_spherical else run_spherical(G, I, args.steps, args.warmup)
    del Bf
    guess = None if args.no_guess else run_guess(G, I, rank, n_states=args.guess_states)
    batched = None
    if not args.no_batched:
        batched, bms, bzones = run_batched(G, I, max(4, min(args.steps, 10)), args.warmup, rank)
        bval, bms_max, _ = aggregate(bms, bzones, batched["steps"], dist if world > 1 else None, "cuda")
        batched["value"] = bval
    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    per_stage = ms / args.steps
    value = world * cells * args.steps / (ms / 1e3)
    fp64_value = world * cells * args.fp64_steps / (ms64 / 1e3)
    # dominant kernel group and its roofline
    per_kernel = {k: v / max(kst, 1) for k, v in kt.items()}
    dom = max(per_kernel, key=per_kernel.get)
    peaks = measured_peaks()
    roof = roofline(dom, per_kernel[dom], n, stats, fp_peaks, per_stage, peaks)
    roof["fp_peaks_tflops"] = {"fp64": fp_peaks[0], "fp32": fp_peaks[1], "how": "grmhd_fp_peaks on this GPU, "
                               "before the timed region"}
    G_cells = (n + 2 * s_mix.ng) ** 3
    h2d = Ph.numel() * Ph.element_size()  # the float primitives copied each way per step
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_stage, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic (seeded random Kerr-Schild primitives)",
        "config": {"workload": f"kerr_schild_random_{n}^3_weno5z_aoah_hll_mixed", "n": n, "ghosts": s_mix.ng,
                   "metric": "kerr_schild a=0.9", "recon": "weno5z_aoah", "riemann": "hll", "precision": "mixed",
                   "cfl": s_mix.cfl, "l2": f"state of {8 * G_cells * 4 / 1e9 + 24 * cells * 8 / 1e9:.1f} GB, "
                   "inputs larger than L2 (no flush needed)", "parallelism": f"replicas x{world}"},
        "fp64": {"value": fp64_value, "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps,
                 "speedup_mixed_over_fp64": value / fp64_value},
        "l1_mixed_vs_fp64": {"after": "one RK2 step", "U": [float(x) for x in l1u], "P": [float(x) for x in l1p],
                             "max": float(max(l1u.max(), l1p.max()))},
        "c2p": {"iterations_per_cell": float(stats[0]) / cells, "eps_floor_cells": int(stats[2]),
                "w_cap_cells": int(stats[3]), "max_iterations": int(stats[6])},
        "kernels_ms_per_stage": per_kernel,
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": world * cells * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": h2d, "call": "grmhd_stage_host_f32: the load's copies beside its prim->cons, "
                "the read-back beside the update, pinned float host buffers"},
        # per stage: 3 flux, EMF, update, the two deferred con2prim passes; the CFL finalisation per step
        "gpu_launches": 7 * args.steps + (args.steps + 1) // 2,
    }
    if face_ct is not None:
        out["face_ct"] = face_ct
    if two_level is not None:
        out["two_level"] = two_level
    if scalar is not None:
        out["scalar"] = scalar
    if spherical is not None:
        out["spherical"] = spherical
    if batched is not None:
        out["batched"] = batched
    if guess is not None:
        out["c2p_guess"] = guess
    if not args.no_cpu_baseline:
        out["cpu_baseline"], ref = cpu_baseline(n)
        out["l1_mixed_vs_oracle"] = l1_vs_oracle(G, ref)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def _iter_summary(iters, status, torch):
    """Mean and 99th percentile of per-state iterations (from their histogram), non-converged fraction."""
    h = torch.bincount(iters.to(torch.int64)).double()
    c = torch.cumsum(h, 0) / h.sum()
    p99 = int(torch.searchsorted(c, torch.tensor([0.99], dtype=torch.float64, device=c.device)).item())
    mean = float((h * torch.arange(len(h), dtype=torch.float64, device=h.device)).sum() / h.sum())
    return {"mean_iterations": mean, "p99_iterations": p99,
            "not_converged_frac": float(((status & 8) != 0).double().mean())}


def run_guess(G, I, rank, n_states=100_000_000, n_train=10_000_000, train_steps=3000, reps=3):
    """Learned con2prim guess: train on pairs solved by the library's FP64 con2prim (standard start), then
    time the flat con2prim batch of n_states fresh states from the standard start and from the network's
    start, with per-state iteration statistics and the agreement of the two solutions."""
    import torch
    dev = torch.device("cuda")
    ctx = G.Context(I.Setup(n=(0, 0, 0)))  # c2p_tol 1e-10
    # ---- training pairs
    P = I.c2p_states_device(n_train, seed=7000 + rank, device=dev)
    U = torch.empty_like(P)
    ctx.p2c(P, U)
    st = torch.empty(n_train, dtype=torch.uint8, device=dev)
    X = torch.empty((n_train, 8), dtype=torch.float32, device=dev)
    T = torch.empty((n_train, 2), dtype=torch.float32, device=dev)
    ctx.c2p_guess(U, P, st, None, X=X, T=T)
    keep = (st & (8 | 16)) == 0
    X, T = X[keep].contiguous(), T[keep].contiguous()
    del P, U, st, keep
    # the same training twice from the same start: gradients on the FP32 cores, then on the tensor cores (the
    # network the rest of this section uses)
    train = {}
    for tc in (False, True):
        net = G.GuessNet(seed=11)
        net.fit_norm(X, T)
        losses = torch.zeros(train_steps, dtype=torch.float32, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        net.train(X, T, batch=152 * 128, steps=train_steps, lr=3e-3, lr_end=3e-5, aux=0.1, losses=losses, tc=tc)
        e1.record()
        torch.cuda.synchronize()
        lh = losses.cpu().numpy()
        train["tensor_cores" if tc else "fp32_cores"] = {"ms": e0.elapsed_time(e1),
                                                          "ms_per_step": e0.elapsed_time(e1) / train_steps,
                                                          "loss_first": float(lh[:10].mean()),
                                                          "loss_last": float(lh[-100:].mean())}
    train_ms = train["tensor_cores"]["ms"]
    n_pairs = X.shape[0]
    del X, T
    torch.cuda.empty_cache()
    # ---- evaluation states (inputs larger than L2)
    P = I.c2p_states_device(n_states, seed=9000 + rank, device=dev)
    U = torch.empty_like(P)
    ctx.p2c(P, U)
    Ps, Pn = P, torch.empty_like(P)
    sts = torch.empty(n_states, dtype=torch.uint8, device=dev)
    stn = torch.empty_like(sts)
    its = torch.empty(n_states, dtype=torch.int32, device=dev)
    itn = torch.empty_like(its)
    guess = torch.empty((2, n_states), dtype=torch.float64, device=dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms_std = timed(lambda: ctx.c2p_guess(U, Ps, sts, its))
    ms_f32 = timed(lambda: ctx.c2p_guess(U, Pn, stn, itn, net=net, guess=guess, fp32=True))
    fall_f32 = int(ctx.stats()[7])
    sum_f32 = _iter_summary(itn, stn, torch)
    mis_f32 = int((sts != stn).sum())
    ms_tc = timed(lambda: ctx.c2p_guess(U, Pn, stn, itn, net=net))
    stats_tc = ctx.stats()
    # backward error |U(P) - U| / (|D| + |tau| + |S|) of each solution on states no solve floored or
    # flagged (forward differences between them are bounded by the conditioning, not the solver)
    plain = (sts == 0) & (stn == 0)
    scale = U[0].abs() + U[4].abs() + torch.linalg.vector_norm(U[1:4], dim=0)
    Ub = torch.empty_like(U)
    berr = []
    for Pd in (Ps, Pn):
        ctx.p2c(Pd, Ub)
        berr.append(float(((Ub - U).abs().amax(dim=0) / scale)[plain].max()))
    del Ub
    mism = _status_mismatch(ctx, U, Ps, Pn, sts, stn, torch)
    out = {"states": n_states, "c2p_tol": 1e-10,
           "train": {"pairs": n_pairs, "source": "the library's FP64 con2prim from the standard start",
                     "steps": train_steps, "batch": 152 * 128, "ms": train_ms,
                     "loss_first": float(lh[:10].mean()), "loss_last": float(lh[-100:].mean()),
                     "gradient": "tensor cores (grmhd_mlp_train_tc): 64 x 64 products and weight gradients as "
                                 "tcgen05 MMAs, BF16 operands, FP32 accumulation", "compare": train},
           "standard": dict(_iter_summary(its, sts, torch), ms=ms_std, states_per_s=n_states / (ms_std / 1e3)),
           "network_tc": dict(_iter_summary(itn, stn, torch), ms=ms_tc, states_per_s=n_states / (ms_tc / 1e3),
                              fallback_frac=int(stats_tc[7]) / n_states, abandoned_tiles=int(stats_tc[6]),
                              kernel="fused: hidden layers as tcgen05 MMAs, FP64 Newton in the same kernel"),
           "network_fp32": dict(sum_f32, ms=ms_f32, states_per_s=n_states / (ms_f32 / 1e3),
                                fallback_frac=fall_f32 / n_states,
                                kernel="network on the FP32 cores, then the FP64 solve (two kernels)"),
           "status_mismatch": {"network_fp32": mis_f32, "network_tc": int((sts != stn).sum()), "network_tc_detail": mism},
           "max_backward_err": {"standard": berr[0], "network_tc": berr[1]}}
    out["speedup_tc"] = ms_std / ms_tc
    out["speedup_fp32"] = ms_std / ms_f32
    del P, U, Pn, guess, sts, stn, its, itn, net, ctx
    torch.cuda.empty_cache()
    return out


def _status_mismatch(ctx, U, Pa, Pb, sta, stb, torch):
    """States whose status bits differ between two solves of the same conserved states (standard start and
    network start): which bits, and how far the solution on which the floor did not fire sits from the
    floor's threshold. A floor decision taken on opposite sides of its threshold by two solutions that both
    meet the root tolerance is a tie at the threshold, within the solve's accuracy at that state."""
    idx = (sta != stb).nonzero().flatten()
    if idx.numel() == 0:
        return {"count": 0}
    a, b = sta[idx].int(), stb[idx].int()
    diff = a ^ b
    bits = {name: int(((diff & m) != 0).sum()) for name, m in (("rho_floor", 1), ("eps_floor", 2), ("w_cap", 4),
                                                                ("not_converged", 8), ("bad_input", 16))}
    p = ctx.p
    Pa_, Pb_ = Pa[:, idx], Pb[:, idx]
    # the eps floor: u >= rho eps_floor0 (flat space); margin of the solution without the floor bit
    free_a = (a & 2) == 0
    Pf = torch.where(free_a[None, :], Pa_, Pb_)
    eps_margin = (Pf[4] / (Pf[0] * p.eps_floor0) - 1.0).abs()
    # the Lorentz-factor cap: W <= w_max; margin of the solution without the cap bit
    free_wa = (a & 4) == 0
    Pw = torch.where(free_wa[None, :], Pa_, Pb_)
    W = torch.sqrt(1.0 + (Pw[1:4] ** 2).sum(0))
    w_margin = (W / p.w_max - 1.0).abs()
    eps_sel = (diff & 2) != 0
    w_sel = (diff & 4) != 0
    # relative difference of mu = 1/(h W) between the two solutions (both meet |d mu| <= 1e-10 mu)
    def mu(P):
        Wp = torch.sqrt(1.0 + (P[1:4] ** 2).sum(0))
        h = 1.0 + ctx.setup.gamma_eos * P[4] / P[0]
        return 1.0 / (h * Wp)
    return {"count": int(idx.numel()), "bits": bits,
            "eps_floor_margin_max": float(eps_margin[eps_sel].max()) if eps_sel.any() else None,
            "w_cap_margin_max": float(w_margin[w_sel].max()) if w_sel.any() else None,
            "mu_rel_diff_max": float(((mu(Pa_) - mu(Pb_)).abs() / mu(Pa_)).max())}


def batched_setups():
    """The 640-block batched workload (inputs.batched_setups): block b's primitives use seed 3 + b."""
    from paper_2410_09146_gb300 import inputs as I
    return I.batched_setups()


def _face_divergence(B, s, torch):
    """max |sum_d (Bf_d(upper) - Bf_d(lower)) / dx_d| x min dx / max |Bf| over the interior cells."""
    ng = s.ng
    nx, ny, nz = s.n
    div = None
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        lo = [slice(ng, ng + nz), slice(ng, ng + ny), slice(ng, ng + nx)]
        hi = list(lo)
        hi[ax] = slice(lo[ax].start + 1, lo[ax].stop + 1)
        t = (B[d][tuple(hi)] - B[d][tuple(lo)]) / s.dx[d]
        div = t if div is None else div + t
    return float(div.abs().max() * min(s.dx) / B.abs().max())


def run_face_ct(G, s_mix, P, Bf, steps, warmup):
    """The same workload with face-centred upwind CT (the field on the faces): stage throughput, per-kernel
    times, and the face divergence before and after the timed stages."""
    import dataclasses
    import torch
    s = dataclasses.replace(s_mix, ct="face")
    ctx = G.Context(s)
    ctx.set_prims(P)
    ctx.set_face_b(Bf)
    B = torch.empty((3,) + tuple(P.shape[1:]), dtype=torch.float64, device="cuda")
    ctx.get(G.GRMHD_GET_FACE_B, out=B)
    div0 = _face_divergence(B, s, torch)
    for k in range(warmup):
        ctx.stage(*stage_coeffs(k), 0.0)
    k0 = warmup + (warmup % 2)
    if warmup % 2:
        ctx.stage(*stage_coeffs(warmup), 0.0)
    torch.cuda.synchronize()
    ms = time_stages(ctx, k0, steps)
    ctx.set_timing(True)
    time_stages(ctx, k0, min(steps, 8))
    kt, kst = ctx.timing()
    ctx.set_timing(False)
    ctx.get(G.GRMHD_GET_FACE_B, out=B)
    torch.cuda.synchronize()
    div = _face_divergence(B, s, torch)
    cells = s.n[0] * s.n[1] * s.n[2]
    out = {"value": cells * steps / (ms / 1e3), "unit": UNIT, "ms_per_stage": ms / steps, "steps": steps,
           "kernels_ms_per_stage": {k: v / max(kst, 1) for k, v in kt.items()},
           "emf_group": "cell-centred EMFs, upwind edge EMFs and the Stokes update of the faces",
           "face_divergence_rel": {"initial": div0, "after": div, "stages": warmup + (warmup % 2) + steps + min(steps, 8)},
           "scheme": "face-centred field, upwind (contact) edge EMFs of Gardiner & Stone 2005"}
    del ctx, B
    torch.cuda.empty_cache()
    return out


def run_scalar(G, s_mix, P, steps, warmup, ms_plain):
    """The same workload with one passive scalar (the electron fraction, say) advanced too: stage
    throughput and the scalar's cost per stage against the plain stage."""
    import dataclasses
    import numpy as np
    import torch
    s = dataclasses.replace(s_mix, scalar=True)
    ctx = G.Context(s)
    ctx.set_prims(P)
    x = s.cell_centres(0)
    X = np.broadcast_to((0.1 + 0.4 * (x > 0.5 * (s.x0[0] + x[-1])))[None, None, :], s.prim_shape()[1:]).copy()
    ctx.set_scalar(X)
    for k in range(warmup + (warmup % 2)):
        ctx.stage(*stage_coeffs(k), 0.0)
    torch.cuda.synchronize()
    ms = time_stages(ctx, 0, steps)
    cells = s.n[0] * s.n[1] * s.n[2]
    out = {"value": cells * steps / (ms / 1e3), "unit": UNIT, "ms_per_stage": ms / steps, "steps": steps,
           "scalar_ms_per_stage": ms / steps - ms_plain, "scheme": "sqrt(gamma) D X carried by the face mass flux, "
           "X reconstructed like the primitives and taken on the upwind side"}
    del ctx
    torch.cuda.empty_cache()
    return out


def run_spherical(G, I, steps, warmup):
    """Spherical Kerr-Schild coordinates (ln r, theta, phi): the stationary torus around the a = 0.9 hole (specific
    angular momentum Keplerian at r = 12, inner edge r = 6) on a full sphere with polar and azimuthal ghosts,
    128 x 96 x 64 cells over r in [2, 40], WENO5-Z-AOAH + HLL; mixed and all-FP64 forms, CFL time step."""
    import torch
    out = {}
    nr, nth, nph = 128, 96, 64
    zones = nr * nth * nph
    for prec in ("mixed", "fp64"):
        s = I.full_sphere_setup(nr, nth, nph, r_lo=2.0, r_hi=40.0, precision=prec)
        ctx = G.Context(s)
        ctx.set_prims(I.torus_prims(s))
        for k in range(warmup + (warmup % 2)):
            ctx.stage(*stage_coeffs(k), 0.0)
        torch.cuda.synchronize()
        n = steps if prec == "mixed" else max(2, steps // 5 // 2 * 2)
        ms = time_stages(ctx, 0, n)
        out[prec] = {"value": zones * n / (ms / 1e3), "unit": UNIT, "ms_per_stage": ms / n, "steps": n}
        del ctx
        torch.cuda.empty_cache()
    out["speedup_mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["workload"] = (f"torus in spherical Kerr-Schild coordinates, full sphere {nr} x {nth} x {nph} (ln r, theta, "
                       "phi), r in [2, 40], a = 0.9, WENO5-Z-AOAH + HLL")
    return out


def two_level_mesh_workload(I, recon, precision):
    """Kerr-Schild two-level mesh: 4 x 4 x 4 root blocks of 32^3 over [3, 23]^3, the 8 roots next to the hole
    refined (56 root blocks + 64 children: 120 blocks of 32^3, 3.93 M zones)."""
    root = I.Setup(n=(32, 32, 32), x0=(3.0, 3.0, 3.0), dx=(20.0 / 128,) * 3, metric="kerr_schild", spin=0.9,
                   mass=1.0, recon=recon, riemann="hll", bc="fixed", precision=precision)
    refined = [(x, y, z) for z in range(2) for y in range(2) for x in range(2)]
    return I.two_level_mesh(root, (4, 4, 4), refined, False)


def run_two_level(G, I, recon, steps, warmup):
    """Stage throughput of the two-level mesh (ghost exchange between levels, refluxing), replayed from CUDA
    graphs, and the same batch with the mesh switched off (blocks with loaded ghosts, no exchange or
    refluxing): the difference is what the mesh costs."""
    import torch
    m = two_level_mesh_workload(I, recon, "mixed")
    setups = [m.setup(b) for b in range(m.nblocks)]
    Ps = I.two_level_prims(m, seed=11)
    res = {}
    for mode in ("mesh", "blocks only"):
        bc = G.BatchContext(setups)
        for b in range(m.nblocks):
            bc.set_prims(b, Ps[b])
        if mode == "mesh":
            bc.set_mesh(m.nb, m.periodic, m.levels, m.pos)
        tile, _ = bc.autotune()
        bc.set_graph(True)
        for k in range(max(warmup, 2)):
            bc.stage(*stage_coeffs(k), 0.0)
        torch.cuda.synchronize()
        res[mode] = time_stages(bc, 0, steps)
        del bc
        torch.cuda.empty_cache()
    zones = m.nblocks * 32 ** 3
    ms = res["mesh"] / steps
    return {"blocks": m.nblocks, "fine_blocks": sum(m.levels), "zones": zones, "ms_per_stage": ms, "steps": steps,
            "zone_updates_per_s": zones / (ms / 1e3), "ms_per_stage_without_mesh": res["blocks only"] / steps,
            "mesh_overhead_ms": ms - res["blocks only"] / steps,
            "scheme": "two-pass ghost exchange (copy, restriction, minmod prolongation), Berger-Colella refluxing",
            "workload": "Kerr-Schild a = 0.9 over [3, 23]^3: 4^3 root blocks of 32^3, the 8 nearest the hole refined"}


def run_batched(G, I, steps, warmup, rank):
    """The 640-block batch: autotuned work items, stages replayed from CUDA graphs."""
    import torch
    setups = batched_setups()
    bc = G.BatchContext(setups)
    for b, s in enumerate(setups):
        bc.set_prims(b, I.kerr_schild_random_prims(s, seed=3 + b + 1000 * rank))
    tile, tune_ms = bc.autotune()
    bc.set_graph(True)
    for k in range(max(warmup, 2)):
        bc.stage(*stage_coeffs(k), 0.0)
    torch.cuda.synchronize()
    ms = time_stages(bc, 0, steps)
    zones = sum(s.n[0] * s.n[1] * s.n[2] for s in setups)
    cells = sum((s.n[0] + 2 * s.ng) * (s.n[1] + 2 * s.ng) * (s.n[2] + 2 * s.ng) for s in setups)
    stats = bc.stats()
    del bc
    torch.cuda.empty_cache()
    return {"blocks": len(setups), "zones": zones, "cells_with_ghosts": cells, "ghost_overhead": cells / zones,
            "tile": tile, "ms_per_stage": ms / steps, "steps": steps,
            "graph": "one CUDA graph per distinct stage, replayed", "zone_updates_per_s": zones * steps / (ms / 1e3),
            "c2p_iterations_per_cell": float(stats[0]) / zones}, ms, zones


# Work and traffic per unit of the mixed-form kernels, measured by ncu (--set full, one kernel per capture)
# on the 96^3 Kerr-Schild random block (summaries under profiles/): double-precision flops (DADD + DMUL +
# 2 DFMA, active lanes) per cell of k_update (mean of the g0 = 0 and g0 != 0 stages), float flops (FADD + FMUL
# + 2 FFMA) per face of k_flux_cc (mean of the three directions), DRAM bytes (read + write) per unit.
UPDATE_FP64_FLOP_PER_CELL = 158.0
UPDATE_DRAM_BYTES_PER_CELL = 324.2
# algorithmic bytes per cell of k_update: P (8 float) + Ucur (8 double) + U0 (8 double, stages with g0 != 0)
# + 3 x 8 face fluxes (float) + 3 EMFs (float) + 6 doubles of cached geometry (the Kerr-Schild f, f/(1+f),
# l_i and 1/sqrt(gamma)) read; Unew (8 double) + P (8 float) + status written; the mean over the two stages
# of an RK2 step
UPDATE_ALGO_BYTES_PER_CELL = 32 + 64 + 32 + 96 + 12 + 48 + 64 + 32 + 1
FLUX_FP32_FLOP_PER_FACE = 1811.2
FLUX_DRAM_BYTES_PER_FACE = 48.4


# Algorithmic bytes per interior zone per stage of the fused-ideal mixed form (primitives in float, state in
# double, metric computed, perfect stencil reuse; the mean of the two stages of an RK2 step at 256^3, where
# the primitive read over the ghosted block is 1.097 zones' worth): 32 f_g (P read) + 64 (U read) + 32
# (U0 read, second stage only) + 64 (U written) + 32 (P written) + 1 (status) bytes.
STAGE_ALGO_BYTES_PER_ZONE = 228.5


def live_fp_peaks(G):
    """(FP64, FP32) dense FMA rates of this GPU in TFLOP/s, measured now by the library (grmhd_fp_peaks)."""
    import torch
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    f64, f32 = G.grmhd_fp_peaks(sink.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return f64, f32


def roofline(dom, ms, n, stats, fp_peaks, ms_stage, peaks):
    """Roofline of the dominant kernel group, and the whole stage against HBM. The update kernel (con2prim
    in double) is bound by the FP64 pipe, the flux kernels by the FP32 pipe; neither is HBM-bound."""
    cells = n ** 3
    f64, f32 = fp_peaks
    hbm = peaks.get("hbm_gbs")
    stage_gbs = STAGE_ALGO_BYTES_PER_ZONE * cells / (ms_stage / 1e3) / 1e9
    stage_hbm = {"achieved": stage_gbs, "peak": hbm, "unit": "GB/s", "frac": stage_gbs / hbm if hbm else None,
                 "bytes_per_zone": STAGE_ALGO_BYTES_PER_ZONE,
                 "note": "whole stage: algorithmic bytes per zone x zones / stage time; peak = MEASURED_PEAKS.json "
                         "hbm_gbs (copy, read + write)"}
    if dom == "update":
        flops = UPDATE_FP64_FLOP_PER_CELL * cells
        achieved = flops / (ms / 1e3) / 1e12
        return {"kernel": "k_update", "bound": "alu", "achieved": achieved, "peak": f64, "unit": "TFLOP/s",
                "frac": achieved / f64, "traffic": UPDATE_DRAM_BYTES_PER_CELL * cells, "ms_per_launch": ms,
                "work_per_unit": f"{UPDATE_FP64_FLOP_PER_CELL} FP64 flop/cell (ncu, 96^3, active lanes)",
                "algorithmic_bytes_per_cell": UPDATE_ALGO_BYTES_PER_CELL,
                "hbm_frac": UPDATE_ALGO_BYTES_PER_CELL * cells / (ms / 1e3) / 1e9 / hbm if hbm else None,
                "stage_hbm": stage_hbm,
                "note": "FP64 pipe (issue-bound: one warp FP64 instruction costs the same pipe time whatever its "
                        "active lanes; ncu: FP64 pipe ~70% busy, the rest of its time float<->double conversions and "
                        "partly active warps); peak = the DFMA rate measured live on this GPU by grmhd_fp_peaks "
                        "(MEASURED_PEAKS.json has no FP64 figure); traffic scaled from the 96^3 ncu capture by "
                        "cell count"}
    faces = 3 * (n + 1) * (n + 2) ** 2 / 3.0
    flops = FLUX_FP32_FLOP_PER_FACE * faces
    achieved = flops / (ms / 1e3) / 1e12
    return {"kernel": f"k_flux_cc ({dom})", "bound": "alu", "achieved": achieved, "peak": f32,
            "unit": "TFLOP/s", "frac": achieved / f32, "traffic": FLUX_DRAM_BYTES_PER_FACE * faces,
            "ms_per_launch": ms, "stage_hbm": stage_hbm,
            "note": "FP32 pipe; peak = the FFMA rate measured live on this GPU by grmhd_fp_peaks"}


# ----------------------------------------------------------------------------- oracle baselines
def _oracle_stage_worker(args):
    n, seed = args
    import oracle
    from paper_2410_09146_gb300 import inputs as I
    s = I.kerr_schild_setup(n, recon="weno5z_aoah", riemann="hll")
    lo = 3.0 + (seed % 4) * 0.5
    s.x0 = (lo, lo, lo)
    p = oracle.params(s)
    P = I.kerr_schild_random_prims(s, seed=seed)
    U = oracle.prim2con_grid(p, P)
    t = time.perf_counter()
    oracle.stage(p, P, None, U, 0.0, 1.0, 1.0, 0.0)
    return n ** 3, time.perf_counter() - t


TILES = ((96, 96, 96), (0, 0, 0))  # 64^3 tiles of the workload: the central one and the one next to the hole


def cpu_baseline(n, tile=64):
    """The oracle as it stands, serial on one host core, on a bounded sample of the workload: one RK2 step of
    each 64^3 tile in TILES of the n^3 block (the block's own primitives, ghosts included). Returns the
    baseline entry and the oracle's states, which the mixed form is then compared with."""
    import oracle
    from paper_2410_09146_gb300 import inputs as I
    oracle.build()
    parent = I.kerr_schild_setup(n, recon="weno5z_aoah", riemann="hll")
    zones, secs, ref = 0, 0.0, []
    for off in TILES:
        if any(o + tile > n for o in off):
            continue
        s = I.kerr_schild_tile(parent, off, (tile,) * 3)
        P = I.kerr_schild_random_prims(s, seed=2)
        p = oracle.params(s)
        Po = P.copy()
        t0 = time.perf_counter()
        Uo, sto, _ = oracle.rk2_step(p, Po, oracle.prim2con_grid(p, Po.copy()), 0.0)
        secs += time.perf_counter() - t0
        zones += 2 * tile ** 3
        ref.append((s, P, Uo, Po))
    return ({"value": zones / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
             "sample": f"one RK2 step (two stages) of each of {len(ref)} {tile}^3 tiles {TILES[:len(ref)]} of the "
                       f"{n}^3 workload block (FP64 oracle, serial, one core)"}, ref)


def l1_vs_oracle(G, ref):
    """The mixed form's per-variable L1 against the oracle after the same RK2 step of the sampled tiles."""
    import dataclasses
    out = []
    for s, P, Uo, Po in ref:
        c = G.Context(dataclasses.replace(s, precision="mixed"))
        c.set_prims(P.copy())
        c.rk2_step(0.0)
        ng = s.ng
        inner = (slice(None),) + (slice(ng, -ng),) * 3
        U, Pm = c.cons(), c.prims()[inner]
        del c
        e_scale = np.abs(Uo[4] + Uo[0]).sum()  # rho eps on the scale con2prim recovers it from (sqrt(gamma) ~ 1)
        out.append({"tile": list(s.tile_of[1]), "U": [float(x) for x in l1_rel(U, Uo)],
                    "P": [float(x) for x in l1_rel(Pm, Po[inner])],
                    "rho_eps_over_tau_plus_D": float(np.abs(Pm[4] - Po[inner][4]).sum() / e_scale)})
    return {"after": "one RK2 step", "tiles": out, "max_U": max(max(o["U"]) for o in out) if out else None}


def run_reference(args):
    """Reference arm: the FP64 oracle on all host cores, each core one independent sample block per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n_sample = 40
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        for w in range(args.warmup):
            pool.map(_oracle_stage_worker, [(n_sample, 100 + w * cores + c) for c in range(cores)])
        t0 = time.perf_counter()
        zones = 0
        for k in range(args.steps):
            res = pool.map(_oracle_stage_worker, [(n_sample, 1000 + k * cores + c) for c in range(cores)])
            zones += sum(r[0] for r in res)
        secs = time.perf_counter() - t0
    value = zones / secs
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded random Kerr-Schild primitives)",
           "config": {"workload": f"kerr_schild_random_{args.n}^3_weno5z_aoah_hll_mixed",
                      "sample": f"{cores} independent {n_sample}^3 blocks per step"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"per step, one RK stage of {cores} independent {n_sample}^3 blocks of the "
                                      "same workload, one FP64 oracle process per core"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.guess_only:
        import torch
        from paper_2410_09146_gb300 import build as B
        B.build()
        from paper_2410_09146_gb300 import grmhd as G
        from paper_2410_09146_gb300 import inputs as I
        torch.cuda.set_device(0)
        print(json.dumps({"c2p_guess": run_guess(G, I, 0, n_states=args.guess_states)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
