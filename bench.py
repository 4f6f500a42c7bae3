#!/usr/bin/env python
"""Benchmark of the disconnected-loop hot path on one GB300 (or N replicas).

Workload (32^3 x 64, eps 0.4, kappa 0.1612, a*mu 0.0055, antiperiodic in t):
the Truncated Solver Method with N_HP = 24 high-precision (CG residual 1e-10,
FP32 Krylov vectors, FP64 reliable updates at delta = 1e-4) and N_LP = 500 low-precision
(residual 1e-2, 16-bit fixed-point Krylov vectors) solves of the even-odd twisted-mass
operator, batched 16 right-hand sides per launch, each solution contracted
into one-end (sigma loop), generalised one-end (isoscalar axial loop) and HPE
(4 exact orders) local loops for all 16 Gamma, every t, |p|^2 <= 9.

One step = one full TSM sweep for the gauge field (24 HP-LP pairs + 500 fresh
LP solves with their contractions: the paper's unit of work per configuration)
on noise vectors no other step has used.

value = loop estimates per second at equal statistical error: the number of
plain high-precision loop estimates (one per noise vector) that would give the
TSM step's error on the isoscalar axial loop (the worse of the two
observables), per second.  Variances come from the per-noise observables of
all steps run.  The plain FP64 CG reference is reported beside it.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (32, 32, 32, 64)
EPS, KAPPA, AMU = 0.4, 0.1612, 0.0055
N_HP, N_LP, SLICES, BLOCK = 24, 500, 1, 16
TOL_HP, TOL_LP = 1e-10, 1e-2
DELTA_HP = 1e-4  # reliable updates every four decades: each costs a high-precision operator application
P2MAX = 9
LINK_SEED, NOISE_SEED = 1002, 2002
WORKLOAD = "tsm_32x32x32x64"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampler over the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(os.environ.get("DL_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[3 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _equal_error(obs_hp, obs_pair, obs_lp, n_hp, n_lp, t_step):
    """Plain-HP-equivalent estimates per second for the two observables."""
    out = {}
    for name, k in (("sigma", 0), ("axial", 2)):
        f_hp = obs_hp[:, k] + 1j * obs_hp[:, k + 1]
        f_pr = obs_pair[:, k] + 1j * obs_pair[:, k + 1]
        f_lp = obs_lp[:, k] + 1j * obs_lp[:, k + 1]
        v_hp = np.var(f_hp, ddof=1)
        v_d = np.var(f_hp - f_pr, ddof=1)
        v_lp = np.var(f_lp, ddof=1)
        e2 = v_d / n_hp + v_lp / n_lp
        n_eq = v_hp / e2 if e2 > 0 else float("nan")
        out[name] = {"v_hp": float(v_hp), "v_diff": float(v_d), "v_lp": float(v_lp), "err2_step": float(e2),
                     "plain_equiv_per_step": float(n_eq), "per_s": float(n_eq / t_step),
                     "r_c": float(np.real(np.corrcoef(np.real(f_hp), np.real(f_pr))[0, 1]))}
    return out


def rank_seed(step: int, rank: int) -> int:
    """Noise seed of a sweep: distinct for every (step, rank), so replicas never share noise."""
    return NOISE_SEED + 1000003 * (step + 1) + 7919 * rank


def max_over_ranks(ms: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's timed region (the job finishes when every replica has)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as tdist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def _nvtx(torch, name):
    """Push (name) or pop (None) an NVTX range around the timed steps, so that a
    profiler can restrict its launch list to them; a no-op where NVTX is absent."""
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def _links():
    import synth
    return synth.gauge_links(DIMS, EPS, LINK_SEED)


def run_ours(args, rank, world, device):
    import torch

    import paper_1309_2256_gb300 as dl

    torch.cuda.set_device(device)
    links = _links()
    n_hp_s, n_lp_s = N_HP // SLICES, N_LP // SLICES
    stream = torch.cuda.current_stream()
    ctx = dl.dl_create(DIMS, device, stream)
    dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
    dl.dl_set_params(ctx, KAPPA, AMU)
    npm = len(dl.dl_momenta(P2MAX))

    def params(step):
        return dl.dl_tsm_params(n_hp=n_hp_s, n_lp=n_lp_s, tol_hp=TOL_HP, tol_lp=TOL_LP, prec_hp_lo=dl.DL_F32,
                                prec_lp_lo=dl.DL_F16, delta_hp=args.delta_hp, block=BLOCK,
                                seed=rank_seed(step, rank), p2max=P2MAX, with_deriv=0,
                                hpe=1, max_iter=200000, chunk=32, hp_guess=1, hpe_diff=1)

    loops = np.zeros((3, DIMS[3], npm, 1, 4, 4), dtype=np.complex128)
    obs = {"hp": [], "pair": [], "lp": []}
    infos = []

    def step(i, record):
        ohp, opr, olp = np.zeros((n_hp_s, 4)), np.zeros((n_hp_s, 4)), np.zeros((n_lp_s, 4))
        st, info = dl.dl_tsm_run(ctx, params(i), loops, ohp, opr, olp)
        obs["hp"].append(ohp)
        obs["pair"].append(opr)
        obs["lp"].append(olp)
        if record:
            infos.append(info)
        return st

    for i in range(args.warmup):
        step(-1 - i, False)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    dl.dl_profile(ctx, 1)
    launches0 = dl.dl_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(device) as clk:
        _nvtx(torch, "dl_timed")
        ev0.record(stream)
        t0 = time.perf_counter()
        for i in range(args.steps):
            step(i, True)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        _nvtx(torch, None)
    if dist:
        tdist.barrier()
    launches = dl.dl_kernel_launches() - launches0
    prof = dl.dl_profile(ctx, 0)
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world)
    t_step = ms / 1e3 / args.steps

    # e2e: the same step through the C ABI from pinned host memory (gauge field
    # uploaded every step, loops and observables copied back)
    pinned = torch.from_numpy(links.view(np.float64)).pin_memory()
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        dl.lib().dl_load_gauge(ctx, pinned.data_ptr(), 0, -1.0, 12, 12)
        step(1000 + i, False)
    torch.cuda.synchronize()
    e2e_t = (time.perf_counter() - t0) / e2e_steps

    # plain FP64 CG reference: one right-hand side at a time, FP64 storage,
    # no reliable updates; timed over a bounded number of iterations and scaled
    # by the measured HP iteration count
    ref = plain_fp64_reference(dl, ctx, device, infos, n_hp_s)
    dl.dl_destroy(ctx)

    ohp, opr, olp = (np.concatenate(obs[k]) for k in ("hp", "pair", "lp"))
    eq = _equal_error(ohp, opr, olp, n_hp_s, n_lp_s, t_step)
    value = min(eq["sigma"]["per_s"], eq["axial"]["per_s"]) * world
    e2e_value = min(eq["sigma"]["plain_equiv_per_step"], eq["axial"]["plain_equiv_per_step"]) / e2e_t * world
    roof = roofline(prof, infos)
    it_hp = sum(i.iters_hp for i in infos) / max(1, len(infos) * n_hp_s)
    it_lp = sum(i.iters_lp for i in infos) / max(1, len(infos) * (n_hp_s + n_lp_s))
    return dict(value=value, t_step=t_step, wall=wall, eq=eq, roof=roof, launches=launches, ref=ref, e2e=e2e_value,
                e2e_t=e2e_t, clocks=clk.summary(), it_hp=it_hp, it_lp=it_lp,
                sec_hp=sum(i.seconds_hp for i in infos) / len(infos),
                sec_lp=sum(i.seconds_lp for i in infos) / len(infos),
                sec_ct=sum(i.seconds_contract for i in infos) / len(infos),
                bytes_h2d=links.nbytes, bytes_d2h=loops.nbytes + 8 * 4 * (2 * n_hp_s + n_lp_s))


def plain_fp64_reference(dl, ctx, device, infos, n_hp_s):
    import torch
    n_it = 64
    V = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]
    eta = torch.empty((1, V * 12), dtype=torch.complex128, device="cuda")
    sol = torch.empty_like(eta)
    dl.dl_noise_z4(ctx, 5, 0, 1, eta, dl.DL_C128)
    per = {}
    for name, pr in (("ieee_f64", dl.DL_F64_IEEE), ("double_float", dl.DL_F64)):
        prm = dl.dl_solve_params(tol=1e-30, max_iter=n_it, prec_hi=pr, prec_lo=pr, delta=0.0, flavour=1, chunk=n_it)
        dl.dl_solve(ctx, eta, sol, 1, dl.DL_C128, prm)  # warm (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dl.dl_solve(ctx, eta, sol, 1, dl.DL_C128, prm)
        torch.cuda.synchronize()
        per[name] = (time.perf_counter() - t0) / n_it
    t_iter = min(per.values())  # the faster FP64 form is the baseline
    it_hp = sum(i.iters_hp for i in infos) / max(1, len(infos) * n_hp_s)
    del eta, sol
    return {"sec_per_iter": t_iter, "sec_per_iter_by_arithmetic": per, "hp_iters": it_hp,
            "sec_per_estimate": t_iter * it_hp, "estimates_per_s": 1.0 / (t_iter * it_hp) if it_hp > 0 else None,
            "how": f"one right-hand side, {n_it} CG iterations timed in IEEE FP64 and in double-float, the faster "
                   "scaled by the mean HP iteration count"}


def roofline(prof, infos):
    """Dominant stencil kernel: algorithmic bytes per launch / average launch duration.

    Durations come from CUDA events recorded inside the solver's graphs around the
    four stencil launches of the first iteration of every chunk (dl_profile).  The
    dominant (stage, precision) is the one with the largest average duration times
    its number of block-iterations in the sweep."""
    peaks, kind = _peaks()
    V = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]
    Vh = V // 2
    link_b = {0: 144, 1: 48, 2: 24}  # FP64 recon 18, FP32 recon 12, 16-bit recon 12 (as loaded)
    sp_b = {0: 192, 1: 96, 2: 52}    # spinor bytes per site (16-bit: 48 + 4-byte scale)
    units = {0: 2, 1: 3, 2: 2, 3: 7}  # spinor streams per stage (in, aux, out, r, y, p ...)
    col_its = {1: sum(i.iters_hp for i in infos), 2: sum(i.iters_lp for i in infos)}
    best = None
    for stage in range(4):
        for prec in range(3):
            n, ms, items = prof[stage, prec]
            if n <= 0:
                continue
            cols = items / n / Vh
            bytes_launch = 4 * V * link_b[prec] + units[stage] * Vh * cols * sp_b[prec]
            avg = ms / n / 1e3
            weight = avg * col_its.get(prec, 0) / max(cols, 1e-9)
            rec = {"stage": stage, "prec": ["f64", "f32", "16-bit"][prec], "launches_sampled": int(n),
                   "avg_ms": avg * 1e3, "cols": cols, "bytes": bytes_launch, "gbs": bytes_launch / avg / 1e9,
                   "weight": weight}
            if best is None or weight > best["weight"]:
                best = rec
    if best is None:
        return None
    peak = peaks["hbm_gbs"]
    # DRAM bytes (read + write) of the 16-bit stage-3 kernel from one ncu capture of the
    # 24^3 x 24, 16-column case (profiles/dslash_staged_16bit_cg_24x24x24x24_16rhs.md),
    # scaled to this launch by its site-columns (traffic is linear in them)
    traffic = None
    if best["stage"] == 3 and best["prec"] == "16-bit":
        per_item = 1002.4e6 / (24 ** 4 // 2 * 16)
        traffic = int(per_item * Vh * best["cols"])
    return {"bound": "hbm", "achieved": round(best["gbs"], 1), "peak": peak, "unit": "GB/s",
            "frac": round(best["gbs"] / peak, 4), "traffic": traffic,
            "kernel": f"dslash stage {best['stage']} ({best['prec']} Krylov, {best['cols']:.1f} columns)",
            "bytes_per_launch": int(best["bytes"]), "avg_launch_ms": round(best["avg_ms"], 4),
            "peak_kind": kind + " (MEASURED_PEAKS.json hbm_gbs)" if kind == "measured" else kind}


def cpu_oracle_sample():
    """The FP64 oracle on the host: one CG iteration (Mhat^dag Mhat + vector updates)
    on the full 32^3 x 64 lattice; returns seconds per iteration and threads used."""
    from oracle import operator as op
    links = _links()
    dims = DIMS
    x = op.project(np.ones((DIMS[3], DIMS[2], DIMS[1], DIMS[0], 4, 3), dtype=np.complex128), dims, 0)
    t0 = time.perf_counter()
    q = op.mhat(links, x, KAPPA, AMU, 1, -1.0, dims)
    ax = op.mhat_dag(links, q, KAPPA, AMU, 1, -1.0, dims)
    a = np.vdot(x.ravel(), ax.ravel()).real
    x = x + (1.0 / a) * ax
    dt = time.perf_counter() - t0
    return dt, 1


def stencil_case():
    """Small case for ncu captures: 24^3 x 24, 16 right-hand sides, one 16-bit and one
    FP32 Krylov solve of 4 CG iterations each (fields 138 MB / 255 MB, above the
    129 MB L2; about 5 GB on the device)."""
    import torch

    import paper_1309_2256_gb300 as dl
    import synth
    dims = (24, 24, 24, 24)
    links = synth.gauge_links(dims, EPS, 77)
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
    dl.dl_set_params(ctx, KAPPA, AMU)
    n = 16
    V = dims[0] * dims[1] * dims[2] * dims[3]
    eta = torch.empty((n, V * 12), dtype=torch.complex64, device="cuda")
    dl.dl_noise_z4(ctx, 9, 0, n, eta, dl.DL_C64)
    sol = torch.empty_like(eta)
    dl.dl_profile(ctx, 1)
    for lo in (dl.DL_F16, dl.DL_F32):
        prm = dl.dl_solve_params(tol=1e-12, max_iter=4, prec_hi=dl.DL_F32, prec_lo=lo, delta=0.0, flavour=1, chunk=4)
        st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C64, prm)
    torch.cuda.synchronize()
    prof = dl.dl_profile(ctx, 0)
    dl.dl_destroy(ctx)
    for prec, name in ((2, "16-bit"), (1, "f32")):
        print(name, "stage ms:", " ".join(f"{prof[k, prec, 1] / max(prof[k, prec, 0], 1):.3f}" for k in range(4)))
    print("stencil case done")


def contract_case():
    """Small case for ncu captures of the contraction kernels: 24^3 x 24, 16 columns,
    one-end loops at |p|^2 <= 9 from complex64 inputs (the low-precision pipeline)."""
    import torch

    import paper_1309_2256_gb300 as dl
    import synth
    dims = (24, 24, 24, 24)
    links = synth.gauge_links(dims, EPS, 78)
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
    dl.dl_set_params(ctx, KAPPA, AMU)
    n = 16
    V = dims[0] * dims[1] * dims[2] * dims[3]
    eta = torch.empty((n, V * 12), dtype=torch.complex64, device="cuda")
    dl.dl_noise_z4(ctx, 9, 0, n, eta, dl.DL_C64)
    sol = torch.empty_like(eta)
    dl.dl_noise_z4(ctx, 10, 0, n, sol, dl.DL_C64)
    npm = len(dl.dl_momenta(P2MAX))
    out = torch.zeros((n, dims[3], npm, 1, 4, 4), dtype=torch.complex128, device="cuda")
    for _ in range(2):
        dl.dl_contract(ctx, dl.DL_EST_ONE_END, eta, sol, n, dl.DL_C64, 0, P2MAX, out)
    torch.cuda.synchronize()
    dl.dl_destroy(ctx)
    print("contract case done")


def learned_case(args):
    """The learned preconditioner on 16^3 x 32 (eps 0.4, kappa 0.161, a*mu 0.0055): a
    4-layer, 16-channel network (FP32 weights, bfloat16 activations) trained with Adam
    on (Z4 noise, FP64-accurate solution) pairs from the plain solver, then on fresh
    noise: flexible GCR on the normal operator M^+ M (preconditioner N N^+) to 1e-10 with and
    without it against the mixed-precision CG,
    and the TSM with the network as its LP map against truncated CG."""
    import torch

    import paper_1309_2256_gb300 as dl
    import synth
    cfg = synth.CONFIGS["learned_16x16x16x32"]
    dims, kappa, amu = cfg["dims"], cfg["kappa"], cfg["amu"]
    V = dims[0] * dims[1] * dims[2] * dims[3]
    links = synth.gauge_links(dims, cfg["eps"], 1000 + cfg["id"])
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, links, -1.0, 12, 8)
    dl.dl_set_params(ctx, kappa, amu)
    out = {"case": "learned_16x16x16x32", "data": "synthetic", "pairs": args.pairs, "fresh": args.fresh}
    t_start = time.perf_counter()

    def progress(what):
        print(f"[learned {time.perf_counter() - t_start:8.1f} s] {what}", file=sys.stderr, flush=True)
    # training pairs from the plain solver (complex64 storage, FP64-accurate solutions)
    eta = torch.empty((args.pairs, V * 12), dtype=torch.complex64, device="cuda")
    sol = torch.empty_like(eta)
    hp = dl.dl_solve_params(tol=1e-10, max_iter=100000, prec_hi=dl.DL_F64, prec_lo=dl.DL_F32, delta=0.01, flavour=1,
                            chunk=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in range(0, args.pairs, 32):
        n = min(32, args.pairs - b)
        dl.dl_noise_z4(ctx, 2000 + cfg["id"], b, n, eta[b:b + n], dl.DL_C64)
        dl.dl_solve(ctx, eta[b:b + n], sol[b:b + n], n, dl.DL_C64, hp)
    torch.cuda.synchronize()
    out["seconds_pairs"] = time.perf_counter() - t0
    progress(f"{args.pairs} training pairs")
    nn = dl.dl_nn_create(ctx, 4, 16, dl.DL_BF16)
    dl.dl_nn_set_weights(nn, synth.network_weights(4, 16, 3000 + cfg["id"]))
    tp = dl.dl_nn_train_params(steps=args.train_steps, batch=args.batch, lr=args.lr, beta1=0.9, beta2=0.999, eps=1e-8,
                               seed=11)
    t0 = time.perf_counter()
    hist = dl.dl_nn_train(nn, tp, args.pairs, eta, sol, dl.DL_C64)
    torch.cuda.synchronize()
    ttrain = time.perf_counter() - t0
    progress(f"trained {args.train_steps} steps")
    k = max(1, min(20, len(hist) // 5))
    out["train"] = {"steps": args.train_steps, "batch": args.batch, "lr": args.lr, "seconds": ttrain,
                    "pair_passes_per_s": args.train_steps * args.batch / ttrain,
                    "loss_first": float(hist[:k].mean()), "loss_last": float(hist[-k:].mean())}
    # inference: one network application, timed with events on the current stream
    one_in = eta[:1].clone()
    one_out = torch.empty_like(one_in)
    ms_by = {}
    for tc in (0, 1):  # CUDA-core and tensor-core channel mixing
        dl.dl_nn_set_tensor_cores(nn, tc)
        for _ in range(3):
            dl.dl_nn_apply(nn, 1, one_in, one_out, dl.DL_C64)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record()
        for _ in range(reps):
            dl.dl_nn_apply(nn, 1, one_in, one_out, dl.DL_C64)
        e1.record()
        torch.cuda.synchronize()
        ms_by["tensor_cores" if tc else "cuda_cores"] = e0.elapsed_time(e1) / reps
    ms_apply = ms_by["tensor_cores"]
    # flops of one application, per site and layer: channel mixing, 9 terms x 12 components x 2
    # complex multiply-adds (8 flops each) per (output, input) channel pair; transports, 8 links x
    # 4 spins x 9 complex multiply-adds per input channel
    flops = 0
    for l in range(4):
        ci = 1 if l == 0 else 16
        co = 1 if l == 3 else 16
        flops += V * (co * ci * 9 * 12 * 2 * 8 + ci * 8 * 4 * 3 * 3 * 8)
    out["apply"] = {"ms": ms_apply, "tflops": flops / ms_apply / 1e9, "flops_per_apply": flops, "ms_by_backend": ms_by}
    progress(f"one application {ms_apply:.2f} ms")
    # fresh noise: FGCR with / without the network, plain mixed-precision CG
    fresh = torch.empty((args.fresh, V * 12), dtype=torch.complex128, device="cuda")
    for b in range(0, args.fresh, 32):
        n = min(32, args.fresh - b)
        dl.dl_noise_z4(ctx, 5000 + cfg["id"], b, n, fresh[b:b + n])
    fg = dl.dl_fgcr_params(tol=1e-10, max_iter=args.fgcr_max_iter, restart=args.fgcr_restart, inner_tol=1e-4,
                           flavour=1, normal=1)
    n_fg = min(args.fresh, args.fgcr_rhs)
    for name, net in (("fgcr_net", nn), ("fgcr_plain", None)):
        x = torch.empty((n_fg, V * 12), dtype=torch.complex128, device="cuda")
        its, secs, ops, nns, res = [], 0.0, 0, 0, []
        for b in range(0, n_fg, 8):
            n = min(8, n_fg - b)
            st, stt = dl.dl_fgcr_solve(ctx, net, fg, n, fresh[b:b + n], x[b:b + n])
            its += list(stt.iters[:n])
            res += list(stt.true_resid[:n])
            secs += stt.seconds
            ops += stt.op_applications
            nns += stt.nn_applications
        progress(f"{name}: {n_fg} solves")
        out[name] = {"rhs": n_fg, "iters_mean": float(np.mean(its)), "true_resid_max": float(np.max(res)),
                     "seconds_per_rhs": secs / n_fg, "op_applications_per_rhs": ops / n_fg,
                     "nn_applications_per_rhs": nns / n_fg}
    x = torch.empty_like(fresh)
    its, secs = [], 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in range(0, args.fresh, 16):
        n = min(16, args.fresh - b)
        stt = dl.dl_solve_stats()
        dl.dl_solve(ctx, fresh[b:b + n], x[b:b + n], n, dl.DL_C128, hp, stt)
        its += list(stt.iters[:n])
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    out["cg_plain"] = {"rhs": args.fresh, "iters_mean": float(np.mean(its)), "seconds_per_rhs": secs / args.fresh,
                       "op_applications_per_rhs": 2.0 * float(np.mean(its)),
                       "how": "even-odd CGNR, FP32 Krylov vectors, FP64 reliable updates, blocks of 16"}
    # TSM: the network as LP map against truncated CG, same HP set
    npm = len(dl.dl_momenta(0))
    for name, net in (("tsm_net_lp", nn), ("tsm_cg_lp", None)):
        prm = dl.dl_tsm_params(n_hp=24, n_lp=args.fresh, tol_hp=1e-10, tol_lp=1e-2, prec_hp_lo=dl.DL_F32,
                               prec_lp_lo=dl.DL_F16, delta_hp=0.01, block=16, seed=7000 + cfg["id"], p2max=0,
                               with_deriv=0, hpe=0, max_iter=100000, chunk=32, lp_net=nn["h"] if net else None)
        loops_ = np.zeros((2, dims[3], npm, 1, 4, 4), dtype=np.complex128)
        ohp, opr, olp = np.zeros((24, 4)), np.zeros((24, 4)), np.zeros((args.fresh, 4))
        st, info = dl.dl_tsm_run(ctx, prm, loops_, ohp, opr, olp)
        progress(f"{name}: TSM")
        ee = _equal_error(ohp, opr, olp, 24, args.fresh, info.seconds_total)
        out[name] = {"seconds": info.seconds_total, "seconds_lp": info.seconds_lp,
                     "sigma_per_s": ee["sigma"]["per_s"], "axial_per_s": ee["axial"]["per_s"],
                     "r_c_sigma": ee["sigma"]["r_c"], "r_c_axial": ee["axial"]["r_c"]}
    dl.dl_nn_destroy(nn)
    dl.dl_destroy(ctx)
    print(json.dumps(out))


def batch_case(args):
    """Six lattices (two each of 12^3 x 24, 16^3 x 32, 24^3 x 48; eps 0.4, kappa 0.161,
    a*mu 0.0055), 32 Z4 noise vectors each, solved together to 1e-8 (FP32 Krylov, FP64
    reliable updates, autotuned right-hand-side tile) with zero-momentum loops."""
    import torch

    import paper_1309_2256_gb300 as dl
    import synth
    dims = [(12, 12, 12, 24)] * 2 + [(16, 16, 16, 32)] * 2 + [(24, 24, 24, 48)] * 2
    n = 32
    ctx = dl.dl_create_multi(dims, 0, torch.cuda.current_stream())
    for i, d in enumerate(dims):
        dl.dl_load_gauge_lat(ctx, i, synth.gauge_links(d, 0.4, 1004 + 10 * i), -1.0, 12, 12)
    dl.dl_set_params(ctx, 0.161, 0.0055)
    out = np.zeros(sum(2 * n * d[3] * 16 for d in dims), dtype=np.complex128)
    res = {"case": "batch_6_lattices", "data": "synthetic", "rhs_per_lattice": n}
    for rep in range(2):
        prm = dl.dl_batch_params(n=n, tol=1e-8, prec_hi=dl.DL_F64, prec_lo=dl.DL_F32, delta=0.01, seed=2004 + rep,
                                 max_iter=20000, tile=0)
        st, info = dl.dl_batch_loops(ctx, prm, out, None)
    res.update({"tile": info.tile, "instances": info.instances, "seconds_tune": info.seconds_tune,
                "seconds_solve": info.seconds_solve, "seconds_contract": info.seconds_contract,
                "iters_max": list(info.iters_max[:6]), "resid_max": list(info.resid_max[:6]),
                "solves_per_s": 6 * n / (info.seconds_solve + info.seconds_contract)})
    dl.dl_destroy(ctx)
    print(json.dumps(res))


def mass_case(args):
    """Cost ratio R_HP/LP of the TSM versus the valence twisted mass (Sec. 4, Table compRatios):
    16^3 x 32 (eps 0.4, kappa 0.161), one-end and generalised one-end loops, per a*mu the cost
    of one noise vector's loops from an HP solve (1e-10, from zero) over that from an LP solve
    (1e-2), each with its contractions; local only and with the one-derivative loops.  The
    masses are a light, a strange-like and a charm-like choice (the paper does not print its
    strange and charm values)."""
    import torch

    import paper_1309_2256_gb300 as dl
    import synth
    dims = (16, 16, 16, 32)
    kappa = 0.161
    masses = [float(m) for m in args.masses.split(",")]
    n_hp, n_lp = 16, 48
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, synth.gauge_links(dims, 0.4, 1001), -1.0, 12, 12)
    rows = []
    for amu in masses:
        dl.dl_set_params(ctx, kappa, amu)
        row = {"amu": amu}
        for deriv in (0, 1):
            prm = dl.dl_tsm_params(n_hp=n_hp, n_lp=n_lp, tol_hp=1e-10, tol_lp=1e-2, prec_hp_lo=dl.DL_F32,
                                   prec_lp_lo=dl.DL_F16, delta_hp=DELTA_HP, block=16, seed=3001, p2max=4,
                                   with_deriv=deriv, hpe=0, max_iter=200000, chunk=32, hp_guess=0, hpe_diff=0)
            for rep in range(2):  # the first run builds this mass's graphs and workspaces
                st, info = dl.dl_tsm_run(ctx, prm, None, None, None, None)
            t_hp = info.seconds_hp / n_hp
            t_lp = info.seconds_lp / (n_hp + n_lp)
            t_c = info.seconds_contract / (2 * n_hp + n_lp)
            key = "one_deriv" if deriv else "local"
            row[key] = {"r_hp_lp": (t_hp + t_c) / (t_lp + t_c), "sec_hp_solve": t_hp, "sec_lp_solve": t_lp,
                        "sec_contract_per_solution": t_c, "iters_hp": info.iters_hp / n_hp,
                        "iters_lp": info.iters_lp / (n_hp + n_lp), "not_converged": info.not_converged}
        rows.append(row)
    dl.dl_destroy(ctx)
    print(json.dumps({"case": "mass_sweep", "data": "synthetic", "lattice": list(dims), "kappa": kappa,
                      "n_hp": n_hp, "n_lp": n_lp, "rows": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default=None, choices=["stencil", "contract", "learned", "batch", "mass"],
                    help="small profiling case instead of the benchmark (for ncu)")
    ap.add_argument("--delta-hp", type=float, default=DELTA_HP,
                    help="reliable-update trigger of the high-precision solves")
    ap.add_argument("--pairs", type=int, default=2000, help="learned case: training pairs")
    ap.add_argument("--fresh", type=int, default=200, help="learned case: fresh noise vectors")
    ap.add_argument("--fgcr-rhs", type=int, default=200, help="learned case: fresh vectors solved by FGCR")
    ap.add_argument("--train-steps", type=int, default=1000, help="learned case: Adam steps")
    ap.add_argument("--fgcr-restart", type=int, default=64, help="learned case: FGCR directions per cycle")
    ap.add_argument("--fgcr-max-iter", type=int, default=600, help="learned case: FGCR iterations per solve")
    ap.add_argument("--batch", type=int, default=4, help="learned case: pairs per Adam step")
    ap.add_argument("--lr", type=float, default=1e-3, help="learned case: Adam learning rate")
    ap.add_argument("--masses", default="0.0055,0.02,0.2", help="mass case: valence a*mu values")
    args = ap.parse_args()
    if args.case == "mass":
        mass_case(args)
        return
    if args.case == "learned":
        learned_case(args)
        return
    if args.case == "batch":
        batch_case(args)
        return
    if args.case == "stencil":
        stencil_case()
        return
    if args.case == "contract":
        contract_case()
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, world)
        return

    import torch
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    r = run_ours(args, rank, world, local)
    if rank != 0:
        return
    ro = r["roof"]
    # CPU baseline: the oracle, bounded sample (one CG iteration at full size), scaled
    t_cpu, cores = cpu_oracle_sample()
    it_hp, it_lp = r["it_hp"], r["it_lp"]
    n_hp_s, n_lp_s = N_HP // SLICES, N_LP // SLICES
    cpu_step = t_cpu * (n_hp_s * (it_hp + it_lp) + n_lp_s * it_lp)
    axial = r["eq"]["axial"]
    cpu_val = min(r["eq"]["sigma"]["plain_equiv_per_step"], axial["plain_equiv_per_step"]) / cpu_step
    line = {
        "metric": "loop estimates/sec at 32^3x64 at equal error (TSM vs plain HP estimates); Dslash HBM GB/s",
        "value": round(r["value"], 4),
        "unit": "loop estimates/s (equal error)",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(r["t_step"] * 1e3, 2),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f16/f32 Krylov, f64 reliable updates and accumulation",
        "data": "synthetic (seeded SU(3) links exp(i eps H), eps 0.4; Z2xiZ2 noise)",
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "kappa": KAPPA, "amu": AMU, "n_hp": N_HP, "n_lp": N_LP,
                   "tol_hp": TOL_HP, "tol_lp": TOL_LP, "delta_hp": args.delta_hp, "hp_from_lp": 1, "hpe_correction_from_difference": 1, "block": BLOCK, "p2max": P2MAX, "hpe_orders": 4,
                   "step": "one TSM sweep: 24 HP-LP pairs + 500 LP solves + contractions",
                   "l2": "inputs larger than L2 (gauge field 0.4-1.2 GB, spinor blocks GBs)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": ro,
        "cpu_baseline": {"value": round(cpu_val, 6), "unit": "loop estimates/s (equal error)", "cores": cores,
                         "kind": "oracle",
                         "sample": f"one FP64 oracle CG iteration on 32^3x64 ({t_cpu:.1f} s), scaled by the measured "
                                   f"iteration counts (HP {it_hp:.0f}, LP {it_lp:.0f}); contractions excluded"},
        "e2e": {"value": round(r["e2e"], 4), "unit": "loop estimates/s (equal error)",
                "h2d_bytes_per_step": int(r["bytes_h2d"]), "d2h_bytes_per_step": int(r["bytes_d2h"])},
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
        "detail": {"equal_error": r["eq"], "iters_hp": it_hp, "iters_lp": it_lp, "sec_hp_per_step": r["sec_hp"],
                   "sec_lp_per_step": r["sec_lp"], "sec_contract_per_step": r["sec_ct"],
                   "plain_fp64_cg": r["ref"],
                   "vs_plain_fp64_cg": (r["value"] / r["ref"]["estimates_per_s"]) if r["ref"]["estimates_per_s"] else None},
    }
    print(json.dumps(line))


# CG iterations of one high-precision (1e-10) solve from a zero start on this
# workload, measured by the GPU path (FP32 Krylov vectors with high-precision
# reliable updates, mean over noise vectors, the TSM's HP solves without the LP
# starting vector); the plain FP64 method needs the same Krylov iterations.
HP_ITERS_MEASURED = 52.0


def run_reference(args, world):
    """The oracle as it stands on the host cores, same metric, config and unit.
    The oracle is the plain method (FP64 CG on every noise vector, no TSM), so each
    of its loop estimates counts one at equal error.  A step is a bounded sample:
    one oracle CG iteration on the full 32^3 x 64 lattice, scaled by the HP
    iteration count of the workload."""
    per = []
    for _ in range(args.warmup):
        cpu_oracle_sample()
    cores = 1
    for _ in range(args.steps):
        dt, cores = cpu_oracle_sample()
        per.append(dt)
    t_it = float(np.median(per))
    value = 1.0 / (t_it * HP_ITERS_MEASURED)
    line = {"impl": "reference",
            "metric": "loop estimates/sec at 32^3x64 at equal error (TSM vs plain HP estimates); Dslash HBM GB/s",
            "value": value, "unit": "loop estimates/s (equal error)", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_it * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": list(DIMS), "kappa": KAPPA, "amu": AMU,
                       "method": "plain FP64 CG per noise vector (the oracle)", "hp_iters": HP_ITERS_MEASURED},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value,
                             "sample": f"one FP64 oracle CG iteration on 32^3x64 per step ({t_it:.1f} s), "
                                       f"x {HP_ITERS_MEASURED:.0f} iterations per HP estimate; contractions excluded"},
            "e2e": {"value": value, "unit": "loop estimates/s (equal error)", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
