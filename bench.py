#!/usr/bin/env python
"""Benchmark of the disconnected-loop hot path on one GB300 (or N replicas).

Workload (32^3 x 64, eps 0.4, kappa 0.1612, a*mu 0.0055, antiperiodic in t):
the Truncated Solver Method with N_HP = 24 high-precision (CG residual 1e-10,
FP32 Krylov vectors, FP64 reliable updates at delta = 1e-4) and N_LP = 500 low-precision
(residual 1e-2, 16-bit fixed-point Krylov vectors) solves of the even-odd twisted-mass
operator, batched in blocks of right-hand sides whose size (8, 16 or 32) the library's
autotuner picks (16 on this workload), each solution contracted
into one-end (sigma loop), generalised one-end (isoscalar axial loop) and HPE
(4 exact orders) local loops for all 16 Gamma, every t, |p|^2 <= 9.

One step = one full TSM sweep for the gauge field (24 HP-LP pairs + 500 fresh
LP solves with their contractions: the paper's unit of work per configuration)
on noise vectors no other step has used.

value = loop estimates per second at equal statistical error: the number of
plain high-precision loop estimates (one per noise vector) that would give the
TSM step's error on the worse of the two observables (sigma and isoscalar axial
loop), per second.  Variances come from the per-noise observables of
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
N_HP, N_LP, SLICES, BLOCK = 24, 500, 1, 0  # BLOCK 0: the library's autotuner picks 8, 16 or 32
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
        if st != 0:  # a solve that hit max_iter or broke down: no valid loops, no valid number
            raise RuntimeError(f"dl_tsm_run status {st}: {dl.dl_last_error(ctx)}")
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
    sprof = dl.dl_profile_stencils()
    dl.dl_profile(ctx, 0)
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
    dl.dl_destroy(ctx)
    block = infos[-1].block  # the TSM's (tuned) block: the comparator batches the same way
    ref_batched = plain_fp64_batched(dl, device, links, block)
    ctx = dl.dl_create(DIMS, device, stream)
    dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
    dl.dl_set_params(ctx, KAPPA, AMU)
    fast = ref_batched["by_arithmetic"][ref_batched["faster"]]
    ref = plain_fp64_reference(dl, ctx, device, ref_batched["iters"], fast["sec_contract"] / ref_batched["columns"])
    dl.dl_destroy(ctx)

    ohp, opr, olp = (np.concatenate(obs[k]) for k in ("hp", "pair", "lp"))
    eq = _equal_error(ohp, opr, olp, n_hp_s, n_lp_s, t_step)
    value = min(eq["sigma"]["per_s"], eq["axial"]["per_s"]) * world
    e2e_value = min(eq["sigma"]["plain_equiv_per_step"], eq["axial"]["plain_equiv_per_step"]) / e2e_t * world
    roof, stencils = roofline(sprof, args.steps)
    it_hp = sum(i.iters_hp for i in infos) / max(1, len(infos) * n_hp_s)
    it_lp = sum(i.iters_lp for i in infos) / max(1, len(infos) * (n_hp_s + n_lp_s))
    return dict(value=value, t_step=t_step, wall=wall, eq=eq, roof=roof, stencils=stencils, launches=launches, ref=ref,
                ref_batched=ref_batched, e2e=e2e_value, block=block,
                e2e_t=e2e_t, clocks=clk.summary(), it_hp=it_hp, it_lp=it_lp,
                sec_hp=sum(i.seconds_hp for i in infos) / len(infos),
                sec_lp=sum(i.seconds_lp for i in infos) / len(infos),
                sec_ct=sum(i.seconds_contract for i in infos) / len(infos),
                bytes_h2d=links.nbytes, bytes_d2h=loops.nbytes + 8 * 4 * (2 * n_hp_s + n_lp_s))


def plain_fp64_reference(dl, ctx, device, iters, sec_contract_per_col):
    """The plain method one right-hand side at a time (FP64 CG from zero, no batching):
    64 CG iterations timed in IEEE FP64 and in double-float, the faster scaled by the
    from-zero iteration count `iters` measured by the batched comparator, plus the
    batched comparator's contraction time per column."""
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
    del eta, sol
    sec = t_iter * iters + sec_contract_per_col
    return {"sec_per_iter": t_iter, "sec_per_iter_by_arithmetic": per, "iters": iters, "sec_per_estimate": sec,
            "estimates_per_s": 1.0 / sec,
            "how": f"one right-hand side, {n_it} CG iterations timed in IEEE FP64 and in double-float, the faster "
                   "scaled by the batched comparator's from-zero iteration count, plus its contraction time per column"}


def plain_fp64_batched(dl, device, links, n):
    """The plain method on this GPU with the TSM's batching: one block of n noise
    vectors solved from zero to 1e-10 in FP64 storage and arithmetic (no mixed precision,
    no reliable updates: every Krylov vector is FP64), timed in double-float and in IEEE
    binary64, each followed by the sweep's contractions (one-end, generalised one-end,
    HPE at |n|^2 <= 9).  Each estimate counts one at equal error.  A context of its own,
    destroyed afterwards, holds its FP64 workspaces."""
    import torch
    V = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]
    npm = len(dl.dl_momenta(P2MAX))
    per = {}
    for name, pr in (("double_float", dl.DL_F64), ("ieee_f64", dl.DL_F64_IEEE)):
        ctx = dl.dl_create(DIMS, device, torch.cuda.current_stream())
        try:
            dl.dl_load_gauge(ctx, links, -1.0, 12, 12)
            dl.dl_set_params(ctx, KAPPA, AMU)
            eta = torch.empty((n, V * 12), dtype=torch.complex128, device="cuda")
            sol = torch.empty_like(eta)
            out = torch.empty((n, DIMS[3], npm, 1, 4, 4), dtype=torch.complex128, device="cuda")
            dl.dl_noise_z4(ctx, NOISE_SEED + 77, 0, n, eta, dl.DL_C128)
            warm = dl.dl_solve_params(tol=1e-30, max_iter=2, prec_hi=pr, prec_lo=pr, delta=0.0, flavour=1, chunk=32)
            dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, warm)  # workspaces and the solver graph
            for est in (dl.DL_EST_ONE_END, dl.DL_EST_GEN, dl.DL_EST_HPE):
                dl.dl_contract(ctx, est, eta, sol, n, dl.DL_C128, 0, P2MAX, out)
            prm = dl.dl_solve_params(tol=TOL_HP, max_iter=200000, prec_hi=pr, prec_lo=pr, delta=0.0, flavour=1,
                                     chunk=32)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, prm)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for est in (dl.DL_EST_ONE_END, dl.DL_EST_GEN, dl.DL_EST_HPE):
                dl.dl_contract(ctx, est, eta, sol, n, dl.DL_C128, 0, P2MAX, out)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            per[name] = {"sec_per_block": t2 - t0, "sec_solve": t1 - t0, "sec_contract": t2 - t1,
                         "iters": float(np.mean(stats.iters[:n])), "max_resid": float(max(stats.resid[:n]))}
            del eta, sol, out
        finally:
            dl.dl_destroy(ctx)
    best = min(per, key=lambda k: per[k]["sec_per_block"])
    return {"by_arithmetic": per, "faster": best, "columns": n, "iters": per[best]["iters"],
            "estimates_per_s": n / per[best]["sec_per_block"],
            "how": f"one block of {n} noise vectors, CG from zero to {TOL_HP:g} with FP64 Krylov vectors (double-float "
                   "and IEEE binary64 timed, the faster kept), then the one-end, generalised one-end and HPE "
                   f"contractions at |n|^2<={P2MAX}"}


# DRAM bytes (read + write) per site-column measured by ncu for stencil classes of the
# current kernels on the 24^3 x 24, 16-column case; a launch's traffic is taken as
# linear in its site-columns (links are read once per launch, every spinor stream once).
# Classes without a capture of the current kernel report no traffic.
#   16-bit CG update (dslash_pair<2, 3, 3, 1>): 736749568 + 251834880 bytes over
#   24^4 / 2 sites x 16 columns (the algorithmic bytes are 997.9 MB)
NCU_DRAM_BYTES_PER_ITEM = {("16-bit", "cg-update"): (736749568 + 251834880) / (24 ** 4 // 2 * 16)}

LINK_BYTES = {"double-float": 144, "f32": 48, "16-bit": 24, "ieee-f64": 144}
SPINOR_BYTES = {"double-float": 192, "f32": 96, "16-bit": 52, "ieee-f64": 192}
STREAMS = {"plain": 2, "aux": 3, "aux+norm": 3, "cg-update": 7}


def stencil_bytes(storage, epilogue, cols):
    """Algorithmic bytes of one stencil launch over the 32^3 x 64 lattice: every link once
    (4 V links), every spinor stream of the output parity once per column."""
    V = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]
    return 4 * V * LINK_BYTES[storage] + STREAMS[epilogue] * (V // 2) * cols * SPINOR_BYTES[storage]


def roofline(st, steps):
    """The stencil class with the largest total time per sweep (launches executed x the
    average CUDA-event duration of its timed launches, from dl_profile_stencils over the
    timed region): algorithmic bytes per launch / average duration against the measured
    HBM copy bandwidth.  Returns (roofline object, per-class table)."""
    peaks, kind = _peaks()
    Vh = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] // 2
    rows = []
    for r in stencil_table(st):
        if not r["timed"] or not r["launches"]:
            continue
        cols = r["items_per_launch"] / Vh
        b = stencil_bytes(r["storage"], r["epilogue"], cols)
        rows.append({"kernel": f"stencil {r['storage']} {r['epilogue']}{' dagger' if r['dagger'] else ''}",
                     "storage": r["storage"], "epilogue": r["epilogue"], "launches_per_step": r["launches"] / steps,
                     "avg_ms": round(r["avg_ms"], 4), "ms_per_step": round(r["total_ms"] / steps, 2),
                     "columns": round(cols, 2), "bytes_per_launch": int(b),
                     "gbs": round(b / (r["avg_ms"] * 1e-3) / 1e9, 1),
                     "frac": round(b / (r["avg_ms"] * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)})
    rows.sort(key=lambda x: -x["ms_per_step"])
    if not rows:
        return None, rows
    top = rows[0]
    per_item = NCU_DRAM_BYTES_PER_ITEM.get((top["storage"], top["epilogue"]))
    traffic = int(per_item * Vh * top["columns"]) if per_item else None
    ro = {"bound": "hbm", "achieved": top["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": top["frac"],
          "traffic": traffic, "kernel": top["kernel"], "columns": top["columns"],
          "bytes_per_launch": top["bytes_per_launch"], "avg_launch_ms": top["avg_ms"],
          "ms_per_step": top["ms_per_step"],
          "peak_kind": kind + " (MEASURED_PEAKS.json hbm_gbs)" if kind == "measured" else kind}
    return ro, rows


# ---- the oracle on the host cores (the reference arm and the cpu_baseline leg) ----
# A bounded sample of the plain method at this workload: the oracle's functions as
# they stand, on the workload's spatial volume (32^3) with SAMPLE_T of its 64 time
# slices, where every step of the oracle (numpy on full-lattice arrays) costs in
# proportion to the volume.  One worker process per host core, each on its own
# noise vector, single-threaded numpy.
SAMPLE_T = 2
# CG iterations of one plain FP64 solve from zero to 1e-10 at this workload, as the
# batched FP64 comparator of the GPU arm measures them (detail.plain_fp64_batched.iters,
# the same on every run: 52 in double-float and in IEEE binary64).
PLAIN_CG_ITERS = 52.0
_SAMPLE = {}


def _oracle_init():
    """Worker start: the oracle's modules and the sample lattice's links (built once per
    worker, outside any timing)."""
    import synth
    from oracle import loops, noise, solver  # noqa: F401
    _SAMPLE["links"] = synth.gauge_links((DIMS[0], DIMS[1], DIMS[2], SAMPLE_T), EPS, LINK_SEED)


def _oracle_sample(idx):
    """On the sample lattice: the even-odd source preparation and odd reconstruction
    (App. A, Eqs. A.2, A.4), one CG iteration of the normal equations (Sec. 2.2; the
    oracle's cg with maxiter = 1), and the contractions of the resulting solution into
    one-end, generalised one-end and HPE loops at |n|^2 <= 9 (Eqs. loopVv, loopStD,
    loopHPE1).  Returns (seconds of the CG iteration, seconds of everything else)."""
    from oracle import loops, noise, solver
    from oracle import operator as op
    dims = (DIMS[0], DIMS[1], DIMS[2], SAMPLE_T)
    if "links" not in _SAMPLE:
        _oracle_init()
    links = _SAMPLE["links"]
    eta = noise.z4_noise(dims, NOISE_SEED, idx)
    t0 = time.perf_counter()
    bhat = op.prep_source(links, eta, KAPPA, AMU, 1, -1.0, dims)
    rhs = op.mhat_dag(links, bhat, KAPPA, AMU, 1, -1.0, dims)
    t1 = time.perf_counter()

    def normal(v):
        return op.mhat_dag(links, op.mhat(links, v, KAPPA, AMU, 1, -1.0, dims), KAPPA, AMU, 1, -1.0, dims)

    x, _, _ = solver.cg(normal, rhs, 0.0, maxiter=1)
    t2 = time.perf_counter()
    s = x + op.reconstruct_odd(links, x, eta, KAPPA, AMU, 1, -1.0, dims)
    for est in ("one_end", "gen_one_end", "hpe"):
        xi, phi = loops.pair(est, links, eta, s, KAPPA, AMU)
        loops.project_momenta(loops.bilinear(xi, phi), dims, P2MAX)
    t3 = time.perf_counter()
    return t2 - t1, (t1 - t0) + (t3 - t2)


class OraclePool:
    """Worker processes (spawned, one per host core, single-threaded numpy) running
    _oracle_sample on distinct noise vectors."""

    def __init__(self, workers=None):
        import multiprocessing as mp
        self.workers = workers or max(1, os.cpu_count() or 1)
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_init)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.next = 0

    def step(self):
        """One sample in every worker at once; returns (wall seconds, per-worker (t_it, t_rest))."""
        idx = list(range(self.next, self.next + self.workers))
        self.next += self.workers
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_sample, idx, chunksize=1)
        return time.perf_counter() - t0, res

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_rate(res, wall, workers):
    """Plain-method loop estimates per second of the whole host from one pool step: each
    worker's full-size estimate costs (64 / SAMPLE_T) (PLAIN_CG_ITERS t_it + t_rest); the
    workers run at once, so the host completes `workers` of them in that time scaled by
    wall / max(worker time) (the contention the concurrent run saw)."""
    scale = DIMS[3] / SAMPLE_T
    per_est = [scale * (PLAIN_CG_ITERS * a + b) for a, b in res]
    busy = max(a + b for a, b in res)
    return workers / (float(np.mean(per_est)) * max(1.0, wall / busy)), per_est


STORAGE = ["double-float", "f32", "16-bit", "ieee-f64"]
EPILOGUE = ["plain", "aux", "aux+norm", "cg-update"]


def stencil_table(st):
    """Rows of dl_profile_stencils: class, launches, average ms (timed launches), total ms."""
    rows = []
    for a in range(4):
        for e in range(4):
            for d in range(2):
                n, nt, ms, items = st[a, e, d]
                if n <= 0 and nt <= 0:
                    continue
                avg = ms / nt if nt > 0 else float("nan")
                rows.append({"storage": STORAGE[a], "epilogue": EPILOGUE[e], "dagger": d, "launches": int(n),
                             "timed": int(nt), "avg_ms": avg, "total_ms": avg * n if nt > 0 else float("nan"),
                             "items_per_launch": items / nt if nt > 0 else float("nan")})
    return rows


def stencil_case():
    """Small case for ncu captures: 24^3 x 24, 16 right-hand sides, one 16-bit, one FP32 and
    one double-float Krylov solve of 4 CG iterations each (fields 138 MB / 255 MB / 510 MB,
    above the 129 MB L2; about 12 GB on the device); prints every stencil class's launches
    and average duration."""
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
    for hi, lo in ((dl.DL_F32, dl.DL_F16), (dl.DL_F32, dl.DL_F32), (dl.DL_F64, dl.DL_F64)):
        prm = dl.dl_solve_params(tol=1e-12, max_iter=4, prec_hi=hi, prec_lo=lo, delta=0.0, flavour=1, chunk=4)
        st, stats = dl.dl_solve(ctx, eta, sol, n, dl.DL_C64, prm)
    torch.cuda.synchronize()
    rows = stencil_table(dl.dl_profile_stencils())
    dl.dl_profile(ctx, 0)
    dl.dl_destroy(ctx)
    for r in rows:
        print(f"{r['storage']:12s} {r['epilogue']:10s} dag {r['dagger']}  launches {r['launches']:4d}  "
              f"avg {r['avg_ms']:.4f} ms  columns {r['items_per_launch'] / (V // 2):.1f}")
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
    # training pairs from the plain solver (complex64 storage, FP64-accurate solutions); the
    # residual loss uses the noise of the pairs only
    residual = args.nn_loss == "residual"
    out["loss"] = args.nn_loss
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
                               seed=11, loss=1 if residual else 0)
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
            # Table compAll analogue: the contractions are the mass-independent overhead
            # (OH) next to the inversion cost of one HP and one LP estimate
            row[key] = {"r_hp_lp": (t_hp + t_c) / (t_lp + t_c), "sec_hp_solve": t_hp, "sec_lp_solve": t_lp,
                        "sec_contract_per_solution": t_c, "overhead_share_hp": t_c / (t_hp + t_c),
                        "overhead_share_lp": t_c / (t_lp + t_c), "iters_hp": info.iters_hp / n_hp,
                        "iters_lp": info.iters_lp / (n_hp + n_lp), "not_converged": info.not_converged}
        rows.append(row)
    dl.dl_destroy(ctx)
    print(json.dumps({"case": "mass_sweep", "data": "synthetic", "lattice": list(dims), "kappa": kappa,
                      "n_hp": n_hp, "n_lp": n_lp, "rows": rows}))


def _gammas16():
    """The 16 Gamma_b of the library's basis (include/discloop.h): chiral Euclidean gammas
    g_k = [[0, -i s_k], [i s_k, 0]] (k = x, y, z), g_t = [[0, 1], [1, 0]];
    Gamma_b = g_x^b0 g_y^b1 g_z^b2 g_t^b3."""
    sig = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], complex)]
    z = np.zeros((2, 2), complex)
    g = [np.block([[z, -1j * sk], [1j * sk, z]]) for sk in sig] + [np.block([[z, np.eye(2)], [np.eye(2), z]])]
    out = []
    for b in range(16):
        m = np.eye(4, dtype=complex)
        for k in range(4):
            if b >> k & 1:
                m = m @ g[k]
        out.append(m)
    return np.stack(out)


def _gamma_loops(out):
    """Loops of the 16 Gamma_b from the [n][T][Np][nd][4][4] bilinear sums:
    l_b = sum_ab (Gamma_b)_ab out_ab."""
    return np.einsum("gab,...ab->...g", _gammas16(), out)


def loop_errors(got, ref):
    """Per Gamma_b and derivative slot: the largest |got - ref| over noise, t and p, and
    that over the largest |ref| of the same Gamma_b and slot."""
    lg, lr = _gamma_loops(got), _gamma_loops(ref)  # [n][T][Np][nd][16]
    d = np.abs(lg - lr).max(axis=(0, 1, 2))
    scale = np.abs(lr).max(axis=(0, 1, 2))
    rel = d / np.maximum(scale, 1e-300)
    return {"max_abs": d.tolist(), "max_rel": rel.tolist(), "worst_rel": float(rel.max()),
            "worst_abs": float(d.max()), "scale_max": float(scale.max())}


def errors_case(args):
    """Per-loop error of the mixed-precision pipeline on 16^3 x 32 (eps 0.4, kappa 0.161,
    a*mu 0.0055, 12 Z4 noise vectors as one block; one-end and generalised one-end loops,
    local and one-derivative, |n|^2 <= 4).  HP map: FP32 Krylov vectors with double-float
    reliable updates every four decades, CG to 1e-10 (the benchmark's HP solve).  LP map:
    16-bit Krylov vectors, CG to 1e-2.  Reference: IEEE binary64 solves to 1e-12 of the
    same noise (no mixed precision; the FP64 operator and contractions are the ones the
    parity tests hold to the oracle within 1e-13), contracted in FP64.  Reports, per
    Gamma and derivative slot, the largest absolute and relative deviation over t and p."""
    import torch

    import paper_1309_2256_gb300 as dl
    import synth
    dims = (16, 16, 16, 32)
    kappa, amu, n, p2 = 0.161, 0.0055, 12, 4
    ctx = dl.dl_create(dims, 0, torch.cuda.current_stream())
    dl.dl_load_gauge(ctx, synth.gauge_links(dims, 0.4, 1001), -1.0, 12, 12)
    dl.dl_set_params(ctx, kappa, amu)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    npm = len(dl.dl_momenta(p2))
    eta = torch.empty((n, V * 12), dtype=torch.complex128, device="cuda")
    dl.dl_noise_z4(ctx, 2001, 0, n, eta, dl.DL_C128)
    maps = {"hp": (1e-10, dl.DL_F64, dl.DL_F32, 1e-4), "lp": (1e-2, dl.DL_F32, dl.DL_F16, 0.0),
            "ref": (1e-12, dl.DL_F64_IEEE, dl.DL_F64_IEEE, 0.0)}
    loops, stats = {}, {}
    for name, (tol, hi, lo, delta) in maps.items():
        sol = torch.empty_like(eta)
        prm = dl.dl_solve_params(tol=tol, max_iter=200000, prec_hi=hi, prec_lo=lo, delta=delta, flavour=1, chunk=32)
        st, ss = dl.dl_solve(ctx, eta, sol, n, dl.DL_C128, prm)
        stats[name] = {"iters": float(np.mean(ss.iters[:n])), "max_resid": float(max(ss.resid[:n])),
                       "max_true_resid": float(max(ss.true_resid[:n]))}
        per = {}
        for est, code in (("one_end", dl.DL_EST_ONE_END), ("gen_one_end", dl.DL_EST_GEN)):
            out = torch.zeros((n, dims[3], npm, 5, 4, 4), dtype=torch.complex128, device="cuda")
            dl.dl_contract(ctx, code, eta, sol, n, dl.DL_C128, 1, p2, out)
            per[est] = out.cpu().numpy()
        loops[name] = per
        del sol
    dl.dl_destroy(ctx)
    res = {}
    for est in ("one_end", "gen_one_end"):
        res[est] = {"hp_vs_fp64": loop_errors(loops["hp"][est], loops["ref"][est]),
                    "lp_vs_hp": loop_errors(loops["lp"][est], loops["hp"][est])}
    print(json.dumps({"case": "loop_errors", "data": "synthetic", "lattice": list(dims), "kappa": kappa, "amu": amu,
                      "noise_vectors": n, "p2max": p2, "derivative_slots": "local, then x, y, z, t",
                      "gamma_order": "b = bitmask of g_x g_y g_z g_t (chiral basis)", "solves": stats,
                      "errors": res}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default=None, choices=["stencil", "contract", "learned", "batch", "mass", "errors"],
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
    ap.add_argument("--nn-loss", default="solution", choices=["solution", "residual"],
                    help="learned case: training loss |N eta - s|^2/|s|^2 or |M N eta - eta|^2/|eta|^2")
    ap.add_argument("--masses", default="0.0055,0.02,0.2", help="mass case: valence a*mu values")
    args = ap.parse_args()
    if args.case == "mass":
        mass_case(args)
        return
    if args.case == "errors":
        errors_case(args)
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

    # the oracle's worker processes start before the first GPU call (spawned, rank 0 only)
    cpu_pool = OraclePool() if rank == 0 else None
    import torch
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    r = run_ours(args, rank, world, local)
    if rank != 0:
        return
    ro = r["roof"]
    # CPU baseline: the oracle on the host cores, one bounded sample per worker (the
    # pool was started before the first GPU call)
    wall, res = cpu_pool.step()
    cpu_pool.close()
    cpu_rate, per_est = oracle_rate(res, wall, cpu_pool.workers)
    it_hp, it_lp = r["it_hp"], r["it_lp"]
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
        "dtype": "int16 fixed point (LP) / f32 (HP) Krylov storage, f32 arithmetic; double-float reliable updates, "
                 "f64 accumulation",
        "data": "synthetic (seeded SU(3) links exp(i eps H), eps 0.4; Z2xiZ2 noise)",
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "kappa": KAPPA, "amu": AMU, "n_hp": N_HP, "n_lp": N_LP,
                   "tol_hp": TOL_HP, "tol_lp": TOL_LP, "delta_hp": args.delta_hp, "hp_from_lp": 1, "hpe_correction_from_difference": 1, "block": r["block"],
                   "block_choice": "autotuned by the library (LP blocks of 8, 16, 32 timed, least time per right-hand side)"
                   if BLOCK == 0 else "fixed", "p2max": P2MAX, "hpe_orders": 4,
                   "step": "one TSM sweep: 24 HP-LP pairs + 500 LP solves + contractions",
                   "l2": "inputs larger than L2 (gauge field 0.4-1.2 GB, spinor blocks GBs)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": ro,
        "cpu_baseline": {"value": round(cpu_rate, 8), "unit": "loop estimates/s (equal error)",
                         "cores": cpu_pool.workers, "kind": "oracle",
                         "sample": f"the plain method (FP64 CG per noise vector, {PLAIN_CG_ITERS:.0f} iterations, and the "
                                   f"same contractions): each of {cpu_pool.workers} worker processes runs the oracle "
                                   f"on 32^3x{SAMPLE_T} (source preparation, one CG iteration, reconstruction, "
                                   f"one-end/generalised/HPE contractions at |n|^2<=9, {wall:.1f} s), scaled "
                                   f"x{DIMS[3] // SAMPLE_T} in volume"},
        "e2e": {"value": round(r["e2e"], 4), "unit": "loop estimates/s (equal error)",
                "h2d_bytes_per_step": int(r["bytes_h2d"]), "d2h_bytes_per_step": int(r["bytes_d2h"])},
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
        "detail": {"stencil_classes": r["stencils"],
                   "equal_error": r["eq"], "iters_hp": it_hp, "iters_lp": it_lp, "sec_hp_per_step": r["sec_hp"],
                   "sec_lp_per_step": r["sec_lp"], "sec_contract_per_step": r["sec_ct"],
                   "plain_fp64_batched": r["ref_batched"],
                   "vs_plain_fp64_batched": r["value"] / r["ref_batched"]["estimates_per_s"],
                   "plain_fp64_single_rhs": r["ref"],
                   "batching_gain_fp64": (r["ref_batched"]["estimates_per_s"] / r["ref"]["estimates_per_s"])
                   if r["ref"]["estimates_per_s"] else None},
    }
    print(json.dumps(line))


def run_reference(args, world):
    """The oracle as it stands on the host cores, same metric, config and unit.
    The oracle is the plain method (FP64 CG on every noise vector to 1e-10, no TSM,
    then the same contractions), so each of its loop estimates counts one at equal
    error.  A step is one bounded sample in every worker (_oracle_sample), scaled to
    the full lattice and the plain method's CG iteration count."""
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.step()
        rates, walls, per_est = [], [], []
        for _ in range(args.steps):
            wall, res = pool.step()
            rate, pe = oracle_rate(res, wall, pool.workers)
            rates.append(rate)
            walls.append(wall)
            per_est += pe
    finally:
        pool.close()
    value = float(np.median(rates))
    sample = (f"per step, each of {pool.workers} worker processes (one per host core, single-threaded numpy) runs the "
              f"oracle on its own noise vector on 32^3x{SAMPLE_T} (the workload's space, {SAMPLE_T} of 64 slices): "
              f"source preparation, one CG iteration of the normal equations, odd reconstruction and the one-end, "
              f"generalised one-end and HPE contractions at |n|^2<=9; scaled x{DIMS[3] // SAMPLE_T} in volume and to "
              f"{PLAIN_CG_ITERS:.0f} CG iterations per estimate (median step {float(np.median(walls)):.1f} s)")
    line = {"impl": "reference",
            "metric": "loop estimates/sec at 32^3x64 at equal error (TSM vs plain HP estimates); Dslash HBM GB/s",
            "value": round(value, 8), "unit": "loop estimates/s (equal error)", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(float(np.median(walls)) * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": list(DIMS), "kappa": KAPPA, "amu": AMU, "p2max": P2MAX,
                       "method": "plain FP64 CG per noise vector + the same contractions (the oracle)",
                       "cg_iters_per_estimate": PLAIN_CG_ITERS},
            "cpu_baseline": {"kind": "oracle", "cores": pool.workers, "value": round(value, 8), "sample": sample,
                             "sec_per_estimate_one_core": round(float(np.median(per_est)), 1)},
            "e2e": {"value": round(value, 8), "unit": "loop estimates/s (equal error)", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
