#!/usr/bin/env python
"""Benchmark of the state-vector ADAPT-VQE hot path on one GB300 (or N
independent replicas under torchrun).

Workload: 32 qubits -- 16 orbitals, 8 alpha + 8 beta electrons, 165,636,900
determinants, seeded synthetic integrals shaped like the H16 STO-3G chain,
the spin-adapted singles+doubles pool (3,376 operators).

One step = one ADAPT-VQE iteration of the mixed-precision driver with the
learned ranker: screen, select, append, re-optimise every parameter with
BFGS (each evaluation: state preparation by exp(theta A) with
double-precision renormalisation, H psi, energy and adjoint gradient, bulk
in float, reductions in double).  While psi has few nonzero amplitudes (the
paper's sparse regime) H psi and the screen run on the sparse-state path
and the screen is exact; later the ranker's top-32 proposals are screened.
The first `warmup` iterations run the full screen and train the ranker; the
next `steps` are timed.  `value` = timed ADAPT iterations per second over all
ranks.  The same run with the dense sweeps only is reported beside it.

Also reported: H|psi> time, algorithmic GB/s and HBM fraction in FP64 and
FP32; one plain FP64 full-screen iteration timed from the same ansatz
("plain vs mixed+ranker"); the double-precision refinement of the final
energy and its gap to the float bulk; the ranker's rank of the true argmax
at the final state.  `e2e` repeats the step through the public API with the
ansatz restored from host memory every step (a stateless-serving step).

Every sweep runs in the library's kernels (libhyperion.so); the FP64 CPU
oracle is timed on a bounded sample for `cpu_baseline` and for the
`--impl reference` arm.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = ("H|psi> GB/s (% of ~8 TB/s) and ADAPT iters/s at 32 qubits, "
          "plain vs mixed+ranker")
TOP_M = 32
# DRAM bytes per launch of k_cpl_tc (the tensor-core phase A of the float
# coupling) at 32 q: the ncu capture at 28 q (profiles/coupling_tc_28q.md:
# 51.5 MB read + 2.30 GB written, the written part being the T intermediate)
# scaled by the size of T (x 18.24) and of the psi rows read (x 14.06).  The
# phase-B gather that the bench's coupling time also covers is not included,
# so the roofline's own "traffic" (both kernels) stays None.
TRAFFIC_CPL_TC = 2.300555e9 * 18.24 + 51.5e6 * 14.06
TRAFFIC_F32 = None
REFRESH = 4        # every 4th ranked iteration selects from the full screen


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="h16_32q")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 iteration")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of oracle work per CPU sample")
    ap.add_argument("--sweeps-only", action="store_true",
                    help="profiling mode: two passes of each sweep (H psi, energy, full screen, "
                         "one exp(theta A)) per dtype on a seeded state, no timing line")
    ap.add_argument("--dtypes", default="f64,f32", help="dtypes of --sweeps-only")
    ap.add_argument("--ranker-eval", action="store_true",
                    help="plain FP64 ADAPT vs mixed+ranker ADAPT with the full screen as judge: "
                         "per-iteration rank of the true argmax and energy gap")
    ap.add_argument("--iters", type=int, default=12, help="iterations of --ranker-eval")
    ap.add_argument("--sparse-eval", action="store_true",
                    help="--ranker-eval on the sparse-state path (plain reference included)")
    ap.add_argument("--top-m", type=int, default=TOP_M,
                    help="operators the ranker proposes for the exact screen")
    ap.add_argument("--adapt-only", action="store_true",
                    help="profiling mode: only the headline ADAPT leg (no sweeps, plain, dense, "
                         "CPU), printing its iterations/s")
    ap.add_argument("--judge-only", action="store_true",
                    help="--ranker-eval without the plain run (ranks of the true argmax only)")
    ap.add_argument("--hmat", action="store_true",
                    help="the Hamiltonian stored explicitly: build it for --rows alpha strings of "
                         "--workload and time H psi streamed from it against the matrix-free sweep")
    ap.add_argument("--rows", default="all",
                    help="--hmat row range 'b:e' in alpha strings, or 'all'")
    ap.add_argument("--hmat-dtypes", default="f32,f64", help="dtypes of --hmat")
    ap.add_argument("--reps", type=int, default=5, help="timed repetitions of --hmat")
    ap.add_argument("--batch", action="store_true",
                    help="64 molecules of 8-12 orbitals: H psi + energies of all in one persistent "
                         "graph-captured launch (autotuned tile) vs one launch sequence per molecule")
    return ap.parse_args()


def batch_bench(args, count=64, reps=5):
    """Batched sweeps over the uneven 64-molecule workload."""
    import torch
    import paper_2604_01176_gb300 as hy
    from paper_2604_01176_gb300 import build as hybuild
    hybuild.build()
    hams = []
    for n, na, nb, seed in synth.batch_molecules(count):
        h1, h2, ec = synth.integrals(n, seed)
        hams.append(hy.Hamiltonian(h1, h2, ec, n, na, nb))
    b = hy.Batch(hams)
    total = sum(h.n_det for h in hams)
    out = {"batch": f"{count} molecules, n = 8..12 at half filling, seeds 2000+i",
           "determinants": total, "tasks": b.n_tasks}
    st = torch.cuda.current_stream()
    for d, dt in (("f64", torch.float64), ("f32", torch.float32)):
        gen = torch.Generator(device="cuda")
        gen.manual_seed(3)
        states = [torch.randn(h.n_det, dtype=dt, device="cuda", generator=gen) for h in hams]
        states = [x / x.norm() for x in states]
        psi = b.pack(states, dt)
        sig = torch.zeros_like(psi)
        en = torch.empty(count, dtype=torch.float64, device="cuda")
        tile, tune_ms = b.tune(psi, sig)
        b.apply_h(psi, sig, en, graph=True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        l0 = hy.launch_count()
        ev[0].record(st)
        for _ in range(reps):
            b.apply_h(psi, sig, en, graph=True)
        ev[1].record(st)
        l1 = hy.launch_count()
        sigs = [torch.empty_like(x) for x in states]
        eo = [torch.empty((), dtype=torch.float64, device="cuda") for _ in hams]
        for h, x, y, e in zip(hams, states, sigs, eo):     # warm the per-molecule path
            h.apply_h(x, out=y)
            h.energy(x, y, out=e)
        torch.cuda.synchronize()
        l2 = hy.launch_count()
        ev[2].record(st)
        for _ in range(reps):
            for h, x, y, e in zip(hams, states, sigs, eo):
                h.apply_h(x, out=y)
                h.energy(x, y, out=e)
        ev[3].record(st)
        torch.cuda.synchronize()
        l3 = hy.launch_count()
        t_b = ev[0].elapsed_time(ev[1]) / reps
        t_l = ev[2].elapsed_time(ev[3]) / reps
        err = max(abs(float(en[m].item()) - float(eo[m].item())) for m in range(count))
        out[d] = {"tile": tile, "tune_ms": round(tune_ms, 3),
                  "batched_ms": round(t_b, 3), "looped_ms": round(t_l, 3),
                  "speedup": round(t_l / t_b, 2),
                  "batched_launches": (l1 - l0) // reps, "looped_launches": (l3 - l2) // reps,
                  "molecules_per_s": round(count / (t_b / 1e3), 1),
                  "max_energy_diff_vs_looped": err}
    print(json.dumps(out), flush=True)


def hmat_bench(args):
    """H psi streamed from the explicitly stored Hamiltonian (a range of its
    rows) against the matrix-free sweep of the same rows: CUDA events on the
    launching stream, inputs resident, the matrix far larger than L2 so every
    repetition streams it from HBM.  Bytes = the stored matrix (16-bit beta
    columns, values, segment partners) + psi rows read + sigma rows written."""
    import torch
    import paper_2604_01176_gb300 as hy
    from paper_2604_01176_gb300 import build as hybuild
    hybuild.build()
    peaks, peak_kind = load_peaks()
    n, na, nb, seed = synth.workload(args.workload)
    h1, h2, ec = synth.integrals(n, seed)
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    NA, NB = ham.n_alpha_str, ham.n_beta_str
    b, e = (0, NA) if args.rows == "all" else tuple(int(x) for x in args.rows.split(":"))
    st = torch.cuda.current_stream()
    out = {"hmat": args.workload, "rows": [b, e], "n_det_rows": (e - b) * NB,
           "row_len": None, "peak_gbs": peaks["hbm_gbs"], "peak_kind": peak_kind}
    for d in args.hmat_dtypes.split(","):
        dt = torch.float64 if d == "f64" else torch.float32
        by, nnz = hy.ExplicitH.size(ham, dt, b, e)
        free, _ = torch.cuda.mem_get_info()
        if by + (1 << 30) + 2 * ham.n_det * (8 if d == "f64" else 4) > free:
            out[d] = {"skipped": f"needs {by} bytes, {free} free"}
            continue
        t0 = time.perf_counter()
        m = hy.ExplicitH(ham, dt, b, e)
        t_build = time.perf_counter() - t0
        out["row_len"] = m.row_len
        gen = torch.Generator(device="cuda")
        gen.manual_seed(2)
        psi = torch.randn(ham.n_det, dtype=dt, device="cuda", generator=gen)
        sig = torch.empty((e - b) * NB, dtype=dt, device="cuda")
        m.apply(psi, out=sig)
        ham.apply_h_rows(psi, b, e, out=sig)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.reps + 2)]
        torch.cuda.synchronize()
        ms_m = []
        for r in range(args.reps):
            ev[2 * r].record(st)
            m.apply(psi, out=sig)
            ev[2 * r + 1].record(st)
        torch.cuda.synchronize()
        ms_m = [ev[2 * r].elapsed_time(ev[2 * r + 1]) for r in range(args.reps)]
        ref = sig.clone()
        ham.apply_h_rows(psi, b, e, out=sig)
        diff = float(torch.max(torch.abs(sig - ref)).item() / torch.max(torch.abs(ref)).item())
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.reps):
            ham.apply_h_rows(psi, b, e, out=sig)
        e1.record(st)
        torch.cuda.synchronize()
        ms_mf = e0.elapsed_time(e1) / args.reps
        es = 8 if d == "f64" else 4
        traffic = by + 2 * (e - b) * NB * es
        ms = statistics.median(ms_m)
        gbs = traffic / (ms / 1e3) / 1e9
        out[d] = {"build_s": round(t_build, 2), "matrix_bytes": by, "nnz": nnz,
                  "ms": round(ms, 4), "ms_all": [round(x, 4) for x in ms_m],
                  "gbs": round(gbs, 1), "frac_of_hbm": round(gbs / peaks["hbm_gbs"], 4),
                  "matrix_free_ms": round(ms_mf, 4),
                  "max_rel_diff_vs_matrix_free": diff}
        del m, psi, sig, ref
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def ranker_eval(args):
    """The ranker judged against the full screen: plain FP64 ADAPT and the
    mixed+ranker ADAPT (double refinement every iteration so energies compare
    at FP64) run side by side; per iteration the rank of the true argmax
    among the ranker's proposals and the energy gap to the plain run."""
    import paper_2604_01176_gb300 as hy
    from paper_2604_01176_gb300 import build as hybuild
    hybuild.build()
    n, na, nb, seed = synth.workload(args.workload)
    h1, h2, ec = synth.integrals(n, seed)
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    pool = hy.Pool(ham)
    it = args.iters
    # the sparse path makes the plain FP64 reference affordable at 32 q; the
    # ranker is asked on every ranked iteration (no exact sparse screen)
    sp = dict(sparse=True, exact_screen_work=-1.0) if args.sparse_eval else {}
    plain = None if args.judge_only else hy.Adapt(ham, pool, "f64", max_iter=it,
                                                  **sp).run(it)
    ranker = hy.Ranker(hidden=256, seed=7)
    ad = hy.Adapt(ham, pool, "mixed", max_iter=it, screen_top_m=args.top_m, judge=True,
                  refine_every=0 if args.judge_only else 1, **sp)
    ad.set_ranker(ranker, warm_iters=args.warmup, epochs=30, refresh_every=REFRESH)
    ranked = ad.run(it)
    rows = []
    for i, r in enumerate(ranked):
        row = {"iter": r["iter"], "e_ranked": r["energy"], "true_rank": r["true_rank"],
               "selected": r["selected"], "true_argmax": r["true_argmax"],
               "t_screen_ranked": round(r["t_screen"], 5), "t_total": round(r["t_total"], 3)}
        if plain is not None:
            p = plain[i]
            row.update({"e_plain": p["energy"], "gap": r["energy"] - p["energy"],
                        "same_op": p["selected"] == r["selected"],
                        "t_screen_plain": round(p["t_screen"], 5)})
        rows.append(row)
    print(json.dumps({"ranker_eval": args.workload, "top_m": args.top_m, "warm": args.warmup,
                      "refresh_every": REFRESH, "pool_ops": len(pool), "rows": rows}), flush=True)


def sweeps_only(args):
    """Two passes of every sweep on a seeded random state, for ncu captures."""
    import torch
    import paper_2604_01176_gb300 as hy
    from paper_2604_01176_gb300 import build as hybuild
    hybuild.build()
    n, na, nb, seed = synth.workload(args.workload)
    h1, h2, ec = synth.integrals(n, seed)
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    pool = hy.Pool(ham)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    for d in args.dtypes.split(","):
        dt = torch.float64 if d == "f64" else torch.float32
        psi = torch.randn(ham.n_det, dtype=dt, device="cuda", generator=gen)
        psi /= psi.norm()
        sig = torch.empty_like(psi)
        for _ in range(2):
            ham.apply_h(psi, out=sig)
            e = ham.energy(psi, sig)
            g = pool.gradients(psi, sig)
            pool.apply_excitation(len(pool) - 1, 0.1, psi)
        torch.cuda.synchronize()
        print(json.dumps({"sweeps": args.workload, "dtype": d, "energy": float(e.item()),
                          "max_grad": float(g.abs().max().item())}), flush=True)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# oracle timing on the host cores (bounded samples of the same workload)
# ---------------------------------------------------------------------------
def oracle_iteration_estimate(n, na, nb, seed, budget_s, ansatz_len, n_evals, state=None):
    """Seconds the FP64 CPU oracle would take for one plain ADAPT iteration
    with `n_evals` energy+gradient evaluations at ansatz length `ansatz_len`,
    extrapolated from a bounded sample: sigma on sampled rows, the gradient
    of a few pool operators (each O(N_det)), and one exp(theta A).
    Returns (seconds, threads, sample description)."""
    import oracle
    h1, h2, ec = synth.integrals(n, seed)
    ref = oracle.System(h1, h2, ec, n, na, nb)
    threads = len(os.sched_getaffinity(0))
    if state is None:
        state = synth.random_state(ref.n_det, 99)
    rng = np.random.default_rng(1)
    rows = rng.integers(0, ref.n_det, 64 * threads)
    t0 = time.perf_counter()
    ref.sigma_rows(state, rows, threads)
    dt = time.perf_counter() - t0
    m = int(min(ref.n_det, max(len(rows), len(rows) * 0.5 * budget_s / max(dt, 1e-6))))
    rows = rng.integers(0, ref.n_det, m)
    t0 = time.perf_counter()
    ref.sigma_rows(state, rows, threads)
    t_rows = time.perf_counter() - t0
    t_sigma = t_rows * ref.n_det / m
    pool = ref.pool()
    nops = max(1, min(threads, 4))
    t0 = time.perf_counter()
    ref.gradients(pool[:nops], state, state, nops)
    t_g = time.perf_counter() - t0
    t_op = t_g / nops            # one operator's gradient, one thread
    t0 = time.perf_counter()
    ref.apply_excitation(pool[len(pool) - 1], 0.1, state)
    t_x = time.perf_counter() - t0
    # screen (all operators, parallel over threads) + per evaluation: prepare
    # (j exps), sigma, energy, adjoint gradient (2j exps + j generator dots)
    t_screen = t_op * len(pool) / threads
    t_eval = t_sigma + ansatz_len * t_x + 2 * ansatz_len * t_x + ansatz_len * t_op
    total = t_screen + n_evals * t_eval
    sample = (f"sigma on {m} sampled rows ({t_rows:.1f} s, {threads} threads), gradients of "
              f"{nops} ops ({t_g:.1f} s), one exp(theta A) ({t_x:.1f} s); extrapolated to one "
              f"plain ADAPT iteration: full screen of {len(pool)} ops + {n_evals} evaluations "
              f"at ansatz length {ansatz_len} over {ref.n_det} determinants")
    return total, threads, sample


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of per-rank timings over the process group (the
    job's time is its slowest replica's)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def job_throughput(world, steps, ms_max):
    """Whole-job iterations per second: every rank ran `steps` iterations of
    its own replica within the slowest rank's `ms_max` milliseconds."""
    return world * steps / (ms_max / 1e3)


def time_sweeps(ham, pool, dt, reps=3):
    """Mean device time (ms) of H psi and of the full screen in dtype dt."""
    import torch
    g = torch.Generator(device=ham.device)
    g.manual_seed(5)
    psi = torch.randn(ham.n_det, dtype=dt, device=ham.device, generator=g)
    psi /= psi.norm()
    sig = torch.empty_like(psi)
    gr = torch.empty(len(pool), dtype=torch.float64, device=ham.device)
    st = torch.cuda.current_stream()
    ham.apply_h(psi, out=sig)
    pool.gradients(psi, sig, out=gr)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record(st)
    for _ in range(reps):
        ham.apply_h(psi, out=sig)
    e[1].record(st)
    for _ in range(reps):
        pool.gradients(psi, sig, out=gr)
    e[2].record(st)
    torch.cuda.synchronize()
    # the dominant kernel alone: events the library records around the
    # alpha-beta coupling launches, on the same stream
    ham.profile_coupling(True)
    cpl = []
    for _ in range(reps):
        ham.apply_h(psi, out=sig)
        cpl.append(ham.coupling_ms())
    ham.profile_coupling(False)
    return e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps, statistics.mean(cpl)


def adapt_leg(ham, pool, hy, torch, args, rank, world, sparse, clocks=None):
    """Mixed precision + ranker ADAPT: W warm-up iterations (full screens that
    train the ranker), S timed iterations, then S end-to-end iterations that
    restore the ansatz from host memory, two judged iterations, the double
    refinement of the final energy, and one plain FP64 full-screen iteration
    from the same ansatz (unless --no-plain)."""
    W, S = args.warmup, args.steps
    stream = torch.cuda.current_stream()
    cap = W + 2 * S + 6
    ranker = hy.Ranker(hidden=256, seed=7 + rank)
    ad = hy.Adapt(ham, pool, "mixed", max_iter=cap, screen_top_m=args.top_m, refine_every=0,
                  sparse=sparse)
    ad.set_ranker(ranker, warm_iters=W, epochs=30, refresh_every=REFRESH)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    warm = [ad.step() for _ in range(W)]
    ops0, th0 = ad.ansatz()
    barrier()
    if clocks:
        clocks.start()
    l0 = hy.launch_count()
    hy.profile_enable(hy.PROFILE_CLASSES)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    timed = [ad.step() for _ in range(S)]
    t1.record(stream)
    barrier()
    launches = hy.launch_count() - l0
    ms = t0.elapsed_time(t1)
    prof = {c: hy.profile_read(c) for c in hy.PROFILE_CLASSES}
    hy.profile_enable([])
    # end to end: the same S iterations again from the ansatz the timed
    # region started from, the ansatz restored from host memory before and
    # read back after every step
    ad.set_ansatz(ops0, th0)
    barrier()
    io0 = ad.io_bytes()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(S):
        ops, th = ad.ansatz()
        ad.set_ansatz(ops, th)
        ad.step()
        ad.ansatz()
    e1.record(stream)
    barrier()
    clk = clocks.stop() if clocks else None
    io1 = ad.io_bytes()
    ms_e2e = e0.elapsed_time(e1)
    ad.set_judge(True)
    judged = [ad.step() for _ in range(2)]
    ad.set_judge(False)
    e_bulk = judged[-1]["energy"]
    e_final = ad.refine(steps=4)
    ops, th = ad.ansatz()
    res = dict(ms=ms, ms_e2e=ms_e2e, launches=launches, clocks=clk, timed=timed, warm=warm, prof=prof,
               io=((io1[0] - io0[0]) / S, (io1[1] - io0[1]) / S), e_final=e_final,
               e_bulk=e_bulk, true_rank=[j["true_rank"] for j in judged], ansatz_len=len(ops))
    del ad
    if not args.no_plain:
        plain = hy.Adapt(ham, pool, "f64", max_iter=len(ops) + 2, sparse=sparse)
        plain.set_ansatz(ops, th)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        p0.record(stream)
        prec = plain.step()
        p1.record(stream)
        torch.cuda.synchronize()
        res.update(plain_ms=p0.elapsed_time(p1), plain_rec=prec)
    if world > 1:
        res["ms"], res["ms_e2e"] = max_over_ranks([ms, ms_e2e], torch.device("cuda"))
    return res


def run_ours(args, rank, world):
    import torch
    import paper_2604_01176_gb300 as hy
    from paper_2604_01176_gb300 import build as hybuild

    hybuild.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    n, na, nb, seed = synth.workload(args.workload)
    h1, h2, ec = synth.integrals(n, seed)
    tb = time.perf_counter()
    ham = hy.Hamiltonian(h1, h2, ec, n, na, nb)
    pool = hy.Pool(ham)
    t_build = time.perf_counter() - tb
    out = dict(N=ham.n_det, K=len(pool), n=n, na=na, nb=nb, seed=seed, t_build=t_build,
               conn=ham.connections_per_det(), n_alpha_str=math.comb(n, na),
               n_beta_str=math.comb(n, nb))
    if args.adapt_only:
        args.no_plain = True
        out["head"] = adapt_leg(ham, pool, hy, torch, args, rank, world, True)
        return out
    out["hpsi_ms_f64"], out["screen_ms_f64"], out["cpl_ms_f64"] = time_sweeps(ham, pool,
                                                                            torch.float64)
    out["hpsi_ms_f32"], out["screen_ms_f32"], out["cpl_ms_f32"] = time_sweeps(ham, pool,
                                                                            torch.float32)
    out["cpl_units"] = (ham.n_alpha * (ham.n_orb - ham.n_alpha) + 1) * \
        (ham.n_beta * (ham.n_orb - ham.n_beta) + 1)
    # headline: the sparse-state path (automatic while psi is sparse)
    out["head"] = adapt_leg(ham, pool, hy, torch, args, rank, world, True, Clocks(dev.index))
    # the same with the dense sweeps only (tracks the dense kernels)
    out["dense"] = adapt_leg(ham, pool, hy, torch, args, rank, world, False)
    return out


# kernels behind each class of the library's event profiler
CLASS_KERNELS = {
    "hpsi": "k_spmm + k_transpose + k_add_transposed + coupling (dense H|psi>)",
    "hpsi_sparse": "sigma memset + k_hpsi_scatter (scatter H|psi>)",
    "excite": "k_excite / k_excite_n (dense pair rotations: 4 s bytes per pair)",
    "sparse_excite": "k_sv_excite, k_sv_prepare (sparse-state rotations)",
    "screen": "k_grad_partial + k_grad_final (dense pool gradients)",
    "screen_sparse": "k_grad_sparse + k_grad_sparse_final (support-restricted gradients)",
    "reduce": "dots, norms, renormalisation",
    "features": "k_pair_weights + k_pair_contract + k_pair_reduce + occupations + k_features",
}


def breakdown(prof, step_ms):
    """Device time per kernel class in the timed region (CUDA events on the
    launching stream), as a share of the region's wall time."""
    return {c: {"launches": v["launches"], "ms": round(v["ms"], 3),
                "share_of_step": round(v["ms"] / step_ms, 4)}
            for c, v in prof.items() if v["launches"]}


# classes bound by arithmetic rather than HBM (the headline's bulk is float)
ALU_CLASSES = ("hpsi",)

# L2 reduction rate of the GB300 (5.61 M reduction sectors = 32.5 % of the
# peak-sustained rate over a 45.8 us launch of k_hpsi_scatter under ncu) and
# the rate of float atomic adds to pseudo-random addresses over 2 M targets
# with the membership-bit test (paper_2604_01176_gb300/probes/l2_atomics.cu);
# both in profiles/scatter_atomics_32q.md
L2_RED_PEAK = 3.77e11
L2_RANDOM_ADDS = 3.33e10


def step_roofline(prof, peaks, peak_kind, fp32_peak):
    """Roofline of the kernel class with the most device time among those
    whose algorithmic work the host knows: bytes / event time against the
    measured HBM copy rate, or flops / event time against the derived FP32
    rate for the arithmetic-bound classes."""
    known = {c: v for c, v in prof.items()
             if v["launches"] and (v["bytes"] > 0 or v["flops"] > 0)}
    estimated = {"sparse_excite": "bytes estimated from the support sizes the host last read back"}
    top_all = max(prof, key=lambda c: prof[c]["ms"])
    if not known:
        return {"bound": "hbm", "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": None, "traffic": None, "dominant_class": top_all}
    c = max(known, key=lambda k: known[k]["ms"])
    v = known[c]
    out = {"kernel_class": c, "kernel": CLASS_KERNELS[c], "launches": v["launches"],
           "ms_per_launch": round(v["ms"] / v["launches"], 4), "dominant_class": top_all,
           "timing": "CUDA events around each launch on its stream, over the timed region",
           "traffic": None}
    if c in ALU_CLASSES and v["flops"] > 0:
        tf = v["flops"] / (v["ms"] / 1e3) / 1e12
        out.update(bound="alu", achieved=round(tf, 3), peak=round(fp32_peak, 3), unit="TFLOP/s",
                   frac=round(tf / fp32_peak, 4), flops_per_launch=round(v["flops"] / v["launches"]),
                   peak_kind="derived FP32 FMA rate: 152 SMs x 128 FMA/clk x 2 x max SM clock")
    else:
        gbs = v["bytes"] / (v["ms"] / 1e3) / 1e9
        out.update(bound="hbm", achieved=round(gbs, 1), peak=peaks["hbm_gbs"], unit="GB/s",
                   frac=round(gbs / peaks["hbm_gbs"], 4),
                   bytes_per_launch=round(v["bytes"] / v["launches"]),
                   peak_kind=f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)")
        if c in estimated:
            out["bytes_note"] = estimated[c]
    if c == "hpsi_sparse" and v["flops"] > 0:
        # the scatter is bound by its gathers and the L2 atomics, not by HBM:
        # its atomic adds against the L2 reduction units' rate (derived from
        # ncu's peak-sustained share of a captured launch) and a probe of
        # pseudo-random adds over a sigma-sized footprint
        adds = v["flops"] / (v["ms"] / 1e3)
        out["l2_atomics"] = {
            "adds_per_launch_est": round(v["flops"] / v["launches"]),
            "achieved_adds_per_s": float(f"{adds:.4g}"),
            "l2_red_peak_sectors_per_s": L2_RED_PEAK,
            "frac_of_l2_red_peak": round(adds / L2_RED_PEAK, 4),
            "probe_random_adds_per_s": L2_RANDOM_ADDS,
            "note": "adds estimated as the couplings per amplitude x the support the host "
                    "last read back; one add is one L2 reduction sector at most",
            "source": "profiles/scatter_atomics_32q.md"}
    return out


def c_tilde(records):
    """The paper's amortised ADAPT coefficient C~ = j / sqrt(T_j) (Numerical
    performance subsection): j iterations from Hartree-Fock, T_j their summed
    wall time in seconds (each iteration's host-measured total)."""
    t = sum(float(r["t_total"]) for r in records)
    j = len(records)
    return {"iterations": j, "t_s": round(t, 6),
            "value": round(j / math.sqrt(t), 3) if t > 0 else None, "unit": "s^-1/2"}


def leg_summary(leg, S):
    out = {"iters_per_s": round(S / (leg["ms"] / 1e3), 5),
           "n_evals": [rec["n_evals"] for rec in leg["timed"]],
           "t_screen_s": [round(rec["t_screen"], 4) for rec in leg["timed"]],
           "support": [rec["support"] for rec in leg["timed"]],
           "sigma_support": [rec["sigma_support"] for rec in leg["timed"]],
           "energy_bulk": [rec["energy"] for rec in leg["timed"]],
           "final_energy_f64": leg["e_final"],
           "final_bulk_minus_f64": leg["e_bulk"] - leg["e_final"],
           "ranker_true_argmax_rank_judged": leg["true_rank"],
           "c_tilde": c_tilde(list(leg["warm"]) + list(leg["timed"]))}
    if "plain_ms" in leg:
        out["plain_f64_full_screen"] = {
            "iters_per_s": round(1e3 / leg["plain_ms"], 5), "ms": round(leg["plain_ms"], 1),
            "n_evals": leg["plain_rec"]["n_evals"], "ansatz_len": leg["plain_rec"]["iter"] + 1}
        out["speedup_vs_plain"] = round(leg["plain_ms"] / (leg["ms"] / S), 3)
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.sweeps_only:
        return sweeps_only(args)
    if args.ranker_eval:
        return ranker_eval(args)
    if args.batch:
        return batch_bench(args)
    if args.hmat:
        return hmat_bench(args)
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world)
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    peaks, peak_kind = load_peaks()
    N, S = r["N"], args.steps
    mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
    fp64_peak = 152 * 2 * 2 * mhz * 1e6 / 1e12

    def hp(ms, s):
        gbs = 2.0 * N * s / (ms / 1e3) / 1e9
        return {"ms": round(ms, 3), "gbs": round(gbs, 3),
                "hbm_frac": round(gbs / peaks["hbm_gbs"], 6),
                "tflops": round(flops / (ms / 1e3) / 1e12, 4)}

    if args.adapt_only:
        print(json.dumps({"adapt_only": args.workload,
                          "iters_per_s": round(S / (r["head"]["ms"] / 1e3), 5),
                          "n_evals": [rec["n_evals"] for rec in r["head"]["timed"]],
                          "support": [rec["support"] for rec in r["head"]["timed"]],
                          "sigma_support": [rec["sigma_support"] for rec in r["head"]["timed"]],
                          "t_total": [round(rec["t_total"], 4) for rec in r["head"]["timed"]],
                          "launches": r["head"]["launches"],
                          "e2e_iters_per_s": round(S / (r["head"]["ms_e2e"] / 1e3), 5),
                          "kernel_breakdown": breakdown(r["head"]["prof"], r["head"]["ms"]),
                          "roofline": step_roofline(r["head"]["prof"], peaks, peak_kind, fp32_peak)}),
              flush=True)
        return
    head, dense = r["head"], r["dense"]
    flops = 2.0 * r["conn"] * N
    cflops = 2.0 * r["cpl_units"] * N      # the coupling kernel's share of the connections
    # tensor-core work of the coupling's phase A: 64 slots x 256 padded types x
    # 3 split products per (alpha string, beta string), 2 flops per MAC
    tc_flops = 2.0 * 3 * 64 * 256 * r["n_alpha_str"] * r["n_beta_str"]
    tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25
    out = {
        "metric": METRIC,
        "value": round(job_throughput(world, S, head["ms"]), 6),
        "unit": "ADAPT iters/s",
        "n_gpus": world,
        "steps": S,
        "warmup": args.warmup,
        "ms_per_step": round(head["ms"] / S, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 bulk + f64 reductions",
        "data": "synthetic (seeded integrals shaped like the H16 STO-3G chain; no PySCF)",
        "config": {"workload": f"{args.workload}: {r['n']} orbitals, {r['na']}a+{r['nb']}b, "
                               f"{N} determinants, seed {r['seed']}",
                   "mode": (f"mixed precision + learned ranker (top-{args.top_m} screened exactly, "
                            f"full-screen refresh every {REFRESH}th ranked iteration); psi kept as a "
                            "sparse vector while its support fits N/256 (float) or N/64 (double), "
                            "exact sparse screen while pool x support <= 5e9"),
                   "pool_ops": r["K"], "replicas": world,
                   "ansatz_len_timed": [rec["iter"] + 1 for rec in head["timed"]],
                   "l2": "inputs larger than L2 (state vector 0.66 GB FP32 / 1.33 GB FP64)",
                   "step": "one ADAPT iteration: screen + select + BFGS re-optimisation"},
        "mixed_ranker": leg_summary(head, S),
        "dense_path": leg_summary(dense, S),
        "hpsi": {"f64": hp(r["hpsi_ms_f64"], 8), "f32": hp(r["hpsi_ms_f32"], 4),
                 "algorithmic_bytes": "2 * N_det * sizeof(amplitude)",
                 "connections_per_det": r["conn"], "state": "dense seeded random state"},
        "screen_ms": {"f64": round(r["screen_ms_f64"], 3), "f32": round(r["screen_ms_f32"], 3)},
        "roofline": step_roofline(head["prof"], peaks, peak_kind, fp32_peak),
        "kernel_breakdown": breakdown(head["prof"], head["ms"]),
        "dense_hpsi_roofline": {
            "bound": "tensor", "kernel": "alpha-beta coupling of dense float H|psi>: k_cpl_tc "
            "(tcgen05 TF32, split hi/lo operands) + k_cpl_gather",
            "achieved": round(tc_flops / (r["cpl_ms_f32"] / 1e3) / 1e12, 3),
            "peak": round(tf32_peak, 1), "unit": "TFLOP/s",
            "frac": round(tc_flops / (r["cpl_ms_f32"] / 1e3) / 1e12 / tf32_peak, 4),
            "traffic": TRAFFIC_F32,
            "traffic_k_cpl_tc_per_launch": round(TRAFFIC_CPL_TC),
            "ms_per_launch": round(r["cpl_ms_f32"], 3),
            "work": (f"3 x 64 x 256 TF32 MACs per (alpha string, column) over "
                     f"{r['n_alpha_str']} x {r['n_beta_str']} (padded types, three split products)"),
            "peak_kind": ("measured bf16 burst x 1.1/2.25 (nominal TF32/BF16 dense ratio); "
                          "2047 TF32 MAC/clk/SM measured by a microbenchmark at M=128"),
            "useful_fp32_tflops": round(cflops / (r["cpl_ms_f32"] / 1e3) / 1e12, 3),
            "f64": {"kernel": "k_coupling<double>",
                    "achieved": round(cflops / (r["cpl_ms_f64"] / 1e3) / 1e12, 4),
                    "peak": round(fp64_peak, 3),
                    "frac": round(cflops / (r["cpl_ms_f64"] / 1e3) / 1e12 / fp64_peak, 4),
                    "ms_per_launch": round(r["cpl_ms_f64"], 3),
                    "peak_kind": f"derived FP64 rate: 152 SMs x 2 FMA/clk x {mhz} MHz"},
            "whole_hpsi_frac": {"f64": round(flops / (r["hpsi_ms_f64"] / 1e3) / 1e12 /
                                             fp64_peak, 4),
                                "f32": round(flops / (r["hpsi_ms_f32"] / 1e3) / 1e12 /
                                             fp32_peak, 4)}},
        "e2e": {"value": round(job_throughput(world, S, head["ms_e2e"]), 6),
                "unit": "ADAPT iters/s",
                "h2d_bytes_per_step": int(head["io"][0]), "d2h_bytes_per_step": int(head["io"][1])},
        "gpu_launches": int(head["launches"]),
        "clocks": head["clocks"],
        "build_s": round(r["t_build"], 2),
    }
    if not args.no_cpu_baseline and world == 1:
        n_evals = dense["plain_rec"]["n_evals"] if "plain_rec" in dense else 10
        jlen = head["ansatz_len"]
        n, na, nb, seed = r["n"], r["na"], r["nb"], r["seed"]
        del r, head, dense
        tot, thr, sample = oracle_iteration_estimate(n, na, nb, seed, args.cpu_budget, jlen,
                                                     n_evals)
        out["cpu_baseline"] = {"value": 1.0 / tot, "unit": "ADAPT iters/s", "cores": thr,
                               "kind": "oracle", "sample": sample}
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


def run_reference(args, rank, world):
    """The oracle as it stands, timed on the host cores: every step is a
    bounded sample of the same workload extrapolated to one plain ADAPT
    iteration (10 evaluations at ansatz length warmup + steps)."""
    if rank != 0:
        return
    import oracle
    n, na, nb, seed = synth.workload(args.workload)
    h1, h2, ec = synth.integrals(n, seed)
    n_det = oracle.System(h1, h2, ec, n, na, nb).n_det
    state = synth.random_state(n_det, 99)
    per = max(2.0, min(args.cpu_budget, 150.0 / max(1, args.steps + args.warmup)))
    jlen = args.warmup + args.steps
    for _ in range(args.warmup):
        oracle_iteration_estimate(n, na, nb, seed, per, jlen, 10, state)
    tots = []
    for _ in range(args.steps):
        tot, thr, sample = oracle_iteration_estimate(n, na, nb, seed, per, jlen, 10, state)
        tots.append(tot)
    t = sum(tots)
    v = args.steps / t
    out = {"metric": METRIC, "value": v, "unit": "ADAPT iters/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"{args.workload}: {n} orbitals, {na}a+{nb}b, "
                                  f"{n_det} determinants, seed {seed}",
                      "mode": "FP64 CPU oracle, plain full screen"},
           "cpu_baseline": {"value": v, "unit": "ADAPT iters/s", "cores": thr,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "ADAPT iters/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
