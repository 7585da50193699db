"""Benchmark of the DMRG sweep engine on one GB300 (or N replicas).

Workload: CAS(16e,16o), S_z = 0, synthetic integrals (gbd_synth, seed 3,
48 Cholesky vectors), bond dimension M = 512.  One "step" is one full
two-site sweep (left-to-right and back, 30 two-site steps: H_eff diagonal,
Davidson with sigma builds, decimation, environment updates), with the state
resident on the device when the timed region starts.  Default precision:
the reduced-precision tiers (BF16 tier 1, skipped in warm sweeps; TF32x3
tier 2 with split-K FP64 sums; FP64 everywhere else); --precision fp64 runs
the plain FP64 path.

value    = algorithmic sigma-build flops of the timed sweeps / wall time of
           the timed sweeps (TFLOP/s, whole job: everything in the sweep
           counts in the denominator); sweep_time_s = wall time per sweep.
fp64_gpu_sweep_s = one further sweep of the FP64 path from the same state.
per_step_energy_error_vs_fp64 = the same two-site problems solved by FP64
           Davidson and by the mixed tiers (FP64 Rayleigh quotients).
e2e      = the same metric through gbd_solve (host integrals in, energies
           out; initial state, sweeps and final energy inside the timed call).
roofline = tc_gemm_kernel (FP64 path: gemm_f64_kernel), CUDA events around
           its launches on the engine stream; tensor and HBM views.
cpu_baseline = the CPU oracle on a bounded sample: one sigma build at the
           central bond pair (7,8) of the same problem (initial MPS at M=512).

Multi-GPU: independent replicas (one problem per rank, seed 3 + rank), no
collective on the data path; value sums the ranks' flops over the max time.
Other modes: --workload batched64 (64 independent active spaces through
gbd_solve_batched), --sigma-probe P (profiling driver, no bench line),
--states K (excited states by penalty deflation, no bench line),
--impl reference (the oracle, timed on the host cores).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from gbd_synth import WORKLOADS, make_integrals  # noqa: E402

PREC = {"fp64": 0, "tf32": 1, "bf16": 2}
PRECOND = {"diag": 0, "olsen": 2, "pcg": 3}
ENV_PREC = {"fp64": 0, "tf32x3": 3, "bf16x3": 4}
METRIC = "sigma-build TFLOP/s; sweep time at CAS(16,16) M=512 vs FP64 GPU at \u22641e-6 Ha"
# DRAM bytes (read + write, ncu) per algorithmic byte of tc_gemm_kernel, from
# one capture of `bench.py --sigma-probe 3 --probe-warm-sweeps 3` (TF32x3
# sigma at the central bond of the CAS(16,16) M=512 state after three mixed
# sweeps: stage A 1051.7 + 928.4 MB, stage B 2761.4 + 160.1 MB, for 2359.8 MB
# of algorithmic bytes).  The launches of a sweep move the same kinds of
# panels, so traffic is reported as this ratio times their algorithmic bytes
# per launch.
TC_DRAM_PER_ALG_BYTE = (1052.990976e6 + 930.154752e6 + 1648.479232e6 + 86.380032e6) / 2359843136.0
DTYPE = {"fp64": "f64", "tf32": "tf32/f32-acc", "bf16": "bf16/f32-acc"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def schedule(nsweeps, tol):
    return [tol] * nsweeps


def run_ours(args, rank, world):
    from paper_2609_09990_gb300 import gbdmrg as G

    wl = WORKLOADS[args.workload]
    n, ne, nq, M = wl["n_orb"], wl["n_elec"], wl["n_chol"], wl["M"]
    seed = wl["seed"] + rank
    h, chol = make_integrals(n, nq, seed)
    prec = PREC[args.precision]
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(dev)
    ctx = G.Context(dev)
    ctx.set_accurate_tier(3 if args.tier2 == "tf32x3" else 4)
    ctx.set_tier_stop(args.floor_mult, args.hard_stag)
    ctx.set_env_precision(ENV_PREC[args.env_prec])
    if args.tc_sout_min is not None:
        ctx.set_tc_sout_split(args.tc_sout_min)
    nsw = args.warmup + args.steps
    ctx.setup(h, chol, ne, 0, [M] * (nsw + 1), schedule(nsw + 1, args.tol), seed=seed, precision=prec,
              fp64_refine=args.refine)
    if args.precond != "diag":
        ctx.set_preconditioner(PRECOND[args.precond])
    ctx.init_state()
    for s in range(args.warmup):
        ctx.run_sweep(s)
    st0 = ctx.stats()
    dist_barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(dev)
    clk.start()
    t0 = time.perf_counter()
    energies, sweep_max_r = [], []
    for s in range(args.warmup, nsw):
        energies.append(ctx.run_sweep(s))
        sweep_max_r.append(ctx.stats()["sweep_max_residual"])   # host counters only
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    dist_barrier(world)
    clocks = clk.stop()
    st1 = ctx.stats()
    dt = t1 - t0
    keys = ["sigma_ms", "tc_ms", "tc_gemm_ms", "tc_build_ms", "env_ms", "enlarge_ms", "enlarge_host_ms",
            "enlarge_dev_ms", "diag_ms",
            "davidson_ms", "truncate_ms", "truncate_rho_ms", "truncate_eig_ms", "env_wall_ms", "step_ms",
            "h2d_wait_ms"]
    breakdown = {k: (st1[k] - st0[k]) / args.steps for k in keys}
    breakdown["sigma_builds"] = (st1["n_sigma"] - st0["n_sigma"]) / args.steps
    breakdown["tc_sigma_builds"] = (st1["n_sigma_tc"] - st0["n_sigma_tc"]) / args.steps
    breakdown["env_gflop"] = (st1["env_flops"] - st0["env_flops"]) / args.steps / 1e9
    breakdown["enlarge_GB"] = (st1["enlarge_bytes"] - st0["enlarge_bytes"]) / args.steps / 1e9
    breakdown["tc_build_phase_ms"] = {
        nm: (st1["tc_build_phase_ms"][i] - st0["tc_build_phase_ms"][i]) / args.steps
        for i, nm in enumerate(["layout_groups", "panels", "tiles", "upload", "maps"])}
    breakdown["tc_gemm_ms_by_stage"] = {
        nm: (st1["tc_gemm_ms_by_stage"][i] - st0["tc_gemm_ms_by_stage"][i]) / args.steps
        for i, nm in enumerate(["A", "B"])}
    breakdown["tc_bytes_by_stage_GB"] = {
        nm: (st1["tc_stage_alg_bytes"][i] - st0["tc_stage_alg_bytes"][i]) / args.steps / 1e9
        for i, nm in enumerate(["A", "B"])}
    breakdown["inner_pcg_matvecs"] = (st1["inner_matvecs"] - st0["inner_matvecs"]) / args.steps
    nsol = st1["n_solves"] - st0["n_solves"]
    breakdown["davidson_final_residual"] = {
        "max_per_sweep": sweep_max_r, "max": max(sweep_max_r),
        "mean": (st1["sum_final_residual"] - st0["sum_final_residual"]) / max(nsol, 1),
        "solves": nsol, "fraction_above_tol": (st1["n_solves_above_tol"] - st0["n_solves_above_tol"]) / max(nsol, 1)}
    breakdown["davidson_iterations_by_tier"] = {
        t: (st1["tier_iterations"][i] - st0["tier_iterations"][i]) / args.steps
        for i, t in enumerate(["bf16_or_tf32", "tf32x3", "fp64"])}
    flops = st1["sigma_flops"] - st0["sigma_flops"]
    sig_ms = st1["sigma_ms"] - st0["sigma_ms"]
    tc_ms = st1["tc_ms"] - st0["tc_ms"]
    tc_flops = st1["tc_flops"] - st0["tc_flops"]
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    e_final = ctx.final_energy()
    fp64 = None
    if prec != 0 and args.compare_fp64:
        # The accuracy gate, like for like: from the warmed state S (saved on
        # the device), one more sweep in the mixed tiers, then, from S again,
        # one sweep of the plain FP64 path at the same tolerance, and one at
        # the residual the mixed sweep actually reached (its tiers stop at
        # their floor when that lies above the tolerance).
        ctx.save_state()

        def one_sweep(precision, tol_sweep):
            ctx.restore_state()
            ctx.set_precision(precision, args.refine if precision else 0)
            ctx.set_sweep_schedule(nsw, M, tol_sweep)
            sa = ctx.stats()
            torch.cuda.synchronize()
            ta = time.perf_counter()
            ctx.run_sweep(nsw)
            torch.cuda.synchronize()
            dt_s = time.perf_counter() - ta
            sb = ctx.stats()
            ns = sb["n_solves"] - sa["n_solves"]
            return dict(sweep_s=dt_s, final_energy=ctx.final_energy(), tol=tol_sweep,
                        max_final_residual=sb["sweep_max_residual"],
                        mean_final_residual=(sb["sum_final_residual"] - sa["sum_final_residual"]) / max(ns, 1),
                        fraction_above_tol=(sb["n_solves_above_tol"] - sa["n_solves_above_tol"]) / max(ns, 1),
                        davidson_iterations=sb["davidson_iterations"] - sa["davidson_iterations"],
                        sigma_builds=sb["n_sigma"] - sa["n_sigma"])
        mixed = one_sweep(prec, args.tol)
        full = one_sweep(0, args.tol)
        floor = one_sweep(0, max(args.tol, mixed["max_final_residual"]))
        ctx.restore_state()
        ctx.set_precision(prec, args.refine)
        fp64 = dict(mixed=mixed, fp64=full, fp64_at_mixed_residual=floor, e_start=e_final)
    # per-step effect of the matvec precision: at a few bonds of a further
    # left-to-right pass, the FP64 Rayleigh quotient of the mixed-precision
    # Davidson solution against the FP64 Davidson solution on the same input
    probes = []
    if prec != 0 and args.probes > 0:
        if fp64:
            ctx.restore_state()
        ks = [int(round(1 + i * (n - 4) / max(args.probes - 1, 1))) for i in range(args.probes)]
        for k in range(max(ks) + 1):
            if k in ks:
                _, e_ref, r_ref = ctx.probe_step(k, 0, 0, 1e-9)
                _, e_mix, r_mix = ctx.probe_step(k, prec, args.refine, args.tol)
                probes.append({"bond": k, "dE": e_mix - e_ref, "r_fp64_solve": r_ref, "r_mixed_solve": r_mix})
            ctx.run_step(k, 0, M, args.tol)
    rdm_times = None
    if args.rdms:
        # RDMs of the current state, each timed on its own (device work
        # synchronised by the call): 1-/2-RDM and orbital entropies with
        # mutual information, contracted through the MPS; where the
        # determinant expansion fits, the same RDMs by that route (time and
        # largest difference) and the 3-RDM where its 2 n^2
        # determinant-length vectors fit
        from math import comb
        rdm_times = {}
        e_final = ctx.final_energy()
        t = time.perf_counter()
        g1, g2 = ctx.rdms(n)
        rdm_times["rdm12_s"] = time.perf_counter() - t
        rdm_times["rdm12_env_gb"] = ctx.stats()["rdm_env_bytes"] / 1e9
        eri = np.einsum("Qpq,Qrs->pqrs", chol, chol)
        e_rdm = float(np.einsum("pq,pq", h, g1) + 0.5 * np.einsum("pqrs,pqrs", eri, g2))
        rdm_times["energy_from_rdms_minus_energy"] = e_rdm - e_final
        t = time.perf_counter()
        s1, mi = ctx.orbital_entropies(n)
        rdm_times["orbital_entropies_s"] = time.perf_counter() - t
        ndet = comb(n, ne // 2) ** 2
        if ndet <= 4e8:
            t = time.perf_counter()
            c1, c2 = ctx.rdms_ci(n)
            rdm_times["rdm12_determinant_route_s"] = time.perf_counter() - t
            rdm_times["routes_max_abs_diff"] = float(max(np.abs(g1 - c1).max(), np.abs(g2 - c2).max()))
        if 2 * n * n * ndet * 8 <= 64e9:
            t = time.perf_counter()
            ctx.rdm3(n)
            rdm_times["rdm3_s"] = time.perf_counter() - t
        rdm_times["determinants"] = ndet
        rdm_times["trace_gamma"] = float(np.trace(g1))
        rdm_times["max_mutual_information"] = float(mi.max())
    ctx.close()
    # end to end through gbd_solve: host integrals in, energies out
    e2e = None
    if not args.no_e2e:
        ctx = G.Context(dev)
        ctx.set_accurate_tier(3 if args.tier2 == "tf32x3" else 4)
        ctx.set_tier_stop(args.floor_mult, args.hard_stag)
        ctx.set_env_precision(ENV_PREC[args.env_prec])
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        r = ctx.solve(h, chol, ne, 0, [M] * args.steps, schedule(args.steps, args.tol), seed=seed,
                      precision=prec, fp64_refine=args.refine)
        t3 = time.perf_counter()
        se = ctx.stats()
        ctx.close()
        e2e = dict(flops=se["sigma_flops"], time=t3 - t2, h2d=int(h.nbytes + chol.nbytes),
                   d2h=int(8 * (1 + args.steps)), energy=r["energy"])
    tc = {k: [b - a for a, b in zip(st0[k], st1[k])] for k in ("tc_flops_by_type", "tc_gemm_ms_by_type")}
    tc["tc_bytes"] = st1["tc_bytes"] - st0["tc_bytes"]
    tc["tc_gemm_ms"] = st1["tc_gemm_ms"] - st0["tc_gemm_ms"]
    return dict(time=dt, flops=flops, sigma_ms=sig_ms, launches=launches, clocks=clocks,
                energies=energies, e2e=e2e, n=n, M=M, st=st1, tc_ms=tc_ms, tc_flops=tc_flops,
                e_final=e_final, fp64=fp64, breakdown=breakdown, tc=tc, probes=probes, rdm_times=rdm_times)


def batched_problems(args):
    """64 independent active spaces: orbital counts U{8..14} and M from
    {128, 256, 512} (seed-1000 stream), half filling, S_z = 0 (1/2 for odd
    electron counts), integrals of problem s from seed s with 3 n Cholesky
    vectors; `batch_sweeps` sweeps each.  The same set on every rank."""
    from gbd_synth import batched_problem_sizes
    out = []
    for s, (n, M) in enumerate(batched_problem_sizes(64)):
        h, chol = make_integrals(n, 3 * n, s)
        # half filling; odd electron counts take S_z = 1/2
        out.append((h, chol, n, n % 2, [M] * args.batch_sweeps, [args.tol] * args.batch_sweeps,
                    {"seed": s, "precision": PREC[args.precision], "fp64_refine": args.refine}))
    return out


def partition_problems(problems, world):
    """Owner rank of every problem: longest-processing-time-first greedy on
    the library's cost estimate (n_orb x M^3 x sweeps), the same on every
    rank without communication."""
    from paper_2609_09990_gb300 import gbdmrg as G
    owner, load = G.host_partition(G.host_batch_costs(problems), world)
    return owner, load


def gather_results(mine, n, world):
    """Rank 0 gets the results of all n problems in problem order from the
    (index, result) pairs each rank solved; the other ranks get None."""
    if world <= 1:
        out = [None] * n
        for i, r in mine:
            out[i] = r
        return out
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    if dist.get_rank() != 0:
        return None
    out = [None] * n
    for part in parts:
        for i, r in part:
            if out[i] is not None:
                raise RuntimeError(f"problem {i} solved by two ranks")
            out[i] = r
    if any(r is None for r in out):
        raise RuntimeError("a problem was solved by no rank")
    return out


def run_batched(args, rank, world):
    """The 64 problems split over the ranks (partition_problems); one step =
    one gbd_solve_batched call per rank over its share (initial state,
    `batch_sweeps` sweeps and final energy of each problem)."""
    from paper_2609_09990_gb300 import gbdmrg as G
    import torch
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    allp = batched_problems(args)
    owner, load = partition_problems(allp, world)
    idx = [i for i in range(len(allp)) if owner[i] == rank]
    probs = [allp[i] for i in idx]
    ctx = G.Context(dev)
    ctx.set_graphs(not args.no_graphs)
    for _ in range(args.warmup):
        rc, _ = ctx.solve_batched(probs, workers=args.workers)
    dist_barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(dev)
    clk.start()
    t0 = time.perf_counter()
    flops, launches, graphs = 0.0, 0, 0
    for _ in range(args.steps):
        rc, res = ctx.solve_batched(probs, workers=args.workers)
        st = ctx.batch_stats()
        flops += st["sigma_flops"]
        launches += st["kernel_launches"]
        graphs += st["graph_launches"]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    dist_barrier(world)
    clocks = clk.stop()
    ctx.close()
    energies = gather_results([(i, r["energy"]) for i, r in zip(idx, res)], len(allp), world)
    return dict(time=t1 - t0, flops=flops, launches=launches, graph_launches=graphs, clocks=clocks,
                energies=energies, n_problems=len(allp), rank_problems=len(idx),
                load_imbalance=float(load.max() / load.mean()) if load.size else 1.0)


def sigma_probe(prec, orders=(1,), warm_sweeps=0, davidson=False, order_a=0):
    """Profiling driver for the tensor-core sigma: CAS(16,16) M=512, initial
    state (or, with warm_sweeps > 0, the state after that many sweeps in the
    mixed tiers), steps up to the central bond (7,8), then three sigma builds
    there with operand type `prec` (1 TF32, 2 BF16, 3 TF32x3).  The first
    build of a new shape runs the tile-shape autotuner (3 candidate plans x 3
    timed runs = 18 tc_gemm_kernel launches), so on the initial state
    `ncu -k regex:tc_gemm_kernel -s 18 -c 2` captures stage A and stage B of
    the tuned plan.  On a warm state one untimed build comes first and the
    CUDA profiler is started right before the timed builds, so
    `ncu --profile-from-start off -k regex:tc_gemm_kernel -c 2` captures the
    first of them.  With several stage-B tile orders, each is timed on three
    more builds.  davidson=True: instead of the sigma builds, one Davidson
    solve of the central problem in the mixed tiers (gbd_probe_step), for
    profiling the vector kernels at the size where the sweep spends its
    time."""
    from paper_2609_09990_gb300 import gbdmrg as G
    import torch
    wl = WORKLOADS["cas16_m512"]
    n, ne, nq, M, seed = wl["n_orb"], wl["n_elec"], wl["n_chol"], wl["M"], wl["seed"]
    h, chol = make_integrals(n, nq, seed)
    ctx = G.Context(0)
    ctx.setup(h, chol, ne, 0, [M] * max(warm_sweeps, 1), [1e-6] * max(warm_sweeps, 1), seed=seed,
              precision=PREC["bf16"] if warm_sweeps else 0, fp64_refine=0)
    ctx.init_state()
    for s in range(warm_sweeps):
        ctx.run_sweep(s)
    k = n // 2 - 1
    for j in range(k):
        ctx.run_step(j, 0, M, 1e-3 if not warm_sweeps else 1e-6)
    x = np.random.default_rng(0).standard_normal(ctx.two_site_size(k))
    if warm_sweeps:
        ctx.apply_heff_prec(k, x, prec)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
    if davidson:
        # one Davidson solve of the central two-site problem in the mixed
        # tiers (plan build, tensor-core sigma builds, vector kernels)
        s0 = ctx.stats()
        t = time.perf_counter()
        theta, e64, r64 = ctx.probe_step(k, PREC["bf16"], 0, 1e-6)
        s1 = ctx.stats()
        print(json.dumps({"davidson_probe": True, "warm_sweeps": warm_sweeps, "bond": k, "psi_len": int(x.size),
                          "seconds": time.perf_counter() - t, "iterations": s1["davidson_iterations"] -
                          s0["davidson_iterations"], "sigma_builds": s1["n_sigma"] - s0["n_sigma"],
                          "final_residual_fp64": r64, "kernel_launches": s1["kernel_launches"] -
                          s0["kernel_launches"]}))
        ctx.close()
        return
    ref = None
    ctx.set_tc_order_a(order_a)
    for order in orders:
        ctx.set_tc_order(order)
        s0 = ctx.stats()
        each = []
        for _ in range(3):
            sa = ctx.stats()["tc_gemm_ms"]
            y = ctx.apply_heff_prec(k, x, prec)
            each.append(ctx.stats()["tc_gemm_ms"] - sa)
        s1 = ctx.stats()
        ref = y if ref is None else ref
        nb = s1["n_sigma_tc"] - s0["n_sigma_tc"]
        per = lambda key: (s1[key] - s0[key]) / nb
        perv = lambda key: [(a - b) / nb for a, b in zip(s1[key], s0[key])]
        print(json.dumps({"sigma_probe": prec, "warm_sweeps": warm_sweeps, "stage_a_order": order_a,
                          "stage_b_order": order, "bond": k,
                          "psi_len": int(x.size),
                          "builds": nb, "identical_to_first_order": bool(np.array_equal(y, ref)),
                          "tc_gemm_ms_per_build": per("tc_gemm_ms"), "tc_gemm_ms_each": each,
                          "tc_ms_per_build": per("tc_ms"),
                          "alg_bytes_per_build": per("tc_bytes"), "alg_flops_per_build": per("tc_flops"),
                          "stage_alg_bytes": perv("tc_stage_alg_bytes"),
                          "stage_box_bytes": perv("tc_stage_box_bytes"),
                          "stage_dense_bytes": perv("tc_stage_dense_bytes"),
                          "stage_ms": perv("tc_gemm_ms_by_stage")}))
    ctx.close()


def rdm_probe(workload, warm_sweeps):
    """Profiling driver for the RDM pass: `workload` after warm_sweeps sweeps
    in the mixed tiers; the CUDA profiler is started right before gbd_rdms
    (1-/2-RDMs contracted through the MPS), so
    `ncu --profile-from-start off` captures that pass alone.  Prints its
    time (CUDA-synchronised by the call) and peak environment bytes."""
    from paper_2609_09990_gb300 import gbdmrg as G
    import torch
    wl = WORKLOADS[workload]
    n, ne, nq, M, seed = wl["n_orb"], wl["n_elec"], wl["n_chol"], wl["M"], wl["seed"]
    h, chol = make_integrals(n, nq, seed)
    ctx = G.Context(0)
    ctx.setup(h, chol, ne, 0, [M] * warm_sweeps, [1e-6] * warm_sweeps, seed=seed, precision=PREC["bf16"],
              fp64_refine=0)
    ctx.init_state()
    for s in range(warm_sweeps):
        ctx.run_sweep(s)
    ctx.final_energy()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    s0 = ctx.stats()
    t = time.perf_counter()
    g1, g2 = ctx.rdms(n)
    dt = time.perf_counter() - t
    torch.cuda.profiler.stop()
    s1 = ctx.stats()
    print(json.dumps({"rdm_probe": workload, "warm_sweeps": warm_sweeps, "seconds": dt,
                      "env_gb": s1["rdm_env_bytes"] / 1e9, "launches": s1["kernel_launches"] - s0["kernel_launches"],
                      "trace_gamma": float(np.trace(g1))}))
    ctx.close()


def precond_probe(n):
    """Profiling driver for the fused learned-preconditioner kernel: n
    elements of (r, diag) and a seeded random network, one application
    (features, MLP with FP16 weights, Jacobi step) through gbd_mlp_precond."""
    from paper_2609_09990_gb300 import gbdmrg as G
    rng = np.random.default_rng(4)
    nparam = 128 * 8 + 128 + 128 + 1
    p = np.concatenate([rng.normal(0, 0.3, 128 * 8), rng.normal(0, 0.1, 128), rng.normal(0, 0.1, 128), [0.05]])
    assert p.size == nparam
    r = rng.normal(size=n) * 1e-3
    d = rng.normal(size=n) * 3 - 10
    ctx = G.Context(0)
    ctx.set_precond_weights(p.astype(np.float32))
    t = ctx.mlp_precond(r, d, -10.5, 3.0)
    ctx.close()
    print(json.dumps({"precond_probe": n, "finite": bool(np.all(np.isfinite(t)))}))


def precond_ab(args):
    """Learned against diagonal Davidson preconditioner at --workload
    (default CAS(20,20) M=1024): the network is trained on the device on
    residuals recorded from CAS(6,6) (4 sweeps), CAS(12,12) (2 sweeps) and
    CAS(16,16) (1 sweep); the workload then runs --warmup mixed sweeps, and at
    five bonds of a further left-to-right pass gbd_probe_step solves the same
    two-site problem to ||r|| < 1e-8 with each preconditioner, in the FP64
    tier and in the mixed tiers with FP64 refinement.  One JSON line with
    Davidson iterations and times; no bench line."""
    from paper_2609_09990_gb300 import gbdmrg as G
    import torch
    ctx = G.Context(0)
    train = []
    for name, nsw in (("cas6_m64", 4), ("cas12_m256", 2), ("cas16_m512", 1)):
        w = WORKLOADS[name]
        h, chol = make_integrals(w["n_orb"], w["n_chol"], w["seed"])
        train.append((h, chol, w["n_elec"], 0, [w["M"]] * nsw, [1e-8] * nsw, {"seed": w["seed"]}))
    t = time.perf_counter()
    loss = ctx.train_precond(train, epochs=400, lr=3e-3)
    train_s = time.perf_counter() - t
    _, _, samples = ctx.davidson_counts()
    wl = WORKLOADS[args.workload]
    n, ne, nq, M, seed = wl["n_orb"], wl["n_elec"], wl["n_chol"], wl["M"], wl["seed"]
    h, chol = make_integrals(n, nq, seed)
    nsw = max(args.warmup, 1)
    ctx.setup(h, chol, ne, 0, [M] * nsw, [1e-6] * nsw, seed=seed, precision=PREC["bf16"], fp64_refine=0)
    ctx.init_state()
    for sweep in range(nsw):
        ctx.run_sweep(sweep)
    ks = [int(round(1 + i * (n - 4) / 4)) for i in range(5)]
    rows = []
    for k in range(max(ks) + 1):
        if k in ks:
            for tier, prec, refine in (("fp64", 0, 0), ("mixed+fp64_refine", PREC["bf16"], 200)):
                for pc in (0, 1):
                    ctx.set_preconditioner(pc)
                    it0 = ctx.davidson_counts()[0]
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    _, e64, r64 = ctx.probe_step(k, prec, refine, 1e-8)
                    dt = time.perf_counter() - t
                    rows.append({"bond": k, "tier": tier, "preconditioner": "learned" if pc else "diagonal",
                                 "iterations": ctx.davidson_counts()[0] - it0, "seconds": dt, "energy": e64,
                                 "final_residual_fp64": r64})
            ctx.set_preconditioner(0)
        ctx.run_step(k, 0, M, 1e-6)
    ctx.close()
    summary = {}
    for tier in ("fp64", "mixed+fp64_refine"):
        for pc in ("diagonal", "learned"):
            sel = [r for r in rows if r["tier"] == tier and r["preconditioner"] == pc]
            summary[f"{tier}/{pc}"] = {"iterations": sum(r["iterations"] for r in sel),
                                       "seconds": sum(r["seconds"] for r in sel)}
    de = max(abs(a["energy"] - b["energy"]) for a in rows for b in rows
             if a["bond"] == b["bond"] and a["tier"] == b["tier"] and a is not b)
    print(json.dumps({"precond_ab": args.workload, "train_s": train_s, "train_loss": loss, "train_samples": samples,
                      "warm_sweeps": nsw, "summary": summary, "max_energy_difference_same_problem_Ha": de,
                      "probes": rows}))


def states_run(args):
    """Excited states by penalty deflation on a workload (gbd_solve_states):
    the lowest `--states` roots of any spin (no <S^2> guard), each from its
    own seeded initial MPS, n_sweeps of the workload at --tol, mixed-precision
    tiers; every root's <S^2> is reported.  One JSON line, no bench line."""
    from paper_2609_09990_gb300 import gbdmrg as G
    wl = WORKLOADS[args.workload]
    n, ne, nq, M, seed, nsw = wl["n_orb"], wl["n_elec"], wl["n_chol"], wl["M"], wl["seed"], wl["n_sweeps"]
    h, chol = make_integrals(n, nq, seed)
    ctx = G.Context(0)
    t0 = time.perf_counter()
    rc, res = ctx.solve_states(h, chol, ne, 0, [M] * nsw, [args.tol] * nsw, args.states, penalty=args.penalty,
                               target_s2=-1.0, max_extra=0, seed=seed, precision=PREC[args.precision],
                               fp64_refine=args.refine, check=False)
    dt = time.perf_counter() - t0
    st = ctx.stats()
    ctx.close()
    print(json.dumps({"states": args.states, "workload": args.workload, "rc": int(rc), "found": len(res),
                      "seconds": dt, "penalty_Ha": args.penalty, "sigma_builds": int(st["n_sigma"]),
                      "roots": [{"energy": r["energy"], "s2": r["s2"], "last_sweep_ritz": float(r["sweep_energies"][-1])}
                                for r in res],
                      "excitation_energies_Ha": [r["energy"] - res[0]["energy"] for r in res]}))


def reduce_over_ranks(tmax, work, world, device="cuda"):
    """Whole-job numbers of a replicas run: the slowest rank's time (MAX) and
    the summed work (SUM) over the process group; unchanged for one rank."""
    if world <= 1:
        return tmax, work
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(tmax)], device=device, dtype=torch.float64)
    f = torch.tensor([float(work)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    return float(t.item()), float(f.item())


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_sample(n_sigma=1, want_flops=True, warmup=0):
    """CPU oracle: sigma builds at the central bond pair (7,8) of CAS(16,16)
    on the seeded initial MPS (M = 512).  Environments are built by the
    oracle with its MPO switch at bond 3 (untimed); the timed part is the
    sigma builds.  Flops per build: the GPU engine's algorithmic count for
    the same sigma on the same state (the oracle's MPS is installed in the
    library and one H_eff application is made), which also checks parity."""
    from oracle import dmrg
    wl = WORKLOADS["cas16_m512"]
    n, ne, nq, M, seed = wl["n_orb"], wl["n_elec"], wl["n_chol"], wl["M"], wl["seed"]
    h, chol = make_integrals(n, nq, seed)
    k = n // 2 - 1
    ts = time.perf_counter()
    d = dmrg.DMRG(h, chol, ne, 0, M, seed=seed, k_switch=3, renv_down_to=k + 2)
    d.move_center(k)
    setup_s = time.perf_counter() - ts
    psi = dmrg.two_site_psi(d.sites[k], d.sites[k + 1], d.dims[k + 1])
    L, W1, W2, R = d.heff_parts(k)
    for _ in range(warmup):
        dmrg.apply_heff(L, W1, W2, R, psi, d.mpo, k)
    times = []
    sig = None
    for _ in range(n_sigma):
        t = time.perf_counter()
        sig = dmrg.apply_heff(L, W1, W2, R, psi, d.mpo, k)
        times.append(time.perf_counter() - t)
    keys = dmrg.psi_keys(d.dims[k], d.dims[k + 2])
    x = dmrg.flatten(psi, keys, d.dims[k], d.dims[k + 2])
    y_ref = dmrg.flatten(sig, keys, d.dims[k], d.dims[k + 2])
    flops, rel = None, None
    if want_flops:
        from paper_2609_09990_gb300 import gbdmrg as G
        ctx = G.Context(int(os.environ.get("LOCAL_RANK", "0")))
        ctx.setup(h, chol, ne, 0, [M], [1e-8], seed=seed)
        ns, tr, data = dmrg.canonical_blocks(d)
        ctx.set_mps(ns, tr, data, k)
        f0 = ctx.stats()["sigma_flops"]
        y = ctx.apply_heff(k, x)
        flops = ctx.stats()["sigma_flops"] - f0
        rel = float(np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref))
        ctx.close()
    return dict(times=times, setup_s=setup_s, flops=flops, parity_rel=rel, psi_len=len(x))


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=list(PREC))
    ap.add_argument("--workload", default="cas16_m512")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--refine", type=int, default=0, help="FP64 Davidson iterations after the tensor-core tiers")
    ap.add_argument("--probes", type=int, default=3, help="bonds probed for the per-step energy error vs FP64")
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false")
    ap.add_argument("--no-batched", dest="with_batched", action="store_false",
                    help="skip the batched64 sub-measurement of the default line")
    ap.add_argument("--rdms", action="store_true", help="also time the RDMs, orbital entropies and (where it "
                    "fits) the 3-RDM of the final state")
    ap.add_argument("--batch-sweeps", type=int, default=2, help="sweeps per problem (batched64)")
    ap.add_argument("--workers", type=int, default=0, help="host worker threads (batched64; 0 = auto)")
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--precond", default="diag", choices=sorted(PRECOND),
                    help="Davidson correction of the timed sweeps (diag = Jacobi)")
    ap.add_argument("--floor-mult", type=float, default=1.0,
                    help="accurate tier stops on a plateau below floor_mult x u x |theta|")
    ap.add_argument("--hard-stag", type=int, default=8,
                    help="accurate tier stops after this many iterations without a 30%% cut (0: off)")
    ap.add_argument("--env-prec", default="fp64", choices=sorted(ENV_PREC),
                    help="environment updates of the mixed sweeps (tensor cores for tf32x3 / bf16x3)")
    ap.add_argument("--tier2", default="tf32x3", choices=["tf32x3", "bf16x3"],
                    help="operands of the accurate Davidson tier")
    ap.add_argument("--sigma-probe", type=int, default=0, help="profiling driver: central sigma of cas16_m512 "
                    "with operand type 1 TF32, 2 BF16, 3 TF32x3 (no bench line)")
    ap.add_argument("--states", type=int, default=0, help="excited-state driver: this many lowest roots of "
                    "--workload by penalty deflation, with <S^2> (no bench line)")
    ap.add_argument("--penalty", type=float, default=2.0, help="deflation penalty (Ha) of --states")
    ap.add_argument("--probe-warm-sweeps", type=int, default=0, help="--sigma-probe on the state after this many "
                    "mixed-precision sweeps (profiler started before the timed builds)")
    ap.add_argument("--precond-ab", action="store_true", help="learned against diagonal preconditioner on "
                    "--workload after --warmup sweeps (probe solves to 1e-8; no bench line)")
    ap.add_argument("--rdm-probe", action="store_true", help="profiling driver: the RDM pass of --workload after "
                    "--probe-warm-sweeps (default 2) mixed sweeps (no bench line)")
    ap.add_argument("--precond-probe", type=int, default=0, help="profiling driver: one fused learned-"
                    "preconditioner application on this many elements (no bench line)")
    ap.add_argument("--probe-davidson", action="store_true", help="--sigma-probe: one mixed-precision Davidson "
                    "solve at the central bond instead of the sigma builds")
    ap.add_argument("--tc-sout-min", type=int, default=None, help="stage-B s_out split threshold on E_L(q) rows "
                    "(library default if omitted)")
    ap.add_argument("--probe-order-a", type=int, default=0, help="stage-A tile order of --sigma-probe (0 the "
                    "library's default, 1 Renl-stack blocks together)")
    ap.add_argument("--probe-orders", default="1", help="stage-B tile orders timed by --sigma-probe, e.g. 0,1,2 "
                    "(1 is the library's default)")
    args = ap.parse_args()
    if args.precond_ab:
        precond_ab(args)
        return
    if args.precond_probe:
        precond_probe(args.precond_probe)
        return
    if args.rdm_probe:
        rdm_probe(args.workload, args.probe_warm_sweeps or 2)
        return
    if args.sigma_probe:
        sigma_probe(args.sigma_probe, tuple(int(o) for o in args.probe_orders.split(",")), args.probe_warm_sweeps,
                    args.probe_davidson, args.probe_order_a)
        return
    if args.states:
        states_run(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.workload == "batched64":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the oracle sample is defined on cas16_m512"}))
            return
        res = run_batched(args, rank, world)
        tmax, flops = res["time"], res["flops"]
        tmax, flops = reduce_over_ranks(tmax, flops, world)
        if rank == 0:
            print(json.dumps({
                "metric": "batched active spaces: sigma-build TFLOP/s", "value": flops / tmax / 1e12,
                "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000 * tmax / args.steps, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
                "config": {"workload": "batched64: 64 active spaces, n_orb U{8..14}, M in {128,256,512}, "
                                       f"half filling (S_z = 0, or 1/2 when odd), {args.batch_sweeps} sweeps each; one step = one batched call",
                           "workers": args.workers, "graphs": not args.no_graphs,
                           "parallelism": f"problems partitioned over {world} rank(s), LPT on n M^3 sweeps",
                           "l2": "per-problem state re-created every step (> L2 in total)"},
                "problems_per_s": res["n_problems"] * args.steps / tmax,
                "load_imbalance_max_over_mean": res["load_imbalance"],
                "energies": res["energies"],
                "clocks": res["clocks"], "gpu_launches": int(res["launches"]),
                "graph_launches": int(res["graph_launches"])}))
        return
    wl = WORKLOADS[args.workload]
    config = {"workload": f"{args.workload}: CAS({wl['n_elec']}e,{wl['n_orb']}o) S_z=0, {wl['n_chol']} Cholesky "
                          f"vectors, M={wl['M']}, one step = one full sweep",
              "n_orb": wl["n_orb"], "bond_dim": wl["M"], "davidson_tol": args.tol,
              "environment_updates": args.env_prec if args.precision != "fp64" else "fp64",
              "davidson_stop": "FP64 path: ||r|| < tol.  Mixed tiers: ||r|| < tol, or the accurate tier's floor "
                               f"(||r|| below {args.floor_mult:g} u max(1,|theta|), u = its measured sigma error, and "
                               f"no 30 % drop over 3 iterations; or no 30 % drop over {args.hard_stag} iterations), "
                               f"then at most {args.refine} FP64 iterations; residuals reached are in "
                               "per_sweep.davidson_final_residual",
              "l2": "inputs larger than L2 (environments of all bonds, > 1 GB)",
              "parallelism": f"replicas x{world}"}
    if args.precond != "diag":
        config["davidson_correction"] = args.precond
    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        s = oracle_sample(n_sigma=args.steps, want_flops=True, warmup=args.warmup)
        ms = 1000 * float(np.mean(s["times"]))
        val = s["flops"] / (ms / 1000) / 1e12
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
                "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores(), "kind": "oracle",
                                 "sample": "one oracle sigma build per step at bond pair (7,8) of "
                                           "CAS(16,16) on the seeded initial MPS (M=512)"},
                "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "oracle_setup_s": s["setup_s"], "wall_s": time.perf_counter() - t0}
        print(json.dumps(line))
        return
    res = run_ours(args, rank, world)
    tmax, flops = res["time"], res["flops"]
    tmax, flops = reduce_over_ranks(tmax, flops, world)
    if rank != 0:
        return
    pk, pk_kind = peaks()
    kern_tflops = res["flops"] / (res["sigma_ms"] / 1000) / 1e12 if res["sigma_ms"] > 0 else 0.0
    if args.precision == "fp64":
        # FP64 runs on the CUDA cores: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
        peak, bound, punit, kind = 152 * 2 * 2 * 2.07e9 / 1e12, "alu", "TFLOP/s", "derived (FP64 unit count x max clock)"
        kname, achieved = "gemm_f64_kernel (sigma stages A+B)", kern_tflops
    else:
        # tc_gemm_kernel (stage A + stage B launches, CUDA events around them
        # on the engine stream).  Tensor view: algorithmic flops per operand
        # type against that type's peak (BF16: measured sustained; TF32:
        # x 1.1/2.25, the nominal ratio; TF32x3 / BF16x3: three passes), i.e. the
        # time the flops need at peak over the time they took.  HBM view:
        # algorithmic bytes (enlarged operators once, Y^T written and read
        # once, psi and sigma) over the same time.  The larger fraction binds.
        tc = res["tc"]
        pb = pk["bf16_tflops_sustained"]
        tpk = [pb, pb * 1.1 / 2.25, pb * 1.1 / 2.25 / 3, pb / 3]   # BF16, TF32, TF32x3, BF16x3
        gms = tc["tc_gemm_ms"]
        at_peak = sum(f / (p * 1e12) for f, p in zip(tc["tc_flops_by_type"], tpk))
        tfrac = at_peak / (gms / 1000) if gms > 0 else 0.0
        tflops = sum(tc["tc_flops_by_type"]) / (gms / 1000) / 1e12 if gms > 0 else 0.0
        gbs = tc["tc_bytes"] / (gms / 1000) / 1e9 if gms > 0 else 0.0
        hfrac = gbs / pk["hbm_gbs"]
        kname = "tc_gemm_kernel (tcgen05 + TMA; sigma stages A and B, all tiers)"
        tview = {"bound": "tensor", "achieved": tflops, "peak": tfrac and tflops / tfrac, "unit": "TFLOP/s",
                 "frac": tfrac, "peak_kind": pk_kind + " bf16 sustained x type ratio (time-weighted over tiers)"}
        hview = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": hfrac,
                 "peak_kind": pk_kind + " copy bandwidth"}
        main_v, alt_v = (hview, tview) if hfrac >= tfrac else (tview, hview)
        peak, bound, punit, kind, achieved = main_v["peak"], main_v["bound"], main_v["unit"], main_v["peak_kind"], \
            main_v["achieved"]
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": punit, "frac": achieved / peak if peak else 0.0,
            "traffic": None, "kernel": kname, "peak_kind": kind}
    if args.precision != "fp64":
        nl = res["breakdown"]["tc_sigma_builds"] * 2 * args.steps   # two tc_gemm_kernel launches per sigma
        if args.tier2 == "tf32x3" and nl > 0:
            roof["traffic"] = TC_DRAM_PER_ALG_BYTE * res["tc"]["tc_bytes"] / nl
            roof["traffic_note"] = ("bytes per launch: ncu DRAM/algorithmic ratio %.2f measured at the central bond of "
                                    "the warm state, times the timed launches' algorithmic bytes" % TC_DRAM_PER_ALG_BYTE)
        roof["other_view"] = alt_v
        roof["tc_gemm_ms_per_sweep"] = res["tc"]["tc_gemm_ms"] / args.steps
        roof["launches_per_sweep"] = res["breakdown"]["tc_sigma_builds"] * 2
    line = {"metric": METRIC, "value": flops / tmax / 1e12,
            "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "config": config,
            "dtype": DTYPE["fp64"] if args.precision == "fp64" else f"{args.precision}+{args.tier2}/f32-acc",
            "sweep_time_s": tmax / args.steps, "sweep_energies": res["energies"],
            "sigma_kernel_tflops": kern_tflops, "final_energy": res["e_final"],
            "per_sweep": res["breakdown"], "roofline": roof,
            "clocks": res["clocks"],
            "gpu_launches": int(res["launches"])}
    if res["rdm_times"]:
        line["rdms"] = res["rdm_times"]
    if res["probes"]:
        line["per_step_energy_error_vs_fp64"] = {
            "max_abs_dE_Ha": max(abs(p["dE"]) for p in res["probes"]), "probes": res["probes"],
            "how": "same input state: FP64 Rayleigh quotient of the mixed-precision Davidson solution minus that "
                   "of an FP64 Davidson solution (residual 1e-9)"}
    if res["fp64"]:
        g = res["fp64"]
        dE = g["mixed"]["final_energy"] - g["fp64"]["final_energy"]
        line["fp64_gpu_sweep_s"] = g["fp64"]["sweep_s"]
        line["speedup_vs_fp64_sweep"] = g["fp64"]["sweep_s"] / (tmax / args.steps)
        line["speedup_vs_fp64_sweep_at_mixed_residual"] = g["fp64_at_mixed_residual"]["sweep_s"] / (tmax / args.steps)
        line["gate"] = {
            "ok": bool(abs(dE) <= 1e-6), "bound_Ha": 1e-6, "E_mixed_minus_E_fp64_Ha": dE,
            "how": "from one saved warmed state: one more sweep in the mixed tiers and one sweep of the plain FP64 "
                   "path at the same Davidson tolerance; final energies <psi|H|psi> in FP64",
            "E_start": g["e_start"], "energy_change_after_mixed_sweep": g["mixed"]["final_energy"] - g["e_start"],
            "energy_change_after_fp64_sweep": g["fp64"]["final_energy"] - g["e_start"],
            "energy_change_after_fp64_sweep_at_mixed_residual":
                g["fp64_at_mixed_residual"]["final_energy"] - g["e_start"],
            "sweeps": {k: g[k] for k in ("mixed", "fp64", "fp64_at_mixed_residual")}}
    if res["e2e"]:
        e = res["e2e"]
        line["e2e"] = {"value": e["flops"] / e["time"] / 1e12, "unit": "TFLOP/s",
                       "h2d_bytes_per_step": e["h2d"] // args.steps, "d2h_bytes_per_step": e["d2h"] // args.steps,
                       "solve_s": e["time"]}
    if world == 1 and args.with_batched and args.workload == "cas16_m512":
        # the batched workload (64 independent active spaces) measured in the
        # same run: one untimed and one timed gbd_solve_batched call
        import copy
        ba = copy.copy(args)
        ba.steps, ba.warmup = 1, 1
        b = run_batched(ba, 0, 1)
        line["batched64"] = {
            "value": b["flops"] / b["time"] / 1e12, "unit": "TFLOP/s", "wall_s": b["time"],
            "problems_per_s": b["n_problems"] / b["time"], "gpu_launches": int(b["launches"]),
            "graph_launches": int(b["graph_launches"]), "clocks": b["clocks"],
            "workload": "64 active spaces, n_orb U{8..14}, M in {128,256,512}, half filling, "
                        f"{ba.batch_sweeps} sweeps each, mixed tiers; one gbd_solve_batched call"}
    if world == 1 and not args.no_cpu_baseline:
        s = oracle_sample(n_sigma=1, want_flops=True)
        v = s["flops"] / s["times"][0] / 1e12
        line["cpu_baseline"] = {"value": v, "unit": "TFLOP/s", "cores": cores(), "kind": "oracle",
                                "sample": f"one oracle sigma build at bond pair (7,8) of the same problem on the "
                                          f"seeded initial MPS (M=512, psi length {s['psi_len']}); "
                                          f"{s['times'][0]:.1f} s; oracle setup {s['setup_s']:.0f} s untimed",
                                "gpu_vs_oracle_sigma_rel_err": s["parity_rel"]}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
