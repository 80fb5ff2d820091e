#!/usr/bin/env python
"""Throughput of the checkerboard Metropolis sweep on one B300 (or N replicas).

A step is one sweep of the whole hot path over the workload: the host
threshold table for beta(t), the colour-0 and colour-1 half-sweeps, and, at
the workload's cadence, the observables (B, M, Q, row and column sums)
recorded on the device -- every 10 sweeps for the large quench (its xi(t) is
logged every 10 sweeps), every sweep for the small workloads; the line also
reports the step recording every sweep.  The default workload is the single
large Ising lattice, L = 2^20 (2^40 spins, 128 GiB of bit-planes), hot start,
quench to beta_c; the lattice is far larger than L2, so no flush is needed
between steps.  The line carries the other large-quench lattice, Blume-Capel
Delta = 0 at L = 2^19 (64 GiB), measured the same way (`blume_capel_large`),
the replica ensemble (`batched`), the served request stream (`served`), the
pre-cooling scan, the row-slab decomposition on one GPU (`decomposition`),
Swendsen-Wang and the oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ising_large|blume_capel_large|ising_small|blume_capel_parity]
                    [--served-requests N] [--served-saturated N]
                    [--no-bc] [--no-batched] [--no-served] [--no-precool] [--no-sw]
                    [--no-decomposition]
                    [--no-cpu-baseline] [--no-calib]

Prints one JSON line.  `value` is the device-timed throughput (spin-flip
attempts per ns, all ranks); `e2e` is the same metric through the public C
ABI with host inputs (the beta of each sweep) and host outputs (each sweep's
record read back, xi_2 computed on the host) inside the timed region.
`roofline.frac` is the dominant half-sweep against the integer-issue peak
(SM count read from the device); `roofline.pipe_bound` is the same launch
against a per-pipe bound from integer rates measured at the start of the run.
With --impl reference the oracle (CPU) is timed on a bounded sample.
"""
import argparse
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

from paper_2503_14688_b300 import workloads as wl  # noqa: E402

METRIC = "spin flips/ns per B300 (Ising, BC) & % roofline; batched/served vs single lattice"
UNIT = "flips/ns"

# Algorithmic integer operations per site update (one 32-lane-issue integer
# operation each; a wide multiply counts once):
#   Philox4x32-10 per 4 sites: 20 wide (32x32->64) multiplies + 20
#   three-input XORs, i.e. 5 + 5 per site;
#   Ising acceptance: 2 threshold compares + 2 bit inserts; the bit-sliced
#   neighbour count and flip logic: about 1 per site (30-40 per 32 sites);
#   total 15;
#   Blume-Capel: the same Philox; per site the table entry's offset (byte
#   permute + mask), the compare (2) and the proposal bit (1); per 32-site
#   word the bit-sliced field sum (~30), the transpose of six planes into
#   index bytes (~56) and the two-plane update (~10), about 3 per site;
#   total 18 (the shared-memory table load is not an integer op).
ALG_OPS_PER_SITE = {wl.ISING: 15.0, wl.BLUME_CAPEL: 18.0}
INT_LANES_PER_SM = 128     # 4 SMSPs x 32 lanes, one warp-instruction per SMSP per clock
# The same algorithmic counts split by execution pipe (pipe-aware bound):
# Philox's 5 wide (32x32->64) multiplies per site run on the FMA-heavy pipe,
# its 5 three-input XORs on the ALU pipe, and the remaining ops (Ising 5,
# Blume-Capel 8) may issue on either pipe.
PIPE_OPS = {wl.ISING: {"wide": 5.0, "alu": 5.0, "either": 5.0},
            wl.BLUME_CAPEL: {"wide": 5.0, "alu": 5.0, "either": 8.0}}
# The kernels fold the launch-uniform parts of Philox's first two rounds:
# 18 wide multiplies per 4 sites instead of 20.
WIDE_MUL_PER_SITE_FOLDED = 18 / 4
# DRAM bytes (read + write) per site of one half-sweep launch, from one ncu
# capture of the current kernels on a smaller lattice (Ising L = 2^16:
# 537.98 + 229.27 MB per 2^31 sites; Blume-Capel L = 2^15: 269.83 + 94.14 MB
# per 2^29 sites), scaled to a full launch by the sites it updates.
DRAM_BYTES_PER_SITE = {wl.ISING: (537.98e6 + 229.27e6) / 2**31,
                       wl.BLUME_CAPEL: (269.83e6 + 94.14e6) / 2**29}


def _l2_note(lattice_bytes):
    if lattice_bytes > 2 * 126e6:
        return "not needed: lattice %.1f GiB >> 126 MB L2" % (lattice_bytes / 2**30)
    return "none: lattice %.1f MiB may stay in the 126 MB L2" % (lattice_bytes / 2**20)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p.get("sm_max_mhz", 2032.0), "measured sm_max_mhz"
    return 2032.0, "fallback (recipe max SM clock)"


def _hbm_peak():
    """Copy bandwidth in GB/s: the measured one, else the recipe's fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        if "hbm_gbs" in p:
            return float(p["hbm_gbs"]), "measured hbm_gbs (MEASURED_PEAKS.json)"
    return 6400.0, "fallback 6.4 TB/s"


def _workload(name):
    return {"ising_large": wl.ising_large, "blume_capel_large": wl.blume_capel_large,
            "ising_small": wl.ising_quench_small,
            "blume_capel_parity": wl.blume_capel_parity}[name]()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = os.path.join("/tmp", "isg_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.out):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.remove(self.out)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(model, beta, delta, budget_s=12.0, seed=wl.BASE_SEED + 99):
    """The oracle, as it stands, on the host cores: a bounded sample of the
    workload (an L = 4096 lattice; the per-site rate of the byte-per-site
    oracle does not depend on L once out of cache)."""
    import oracle

    threads = oracle.default_threads()
    L = 4096
    s = oracle.init_random(L, model, seed)
    oracle.run(s, model, seed, 0, [beta], delta=delta, nthreads=threads)  # warm-up (threads, pages)
    t0 = time.perf_counter()
    oracle.run(s, model, seed, 1, [beta] * 3, delta=delta, nthreads=threads)
    one = (time.perf_counter() - t0) / 3
    n = max(1, min(4000, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(s, model, seed, 4, [beta] * n, delta=delta, record_every=n, nthreads=threads)
    dt = time.perf_counter() - t0
    return {"value": L * L * n / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{'Ising' if model == 0 else 'Blume-Capel'} L={L} hot start, {n} sweeps "
                      f"at the workload's beta with the observables of the last sweep, "
                      f"{dt:.1f} s on {threads} threads"}


def batched_bench(sweeps=10000, n_rep=4096, record_every=1000):
    """The replica-ensemble workload: n_rep independent Ising replicas, L drawn
    uniformly from {64, 128, 256, 512, 1024}, hot start quenched to beta_c,
    `sweeps` sweeps in one persistent graph-captured launch (records every
    `record_every` sweeps), against one L = 32768 lattice (about the same
    number of spins) swept alone."""
    import torch

    import paper_2503_14688_b300 as P

    Ls = wl.ensemble_sizes(n_rep)
    seeds = [wl.BASE_SEED + 3 + r for r in range(n_rep)]
    stream = torch.cuda.Stream()
    ens = P.Ensemble(Ls, seeds, stream=stream, record_capacity=sweeps // record_every + 1)
    ens.init_random()
    tune, cands = ens.autotune(50, with_candidates=True)
    ens.sweep(4, beta=wl.BETA_C_ISING)  # warm-up (graph instantiation)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    ens.sweep(sweeps, beta=wl.BETA_C_ISING, record_every=record_every)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    spins = float(np.sum(Ls.astype(np.float64) ** 2))
    rows = ens.read_records(with_sums=False)
    ens.close()
    batched = spins * sweeps / (ms * 1e6)
    # one lattice of about the same number of spins
    Ls1, n1 = 32768, 200
    lat = P.Lattice(Ls1, wl.ISING, seed=wl.BASE_SEED + 3, stream=stream)
    lat.init_random()
    lat.sweep(3, beta=wl.BETA_C_ISING)
    torch.cuda.synchronize()
    a.record(stream)
    lat.sweep(n1, beta=wl.BETA_C_ISING)
    b.record(stream)
    torch.cuda.synchronize()
    single = float(Ls1) ** 2 * n1 / (a.elapsed_time(b) * 1e6)
    lat.close()
    # the same replicas swept one lattice at a time through the single-lattice
    # path (sweeps_alone sweeps each, one after another on one stream)
    sweeps_alone = 100
    lats = [P.Lattice(int(L), wl.ISING, seed=s_, stream=stream) for L, s_ in zip(Ls, seeds)]
    for x in lats:
        x.init_random()
    torch.cuda.synchronize()
    a.record(stream)
    for x in lats:
        x.sweep(sweeps_alone, beta=wl.BETA_C_ISING)
    b.record(stream)
    torch.cuda.synchronize()
    one_at_a_time = spins * sweeps_alone / (a.elapsed_time(b) * 1e6)
    for x in lats:
        x.close()
    return {"workload": f"{n_rep} Ising replicas, L uniform in {{64..1024}}, beta_c, "
                        f"{sweeps} sweeps in one persistent launch, records every {record_every}",
            "value": batched, "unit": UNIT, "ms": ms, "spins": spins, "record_rows": len(rows),
            "tuning": tune,
            "tuning_candidates": [[c["threads_per_cta"], c["half_teams"], c["sweeps_per_launch"],
                                   c["multi_words"], c["multi_band"], round(c["ms"], 3)]
                                  for c in cands],
            "tuning_candidates_fields": "threads_per_cta, half_teams, sweeps_per_launch, "
                                        "multi_words, multi_band, ms over 50 sweeps",
            "single_lattice_equal_spins": {"L": Ls1, "value": single, "unit": UNIT},
            "ratio_vs_single": batched / single,
            "one_lattice_at_a_time": {"sweeps": sweeps_alone, "value": one_at_a_time,
                                      "unit": UNIT, "batched_speedup": batched / one_at_a_time}}


def precool_bench(n_rep=4096):
    """The pre-cooling scan at scaled size (Ising, T1 = 0.73 T_c, T2 = 1.04 T_c,
    L = 512 replicas): xi_eq(T2), the switch times, the protocol ensembles for
    four f and the joint fit of Eq. (8); the zero f* of b(f) against the
    paper's 0.59(5)."""
    from paper_2503_14688_b300 import precooling as pc

    t0 = time.perf_counter()
    res = pc.scan(wl.ISING, [0.3, 0.45, 0.6, 0.75], n_replicas=n_rep, n_xi=16, t_after=1000)
    return {"workload": "Ising pre-cooling scan: T1 = 0.73 T_c, T2 = 1.04 T_c, %d replicas of "
                        "L = 512, f in {0.3, 0.45, 0.6, 0.75}, 1000 sweeps at T2" % n_rep,
            "xi_eq": res["xi_eq"], "t_switch": res["t_switch"], "tau": res["fit"]["tau"],
            "b": res["fit"]["b"], "b_err": res["fit"]["b_err"],
            "fit_window": [res["fit"]["t_min"], res["fit"]["t_max"]],
            "chi2_per_dof": res["fit"]["chi2_per_dof"],
            "f_star": res["f_star"], "f_star_err": res["f_star_err"], "f_star_paper": 0.59,
            "ensemble_flips_per_ns": res["ensemble_flips_per_ns"],
            "seconds": time.perf_counter() - t0}


def decomposition_bench(L=1 << 19, P=4, sweeps=6):
    """The row-slab domain decomposition on one GPU: one Ising lattice cut
    into P slabs in this process (halo rows copied device to device before
    every half-sweep), against the same lattice swept whole.  Several GPUs
    would each hold one slab; here the slabs share one."""
    import torch

    import paper_2503_14688_b300 as P_
    from paper_2503_14688_b300 import decomposition as dd

    beta = wl.BETA_C_ISING
    parts = dd.partition(L, P)
    slabs = {r: dd.Slab(wl.ISING, L, y0, rows, wl.BASE_SEED + 8) for r, (y0, rows) in enumerate(parts)}
    for sl in slabs.values():
        sl.init_random()
    run = dd.Decomposition(slabs, dd.LocalExchange(P))
    run.sweep(2, beta=beta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run.sweep(sweeps, beta=beta)
    torch.cuda.synchronize()
    slab_s = time.perf_counter() - t0
    rec = run.record()
    for sl in slabs.values():
        sl.close()
    lat = P_.Lattice(L, wl.ISING, seed=wl.BASE_SEED + 8)
    lat.init_random()
    lat.sweep(2, beta=beta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.sweep(sweeps, beta=beta)
    torch.cuda.synchronize()
    whole_s = time.perf_counter() - t0
    wrec = lat.measure()
    lat.close()
    sites = float(L) ** 2
    return {"workload": f"Ising L={L} as {P} row slabs in one process, halos exchanged device to "
                        f"device before every half-sweep, {sweeps} sweeps (host-timed)",
            "slabs": [r for _, r in parts],
            "value": sites * sweeps / slab_s / 1e9, "unit": UNIT,
            "whole_lattice": sites * sweeps / whole_s / 1e9,
            "ratio": whole_s / slab_s,
            "halo_bytes_per_half_sweep_per_slab": 2 * L // 16,
            "same_record_as_whole": (rec.B, rec.M, rec.Q) == (wrec.B, wrec.M, wrec.Q)}


def sw_bench(Ls=(4096, 16384), reps=20):
    """Swendsen-Wang iteration (Appendix B) on a Blume-Capel lattice at the
    paper's T_c, and the elementary Monte Carlo step (10 Metropolis sweeps +
    one Swendsen-Wang iteration).  Algorithmic bytes per site of one
    iteration: labels written (init), read and written (link, flatten),
    read (coin), read twice (flip: own label, root's coin) = 24 B, plus the
    spin planes read twice and written once (0.75 B)."""
    import torch

    import paper_2503_14688_b300 as P

    beta = 1.0 / wl.T_C_BLUME_CAPEL
    out = []
    for L in Ls:
        lat = P.Lattice(L, wl.BLUME_CAPEL, seed=wl.BASE_SEED + 4100)
        lat.init_random()
        lat.emcs(3, beta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.swendsen_wang(beta, n=reps)
        sw_s = (time.perf_counter() - t0) / reps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.sweep(10 * reps, beta=beta)
        torch.cuda.synchronize()
        sweep_s = (time.perf_counter() - t0) / (10 * reps)
        lat.close()
        n = float(L) * L
        out.append({"L": L, "sw_ms": 1e3 * sw_s, "metropolis_sweep_ms": 1e3 * sweep_s,
                    "emcs_ms": 1e3 * (sw_s + 10 * sweep_s),
                    "sw_sites_per_ns": n / sw_s / 1e9,
                    "sw_GB_per_s": 24.75 * n / sw_s / 1e9,
                    "labels_MiB": 4 * n / 2**20})
    return {"workload": "Blume-Capel at T_c (Delta = 0), hot start + 3 EMCS, then 20 "
                        "Swendsen-Wang iterations (host-timed, each synchronises) and 200 sweeps",
            "bytes_per_site": 24.75, "sizes": out}


def served_bench(n_req=2000, n_saturated=200, load=0.9, chunk=100, max_active=48):
    """The served stream: requests of the served workload (workloads.py)
    through the continuous-batching server.  Capacity: the stream's first
    `n_saturated` requests submitted at once (saturated throughput and its
    ratio to the same mix run as single lattices).  Latency: all `n_req`
    requests with Poisson arrivals at `load` x that capacity -- p50/p99 of
    arrival-to-completion, and of the slowdown (latency over the request's
    time alone at the single-lattice rate of its model); under processor
    sharing the mean slowdown at load rho is 1 / (1 - rho)."""
    import paper_2503_14688_b300 as P

    reqs = wl.served_requests(n_req)
    flips = np.array([float(r["L"]) ** 2 * r["sweeps"] for r in reqs])
    budget = 96 << 30

    def run(sub, arrivals):
        srv = P.Server(hbm_budget=budget, max_active=max_active, chunk_sweeps=chunk)
        ids = []
        for r, a in zip(sub, arrivals):
            ids.append(srv.submit(r["model"], r["L"], r["seed"], r["sweeps"], r["t_start"],
                                  r["beta"], arrival_time=a))
        srv.drain()
        res = [srv.poll(i) for i in ids]
        srv.close()
        lat = np.array([x.t_done - x.t_arrival for x in res])
        t_first = min(x.t_arrival for x in res)
        t_last = max(x.t_done for x in res)
        return lat, t_last - t_first

    # single-lattice reference at equal spins: each model's rate on one
    # L = 32768 lattice, combined with the mix's flips of that model
    import torch

    ref_rate = {}
    for model in (wl.ISING, wl.BLUME_CAPEL):
        lat = P.Lattice(32768, model, seed=wl.BASE_SEED + 5)
        lat.init_random()
        beta = wl.BETA_C_ISING if model == wl.ISING else 1.0 / wl.T_C_BLUME_CAPEL
        lat.sweep(2, beta=beta)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        lat.sweep(50, beta=beta)
        b.record()
        torch.cuda.synchronize()
        ref_rate[model] = 32768.0 ** 2 * 50 / (a.elapsed_time(b) * 1e-3)
        lat.close()
    # each request's time alone on the idle GPU: its flips at the measured
    # single-lattice rate of its own (model, L), as isg_sweep runs it
    own_rate = {}
    for model, L in sorted({(r["model"], r["L"]) for r in reqs}):
        k = int(min(2000, max(20, 5e9 / float(L) ** 2)))
        lat = P.Lattice(L, model, seed=wl.BASE_SEED + 6)
        lat.init_random()
        beta = wl.BETA_C_ISING if model == wl.ISING else 1.0 / wl.T_C_BLUME_CAPEL
        lat.sweep(2, beta=beta)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        lat.sweep(k, beta=beta)
        b.record()
        torch.cuda.synchronize()
        own_rate[(model, L)] = float(L) ** 2 * k / (a.elapsed_time(b) * 1e-3)
        lat.close()
    alone = np.array([f / own_rate[(r["model"], r["L"])] for f, r in zip(flips, reqs)])
    full = np.array([f / ref_rate[r["model"]] for f, r in zip(flips, reqs)])  # at the L=32768 rate

    sat = reqs[:n_saturated]
    sat_total = float(flips[:n_saturated].sum())
    ref = sat_total / float(full[:n_saturated].sum())
    _, span0 = run(sat, [0.0] * len(sat))
    capacity = sat_total / span0  # flips/s with the queue always full
    total = float(flips.sum())
    rate = load * capacity / (total / n_req)
    arrivals = wl.poisson_arrivals(n_req, rate)
    lat, span = run(reqs, list(arrivals))
    slow = lat / alone
    return {"workload": f"{n_req} requests: Ising or Blume-Capel (p=1/2), L=2^k, k in 8..14, "
                        f"sweeps log-uniform in [1e3, 1e4], 10-step bath 1.5 T_c -> 1.01 T_c; "
                        f"chunk {chunk} sweeps, {max_active} slots",
            "saturated": {"requests": len(sat), "value": capacity / 1e9, "unit": UNIT,
                          "makespan_s": span0, "flips": sat_total,
                          "single_lattice_mix": {"value": ref / 1e9, "unit": UNIT,
                                                 "ising_L32768": ref_rate[wl.ISING] / 1e9,
                                                 "blume_capel_L32768":
                                                     ref_rate[wl.BLUME_CAPEL] / 1e9},
                          "ratio_vs_single": capacity / ref},
            "poisson": {"requests": n_req, "load": load, "rate_per_s": rate,
                        "value": total / span / 1e9, "unit": UNIT,
                        "p50_s": float(np.percentile(lat, 50)),
                        "p99_s": float(np.percentile(lat, 99)), "makespan_s": span,
                        "slowdown_basis": "latency / the request's time alone on the idle GPU "
                                          "(its flips at the single-lattice rate of its model and L)",
                        "slowdown_p50": float(np.percentile(slow, 50)),
                        "slowdown_p99": float(np.percentile(slow, 99)),
                        "slowdown_mean": float(slow.mean()),
                        "slowdown_p50_by_L": {str(L): float(np.percentile(
                            slow[[r["L"] == L for r in reqs]], 50))
                            for L in sorted({r["L"] for r in reqs})},
                        "slowdown_processor_sharing": 1.0 / (1.0 - load),
                        "alone_rate_by_model_L": {f"{m}:{L}": v / 1e9
                                                  for (m, L), v in sorted(own_rate.items())}},
            "total_flips": total}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    threads = oracle.default_threads()
    L = 4096
    seed = w.seed
    s = oracle.init_random(L, w.model, seed)
    for i in range(args.warmup):
        oracle.run(s, w.model, seed, i, [w.beta], delta=w.delta, nthreads=threads)
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(s, w.model, seed, args.warmup + i, [w.beta], delta=w.delta, record_every=1,
                   nthreads=threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = L * L * args.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": w.name, "sample_L": L, "note": "oracle on host cores, one "
                       "sweep of an L=4096 sample of the same model/beta per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"L={L}, {args.steps} sweeps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def roofline(model, sites, dom_ms, which, half_ms, sms, sm_max, peak_src, rates):
    """The dominant half-sweep launch against the integer-issue peak (the
    headline `frac`) and against the pipe-aware bound from the rates measured
    in this run (`pipe_bound`)."""
    peak = sms * INT_LANES_PER_SM * sm_max * 1e6 / 1e12  # Tops/s
    per_launch = sites / 2
    achieved = ALG_OPS_PER_SITE[model] * per_launch / (dom_ms * 1e-3) / 1e12
    sites_per_ns = per_launch / (dom_ms * 1e6)
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
           "frac": achieved / peak,
           "traffic": DRAM_BYTES_PER_SITE[model] * per_launch,
           "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one half-sweep at "
                            "L=2^16 (Ising) / 2^15 (Blume-Capel), scaled by sites per launch; "
                            f"algorithmic {0.375 if model == wl.ISING else 0.75} B/site",
           "kernel": "half-sweep colour %d" % which,
           "ops_per_site": ALG_OPS_PER_SITE[model],
           "peak_basis": f"{sms} SMs (device) x {INT_LANES_PER_SM} int lanes x {sm_max:.0f} MHz "
                         f"({peak_src})",
           "half_sweep_ms": half_ms,
           "achieved_sites_per_ns": sites_per_ns}
    if rates:
        rw = rates["wide_multiply"]["per_sm_per_clk"]
        ra = rates["alu_op"]["per_sm_per_clk"]
        ops = PIPE_OPS[model]
        t_fma = ops["wide"] / rw
        t_alu = ops["alu"] / ra
        t_all = (ops["wide"] / rw + (ops["alu"] + ops["either"]) / ra) / 2
        t = max(t_fma, t_alu, t_all)
        bound = sms * sm_max * 1e6 / t / 1e9
        wide_bound = sms * sm_max * 1e6 * rw / ops["wide"] / 1e9
        folded = sms * sm_max * 1e6 * rw / WIDE_MUL_PER_SITE_FOLDED / 1e9
        out["pipe_bound"] = {
            "basis": "per site: max(wide/r_wide, alu/r_alu, (wide/r_wide + (alu + either)/r_alu)/2) "
                     "SM-clocks with the algorithmic counts and the rates measured in this run",
            "ops_per_site": ops, "rates_per_sm_per_clk": {"wide_multiply": rw, "alu_op": ra,
                                                          "fma_op": rates["fma_op"]["per_sm_per_clk"]},
            "sms": sms, "sm_mhz": sm_max,
            "sites_per_ns": bound, "frac": sites_per_ns / bound}
        out["wide_multiply_bound"] = {
            "basis": f"{ops['wide']:.0f} wide multiplies per site (Philox4x32-10, 20 per 4 sites) "
                     f"at the measured {rw:.2f} per SM per clock (FMA-heavy pipe)",
            "sites_per_ns": wide_bound, "frac": sites_per_ns / wide_bound,
            "folded": {"wide_per_site": WIDE_MUL_PER_SITE_FOLDED, "sites_per_ns": folded,
                       "frac": sites_per_ns / folded}}
    return out


def single_lattice(args, w, rank, world, stream, rates, sms, with_corr):
    """One lattice of the workload: device-timed steps, the step recording
    every sweep, the end-to-end leg through the C ABI, and the roofline of
    the dominant half-sweep."""
    import torch

    import paper_2503_14688_b300 as P

    from paper_2503_14688_b300 import replicas

    seed = replicas.replica_seed(w.seed, rank)  # replicas: independent lattices, one per rank
    lat = P.Lattice(w.L, w.model, seed=seed, delta=w.delta, stream=stream,
                    record_capacity=args.steps + args.warmup + 4)
    lat.init_random()
    beta = w.beta
    # observables (B, M, Q, R, C) recorded on the device at the workload's
    # cadence: every 10 sweeps for the large quench ("xi(t) growth logged
    # every 10 sweeps"), every sweep for the small ones
    every = max(1, int(w.record_every))

    def step(i, events=None, record_every=every):
        if events is not None:
            events[0].record(stream)
        lat.half_sweep(0, beta)
        if events is not None:
            events[1].record(stream)
        lat.half_sweep(1, beta)
        if events is not None:
            events[2].record(stream)
        if (i + 1) % record_every == 0:
            lat.record()

    for i in range(args.warmup):
        step(i)
    lat.read_records(with_sums=False)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    start.record(stream)
    for i in range(args.steps):
        step(i, evs[i])
    stop.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = start.elapsed_time(stop)
    half0 = [e[0].elapsed_time(e[1]) for e in evs]
    half1 = [e[1].elapsed_time(e[2]) for e in evs]
    recs = lat.read_records()
    assert len(recs) == args.steps // every
    xi = P.xi2([recs[-1].M], recs[-1].R[None], recs[-1].C[None]) if recs else None

    # the same step recording every sweep, for comparison (5 steps)
    n_each = min(args.steps, 5)
    a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a_ev.record(stream)
    for i in range(n_each):
        step(i, record_every=1)
    b_ev.record(stream)
    torch.cuda.synchronize()
    ms_each = a_ev.elapsed_time(b_ev) / n_each
    lat.read_records(with_sums=False)

    # the record pass alone: it reads the lattice once (plus the sums it
    # writes), so its bound is the copy bandwidth
    rec_ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    torch.cuda.synchronize()
    rec_ev[0].record(stream)
    for k in range(5):
        lat.record()
        rec_ev[k + 1].record(stream)
    torch.cuda.synchronize()
    rec_ms = statistics.median(rec_ev[k].elapsed_time(rec_ev[k + 1]) for k in range(5))
    lat.read_records(with_sums=False)
    rec_bytes = P.Lattice.nbytes(w.model, w.L) + 8 * w.L
    hbm, hbm_src = _hbm_peak()
    record = {"ms": rec_ms, "bytes": rec_bytes, "GB_per_s": rec_bytes / rec_ms / 1e6,
              "peak_GB_per_s": hbm, "peak_basis": hbm_src, "frac": rec_bytes / rec_ms / 1e6 / hbm,
              "kernel": "k_measure_stream" if w.L % 16384 == 0 else "k_measure",
              "basis": "lattice bytes read once + row and column sums written, per record "
                       "(median of 5, CUDA events, each after a slot clear)"}

    # end to end through the C ABI: host beta in, host record out, xi_2 on host
    # (per call: `every` sweeps with their betas from a host array, the
    # record read back to host arrays)
    e2e_calls = max(1, min(args.steps // every, 2)) if every > 1 else max(2, min(args.steps, 5))
    e2e_steps = e2e_calls * every
    betas_host = np.full(every, beta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_calls):
        lat.sweep(every, betas=betas_host, record_every=every)
        r = lat.read_records()[0]
        P.xi2([r.M], r.R[None], r.C[None])
    e2e_s = time.perf_counter() - t0

    corr = None
    if with_corr:
        # axis correlation function C(r) (Eq. (2)) at 12 distances, one pass each
        corr_r = [1 << k for k in range(12)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sx, sy = lat.correlation(corr_r)
        corr_s = time.perf_counter() - t0
        corr = {"distances": corr_r, "ms": 1e3 * corr_s,
                "lattice_GB_read_per_s": len(corr_r) * 2 * P.Lattice.nbytes(w.model, w.L) / corr_s / 1e9,
                "C_r": [float(a + b) / (2.0 * float(w.L) ** 2) for a, b in zip(sx, sy)]}
    lat.close()

    ms, e2e_s = replicas.max_over_ranks([ms, e2e_s], device="cuda")
    sites = float(w.L) * float(w.L)
    value = replicas.weak_scaling_value(world, sites, args.steps, ms)
    weak_each = replicas.weak_scaling_value(world, sites, 1, ms_each)
    e2e_value = replicas.weak_scaling_value(world, sites, e2e_steps, e2e_s * 1e3)
    sm_max, peak_src = _peaks()
    m0, m1 = statistics.mean(half0), statistics.mean(half1)
    which = 1 if m1 >= m0 else 0
    roof = roofline(w.model, sites, max(m0, m1), which, [m0, m1], sms, sm_max, peak_src, rates)
    return {
        "value": value, "ms_per_step": ms / args.steps, "steps": args.steps,
        "config": {"workload": w.name, "model": "ising" if w.model == 0 else "blume_capel",
                   "L": w.L, "spins": int(sites), "beta": beta, "delta": w.delta,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2_flush": _l2_note(P.Lattice.nbytes(w.model, w.L)),
                   "step": "host thresholds + half-sweep colour 0 + half-sweep colour 1; "
                           "every record_every steps an on-device record of B, M, Q, "
                           "row and column sums",
                   "record_every": every},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8,
                "d2h_bytes_per_step": (32 + 8 * w.L) / every, "steps": e2e_steps},
        "gpu_launches": 2 * args.steps + args.steps // every,
        "record_every_sweep": {"ms_per_step": ms_each, "value": weak_each, "unit": UNIT,
                               "steps": n_each,
                               "overhead_vs_value": value / weak_each - 1.0},
        "clocks": clk, "xi2_last": xi, "correlation": corr, "record": record,
    }


def run_ours(args, w):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    rates = None
    if not args.no_calib:
        from paper_2503_14688_b300 import calibrate

        rates = calibrate.measure_rates()
    stream = torch.cuda.Stream()
    main = single_lattice(args, w, rank, world, stream, rates, sms, with_corr=True)
    if rank == 0:
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic (hot-start lattice from the seeded Philox)",
            "config": main["config"], "roofline": main["roofline"], "e2e": main["e2e"],
            "gpu_launches": main["gpu_launches"],
            "record_every_sweep": main["record_every_sweep"], "record": main["record"],
            "clocks": main["clocks"],
            "xi2_last": main["xi2_last"], "correlation": main["correlation"],
            "calibration": rates,
        }
    # the other single-lattice workload of the large quench: Blume-Capel
    # Delta = 0 at L = 2^19 (its own roofline, e2e and CPU baseline)
    if not args.no_bc and w.name.startswith("ising_L1048576"):
        wb = wl.blume_capel_large()
        bc = single_lattice(args, wb, rank, world, stream, rates, sms, with_corr=False)
        if rank == 0:
            bc.pop("correlation")
            line["gpu_launches"] += bc["gpu_launches"]
            if not args.no_cpu_baseline:
                bc["cpu_baseline"] = cpu_baseline(wb.model, wb.beta, wb.delta)
            line["blume_capel_large"] = bc
    if rank == 0:
        if not args.no_batched and world == 1:
            line["batched"] = batched_bench(sweeps=args.batched_sweeps, n_rep=args.batched_replicas)
        if not args.no_served and world == 1:
            line["served"] = served_bench(n_req=args.served_requests,
                                          n_saturated=args.served_saturated)
        if not args.no_precool and world == 1:
            line["precool"] = precool_bench()
        if not args.no_decomposition and world == 1:
            line["decomposition"] = decomposition_bench()
        if not args.no_sw and world == 1:
            line["swendsen_wang"] = sw_bench()
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w.model, w.beta, w.delta)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ising_large")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sw", action="store_true",
                    help="skip the Swendsen-Wang sub-object")
    ap.add_argument("--no-precool", action="store_true",
                    help="skip the pre-cooling scan (Eq. (8)) sub-object")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the replica-ensemble measurement")
    ap.add_argument("--L", type=int, default=0, help="override the workload's L (profiling)")
    ap.add_argument("--batched-replicas", type=int, default=4096)
    ap.add_argument("--batched-sweeps", type=int, default=10000)
    ap.add_argument("--served-requests", type=int, default=2000,
                    help="requests of the served stream's Poisson leg")
    ap.add_argument("--served-saturated", type=int, default=200,
                    help="requests (the stream's first) of the saturated capacity leg")
    ap.add_argument("--no-served", action="store_true", help="skip the served stream")
    ap.add_argument("--no-decomposition", action="store_true",
                    help="skip the row-slab decomposition sub-object")
    ap.add_argument("--no-bc", action="store_true",
                    help="skip the Blume-Capel L=2^19 single-lattice sub-object")
    ap.add_argument("--no-calib", action="store_true",
                    help="skip the run-time integer-rate calibration (no pipe-aware bound)")
    ap.add_argument("--only-batched", action="store_true",
                    help="print only the replica-ensemble measurement (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.only_batched:
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(batched_bench(sweeps=args.batched_sweeps, n_rep=args.batched_replicas,
                                       record_every=max(1, args.batched_sweeps // 10))), flush=True)
        return
    w = _workload(args.workload)
    if args.L:
        w.L = args.L
        w.name = f"{w.name}@L={args.L}"
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
