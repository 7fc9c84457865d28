#!/usr/bin/env python
"""Fock builds/s of the density-fitted RHF Fock build at (H2O)_64 on GB300.

One step = one Fock build F = H + 2J - K from C_occ (bqc_jk): the X pass
(X_P = B_P C_occ with the fused Coulomb contraction w_P), the J pass and the
K contraction, with B (N = 1600, Naux = 4800, nocc = 320) resident in HBM.
The headline runs in mixed precision (TF32 tcgen05 tensor cores, FP32
accumulation, FP64 chunk sums); the plain-FP64 build is timed beside it.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torchrun, each rank runs an independent replica (weak scaling, no
collective on the data path).  --impl reference times the CPU oracle on a
bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Fock builds/s at (H2O)_64, mixed vs FP64 at <=1e-6 Eh; serve p50/p99 ms"
UNIT = "Fock builds/s"
# TF32 dense peak = measured bf16 x nominal (1.1 / 2.25) ratio of the recipe
TF32_OVER_BF16 = 1.1 / 2.25
# DRAM bytes / algorithmic bytes of k_xpass_tf32<.,3> in an ncu capture at
# (H2O)_16 (1.905 GB / 1.843 GB); both grow as Naux x N x (N + nocc)
XPASS_TRAFFIC_RATIO = 1.034
# the same ratio for the split-FP16 X pass in two-CTA clusters (k_xpass_mc,
# full capture of one aux piece at (H2O)_20: 457.0 MB of DRAM traffic against
# 474.0 MB of algorithmic bytes); the operand layout sets it per unit of work
XPASS_F16_TRAFFIC_RATIO = 0.964


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--waters", type=int, default=64)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--prec", choices=["f16x3", "tf32x3"], default="f16x3",
                    help="precision of the timed mixed build (split FP16 or split TF32)")
    ap.add_argument("--no-scf-check", action="store_true",
                    help="skip the staged-vs-plain-FP64 SCF energy check at the workload size")
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve", action="store_true",
                    help="serving run: Poisson stream of (H2O)_n solves, p50/p99 latency")
    ap.add_argument("--serve-requests", type=int, default=60)
    ap.add_argument("--serve-leg", type=int, default=6,
                    help="requests per offered rate in the default line's serving leg (0: skip)")
    ap.add_argument("--serve-low-rate", type=float, default=0.1,
                    help="the sub-capacity offered rate of the serving leg (req/s)")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-policy", choices=["backfill", "fifo"], default="backfill")
    ap.add_argument("--serve-precs", default="mixed_f16x3,fp64")
    ap.add_argument("--scf", action="store_true",
                    help="time one precision-staged SCF (--prec, then FP64) at --waters")
    ap.add_argument("--incremental", action="store_true",
                    help="--scf: anchored incremental FP64 stage")
    ap.add_argument("--direct", action="store_true",
                    help="direct (on-the-fly) DF run, default (H2O)_128")
    ap.add_argument("--screen-ablation", action="store_true",
                    help="time the three survivor compactions of the screened 3-centre "
                         "integrals on one aux block of (H2O)_128 (default) at tau = 1e-10")
    ap.add_argument("--mp2", action="store_true",
                    help="DF-MP2 energy after a staged SCF at --mp2-waters")
    ap.add_argument("--mp2-waters", type=int, default=32, help="--mp2: cluster size")
    ap.add_argument("--mp2-prec", choices=["f64", "f16x3"], default="f16x3",
                    help="--mp2: FP64 DFMA pair blocks or split-FP16 tensor-core pair blocks")
    return ap.parse_args()


def max_over_ranks(x: float, dist, device: str) -> float:
    """The slowest rank's time: all-reduce(MAX) of one float."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, seconds: float) -> float:
    """Fock builds per second of the whole job: every rank (an independent
    replica) ran `steps` builds within the slowest rank's `seconds`."""
    return world * steps / seconds


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() in ("active", "0x1", "1"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if ids and all(v.strip().isdigit() for v in ids) and local_rank < len(ids):
        return int(ids[local_rank])
    return local_rank


def _seeded_sample(n, nocc, nsample, seed=2025):
    """Seeded symmetric B rows and C_occ of the workload's shape (the oracle's
    dense contractions take the same time whatever the values)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    base = rng.standard_normal((min(nsample, 16), n, n))
    base = 0.5 * (base + base.transpose(0, 2, 1))
    B = np.empty((nsample, n, n))
    for i in range(nsample):  # repeat the seeded rows: filling by copy is fast
        B[i] = base[i % len(base)]
    C = rng.standard_normal((n, nocc)) * 0.05
    return B, C


def cpu_baseline(mol, samples=(64, 128, 256), reps: int = 3):
    """Oracle Fock build (numpy/BLAS FP64, oracle.jk_df as it stands) timed on
    seeded B rows of the workload's shape at several aux sample sizes, `reps`
    times each (median); t(nsample) = a + b * nsample is fitted by least squares
    and evaluated at the workload's Naux (the build is a sum over P)."""
    import numpy as np

    import oracle
    n = sum((s.l + 1) * (s.l + 2) // 2 for s in mol.orb)
    naux = sum((s.l + 1) * (s.l + 2) // 2 for s in mol.aux)
    Bmax, C = _seeded_sample(n, mol.nocc, max(samples))
    oracle.jk_df(Bmax[:2], C)  # warm the BLAS
    pts = []
    for ns in samples:
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            oracle.jk_df(Bmax[:ns], C)
            ts.append(time.perf_counter() - t0)
        pts.append((ns, statistics.median(ts), min(ts), max(ts)))
    x = np.array([p[0] for p in pts], dtype=float)
    y = np.array([p[1] for p in pts])
    b, a = np.polyfit(x, y, 1)
    resid = y - (a + b * x)
    per_build = a + b * naux
    return {"value": 1.0 / per_build, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle.jk_df on {', '.join(str(p[0]) for p in pts)} of {naux} aux "
                      f"functions (N={n}, nocc={mol.nocc}), seeded B rows, {reps} reps each; "
                      f"t = a + b*Naux fitted and evaluated at Naux={naux}",
            "fit": {"a_s": a, "b_s_per_aux": b, "max_abs_residual_s": float(np.abs(resid).max()),
                    "points_naux_median_min_max_s": [list(p) for p in pts],
                    "seconds_per_build": per_build}}


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores: each step is a bounded
    sample (nsample of the Naux aux functions) of one Fock build of the
    workload; value = builds/s = (nsample / Naux) / seconds per step."""
    import oracle
    import workload
    mol = workload.water_cluster(args.waters)
    if rank != 0:
        return
    n = sum((s.l + 1) * (s.l + 2) // 2 for s in mol.orb)
    naux = sum((s.l + 1) * (s.l + 2) // 2 for s in mol.aux)
    nsample = 64
    B, C = _seeded_sample(n, mol.nocc, nsample)
    oracle.jk_df(B[:2], C)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.jk_df(B, C)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    per = statistics.mean(times)
    v = (nsample / naux) / per
    sample = (f"oracle.jk_df on {nsample} of {naux} aux functions (N={n}, nocc={mol.nocc}) per "
              f"step, seeded B rows; builds/s = ({nsample}/{naux}) / step time")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(mol, "mixed_" + args.prec),
            "reference_is": "the FP64 CPU oracle (oracle.jk_df), timed on the host cores",
            "step_is": f"a {nsample}/{naux} sample of one Fock build",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config(mol, prec):
    n = sum((s.l + 1) * (s.l + 2) // 2 for s in mol.orb)
    naux = sum((s.l + 1) * (s.l + 2) // 2 for s in mol.aux)
    esz = 2 if "f16" in prec else 4
    return {"workload": f"{mol.name} DF-RHF Fock build, stored B, N={n}, Naux={naux}, "
                        f"nocc={mol.nocc}", "prec": prec, "seed": len(mol.Z) // 3,
            "l2": f"inputs larger than L2 (per step: {naux * n * n * 2 * esz / 1e9:.1f} GB "
                  f"of split B shadows read by the X pass, {naux * n * (n + 1) / 2 * 8 / 1e9:.1f} GB "
                  + ("of float-pair B by the J pass)" if esz == 2 else "of FP64 B by the J pass)"),
            "parallelism": "replicas"}


def serve_leg(bqc, ctx, workload, nreq, rate, slots=8, prec=None, incremental=True,
              policy=0, budget=150 * 10 ** 9, log=None, grouped=False):
    """Submits the first `nreq` requests of the seed-2025 Poisson stream at
    their arrival times (offered `rate` req/s) to one server and waits for
    all; latency = completion - arrival (the server's submit time).  With
    grouped, the mixed-stage Fock builds of the solves in flight run as
    grouped launches."""
    stream = workload.serving_stream(nreq=nreq, rate_hz=rate)
    srv = bqc.Server(ctx, max_slots=slots, hbm_budget=budget, prec=prec, policy=policy,
                     incremental=incremental, grouped=grouped)
    t0 = time.perf_counter()
    tickets = []
    for (ta, n, rid) in stream:
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append((ta, n, srv.submit(workload.water_cluster(n, seed=rid))))
    done = {}
    while len(done) < len(tickets):
        for (ta, n, t) in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
                    if log:
                        print(f"[serve {rate} req/s] n={n} nbf={r['nbf']} status={r['status']} "
                              f"iters={r['iterations']} (mixed {r['iterations_mixed']}) "
                              f"wait={r['t_admit'] - r['t_submit']:.2f}s "
                              f"run={r['t_done'] - r['t_admit']:.2f}s", file=log, flush=True)
        time.sleep(0.02)
    wall = time.perf_counter() - t0
    gst = srv.group_stats()
    srv.close()
    lat = sorted(done[t]["t_done"] - done[t]["t_submit"] for (_, _, t) in tickets)
    q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
    out = {"offered_req_per_s": rate, "requests": len(lat), "p50_ms": q(0.5) * 1e3,
           "p99_ms": q(0.99) * 1e3, "solves_per_s": len(lat) / wall, "wall_s": wall,
           "converged": sum(1 for t in done.values() if t["status"] == 0),
           "sizes_n": [n for (_, n, _) in tickets]}
    if grouped:
        out["grouped"] = gst
    return out


def run_serve(args):
    """Continuous batching on the seeded Poisson stream (mean 20 req/s,
    n ~ U{2..48}); the first --serve-requests requests, submitted at their
    arrival times; latency = completion - arrival."""
    import torch

    import paper_2502_17963_gb300 as bqc
    import workload
    from paper_2502_17963_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    ctx = bqc.Context(0)
    stream = workload.serving_stream(nreq=args.serve_requests, rate_hz=args.serve_rate)
    out = {}
    precs = {"mixed_tf32x3": bqc.PREC_MIXED_TF32X3, "mixed_f16x3": bqc.PREC_MIXED_F16X3,
             "fp64": bqc.PREC_FP64}
    for label in args.serve_precs.split(","):
        prec = precs[label]
        policy = {"backfill": bqc.SERVE_BACKFILL, "fifo": bqc.SERVE_FIFO}[args.serve_policy]
        srv = bqc.Server(ctx, max_slots=args.serve_slots, hbm_budget=150 * 10 ** 9, prec=prec,
                         policy=policy)
        clocks = ClockSampler(gpu_index(0))
        clocks.start()
        t0 = time.perf_counter()
        tickets = []
        for (ta, n, rid) in stream:
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            mol = workload.water_cluster(n, seed=rid)
            tickets.append((ta, n, srv.submit(mol)))
        done = set()
        while len(done) < len(tickets):
            for (ta, n, t) in tickets:
                if t in done:
                    continue
                r = srv.poll(t)
                if r is not None:
                    done.add(t)
                    print(f"[serve {label}] n={n} nbf={r['nbf']} status={r['status']} "
                          f"iters={r['iterations']} (mixed {r['iterations_mixed']}) "
                          f"prio={r['priority']} wait={r['t_admit'] - r['t_submit']:.2f}s "
                          f"run={r['t_done'] - r['t_admit']:.2f}s", file=sys.stderr, flush=True)
            time.sleep(0.05)
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        lat, ok, nbf, per = [], 0, [], []
        for (ta, n, t) in tickets:
            r = srv.poll(t)
            lat.append(r["t_done"] - r["t_submit"])
            ok += r["status"] == 0
            nbf.append(r["nbf"])
            per.append([n, round(r["t_admit"] - r["t_submit"], 3), round(r["t_done"] - r["t_admit"], 3),
                        r["iterations"], r["iterations_mixed"]])
        srv.close()
        lat.sort()
        q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))]
        out[label] = {"p50_ms": q(0.5) * 1e3, "p99_ms": q(0.99) * 1e3, "solves_per_s": len(lat) / wall,
                      "converged": ok, "requests": len(lat), "wall_s": wall, "clocks": clk,
                      "offered_req_per_s": args.serve_rate,
                      "requests_n_wait_run_iters_mixed": per}
    first = args.serve_precs.split(",")[0]
    line = {"metric": "serve p50/p99 ms (DF-RHF solves, Poisson arrivals)", "value": out[first]["p99_ms"],
            "unit": "ms (p99 latency)", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
            "config": {"workload": f"Poisson {args.serve_rate} req/s, (H2O)_n n~U{{2..48}}, first "
                                   f"{args.serve_requests} of the seed-2025 stream",
                       "slots": args.serve_slots, "policy": args.serve_policy, "hbm_budget_gb": 150,
                       "prec": first}, "serve": out}
    print(json.dumps(line), flush=True)


def run_scf(args):
    """One precision-staged SCF (3xTF32 first stage, FP64 to DIIS 1e-8) from the
    core guess at --waters: wall time, Fock builds per stage, energy."""
    import torch

    import paper_2502_17963_gb300 as bqc
    import workload
    from paper_2502_17963_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    mol = workload.water_cluster(args.waters)
    ctx = bqc.Context(0)
    basis = bqc.Basis(ctx, mol)
    f16 = args.prec == "f16x3"
    prec = bqc.PREC_MIXED_F16X3 if f16 else bqc.PREC_MIXED_TF32X3
    t0 = time.perf_counter()
    df = bqc.DF(ctx, basis, mode=bqc.DF_STORED,
                keep_fp32=bqc.SHADOW_F16 if f16 else bqc.SHADOW_TF32)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    clocks = ClockSampler(gpu_index(0))
    clocks.start()
    t0 = time.perf_counter()
    r = bqc.scf_run(ctx, df, prec=prec, incremental=args.incremental)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    h = r["history"]
    nmix = sum(1 for p, _, _ in h if p != bqc.PREC_FP64)
    line = {"metric": "s per precision-staged DF-RHF SCF", "value": wall, "unit": "s",
            "n_gpus": 1, "higher_is_better": False, "dtype": f"{args.prec} then f64",
            "data": "synthetic", "fp64_stage": "incremental" if args.incremental else "full",
            "builds": r["builds"],
            "config": {"workload": f"{mol.name} staged SCF from the core guess, N={basis.nbf}, "
                                   f"Naux={basis.naux}, nocc={basis.nocc}",
                       "stage_tol": 1e-5, "diis_tol": 1e-8},
            "energy": r["energy"], "converged": r["converged"], "diis_err": r["diis_err"],
            "fock_builds": {"mixed": nmix, "fp64": len(h) - nmix},
            "switch_rule": r["switch_rule"], "switch_err": r["switch_err"],
            "history": [[p, e, en] for p, e, en in h], "setup_s": setup, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_direct(args):
    """Direct (on-the-fly) DF Fock build: s per build and its phases."""
    import torch

    import paper_2502_17963_gb300 as bqc
    import workload
    from paper_2502_17963_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    nw = args.waters if args.waters != 64 else 128
    mol = workload.water_cluster(nw)
    ctx = bqc.Context(0)
    basis = bqc.Basis(ctx, mol)
    t0 = time.perf_counter()
    df = bqc.DF(ctx, basis, mode=bqc.DF_DIRECT, aux_block=1024, keep_fp32=True)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    C = torch.linalg.qr(torch.randn((basis.nbf, basis.nocc), dtype=torch.float64,
                                    generator=torch.Generator().manual_seed(5)))[0].cuda() * 0.5
    J = torch.empty((basis.nbf, basis.nbf), dtype=torch.float64, device="cuda")
    K = torch.empty_like(J)
    df.jk(C, bqc.PREC_MIXED_TF32X3, J, K)
    torch.cuda.synchronize()
    df.timing(True)
    steps = max(1, min(args.steps, 3))
    clocks = ClockSampler(gpu_index(0))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ph = []
    for _ in range(steps):
        df.jk(C, bqc.PREC_MIXED_TF32X3, J, K)
        ph.append(df.phase_ms())
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    pm = np.mean(np.array(ph), axis=0).tolist()
    line = {"metric": "s per Fock build, direct DF", "value": ms / 1e3, "unit": "s/build",
            "n_gpus": 1, "steps": steps, "higher_is_better": False, "dtype": "f64 integrals, tf32x3",
            "data": "synthetic", "config": {"workload": f"{mol.name} direct DF, N={basis.nbf}, "
                                            f"Naux={basis.naux}, nocc={basis.nocc}, aux block 1024, "
                                            "Schwarz 1e-10"},
            "phases_ms": {"pass1_integrals_gamma_X": pm[0], "metric_solve_and_K": pm[1],
                          "pass2_integrals_J": pm[2], "prep": pm[3]},
            "setup_s": setup, "device_bytes": df.device_bytes, "clocks": clk,
            "screening": dict(zip(("triplets_considered", "triplets_kept"), df.screening()))}
    sc = line["screening"]
    sc["survival"] = sc["triplets_kept"] / max(1, sc["triplets_considered"])
    print(json.dumps(line), flush=True)


def staged_scf_check(bqc, ctx, df, torch, prec):
    """Staged SCF (mixed first stage, then the anchored incremental FP64
    stage, converged on a full FP64 build) and plain FP64 SCF from the core
    guess on one DF handle: wall times, Fock builds by kind, the stage switch
    rule, and |E_staged - E_FP64|."""
    no = df.basis.nocc
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rs = bqc.scf_run(ctx, df, prec=prec, keep_arrays=True, incremental=True)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    t0 = time.perf_counter()
    r64 = bqc.scf_run(ctx, df, prec=bqc.PREC_FP64)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    dE = abs(rs["energy"] - r64["energy"])
    return {"E_staged_Eh": rs["energy"], "E_fp64_scf_Eh": r64["energy"], "abs_dE_Eh": dE,
            "meets_1e-6_Eh": bool(dE <= 1e-6 and rs["converged"] and r64["converged"]),
            "staged": {"wall_s": ts, "fock_builds": rs["builds"], "first_stage_prec": prec,
                       "fp64_stage": "anchored incremental (final build full FP64)",
                       "converged": rs["converged"], "diis_err": rs["diis_err"],
                       "switch_rule": rs["switch_rule"], "switch_err": rs["switch_err"],
                       "stage_tol": 1e-5,
                       # per build: precision (3 split FP16, 2 split TF32, 0 full FP64,
                       # -1 incremental FP64) and the DIIS error max|e| after it
                       "history": [[int(p), float(f"{e:.3g}")] for p, e, _ in rs["history"]]},
            "fp64_scf": {"wall_s": t64, "fock_builds": len(r64["history"]),
                         "converged": r64["converged"], "diis_err": r64["diis_err"]},
            "protocol": "core-Hamiltonian guess, DIIS(8), converged at max|e| < 1e-8 and "
                        "|dE| < max(1e-10, eps*N*|E|) Eh; wall times exclude the DF setup",
            "_C": rs["C"][:, :no].contiguous()}


def run_screen_ablation(args):
    """One aux block of 1024 functions of the direct-mode integrals, computed
    with each survivor compaction (0 sorted prefix, 1 the paper's warp loop
    buffer, 2 a two-kernel global index list): CUDA-event time per variant
    (median of 3 after a warm-up), and a bitwise comparison of the outputs."""
    import torch

    import paper_2502_17963_gb300 as bqc
    import workload
    from paper_2502_17963_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    nw = args.waters if args.waters != 64 else 128
    mol = workload.water_cluster(nw)
    ctx = bqc.Context(0)
    basis = bqc.Basis(ctx, mol)
    df = bqc.DF(ctx, basis, mode=bqc.DF_DIRECT, schwarz=1e-10, aux_block=1024, keep_fp32=False)
    p1 = min(1024, basis.naux)
    outs, times = [], {}
    names = {0: "sorted_prefix", 1: "warp_loop_buffer", 2: "global_index_list"}
    stream = torch.cuda.current_stream()
    for v in range(3):
        out = torch.zeros((p1, basis.npair), dtype=torch.float64, device="cuda")
        df.int3c_screened(0, p1, v, out)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            df.int3c_screened(0, p1, v, out)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        times[names[v]] = statistics.median(ts)
        outs.append(out.cpu() if v == 0 else out)
    same = [bool(torch.equal(outs[v].cpu(), outs[0])) for v in (1, 2)]
    maxdiff = [float((outs[v].cpu() - outs[0]).abs().max()) for v in (1, 2)]
    cand, kept = df.screening()
    line = {"metric": "ms per screened 3-centre integral block", "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"{mol.name} aux functions [0, {p1}) of Naux={basis.naux}, "
                                   f"N={basis.nbf}, Schwarz 1e-10 (direct-mode block)"},
            "ms": times, "bitwise_equal_to_sorted_prefix": same,
            "max_abs_diff_to_sorted_prefix": maxdiff,
            "triplets_kept_fraction_all_aux": kept / max(1, cand),
            "speed_vs_sorted_prefix": {k: times["sorted_prefix"] / v for k, v in times.items()}}
    print(json.dumps(line), flush=True)


def run_mp2(args):
    """DF-MP2 (FP64 DFMA path) after a staged SCF: seconds, flop rate against
    the FP64 peak, and the energy."""
    import torch

    import paper_2502_17963_gb300 as bqc
    import workload
    from paper_2502_17963_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    nw = args.mp2_waters
    mol = workload.water_cluster(nw)
    ctx = bqc.Context(0)
    basis = bqc.Basis(ctx, mol)
    df = bqc.DF(ctx, basis, mode=bqc.DF_STORED, keep_fp32=bqc.SHADOW_F16)
    r = bqc.scf_run(ctx, df, prec=bqc.PREC_MIXED_F16X3, incremental=True, keep_arrays=True)
    C, eps = r["C"].contiguous(), r["eps"].contiguous()
    mp = bqc.PREC_MIXED_F16X3 if args.mp2_prec == "f16x3" else bqc.PREC_FP64
    bqc.mp2(df, C, eps, prec=mp)  # warm
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_index(0))
    clocks.start()
    t0 = time.perf_counter()
    e2 = bqc.mp2(df, C, eps, prec=mp)
    dt = time.perf_counter() - t0
    clk = clocks.stop()
    e2_64, dt64 = None, None
    if mp != bqc.PREC_FP64 and nw <= 32:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e2_64 = bqc.mp2(df, C, eps, prec=bqc.PREC_FP64)
        dt64 = time.perf_counter() - t1
    n, naux, no = basis.nbf, basis.naux, basis.nocc
    nv = r["nmo"] - no
    bi = max(1, min(16, no, int((1 << 27) ** 0.5 / max(1, nv))))
    pair_flops = 0.0
    for i0 in range(0, no, bi):
        ni = min(bi, no - i0)
        for j0 in range(0, i0 + 1, bi):
            nj = min(bi, no - j0)
            pair_flops += 2.0 * ni * nv * nj * nv * naux
    tflops = 2.0 * naux * n * n * no + 2.0 * naux * n * no * nv  # FP64 MO transform
    flops = tflops + pair_flops
    fp64_peak = 152 * 2 * 2 * 2.07e9 / 1e12  # 2 DFMA units per SM at the max SM clock
    pk, pk_src = peaks()
    if mp == bqc.PREC_FP64:
        roof = {"bound": "alu", "achieved": flops / dt / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": flops / dt / 1e12 / fp64_peak,
                "peak_source": "FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                "algorithmic_flop": flops}
    else:
        t_tr = tflops / (fp64_peak * 1e12 * 0.9)  # the FP64 transform at the DFMA rate
        t_pair = max(1e-9, dt - t_tr)
        sust = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        roof = {"bound": "tensor", "kernel": "k_gemm_nt<f16> (pair blocks, 3 products)",
                "achieved": pair_flops / t_pair / 1e12, "peak": sust, "unit": "TFLOP/s",
                "frac": pair_flops / t_pair / 1e12 / sust,
                "frac_issued": 3 * pair_flops / t_pair / 1e12 / sust,
                "note": "pair-block time = total - FP64 transform at 0.9 of the DFMA rate "
                        f"({t_tr:.2f} s estimated)", "peak_source": f"{pk_src}: bf16 sustained"}
    line = {"metric": f"s per DF-MP2 energy ({args.mp2_prec})", "value": dt, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "dtype": args.mp2_prec,
            "config": {"workload": f"{mol.name} DF-MP2 after the staged SCF, N={n}, Naux={naux}, "
                                   f"nocc={no}, nvir={nv}"},
            "e2_Eh": e2, "e2_fp64_Eh": e2_64, "fp64_s": dt64,
            "e_scf_Eh": r["energy"], "roofline": roof, "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.serve:
        return run_serve(args)
    if args.screen_ablation:
        return run_screen_ablation(args)
    if args.mp2:
        return run_mp2(args)
    if args.direct:
        return run_direct(args)
    if args.scf:
        return run_scf(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import paper_2502_17963_gb300 as bqc
    import workload
    from paper_2502_17963_gb300 import _build
    _build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    mol = workload.water_cluster(args.waters)
    ctx = bqc.Context(local)
    basis = bqc.Basis(ctx, mol)
    n, no = basis.nbf, basis.nocc
    MIX = bqc.PREC_MIXED_F16X3 if args.prec == "f16x3" else bqc.PREC_MIXED_TF32X3
    t0 = time.perf_counter()
    df = bqc.DF(ctx, basis, mode=bqc.DF_STORED,
                keep_fp32=bqc.SHADOW_F16 if args.prec == "f16x3" else bqc.SHADOW_TF32)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    scf = None
    if not args.no_scf_check:
        # the metric's accuracy condition, measured at this size: the staged
        # SCF (mixed, then FP64) against a plain FP64 SCF on the same DF
        # handle, both from the core guess; the timed builds below then run
        # at the converged occupied orbitals
        scf = staged_scf_check(bqc, ctx, df, torch, MIX)
        C = scf.pop("_C")
    else:
        # occupied orbitals of a physical state: two mixed SCF iterations from the core guess
        r = bqc.scf_run(ctx, df, prec=MIX, max_iter=2, keep_arrays=True)
        C = r["C"][:, :no].contiguous()
    J = torch.empty((n, n), dtype=torch.float64, device="cuda")
    K = torch.empty_like(J)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        df.jk(C, MIX, J, K)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_index(local))
    clocks.start()
    df.timing(True)
    phases = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        df.jk(C, MIX, J, K)
        phases.append(df.phase_ms())
    e1.record(stream)
    torch.cuda.synchronize()
    elapsed_ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    df.timing(False)
    if dist:
        elapsed_ms = max_over_ranks(elapsed_ms, dist, "cuda")
        dist.barrier()
    ms_per_step = elapsed_ms / args.steps
    value = whole_job_rate(world, args.steps, elapsed_ms * 1e-3)
    ph = np.array(phases)
    ph_mean = ph.mean(axis=0).tolist()

    tf1 = None
    if args.prec == "tf32x3":
        # single-pass TF32 (one product per term) for comparison
        df.jk(C, bqc.PREC_MIXED_TF32, J, K)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            df.jk(C, bqc.PREC_MIXED_TF32, J, K)
        a1.record(stream)
        torch.cuda.synchronize()
        tf1 = {"builds_per_s": args.steps / (a0.elapsed_time(a1) * 1e-3),
               "ms_per_build": a0.elapsed_time(a1) / args.steps}
    # plain FP64 build at the same C_occ, and the Fock-matrix difference
    J64 = torch.empty_like(J)
    K64 = torch.empty_like(J)
    fp64 = None
    if args.fp64_steps > 0:
        df.jk(C, bqc.PREC_FP64, J64, K64)  # warm
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.fp64_steps + 1)]
        ev[0].record(stream)
        for k in range(args.fp64_steps):
            df.jk(C, bqc.PREC_FP64, J64, K64)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        per_step = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.fp64_steps)]
        fms = statistics.median(per_step)
        D = C @ C.T  # E = sum D (H + F) + E_nn, so a build's energy error is sum D dF
        if tf1 is not None:
            df.jk(C, bqc.PREC_MIXED_TF32, J, K)
            dF1 = 2.0 * (J - J64) - (K - K64)
            tf1["max_abs_dF_vs_fp64"] = dF1.abs().max().item()
            tf1["dE_vs_fp64_Eh"] = (D * dF1).sum().item()
        df.jk(C, MIX, J, K)
        dFm = 2.0 * (J - J64) - (K - K64)
        dF = dFm.abs().max().item()
        fp64 = {"builds_per_s": 1e3 / fms, "ms_per_build": fms, "steps": args.fp64_steps,
                "ms_per_build_median_min_max": [fms, min(per_step), max(per_step)],
                "max_abs_dF_mixed_vs_fp64": dF, "dE_mixed_vs_fp64_Eh": (D * dFm).sum().item(),
                "density": "converged SCF" if scf else "two mixed SCF iterations",
                "note": "error of ONE mixed build at this density (E is linear in dF); the "
                        "<=1e-6 Eh condition applies to the staged SCF's final energy "
                        "(staged_scf)",
                "speedup_mixed_over_fp64": fms / ms_per_step}

    # the Coulomb matrix alone by the two passes over B (w = B.D, J = sum w_P
    # B_P): FP64 FMAs vs float-float on the FP32 pipe, on achieved HBM GB/s
    coul = None
    if args.prec == "f16x3":
        Dm = C @ C.T
        Jc = torch.empty_like(J)
        coul = {}
        for label, var in (("fp64", bqc.COULOMB_FP64), ("float_float", bqc.COULOMB_FF)):
            df.coulomb(Dm, var, Jc)
            torch.cuda.synchronize()
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(5):
                df.coulomb(Dm, var, Jc)
            c1.record(stream)
            torch.cuda.synchronize()
            cms = c0.elapsed_time(c1) / 5
            cbytes = 2.0 * basis.naux * n * (n + 1) / 2 * 8  # two reads of the packed B
            coul[label] = {"ms": cms, "gbs": cbytes / (cms * 1e-3) / 1e9,
                           "frac_of_hbm": cbytes / (cms * 1e-3) / 1e9 / peaks()[0]["hbm_gbs"]}
        coul["bytes_per_call"] = 2.0 * basis.naux * n * (n + 1) / 2 * 8
        coul["note"] = ("bqc_df_coulomb at the benchmark density: w = B.D then J = sum_P w_P B_P, "
                        "each pass one read of the packed B (8 bytes per element: FP64, or the "
                        "float-pair copy); CUDA events, mean of 5, inputs larger than L2")

    # end to end through the C ABI with host buffers (H2D of C_occ, D2H of J, K)
    e2e = None
    if not args.no_e2e:
        Ch = torch.empty((n, no), dtype=torch.float64, pin_memory=True)
        Ch.copy_(C.cpu())
        Jh = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        Kh = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        Cn, Jn, Kn = Ch.numpy(), Jh.numpy(), Kh.numpy()
        for _ in range(2):
            df.jk_host(Cn, MIX, Jn, Kn)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            df.jk_host(Cn, MIX, Jn, Kn)
        dt = time.perf_counter() - t0
        if dist:
            dt = max_over_ranks(dt, dist, "cuda")
        e2e = {"value": whole_job_rate(world, args.steps, dt), "unit": UNIT,
               "h2d_bytes_per_step": n * no * 8, "d2h_bytes_per_step": 2 * n * n * 8}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    pk, pk_src = peaks()
    naux = basis.naux
    xalg = 2.0 * naux * n * n * no          # algorithmic flops of one X pass (2 Naux N^2 nocc)
    xissued = 3 * xalg                      # the split issues three products per term
    xs = ph_mean[0] * 1e-3
    sust = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    if args.prec == "f16x3":
        esz = 2
        peak = sust  # dense fp16 and bf16 run at the same tensor rate
        kern = "k_xpass_mc<XN> (X = B C, split FP16, 3 products, two-CTA clusters)"
        peak_src = f"{pk_src}: bf16 sustained (the fp16 dense rate equals bf16's)"
        xb16 = naux * n * n * 2 * esz + naux * n * no * 2 * esz
        traffic = XPASS_F16_TRAFFIC_RATIO * xb16
        traffic_src = ("ncu dram__bytes_read+write / algorithmic bytes of k_xpass_mc at (H2O)_20 "
                       f"({XPASS_F16_TRAFFIC_RATIO}, one aux piece) x this X pass's bytes "
                       f"({xb16:.4g} B, all four pieces)")
    else:
        esz = 4
        peak = sust * TF32_OVER_BF16
        kern = "k_xpass<tf32,XN,3,0> (X = B C, split TF32, 3 products)"
        peak_src = f"{pk_src}: bf16 sustained x nominal tf32/bf16 (1.1/2.25)"
        traffic = None  # the kernel changed (TMEM chain sums) since its (H2O)_16 capture
        traffic_src = ("none: the TF32 X pass changed since its ncu capture "
                       f"(ratio {XPASS_TRAFFIC_RATIO} then)")
    xbytes = naux * n * n * 2 * esz + naux * n * no * 2 * esz  # hi+lo B shadows read, hi+lo X written
    achieved = xalg / xs / 1e12
    roofline = {"bound": "tensor", "kernel": kern,
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "frac_issued": xissued / xs / 1e12 / peak,
                "traffic": traffic, "traffic_source": traffic_src,
                "bytes_per_launch": xbytes,
                "peak_source": peak_src,
                "algorithmic_per_launch": f"2*Naux*N^2*nocc = {xalg:.4g} flop (frac); "
                                          f"3 products issued = {xissued:.4g} flop (frac_issued)"}
    tf32_peak = peak
    jbytes = naux * n * (n + 1) / 2 * 8  # J pass: one read of the packed FP64 B
    kflops = n * n * naux * no           # SYRK half (algorithmic; 3 products issued)
    extra = {
        "coulomb": coul,
        "phases_ms": {"x_pass": ph_mean[0], "j_pass": ph_mean[1], "k_syrk": ph_mean[2],
                      "prep": ph_mean[3]},
        "j_pass_gbs_beside_syrk": jbytes / (ph_mean[1] * 1e-3) / 1e9,
        "j_note": ("J pass (split-FP16 build: float-float FMAs on the FP32 pipe over the "
                   "float-pair copy of B, in four aux pieces on a side stream beside the X-pass "
                   "pieces and the SYRK), timed from the end of the first X piece to its end, so "
                   "the rate includes the contention; alone see coulomb"),
        "k_syrk_tflops": kflops / (ph_mean[2] * 1e-3) / 1e12,
        "k_syrk_frac": kflops / (ph_mean[2] * 1e-3) / 1e12 / tf32_peak,
        "tensor_peak_tflops": tf32_peak,
        "k_syrk_frac_issued": 3 * kflops / (ph_mean[2] * 1e-3) / 1e12 / tf32_peak,
        "staged_scf": scf,
        "setup_s": setup_s,
        "fp64": fp64,
        "tf32_single_pass": tf1,
    }
    # kernels of one build: split-FP16 = C split (3), four X-pass pieces with
    # their w reductions (8), four float-float J pieces and the unpack (5), the
    # SYRK and its reduction (2); split-TF32 = C split, X pass, w, J, unpack,
    # SYRK, reduction
    launches_per_build = 18 if args.prec == "f16x3" else 7
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": config(mol, "mixed_" + args.prec), "roofline": roofline,
            "gpu_launches": launches_per_build * args.steps, "clocks": clk, "e2e": e2e}
    line.update(extra)
    if not args.no_baseline and world >= 1:
        line["cpu_baseline"] = cpu_baseline(mol)
    if args.serve_leg > 0 and world == 1:
        # serving on a bounded prefix of the seed-2025 stream, after the
        # (H2O)_64 handle is released (the 150 GB arena would not fit beside it)
        df.close()
        del J, K, J64, K64, C
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        sv = {}
        for rate in (args.serve_rate, args.serve_low_rate):
            sv[f"{rate:g}_req_per_s"] = serve_leg(bqc, ctx, workload, args.serve_leg, rate,
                                                  prec=MIX, log=sys.stderr)
        if MIX == bqc.PREC_MIXED_F16X3:
            # the same offered load with the mixed-stage builds of the solves
            # in flight batched into grouped launches
            sv[f"{args.serve_rate:g}_req_per_s_grouped"] = serve_leg(
                bqc, ctx, workload, args.serve_leg, args.serve_rate, prec=MIX, log=sys.stderr,
                grouped=True)
        line["serve"] = {"prec": args.prec + " staged, incremental FP64 stage", "slots": 8,
                         "hbm_budget_gb": 150, "policy": "backfill",
                         "workload": f"first {args.serve_leg} requests of the seed-2025 Poisson "
                                     "stream, (H2O)_n with n ~ U{2..48}, submitted at their "
                                     "arrival times scaled to each offered rate",
                         "legs": sv}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
