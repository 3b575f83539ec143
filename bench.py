"""PT2 throughput benchmark (terms/s) of the GB300 path, one JSON line.

Headline workload: PT2 at "trillions of contributions" scale, 24 electrons
(12 alpha, 12 beta) in 60 orbitals, N_det = 1,000,000 reference determinants
up to quadruple excitations, seeded synthetic FP64 integrals: 4.818e11
generated terms per complete solve, streamed through HBM in memory-bounded
passes.  The solve is split into SLICES = 20 contiguous slices of the 4096
alpha-hash classes (non-overlapping, complete constraint classes of
Algorithm 2); a step is the complete path (work list, every pass of generate /
tile sort-reduce / filter / energy, final sum) over one slice, on inputs
already resident in device memory.  Step k takes slice k mod 20, warm-up steps
included, so any 20 consecutive steps are exactly one complete solve, whose
E2 is the sum of their slice energies.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 (under torchrun) every rank solves its own replica of the
workload ("replicas only": the path needs no exchange between GPUs); value
is the sum of terms over ranks divided by the slowest rank's time.
--impl reference times the CPU oracle on a bounded sample of the same
workload on all host cores instead.
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PT2 terms/sec"
UNIT = "terms/s"
WORKLOAD = ("plain PT2 at trillions-of-contributions scale: 24 electrons (12a,12b) in 60 orbitals, "
            "N_det=1000000 (HF + excitations up to quadruples), seeded synthetic FP64 integrals")
SLICES = 20            # alpha-class slices of one complete solve (one per step)
E2E_SLICES = 4         # slices of the end-to-end measurement (one load, these slices, one unload)
CPU_DETS_ALL = 200     # reference determinants of the all-cores oracle sample
CPU_DETS_ONE = 20      # reference determinants of the single-thread oracle sample
REF_DETS_STEP = 40     # reference determinants per step of the reference arm


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(name="million", n_det=None):
    from paper_1808_02049_gb300 import inputs

    return inputs.make_workload(name, n_det=n_det or None)


def workload_name(n_det):
    if not n_det:
        return WORKLOAD
    return WORKLOAD.replace("N_det=1000000", f"N_det={n_det} (reduced case)")


def oracle_all_cores(s, r, e0, n_dets, cores):
    """The oracle on the first n_dets reference determinants, its constraint
    classes alpha % m == k (m prime, several per core) solved by `cores` host
    threads (the C oracle releases the interpreter lock); the classes
    partition the sum, so the class results add up to the sample's PT2."""
    import oracle

    oracle.build()
    m = 4 * cores + 1
    while any(m % q == 0 for q in range(2, int(m ** 0.5) + 1)):
        m += 1
    keys, coef = r.keys[: 2 * n_dets], r.coef[:n_dets]
    t = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        res = list(ex.map(lambda k: oracle.pt2(s.h, s.eri, keys, coef, e0, constraint=(m, k)), range(m)))
    dt = time.perf_counter() - t
    return sum(x["n_terms"] for x in res), sum(x["e2"] for x in res), dt, m


def cpu_baseline(s, r, e0):
    """The oracle as it stands on the host cores: all cores on a sample of
    CPU_DETS_ALL determinants, one thread on CPU_DETS_ONE."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    terms_all, _, dt_all, m = oracle_all_cores(s, r, e0, CPU_DETS_ALL, cores)
    t = time.perf_counter()
    one = oracle.pt2(s.h, s.eri, r.keys[: 2 * CPU_DETS_ONE], r.coef[:CPU_DETS_ONE], e0)
    dt_one = time.perf_counter() - t
    return {"value": terms_all / dt_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": one["n_terms"] / dt_one,
            "sample": f"PT2 of the first {CPU_DETS_ALL} reference determinants of the workload "
                      f"({terms_all} terms, {dt_all:.1f} s on {cores} threads: constraint classes alpha % {m}); "
                      f"single thread: the first {CPU_DETS_ONE} ({one['n_terms']} terms, {dt_one:.1f} s)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(), f"pt2_bench_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_fleet(ctx, n=64):
    """The 64 uneven instances of the batched workload, loaded and resident."""
    from paper_1808_02049_gb300 import inputs

    fleet = []
    for k in range(n):
        prm = inputs.batch_instance_params(k)
        s, r = inputs.make_instance(prm)
        sid = ctx.load_system(s.h, s.eri)
        e0 = float(ctx.diagonal(sid, r.keys).min() - 0.1)
        fleet.append(dict(sid=sid, rid=ctx.load_reference(sid, r.keys, r.coef, e0), prm=prm))
    return fleet


SAME = ("e2", "n_terms", "n_unique", "n_in_ref", "n_external", "digest_sum", "digest_xor", "n_pos_denom")


def timed_run(ctx, rid, **kw):
    t = time.perf_counter()
    res = ctx.run(rid, **kw)
    return res, time.perf_counter() - t


def best_of(ctx, rid, reps, **kw):
    ctx.run(rid, **kw)  # warm-up
    best, res = None, None
    for _ in range(reps):
        res, dt = timed_run(ctx, rid, **kw)
        best = dt if best is None or dt < best else best
    return res, best


def bench_large(ctx, reps=2):
    """The one-large-solve workload (20e in 40 orbitals, N_det = 100,000,
    1.2975e10 terms) as a complete solve per call: wall time of the blocking
    call (best of `reps`) and the phase split of a profiled run."""
    s, r = workload("large")
    sid = ctx.load_system(s.h, s.eri)
    e0 = float(ctx.diagonal(sid, r.keys).min() - 0.1)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    res, dt = best_of(ctx, rid, reps)
    ctx.run(rid, profile=True)
    ph, _ = ctx.phase_times()
    out = {"workload": "plain PT2, one large solve: 20 electrons (10a,10b) in 40 orbitals, N_det=100000",
           "terms": res["n_terms"], "ms_per_solve": dt * 1e3, "terms_per_s": res["n_terms"] / dt,
           "passes": res["n_passes"], "e2": res["e2"],
           "phase_ms": {k: round(v, 3) for k, v in ph.items()},
           "tile_kernel_gbs": res["n_terms"] * 32 / (ph["tile_sort_reduce"] * 1e-3) / 1e9,
           "timing": "wall time of the blocking C-ABI call, best of %d" % reps}
    return sid, rid, res, dt, out


def bench_cutoff(ctx, rid, exact, cut=1e-8):
    """The paper's numerator cutoff on slices of the headline workload: the
    slices' exact solves (timed in the measured steps) against the same
    slices with contributions |c_i H_ai| < cut dropped before they get a
    record (wall time of the blocking call)."""
    ks = sorted(exact)[:2]
    t_ex = sum(exact[k][1] for k in ks)
    res, t_ct = [], 0.0
    for k in ks:
        ctx.run(rid, class_slice=(k, SLICES), cutoff=cut)  # warm-up
        r, dt = timed_run(ctx, rid, class_slice=(k, SLICES), cutoff=cut)
        res.append(r)
        t_ct += dt
    ctx.run(rid, class_slice=(ks[0], SLICES), cutoff=cut, profile=True)
    ph, _ = ctx.phase_times()
    ex_terms = sum(exact[k][0]["n_terms"] for k in ks)
    ct_terms = sum(r["n_terms"] for r in res)
    return {"cutoff": cut, "slices": [f"{k}/{SLICES}" for k in ks], "ms_exact": t_ex * 1e3, "ms_cutoff": t_ct * 1e3,
            "speedup": t_ex / t_ct, "phase_ms_cutoff_first_slice": {k: round(v, 3) for k, v in ph.items()},
            "terms_exact": ex_terms, "terms_kept": ct_terms, "kept_fraction": ct_terms / ex_terms,
            "external_exact": sum(exact[k][0]["n_external"] for k in ks),
            "external_kept": sum(r["n_external"] for r in res),
            "delta_e2": sum(r["e2"] for r in res) - sum(exact[k][0]["e2"] for k in ks)}


def bench_hashed_keys(ctx, rid, exact):
    """Keys of a tile identified by a 54-bit hash (the hashing section) on two
    slices of the headline workload, against the same slices' timed exact
    solves: time, and whether the hash merged different keys."""
    ks = sorted(exact)[:2]
    t_ex = sum(exact[k][1] for k in ks)
    t_h, res = 0.0, []
    for k in ks:
        ctx.run(rid, class_slice=(k, SLICES), hashed_keys=True)
        r, dt = timed_run(ctx, rid, class_slice=(k, SLICES), hashed_keys=True)
        res.append(r)
        t_h += dt
    same = all(r["e2"] == exact[k][0]["e2"] and r["n_external"] == exact[k][0]["n_external"]
               and r["digest_sum"] == exact[k][0]["digest_sum"] for r, k in zip(res, ks))
    return {"slices": [f"{k}/{SLICES}" for k in ks], "ms_exact": t_ex * 1e3, "ms_hashed": t_h * 1e3,
            "speedup": t_ex / t_h, "merged_records": sum(r["n_hash_collisions"] for r in res),
            "identical_to_exact": bool(same)}


def bench_subtraction(ctx, rid, exact):
    """Duplicate subtraction on slices of the headline workload against the
    explicit filter (timed in the measured steps).  The synthetic reference is
    not an eigenvector of H in its space, so the energies differ by the
    residual; their equality for eigenvector references is a parity test."""
    ks = sorted(exact)[:2]
    t_f = sum(exact[k][1] for k in ks)
    t_s = 0.0
    for k in ks:
        ctx.run(rid, class_slice=(k, SLICES), subtract_ref=True)
        _, dt = timed_run(ctx, rid, class_slice=(k, SLICES), subtract_ref=True)
        t_s += dt
    return {"slices": [f"{k}/{SLICES}" for k in ks], "ms_filtered": t_f * 1e3, "ms_subtracted": t_s * 1e3,
            "speedup": t_f / t_s,
            "note": "timing only: the synthetic reference is not an eigenvector, so E2 differs"}


def bench_triplets(ctx, reps=3):
    """The small workload (4+4 electrons in 16 orbitals, 1,000 determinants)
    solved as the sum of its triplet constraints, one run per triplet T (the
    "Triplet constraints" section: every run regenerates the terms of all
    determinants and keeps those whose three highest occupied alpha orbitals
    are T, with Algorithm 3 for the alpha-alpha doubles), against one run whose
    passes are ranges of alpha-hash classes (wall time of the blocking calls)."""
    import itertools

    s, r = workload("small")
    sid = ctx.load_system(s.h, s.eri)
    e0 = float(ctx.diagonal(sid, r.keys).min() - 0.1)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    try:
        full, t_full = best_of(ctx, rid, reps)
        masks = [sum(1 << q for q in o) for o in itertools.combinations(range(16), 3)]
        for T in masks[:20]:
            ctx.run(rid, top_alpha=T)  # warm-up
        t0 = time.perf_counter()
        parts = [ctx.run(rid, top_alpha=T) for T in masks]
        t_trip = time.perf_counter() - t0
    finally:
        ctx.unload(rid)
        ctx.unload(sid)
    return {"workload": "small: 4+4 electrons in 16 orbitals, N_det=1000", "triplets": len(masks),
            "nonempty_triplets": sum(1 for p in parts if p["n_terms"]),
            "ms_hash_classes": t_full * 1e3, "ms_all_triplets": t_trip * 1e3, "ratio": t_trip / t_full,
            "terms": full["n_terms"], "terms_sum_triplets": sum(p["n_terms"] for p in parts),
            "e2_rel_diff": abs(sum(p["e2"] for p in parts) - full["e2"]) / abs(full["e2"]),
            "note": "per-constraint regeneration: each triplet run enumerates every determinant's excitations"}


def bench_spin_symmetric(ctx, reps=2):
    """The 40-orbital system with a reference closed under alpha <-> beta
    exchange (100,000 determinants with their mirrors, equal coefficients):
    the ordinary solve against the spin-flip symmetric one, which generates,
    sorts and reduces only the alpha' >= beta' half (best of `reps` each)."""
    from paper_1808_02049_gb300 import inputs

    w = inputs.WORKLOADS["large"]
    seed = inputs.workload_seed(w["seed_index"])
    s = inputs.make_integrals(w["n_orb"], seed)
    r = inputs.make_symmetric_reference(w["n_orb"], w["n_elec_per_spin"], w["n_det"], w["max_level"], seed + 1)
    sid = ctx.load_system(s.h, s.eri)
    e0 = float(ctx.diagonal(sid, r.keys).min() - 0.1)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    try:
        full, tf = best_of(ctx, rid, reps)
        sym, ts = best_of(ctx, rid, reps, spin_symmetric=True)
    finally:
        ctx.unload(rid)
        ctx.unload(sid)
    return {"workload": "20e in 40 orbitals, symmetric reference N_det=100000 (mirrors included)",
            "ms_full": tf * 1e3, "ms_symmetric": ts * 1e3, "speedup": tf / ts,
            "terms_full": full["n_terms"], "terms_symmetric": sym["n_terms"],
            # the full solve's terms over the symmetric solve's time
            "equivalent_terms_per_s": full["n_terms"] / ts,
            "e2_full": full["e2"], "e2_symmetric": sym["e2"],
            "e2_rel_diff": abs(sym["e2"] - full["e2"]) / abs(full["e2"])}


def bench_batched(ctx, fleet, reps):
    """64 instances: one captured batch (autotuned) against pt2_run of each
    instance one after the other (wall time of the blocking calls)."""
    for x in fleet:  # warm-up, and each instance's result alone
        x["alone"], _ = timed_run(ctx, x["rid"])
    serial = []
    for _ in range(reps):
        t = 0.0
        for x in fleet:
            _, dt = timed_run(ctx, x["rid"])
            x["alone_s"] = dt
            t += dt
        serial.append(t)
    ids = [x["rid"] for x in fleet]
    t0 = time.perf_counter()
    bid = ctx.batch_create(ids, autotune=True)
    create_s = time.perf_counter() - t0
    try:
        info = ctx.batch_info(bid)
        res = ctx.batch_run(bid, len(ids))  # warm-up replay
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            res = ctx.batch_run(bid, len(ids))
            times.append(time.perf_counter() - t0)
    finally:
        ctx.batch_destroy(bid)
    terms = sum(x["alone"]["n_terms"] for x in fleet)
    identical = all(all(g[k] == x["alone"][k] for k in SAME) for g, x in zip(res, fleet))
    d_e2 = max(abs(g["e2"] - x["alone"]["e2"]) for g, x in zip(res, fleet))
    tb, ts = min(times), min(serial)
    return {"workload": "64 independent instances, n_orb U{16..40}, 4-10 electrons per spin, "
                        "N_det log-uniform in [1e3, 5e4], seeded synthetic FP64 integrals",
            "terms": terms, "steps": info["steps"], "gpu_launches": info["launches"],
            "batched_terms_per_s": terms / tb, "batched_s": tb,
            "serial_terms_per_s": terms / ts, "serial_s": ts, "speedup_vs_serial": ts / tb,
            "capture_and_autotune_s": create_s, "max_abs_dE2_vs_alone": d_e2,
            "bit_identical_to_alone": identical,
            "timing": "wall time of the blocking C-ABI calls, best of %d" % reps}


def bench_served(ctx, fleet, big, n_req, load, seed=20185000):
    """Poisson stream of solves: 90% instances of the batched workload, 10% the
    one-large-solve workload.  Served: every request submitted at its arrival
    time to the continuous-batching engine (pt2_submit), latency = submission
    to completion.  Plain: the same arrivals run first-come first-served by
    pt2_run in one host thread (a request starts when it has arrived and the
    previous one has finished), latency = arrival to completion."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pool = [(x["rid"], x["alone"], x["alone_s"]) for x in fleet]
    reqs = [big if rng.random() < 0.1 else pool[int(rng.integers(len(pool)))] for _ in range(n_req)]
    mean_service = float(np.mean([r[2] for r in reqs]))
    rate = load / mean_service  # offered load relative to the plain path's capacity
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    arrivals -= arrivals[0]
    # served
    tickets = []
    t0 = time.perf_counter()
    for (rid, _, _), ta in zip(reqs, arrivals):
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append((ctx.submit(rid), time.perf_counter() - t0))
    lat, done, identical, d_e2 = [], [], True, 0.0
    for (t, ts), (_, alone, _) in zip(tickets, reqs):
        got = ctx.wait(t, timeout_s=3600)
        lat.append(got["seconds"])
        done.append(ts + got["seconds"])
        identical &= all(got[k] == alone[k] for k in SAME)
        d_e2 = max(d_e2, abs(got["e2"] - alone["e2"]))
    terms = sum(r[1]["n_terms"] for r in reqs)
    span = max(done)
    # plain: one host thread, pt2_run in arrival order
    plat, pdone = [], []
    t0 = time.perf_counter()
    for (rid, _, _), ta in zip(reqs, arrivals):
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ctx.run(rid)
        tc = time.perf_counter() - t0
        plat.append(tc - ta)
        pdone.append(tc)
    pspan = max(pdone)
    return {"workload": f"{n_req} requests, Poisson arrivals at {rate:.2f}/s "
                        f"({load:.2f}x the plain path's capacity); 90% batched-workload instances, "
                        "10% the one-large-solve workload",
            "requests": n_req, "terms": terms,
            "served_terms_per_s": terms / span, "plain_terms_per_s": terms / pspan,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "plain_p50_s": float(np.percentile(plat, 50)), "plain_p99_s": float(np.percentile(plat, 99)),
            "max_abs_dE2_vs_alone": d_e2, "bit_identical_to_alone": bool(identical),
            "plain": "measured: first-come first-served pt2_run of the same arrivals in one host thread"}


# DRAM bytes per term of the two large kernels from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum over the records of the
# captured launch; summaries under profiles/), valid only for the kernel
# source they were taken on.
PROFILED_TRAFFIC = {
    # code hash (kernel_sources_sha256) of the captured source; pt2_kernels.cu's file sha256 at capture began 75947701
    "kernels_sha256": "96533fcab6611371da770b2a79168fbacaec410796a262b37371bde2b538fe83",
    "tile_kernel": (1.444991e9 + 3.737088e6) / 45_176_097,     # 32.07 B per term
    "gen_kernel<Emit>": (0.172486e9 + 1.392777e9) / 45_176_097,  # 34.65 B per term
}


def kernel_code_sha256(text):
    """sha256 of the kernel source with // comments and blank space removed:
    the code the capture measured, whatever its comments say."""
    import hashlib
    import re

    lines = (re.sub(r"//.*$", "", ln).strip() for ln in text.splitlines())
    return hashlib.sha256("\n".join(ln for ln in lines if ln).encode()).hexdigest()


def kernel_sources_sha256():
    """kernel_code_sha256 of the kernels and the header of their constants."""
    csrc = os.path.join(ROOT, "paper_1808_02049_gb300", "csrc")
    text = "\n".join(open(os.path.join(csrc, f)).read() for f in ("pt2_kernels.cu", "pt2_internal.cuh"))
    return kernel_code_sha256(text)


def profiled_traffic_per_term(kernel):
    """Bytes per term from the capture, or None if the kernel code changed since."""
    try:
        sha = kernel_sources_sha256()
    except OSError:
        return None
    if sha != PROFILED_TRAFFIC["kernels_sha256"]:
        return None
    return PROFILED_TRAFFIC.get(kernel)


def replica_totals(elapsed, units, device):
    """Whole-job figures of N independent replicas: the slowest rank's time
    and the units all ranks processed (one all-reduce each; no-op alone)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed), float(units)
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    s, r = workload("million", args.n_det)
    oracle.build()
    e0 = oracle.e0_of(s.h, s.eri, r.keys)
    cores = os.cpu_count() or 1
    n = REF_DETS_STEP
    for _ in range(args.warmup):
        oracle_all_cores(s, r, e0, 4, cores)
    terms, dt = 0, 0.0
    for _ in range(args.steps):
        t_, _, d_, m = oracle_all_cores(s, r, e0, n, cores)
        terms += t_
        dt += d_
    value = terms / dt
    sample = (f"bounded sample per step: PT2 of the first {n} reference determinants "
              f"({terms // args.steps} terms) on {cores} host threads (constraint classes alpha % {m})")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args.n_det), "sample": sample, "l2": "CPU run"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    from paper_1808_02049_gb300 import build, pt2

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build_library()
    s, r = workload("million", args.n_det)
    ctx = pt2.Context(local)
    sid = ctx.load_system(s.h, s.eri)
    e0 = float(ctx.diagonal(sid, r.keys).min() - 0.1)
    rid = ctx.load_reference(sid, r.keys, r.coef, e0)
    print(f"[bench] device memory: {ctx.memory_info()}", file=sys.stderr)
    stream = torch.cuda.ExternalStream(ctx.stream, device=local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    M = SLICES
    for k in range(args.warmup):
        ctx.run(rid, class_slice=(k % M, M), profile=True)
    # timed region: K slices, L2 flushed between them, CUDA events on the library stream
    sampler = ClockSampler(local)
    sampler.start()
    step_ms, phases, launches, results, passes = [], {}, 0, [], 0
    per_slice = {}
    barrier()
    torch.cuda.synchronize()
    for k in range(args.warmup, args.warmup + args.steps):
        flush.random_(0, 255)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        res = ctx.run(rid, class_slice=(k % M, M), profile=True)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        step_ms.append(ms)
        ph, nl = ctx.phase_times()
        for key, v in ph.items():
            phases[key] = phases.get(key, 0.0) + v
        launches += nl
        passes += res["n_passes"]
        results.append(res)
        per_slice[k % M] = (res, ms * 1e-3)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    total_ms = float(sum(step_ms))
    terms = sum(x["n_terms"] for x in results)
    total_ms_all, terms_all = replica_totals(total_ms, terms, f"cuda:{local}")

    # end to end through the C ABI with host buffers: load the system and the
    # reference from host memory, solve E2E_SLICES slices, read each result
    # back, unload; the input bytes are copied once per E2E_SLICES steps
    h2d = s.h.nbytes + s.eri.nbytes + r.keys.nbytes + r.coef.nbytes
    d2h = 4096 * 8 + 256
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_terms = 0
    sid2 = ctx.load_system(s.h, s.eri)
    rid2 = ctx.load_reference(sid2, r.keys, r.coef, e0)
    for k in range(E2E_SLICES):
        out = ctx.run(rid2, class_slice=(k, M))
        e2e_terms += out["n_terms"]
    ctx.unload(rid2)
    ctx.unload(sid2)
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s, e2e_terms = replica_totals(e2e_s, e2e_terms, f"cuda:{local}")

    extra = {}
    if rank == 0 and not args.no_batch:
        extra["cutoff"] = bench_cutoff(ctx, rid, per_slice)
        extra["subtraction"] = bench_subtraction(ctx, rid, per_slice)
        extra["hashed_keys"] = bench_hashed_keys(ctx, rid, per_slice)
        lsid, lrid, lres, lsec, extra["large"] = bench_large(ctx)
        extra["spin_symmetric"] = bench_spin_symmetric(ctx)
        extra["triplets"] = bench_triplets(ctx)
        fleet = load_fleet(ctx)
        extra["batched"] = bench_batched(ctx, fleet, reps=2)
        if args.served_requests > 0:
            extra["served"] = bench_served(ctx, fleet, (lrid, lres, lsec), args.served_requests,
                                           args.served_load)

    if rank == 0:
        value = terms_all / (total_ms_all * 1e-3)
        peaks = measured_peaks()
        # dominant kernel and its roofline: algorithmic bytes (32 B per record
        # written by the emission or read by the tile kernel) over the
        # kernel's device time, summed over the passes of the timed steps
        dom = max(("emit", "tile_sort_reduce"), key=lambda k: phases.get(k, 0.0))
        bytes_per_term = 32
        achieved = terms * bytes_per_term / (phases[dom] * 1e-3) / 1e9
        peak = peaks["hbm_gbs"] if peaks else 6800.0
        kname = {"emit": "gen_kernel<Emit>", "tile_sort_reduce": "tile_kernel"}[dom]
        tpt = profiled_traffic_per_term(kname)
        other = "tile_sort_reduce" if dom == "emit" else "emit"
        roof = {"kernel": kname,
                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": None if tpt is None else tpt * terms / passes,
                "traffic_note": "DRAM bytes per launch (one pass) from an ncu capture of the same kernel code, "
                                "scaled by records; null when the kernel changed since the capture",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_term": bytes_per_term,
                "launches": passes,
                "phase_ms_per_step": {k: round(v / args.steps, 3) for k, v in phases.items()},
                "second_kernel": {"kernel": {"emit": "gen_kernel<Emit>", "tile_sort_reduce": "tile_kernel"}[other],
                                  "achieved": terms * bytes_per_term / (phases[other] * 1e-3) / 1e9,
                                  "frac": terms * bytes_per_term / (phases[other] * 1e-3) / 1e9 / peak},
                # the path against the floor of a global-memory sort (write 24 B,
                # permute 48 B, read 24 B per term)
                "path": {"bytes_per_term": 96, "achieved": value / world * 96 / 1e9,
                         "frac": value / world * 96 / 1e9 / peak}}
        covered = sorted(per_slice) == list(range(M))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(args.n_det),
                           "step": f"one of {M} alpha-class slices of the solve (step k: slice k mod {M}); "
                                   f"{M} consecutive steps are one complete solve",
                           "terms_timed": terms, "passes_timed": passes,
                           "complete_solves_timed": round(args.steps / M, 3),
                           "e2_complete_solve": sum(per_slice[k][0]["e2"] for k in range(M)) if covered else None,
                           "terms_complete_solve": sum(per_slice[k][0]["n_terms"] for k in range(M)) if covered
                           else None,
                           "l2": "inputs larger than L2 (32-byte records, up to 64 GiB per pass, stream through "
                                 "HBM) and a 256 MB L2 flush between steps",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roof,
                "clocks": clocks,
                "e2e": {"value": e2e_terms / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d // E2E_SLICES,
                        "d2h_bytes_per_step": d2h,
                        "note": f"one load of system and reference from host memory, {E2E_SLICES} slices solved "
                                "and read back, one unload; input bytes per step = inputs / slices"},
                "gpu_launches": launches}
        line.update(extra)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(s, r, e0)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=SLICES)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the secondary measurements (cutoff, subtraction, large, spin, batched, served)")
    ap.add_argument("--n-det", type=int, default=0,
                    help="reference size of the headline workload (0: 1000000); smaller values give the "
                         "reduced cases used for profiling")
    ap.add_argument("--served-requests", type=int, default=1000)
    ap.add_argument("--served-load", type=float, default=1.5,
                    help="offered load of the served stream relative to the plain path's capacity")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
