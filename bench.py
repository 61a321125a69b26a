#!/usr/bin/env python
"""Benchmark: sphere-steps/s of the 100,000-sphere self-gravitating collapse.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (synthetic, seeded): 100,000 spheres bonded into 30,787 rigid
aggregates drawn uniformly from dumbbell / 3-rod / tetrahedron / square,
radii lognormal (median 5 m, sigma 0.2, per aggregate), COMs uniform in a
2 km ball at rest, spring-dashpot contacts (max overlap ~1% R, e = 0.5,
mu_s = 0.5, mu_r = 0.1), Plummer-softened direct-sum self-gravity
(eps = 0.5 m), h = t_contact / 50.  One step = the whole per-step path
(kick/drift/rotation, expansion, cell sort, contact pass, gravity,
aggregate reduction, closing kick) as one CUDA-graph launch.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the library's stream, with a 512 MiB write between steps to flush L2 (the
working set, ~40 MB, would otherwise stay in the 129 MB L2).  The gravity
kernel is timed by event nodes inside the same graph launches.  With N GPUs
(torchrun), each rank runs an independent replica (seed = rank); the job
value is all spheres x steps / the slowest rank's time.

One JSON line on rank 0.  Extra keys: fp64_path (the all-FP64 GPU path on
the same workload), roofline_contact (the contact pass on a 1M-sphere dense
lattice), batched (256 piles in one graph launch vs one pile at a time),
serving_config5 (p50/p99 time-to-finish and throughput of configuration 5's
served Poisson trace, direct sum; serving_config5_tree beside it),
accuracy_* (GPU vs stored FP64-oracle trajectories), e2e (through the public
API with host buffers).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sphere-steps/s at 100k spheres, mixed vs FP64 form; batched p50/p99 sim latency"
UNIT = "sphere-steps/s"
N_SPHERES = 100_000
# Gravity arithmetic.  One-sided (gather) form: 20 flop per ordered pair (3 sub,
# 3 FMA, rsqrt counted as 2, 3 mul, 3 FMA).  Symmetric form, which the mixed
# path runs: each unordered pair once, 27 flop (3 sub, 3 FMA, rsqrt as 2,
# 2 mul for r^-3, 2 mul for the two mass factors, 6 FMA for the two sums).
FLOP_PER_INTERACTION = 20.0
FLOP_PER_PAIR_SYM = 27.0
# Contact pass, algorithmic bytes per sphere-step (the hot-path scope's count):
# read position+radius, predicted velocity+aggregate, spin (16 B each) and the
# cell range (4 B), write F and tau (16 B each); per canonical pair (one per
# contact, z / 2 per sphere) read and write one 16-byte history record
# (partner 4 B, S 12 B).
CONTACT_BYTES_PER_SPHERE = 16 + 16 + 16 + 4 + 32
CONTACT_BYTES_PER_PAIR = 16 + 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-contact", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-e2-collapse", action="store_true")
    ap.add_argument("--no-tree", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--part", default="all",
                    choices=["all", "contact", "e2", "tree", "analysis", "probe", "serving"],
                    help="contact: only the contact-pass roofline on the 1M-sphere lattice; "
                         "e2: only the paper's 2e4-sphere profiling collapse; "
                         "tree: only tree vs direct gravity; "
                         "analysis: only the spin-up and encounter runs with device-side watches "
                         "(not part of all); probe: only the peak-rate probes; serving: only "
                         "the served traces of configuration 5")
    ap.add_argument("--contact-n", type=int, default=1_048_576)
    ap.add_argument("--contact-mode", type=int, default=None, choices=[0, 1],
                    help="contact part: 0 = one thread per sphere, 1 = tiles with a shared-memory inbox")
    return ap.parse_args()


def workload_config(ic, precision="mixed"):
    return {"workload": "collapse-100k: 100,000 spheres in %d rigid aggregates (dumbbell, rod3, "
                        "tetra, square; radii lognormal median 5 m sigma 0.2) uniform in a 2 km "
                        "ball at rest, contacts + softened direct-sum self-gravity" % ic.n_agg,
            "n_spheres": int(ic.n_sph), "n_aggregates": int(ic.n_agg), "precision": precision,
            "l2": "flushed between timed steps (512 MiB write on the library stream)",
            "seed": 0}


def interactions(ic):
    """Ordered gravity pairs evaluated per step: spheres of other aggregates."""
    n = ic.n_sph
    return float(n) * n - float(np.sum(ic.counts.astype(np.float64) ** 2))


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- pieces
def traffic_for(kernel_file, kernel):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source has not changed since the counters were taken; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    src = os.path.join(ROOT, "paper_2311_11322_gb300", "csrc", kernel_file)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != h:
        return None
    return rec.get("dram_bytes_per_launch")


def run_fp64(dem, W, steps):
    ic, p = W.config2(0, precision=W.PRECISION_FP64)
    with dem.World() as w:
        w.add_pile(ic, p)
        w.step_timed()
        ms = [w.step_timed()[0] for _ in range(steps)]
    t = sum(ms) / 1e3
    return {"value": ic.n_sph * steps / t, "unit": UNIT, "ms_per_step": 1e3 * t / steps,
            "steps": steps, "dtype": "f64"}


def run_contact_roofline(dem, W, peak_gbs, steps=5, n=1_048_576, warmup=3, mode=None):
    """Contact pass on a dense FCC-tetrahedra lattice (0.5% R overlaps, 9 contacts
    per sphere), gravity off, working set far above L2.  Steady state: the pair
    pass over the candidate lists kept since the last rebuild (the lattice moves
    ~1e-4 R per step, so its lists are rebuilt every few hundred steps); the
    rebuild step (cell sort + candidate filter + pair pass) is timed separately."""
    import torch
    ic, p = W.dense_lattice(n_spheres=n, seed=0, precision=W.PRECISION_MIXED)
    p = p.replace(G=0.0)
    with dem.World() as w:
        if mode is not None:
            w.set_tuning("contact_mode", mode)
        mode_used = int(w.get_tuning("contact_mode"))
        pid = w.add_pile(ic, p)
        w.set_timed_kernel("CONTACT")
        flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        st = torch.cuda.ExternalStream(w.stream)
        for _ in range(warmup):
            w.step_timed()
        r0 = w.info(pid)["rebuilds"]
        ks = []
        for _ in range(steps):
            with torch.cuda.stream(st):
                flush.zero_()
            ks.append(w.step_timed()[1])
        info = w.info(pid)
        # the other kernels of the same steps, each between event nodes in the graph
        others = {}
        step_ms = []
        for kname in ("AGG_BEGIN", "PILE_BEGIN", "KEYS", "GATHER", "AGG_END", "PILE_END"):
            w.set_timed_kernel(kname)
            km = []
            for _ in range(steps):
                with torch.cuda.stream(st):
                    flush.zero_()
                sm_, k_ = w.step_timed()
                km.append(k_)
                step_ms.append(sm_)
            others[kname] = statistics.median(km) * 1e3
        w.set_timed_kernel("CONTACT")
        cnt = w.read(pid, "CONTACTS")[:, 0]
        # rebuild steps: a state write (the same velocities) forces one
        vel = w.read(pid, "VEL")
        rb = []
        for _ in range(3):
            w.write(pid, "VEL", vel)
            with torch.cuda.stream(st):
                flush.zero_()
            rb.append(w.step_timed()[1])
    z = float(cnt.sum())
    N = ic.n_sph
    # this library's own compulsory bytes per step: own sorted records (fixed-
    # point position with its rounding remainders 32 B, velocity and spin 32 B),
    # list offset and length (8 B), F and tau out (32 B); per list entry the
    # entry (partner, mirror: 8 B); per pair its history record read and written
    # (16 B each)
    layout = N * (64 + 8 + 32) + z * 8 + (z / 2) * 32
    algo = N * CONTACT_BYTES_PER_SPHERE + (z / 2) * CONTACT_BYTES_PER_PAIR
    ms = statistics.median(ks)
    achieved = algo / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
            "frac": achieved / peak_gbs, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": traffic_for("kernels_contact.cu", "k_contact_sphere" if mode_used == 0 else "k_contact"),
            "kernel": ("k_contact_sphere (one thread per sphere over its kept candidate list)" if mode_used == 0
                       else "k_contact (128-sphere tiles, each inner pair once, shared-memory inbox)"),
            "kernel_ms": ms, "rebuilds_in_timed_steps": info["rebuilds"] - r0,
            "rebuild_step_contact_ms": statistics.median(rb),
            "n_spheres": N, "contacts_per_sphere": z / N,
            "algorithmic_bytes_per_launch": algo,
            "algorithmic_bytes": "84 B per sphere (position, velocity, spin 16 B each, cell range 4 B "
                                 "read; F, tau 32 B written) + 32 B per contact pair (16-byte history "
                                 "record read and written)",
            "layout_bytes_per_launch": layout, "frac_on_layout_bytes": layout / (ms / 1e3) / 1e9 / peak_gbs,
            "layout_bytes": "this library's own layout: 104 B per sphere + 8 B per list entry + 32 B per "
                            "contact pair",
            "other_kernels_us": others, "step_ms": statistics.median(step_ms),
            "other_kernels": "CUDA events around each kernel inside the step graph, median over the steps "
                             "(the rebuild-only kernels return at once in these steps)",
            "workload": "dense FCC tetrahedra lattice, %d spheres, overlaps 0.5%% R, gravity off" % N}


PHASES = {"aggregate": ("AGG_BEGIN", "PILE_BEGIN", "AGG_END", "PILE_END"),
          "search_and_contact": ("KEYS", "SCAN", "SCATTER", "CELL_ORDER", "GATHER", "CONTACT"),
          "gravity": ("GRAVITY",)}


def run_e2_collapse(dem, W, steps=10, warmup=3):
    """The paper's self-gravity profiling collapse (Sec. 3): 2e4 spheres of 50 m as free
    spheres, mixed grain shapes, dumbbells and cubes, each one pile; sphere-steps/s, and
    for the mixed population the share of the step per group of kernels (the paper's
    profile groups: aggregate operations, neighbour search and contacts, gravity)."""
    import torch
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for kind in ("spheres", "mixed", "dumbbell", "cube8"):
        ic, p = W.e2_collapse(kind, seed=0)
        with dem.World() as w:
            pid = w.add_pile(ic, p)
            st = torch.cuda.ExternalStream(w.stream)
            for _ in range(warmup):
                w.step_timed()
            ms = []
            for _ in range(steps):
                with torch.cuda.stream(st):
                    flush.zero_()
                ms.append(w.step_timed()[0])
            rec = {"n_aggregates": ic.n_agg, "ms_per_step": statistics.median(ms),
                   "value": ic.n_sph / (statistics.median(ms) / 1e3), "unit": UNIT}
            if kind == "mixed":
                share = {}
                for grp, names in PHASES.items():
                    tot = 0.0
                    for nm in names:
                        w.set_timed_kernel(nm)
                        w.step_timed()
                        tot += statistics.median([w.step_timed()[1] for _ in range(3)])
                    share[grp] = tot
                w.set_timed_kernel(None)
                step = statistics.median([w.step_timed()[0] for _ in range(3)])
                rec["phase_ms"] = share
                rec["phase_share"] = {k: v / step for k, v in share.items()}
            out[kind] = rec
    out["n_spheres"] = 20_000
    out["paper_context"] = ("pkdgrav on 1 core, mixed-aggregate collapse of 2e4 spheres, 1e4 steps: "
                            "1.8e4 s before and 6.4e3 s after the paper's aggregate bookkeeping "
                            "(1.1e4 -> 3.1e4 sphere-steps/s); aggregate operations 65.4% -> 0.3% of "
                            "the time (Sec. 3); tree gravity there, direct sum here")
    return out


TREE_MODES = (("hexadecapole, theta 0.7", 0.7, 4), ("hexadecapole, theta 0.5", 0.5, 4),
              ("quadrupole, theta 0.5", 0.5, 2))


def run_tree_gravity(dem, W, steps=5):
    """The tree-gravity option (multipoles up to the hexadecapole, the paper's
    order, or up to the quadrupole; opening angle theta) against the direct sum
    on collapse-100k and on the 200,000-sphere spin-up pile: step and
    gravity-phase times, and per-sphere relative force errors after one step."""
    import torch
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for name, (ic, p) in (("collapse-100k", W.config2(0)), ("spinup-200k", W.config3(0))):
        rec = {}
        fg = {}
        for mode, th, order in (("direct", 0.0, 0),) + TREE_MODES:
            with dem.World() as w:
                if th:
                    w.set_tuning("grav_theta", th)
                    w.set_tuning("grav_order", order)
                pid = w.add_pile(ic, p)
                w.set_timed_kernel("GRAVITY")
                w.step_timed()
                fg[mode] = w.read(pid, "SPHERE_FG")
                st = torch.cuda.ExternalStream(w.stream)
                ss, gg = [], []
                for _ in range(steps):
                    with torch.cuda.stream(st):
                        flush.zero_()
                    s_, g_ = w.step_timed()
                    ss.append(s_)
                    gg.append(g_)
                rec[mode] = {"ms_per_step": statistics.median(ss), "gravity_ms": statistics.median(gg),
                             "value": ic.n_sph / (statistics.median(ss) / 1e3), "unit": UNIT,
                             "flags": w.flags(pid)}
            if th:
                e = (np.linalg.norm(fg[mode] - fg["direct"], axis=1) /
                     np.linalg.norm(fg["direct"], axis=1))
                rec[mode]["force_rel_error"] = {"median": float(np.median(e)),
                                                "p99": float(np.quantile(e, 0.99)), "max": float(e.max())}
        rec["n_spheres"] = ic.n_sph
        out[name] = rec
    return out


def run_analysis(dem, W, n_agg=250, settle=150_000, omega_target=1.5, ramp_pcrit=2.0,
                 max_steps=600_000, chunk=20_000):
    """The spin-up and tidal-encounter analyses (Sec. 4.1, 4.2) on the device: a
    lattice pile of n_agg tetrahedra settles under self-gravity; then two copies
    step together in one world (one graph per step), one spun up by a constant
    spin increment reaching omega_target x the nominal critical spin over
    ramp_pcrit critical periods, one on a flyby of an Earth-mass planet (close
    approach 1.2 Earth radii, v_inf 3 km/s, started 3 Roche distances out),
    each with a radius-growth watch (5% and 0.5%) evaluated every 10 steps
    inside the graph."""
    from paper_2311_11322_gb300 import analysis
    rng = np.random.default_rng(0)
    ic = W.lattice_pile(rng, n_agg, shapes=("tetra",))
    p = W.settled_params(ic, 1.0)
    t0 = time.perf_counter()
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        b_lat = w.bulk(pid)
        ic_s = analysis.settled(w, pid, settle, chunk)
        b_set = w.bulk(pid)
    t_settle = time.perf_counter() - t0
    P_steps = b_set["p_crit"] / p.dt
    ps = analysis.spinup_params(p, ic_s, omega_target * 2 * math.pi / b_set["p_crit"],
                                int(ramp_pcrit * P_steps))
    pe, orb = analysis.encounter_params(p, ic_s)
    out = {"n_spheres": ic.n_sph, "n_aggregates": ic.n_agg, "dt_s": p.dt, "settle_steps": settle,
           "settle_s": t_settle, "settle_value": ic.n_sph * settle / t_settle, "unit": UNIT,
           "lattice_radius_m": b_lat["radius"], "settled_radius_m": b_set["radius"],
           "settled_density": b_set["density"], "p_crit_s": b_set["p_crit"],
           "spin_ramp": f"{omega_target} x nominal critical spin over {ramp_pcrit} critical periods",
           "encounter": {"periapsis_earth_radii": orb["q"] / W.EARTH_RADIUS, "v_inf_kms": orb["vinf"] / 1e3}}
    with dem.World() as w:
        a, b = w.add_pile(ic_s, ps), w.add_pile(ic_s, pe)
        w.watch(a, 0.05, 10)
        w.watch(b, 0.005, 10)
        live, taken, sph_steps = [a, b], 0, 0
        t0 = time.perf_counter()
        while live and taken < max_steps:
            w.step(chunk, piles=live)
            taken += chunk
            sph_steps += chunk * ic.n_sph * len(live)
            live = [x for x in live if w.watch_result(x)["fired_step"] is None]
        w.sync()
        t = time.perf_counter() - t0
        ra, rb = w.watch_result(a), w.watch_result(b)
    out["runs_s"] = t
    out["runs_value"] = sph_steps / t
    out["spinup"] = {"fired_step": ra["fired_step"], "critical_spin_ratio": analysis.critical_spin_ratio(ra),
                     "period_at_fire_s": ra["at_fire"]["period"] if ra["at_fire"] else None}
    out["encounter_run"] = {"fired_step": rb["fired_step"], "disruption_ratio": analysis.disruption_ratio(rb),
                            "distance_at_fire_km": rb["at_fire"]["planet_dist"] / 1e3 if rb["at_fire"] else None}
    out["paper_context"] = ("Sec. 4.1 / 4.2 tables: critical spin ratios 100-120% and disruption ratios "
                            "55-85% for 2,500-20,000-grain piles; their initial conditions and spin-up "
                            "rate are not published, so the ratios here are not comparable")
    return out


def run_batched(dem, W, steps=5, n_piles=256):
    """256 independent piles of tetrahedra (sizes lognormal in [500, 20000]):
    all stepped by one graph launch per step after autotuning, against looping
    the plain path one pile at a time (each pile alone in its own world)."""
    piles = W.config4(0, n_piles=n_piles)
    n_tot = sum(ic.n_sph for ic, _ in piles)
    with dem.World() as w:
        for ic, p in piles:
            w.add_pile(ic, p)
        best = w.autotune(2)
        for _ in range(2):
            w.step_timed()
        ms = [w.step_timed()[0] for _ in range(steps)]
    t_batch = sum(ms) / 1e3 / steps
    t_loop = 0.0
    for ic, p in piles:
        with dem.World() as w:
            w.add_pile(ic, p)
            w.step_timed()
            t_loop += statistics.median([w.step_timed()[0] for _ in range(3)]) / 1e3
    return {"value": n_tot / t_batch, "unit": UNIT, "ms_per_step": 1e3 * t_batch,
            "n_piles": n_piles, "n_spheres": n_tot, "autotune_best_ms": best,
            "loop_one_pile_at_a_time": {"value": n_tot / t_loop, "ms_per_step": 1e3 * t_loop},
            "batched_over_loop": t_loop / t_batch,
            "workload": "256 piles of tetrahedra, sizes lognormal median 3,000 in [500, 20,000], "
                        "each on a jittered lattice in a ball, mixed precision"}


def run_serving(dem, W, n_req=64, steps=20_000, n_hi=100_000, theta=0.0, rate=4.0):
    """Served tidal encounters: a Poisson trace (`rate` arrivals/s) of `n_req`
    flyby piles, sizes log-uniform in [1,000, n_hi] spheres, `steps` steps each,
    served by continuous batching in one world (admission by footprint, state
    resident on the device), direct-sum gravity unless theta > 0 (tree)."""
    from paper_2311_11322_gb300 import serve
    trace = W.config5_trace(0, n_arrivals=n_req, rate=rate, n_hi=n_hi, steps=steps)
    t0 = time.perf_counter()
    reqs = serve.trace_requests(trace, W.config5_pile)
    t_gen = time.perf_counter() - t0
    with dem.World() as w:
        if theta:
            w.set_tuning("grav_theta", theta)
        srv = serve.Server(w, dem.dem_footprint_bytes, budget_bytes=64 << 30, max_piles=64,
                           chunk=250)
        st = srv.run(reqs)
    n = np.array([r.n_spheres for r in reqs], float)
    st["mean_request_sphere_steps"] = float(np.mean(n * steps))
    st["host_generation_s"] = t_gen
    st.update({"trace": "%d Poisson arrivals at %.2f/s, sizes log-uniform [1000, %d] spheres "
                        "(drawn: min %d, median %d, max %d), %d steps each, settled lattice piles "
                        "of tetrahedra on a hyperbolic flyby of an Earth-mass planet (periapsis "
                        "1.5-4 planet radii, v_inf 1-10 km/s)"
                        % (n_req, rate, n_hi, n.min(), np.median(n), n.max(), steps),
               "gravity": "tree (hexadecapole), theta %.2f" % theta if theta else "direct sum",
               "batching": "every resident pile in one step graph; rounds of <= 250 steps; "
                           "up to 64 piles, 64 GiB footprint budget"})
    return st


def run_accuracy(dem, W, name="collapse100k"):
    """GPU (mixed and all-FP64) side by side with a stored FP64-oracle trajectory
    (tests/golden, written by scripts that call only the oracle): 100 steps of
    collapse-100k, or 30 steps of the pre-settled 200,000-sphere spin-up pile
    (~940,000 contact pairs under the spin ramp).  Per-step condition-relative
    and |X|-relative force and torque errors of 256 sampled aggregates, COM and
    quaternion deviations, and for the pile the contact-pair counts."""
    from tests.parity_util import (contact_pair_count, same_inputs, summarize_trajectory,
                                   trajectory_errors)
    if name == "collapse100k":
        path = os.path.join(ROOT, "tests", "golden", "collapse100k_100steps.npz")
        make, steps = W.config2, 100
        what = "collapse-100k (100,000 spheres, no contacts yet)"
    else:
        path = os.path.join(ROOT, "tests", "golden", "config3_settled_30steps.npz")
        make, steps = W.config3_settled, 30
        what = ("pre-settled spin-up pile (200,000 equal spheres of a 3:2:1.5 FCC packing in "
                "2-8-sphere aggregates, neighbours overlapping 1e-5 s, spin ramp 1e-9 rad/s per step)")
    if not os.path.exists(path):
        return {"unavailable": "stored oracle trajectory missing"}
    gold = np.load(path)
    out = {"reference": "FP64 oracle, %d full steps of %s, 256 sampled aggregates" % (steps, what),
           "bound": {"mixed": 1e-5, "fp64": 1e-9},
           "measure": "condition-relative: |X_gpu - X_oracle| / sum of the magnitudes of the summed "
                      "terms; abs_rel: / |X_oracle|"}
    for prec_name, prec in (("mixed", W.PRECISION_MIXED), ("fp64", W.PRECISION_FP64)):
        ic, p = make(0, precision=prec)
        if not same_inputs(ic, gold):
            out[prec_name] = {"unavailable": "input generator differs from the stored run"}
            continue
        with dem.World() as w:
            pid = w.add_pile(ic, p)
            rows = trajectory_errors(w, pid, gold)
            pairs = contact_pair_count(w, pid)
        out[prec_name] = summarize_trajectory(rows)
        out[prec_name]["contact_pairs_last_step"] = {"gpu": pairs, "oracle": int(gold["n_pairs"][-1])}
    return out


def run_e2e(dem, W, ic, p, steps):
    """Through the public API with pinned host buffers: add the pile (host->device
    copy of the initial conditions), then per step dem_step + read the COMs back
    (asynchronously: each step's result is waited for while the next step runs)."""
    import torch

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t.numpy()

    hic = W.PileIC(pinned(ic.counts), pinned(ic.pos), pinned(ic.radius), pinned(ic.density),
                   pinned(ic.vel), pinned(ic.omega))
    h2d = sum(a.nbytes for a in (hic.counts, hic.pos, hic.radius, hic.density, hic.vel, hic.omega))
    with dem.World() as w:
        pid = w.add_pile(hic, p)      # warm the allocator and the code paths
        w.step(1)
        coms = [pinned(w.read(pid, "COM")) for _ in range(2)]   # each step's result, in pinned memory
        w.remove(pid)
        w.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pid = w.add_pile(hic, p)
        d2h = coms[0].nbytes
        for s in range(steps):
            w.step(1)              # step s is issued; result s - 1 is waited for while it runs
            if s > 0:
                w.read_wait()
            w.read_async(pid, "COM", coms[s % 2])
        w.read_wait()
        w.remove(pid)
        w.sync()
        t = time.perf_counter() - t0
    return {"value": ic.n_sph * steps / t, "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h, "steps": steps,
            "definition": "add_pile from pinned host arrays + steps x (dem_step(1) + read of the COMs "
                          "into a pinned host array, waited for while the next step runs) + remove, "
                          "wall clock"}


def cpu_baseline(W, ic, p, rows_frac=1.0):
    import oracle
    oracle.build()
    pile = oracle.Pile(ic, p)
    n = ic.n_sph
    rows = np.arange(0, n, max(1, int(round(1.0 / rows_frac))), dtype=np.int64)
    t0 = time.perf_counter()
    pile.step_sampled(rows)
    t = time.perf_counter() - t0
    return {"value": len(rows) / t, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "one FP64 oracle step of the same 100k-sphere workload, forces of %d of "
                      "its %d spheres (every %d-th; brute-force contacts + direct gravity over "
                      "all spheres), %.1f s" % (len(rows), n, n // len(rows), t)}


def run_probes(dem, clocks_index=0):
    """Peak rates of this GPU measured in this run (dem_probe_peak): FP32 FMA
    (scalar and packed f32x2), FP64 FMA and HBM copy, with nvidia-smi clocks
    sampled while the probes run."""
    import torch
    sink = torch.zeros(64, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    ck = Clocks(clocks_index)
    ck.start()
    out = {}
    for kind, size, reps in (("FMA32", 300_000, 10), ("FMA32X2", 150_000, 10), ("FMA64", 5_000, 5)):
        rate, ms, sms = dem.dem_probe_peak(kind, size, reps, 0, sink.data_ptr(), st)
        out[kind] = {"tflops": rate / 1e12, "ms": ms}
    nbytes = 4 << 30
    src = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dst = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    src.fill_(1)
    rate, ms, sms = dem.dem_probe_peak("COPY", nbytes, 10, src.data_ptr(), dst.data_ptr(), st)
    out["COPY"] = {"gbs": rate / 1e9, "ms": ms, "bytes_per_buffer": nbytes}
    del src, dst
    torch.cuda.synchronize()
    out["clocks"] = ck.stop()
    out["sm_count"] = int(sms)
    out["sm_count_torch"] = int(torch.cuda.get_device_properties(0).multi_processor_count)
    out["fp32_peak_tflops"] = max(out["FMA32"]["tflops"], out["FMA32X2"]["tflops"])
    out["fp32_peak_form"] = ("packed f32x2 FMA" if out["FMA32X2"]["tflops"] > out["FMA32"]["tflops"]
                             else "scalar FMA")
    out["what"] = ("dem_probe_peak: 4 blocks x 256 threads per SM, 8 independent FMA chains per thread "
                   "(2 flop per FMA, 4 per packed f32x2 FMA), fastest of the launches; copy: float4 "
                   "streaming copy of 4 GiB, read + write bytes")
    return out


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- arms
def run_ours(args):
    import torch
    from paper_2311_11322_gb300 import dem
    from paper_2311_11322_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier(ws)
    dem.load()

    ic, p = W.config2(rank)
    pk = peaks()
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    w = dem.World()
    pid = w.add_pile(ic, p)
    w.set_timed_kernel("GRAVITY")
    n_kern = w.graph_kernel_count()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.ExternalStream(w.stream)
    for _ in range(max(args.warmup, 0)):
        w.step_timed()
    barrier(ws)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    wall0 = time.perf_counter()
    step_ms, grav_ms = [], []
    for _ in range(args.steps):
        with torch.cuda.stream(st):
            flush.zero_()
        s, g = w.step_timed()
        step_ms.append(s)
        grav_ms.append(g)
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - wall0
    ck = clocks.stop()
    w.sync()
    t_rank = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_rank, ws, device="cuda")
    value = ws * ic.n_sph * args.steps / t_max
    g_ms = statistics.mean(grav_ms)
    n_int = interactions(ic)
    flops = FLOP_PER_INTERACTION * n_int
    achieved = flops / (g_ms / 1e3) / 1e12
    executed = FLOP_PER_PAIR_SYM * n_int / 2.0
    w.close()
    probes = run_probes(dem, local)
    fp32_peak = probes["fp32_peak_tflops"]

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32/f64", "data": "synthetic (seeded generator, no dataset)",
           "config": workload_config(ic), "wall_s_timed_region": wall,
           "gpu_launches": n_kern * args.steps,
           "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak,
                        "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                        "traffic": traffic_for("kernels_gravity.cu", "k_gravity32s"),
                        "kernel": "k_gravity32s (softened direct-sum gravity, symmetric "
                                  "tile pairs, packed f32x2) + k_grav_acc_to_force (its integer sums to forces)",
                        "kernel_ms": g_ms, "share_of_step": g_ms / statistics.mean(step_ms),
                        "flops_per_launch": flops,
                        "flop_count": "20 per ordered pair of spheres in different aggregates "
                                      "(the direct-sum convention: 3 sub, 3 FMA, rsqrt as 2, 3 mul, "
                                      "3 FMA)",
                        "interactions_per_s": n_int / (g_ms / 1e3),
                        "executed_flops_per_launch": executed,
                        "executed_tflops": executed / (g_ms / 1e3) / 1e12,
                        "executed_frac": executed / (g_ms / 1e3) / 1e12 / fp32_peak,
                        "executed_flop_count": "27 per unordered pair: each pair is evaluated once "
                                               "and applied to both spheres",
                        "peak_source": "measured in this run: %s probe (dem_probe_peak) on %d SMs, "
                                       "median SM clock %s MHz during the probes"
                                       % (probes["fp32_peak_form"], probes["sm_count"],
                                          probes["clocks"].get("sm_mhz"))},
           "peaks_measured": probes,
           "clocks": ck}
    if rank == 0 and ws == 1 and not args.no_accuracy:
        out["accuracy_collapse100k"] = run_accuracy(dem, W)
        out["accuracy_config3_settled"] = run_accuracy(dem, W, "config3_settled")
    if rank == 0 and not args.no_fp64:
        out["fp64_path"] = run_fp64(dem, W, steps=3)
        out["fp64_path"]["mixed_over_fp64"] = value / ws / out["fp64_path"]["value"]
    if rank == 0 and not args.no_contact:
        out["roofline_contact"] = run_contact_roofline(dem, W, hbm_peak)
        # the same pass at 2M and 4M spheres (working sets of 0.9 and 1.8 GB)
        out["roofline_contact_sweep"] = []
        for n in (2 * 1_048_576, 4 * 1_048_576):
            r = run_contact_roofline(dem, W, hbm_peak, n=n)
            out["roofline_contact_sweep"].append({k: r[k] for k in ("n_spheres", "kernel_ms", "achieved",
                                                                    "frac", "rebuild_step_contact_ms")})
    if rank == 0 and not args.no_batched:
        out["batched"] = run_batched(dem, W)
    if rank == 0 and ws == 1 and not args.no_serving:
        # configuration 5 as stated: 64 arrivals at 4/s, 1,000-100,000 spheres, 20,000
        # steps each, direct sum (about 7 minutes of GPU time)
        out["serving_config5"] = run_serving(dem, W)
        # the same trace with tree gravity, 2,000 steps per request
        out["serving_config5_tree"] = run_serving(dem, W, steps=2000, theta=0.7)
    if rank == 0 and not args.no_e2_collapse:
        out["e2_collapse"] = run_e2_collapse(dem, W)
    if rank == 0 and not args.no_tree:
        out["tree_gravity"] = run_tree_gravity(dem, W)
    if not args.no_e2e:
        e = run_e2e(dem, W, ic, p, steps=args.steps)
        e_t = max_over_ranks(ic.n_sph * args.steps / e["value"], ws, device="cuda")
        e["value"] = ws * ic.n_sph * args.steps / e_t
        out["e2e"] = e
    if rank == 0 and ws == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(W, ic, p, rows_frac=1.0)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """The oracle (plain FP64 CPU program) timed on the host cores, on bounded
    samples of the same workload: each step computes the forces of 1/8 of the
    spheres against all spheres."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2311_11322_gb300 import workloads as W
    import oracle
    oracle.build()
    ic, p = W.config2(0)
    pile = oracle.Pile(ic, p)
    rows = np.arange(0, ic.n_sph, 8, dtype=np.int64)
    for _ in range(max(args.warmup, 0)):
        pile.step_sampled(rows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pile.step_sampled(rows)
    t = time.perf_counter() - t0
    value = len(rows) * args.steps / t
    cb = {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
          "sample": "per step: FP64 oracle forces of %d of the %d spheres (every 8th) against "
                    "all spheres, brute-force contacts + direct gravity" % (len(rows), ic.n_sph)}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded generator, no dataset)",
           "config": workload_config(ic, precision="fp64 (the oracle)"), "cpu_baseline": cb,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_contact_only(args):
    import torch
    from paper_2311_11322_gb300 import dem
    from paper_2311_11322_gb300 import workloads as W
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    r = run_contact_roofline(dem, W, float(peaks().get("hbm_gbs", 6800.0)), steps=args.steps,
                             n=args.contact_n, warmup=args.warmup, mode=args.contact_mode)
    print(json.dumps({"part": "contact", "roofline_contact": r}), flush=True)


def run_e2_only(args):
    import torch
    from paper_2311_11322_gb300 import dem
    from paper_2311_11322_gb300 import workloads as W
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    print(json.dumps({"part": "e2", "e2_collapse": run_e2_collapse(dem, W, steps=args.steps,
                                                                    warmup=args.warmup)}), flush=True)


def run_tree_only(args):
    import torch
    from paper_2311_11322_gb300 import dem
    from paper_2311_11322_gb300 import workloads as W
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    print(json.dumps({"part": "tree", "tree_gravity": run_tree_gravity(dem, W, steps=args.steps)}),
          flush=True)


def run_probe_only(args):
    import torch
    from paper_2311_11322_gb300 import dem
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    dem.load()
    print(json.dumps({"part": "probe", "peaks_measured": run_probes(dem)}), flush=True)


def run_serving_only(args):
    import torch
    from paper_2311_11322_gb300 import dem
    from paper_2311_11322_gb300 import workloads as W
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    dem.load()
    out = {"part": "serving", "serving_config5": run_serving(dem, W)}
    out["serving_config5_tree"] = run_serving(dem, W, steps=2000, theta=0.7)
    print(json.dumps(out), flush=True)


def run_analysis_only(args):
    import torch
    from paper_2311_11322_gb300 import dem
    from paper_2311_11322_gb300 import workloads as W
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    print(json.dumps({"part": "analysis", "analysis": run_analysis(dem, W)}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.part == "contact":
        run_contact_only(a)
    elif a.part == "e2":
        run_e2_only(a)
    elif a.part == "tree":
        run_tree_only(a)
    elif a.part == "analysis":
        run_analysis_only(a)
    elif a.part == "probe":
        run_probe_only(a)
    elif a.part == "serving":
        run_serving_only(a)
    else:
        run_ours(a)
