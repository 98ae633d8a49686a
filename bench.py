#!/usr/bin/env python3
"""Throughput benchmark of the VBC path on B300.

One bench step = one BAOAB Langevin timestep of the whole path: neighbour-list
rebuild when due (amortised), pass 1 counts, chain-rule pass, pass 2 forces
fused with the integrator update.  Workload: N = 1,000,000 identical particles,
uniform random in a periodic cube at number density 0.5, standard VBC(1.5, 2.0, 0)
on the polynomial soft core (E_r = 20, E_a = 8), valency 2, dt = 0.005, kT = 1,
gamma = 1, skin 0.4; FP32 pair arithmetic with FP64 state and reductions.
The system is equilibrated (untimed) before the W warm-up and K timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs an
independent replica of the workload on its own GPU (the path has no exchange
step between systems), and value = total timesteps of all replicas / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VBC pair-interactions/s and MD timesteps/s at N=1M on 1 B300, % HBM roofline; p50/p99 served"
UNIT = "timesteps/s"
FALLBACK_HBM_GBS = 6400.0
KERNELS_OF = {"count": "k_count_near", "chain": "k_chain", "force": "k_force_rows + k_step",
              "rebuild": "k_bin, k_scan_sums, k_scan_apply, k_scatter, k_cellsort, k_permute, k_copyback, k_nlist"}
KERNEL_SOURCES = ("paper_2609_07842_b300/csrc/vbc_kernels.cuh", "paper_2609_07842_b300/csrc/vbc_device.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "kernel_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("b300", "reference"), default="b300")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--rho", type=float, default=0.5)
    ap.add_argument("--valency", type=float, default=2.0)
    ap.add_argument("--E_a", type=float, default=8.0)
    ap.add_argument("--equil", type=int, default=500, help="untimed equilibration steps")
    ap.add_argument("--e2e-chunk", type=int, default=1000, help="steps per host round trip in the e2e leg")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-valency8", action="store_true", help="skip the valency-8 measurement of the same system")
    ap.add_argument("--no-served", action="store_true", help="skip the served leg (p50/p99 latency)")
    ap.add_argument("--served-requests", type=int, default=24)
    ap.add_argument("--served-steps", type=int, default=50_000, help="Langevin steps per served request")
    ap.add_argument("--served-slots", type=int, default=16)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched leg (many uneven systems)")
    ap.add_argument("--batched-systems", type=int, default=256)
    ap.add_argument("--batched-steps", type=int, default=1000)
    ap.add_argument("--sweep", action="store_true",
                    help="cost-vs-valency curve (N=100k, rho 0.5, E_a 8, v in 1,2,4,6,8) and the paper-shape "
                         "point (N=10k, rho 0.05, E_a 2, dt 0.01, gamma 0.1, f = 1..6); one JSON line each")
    ap.add_argument("--stickers", action="store_true",
                    help="the multi-type sticker-chain workload (31,250 chains of 64 beads at bead density 0.3, "
                         "stickers every 4th bead, FP64 typed path); one JSON line")
    ap.add_argument("--sticker-chains", type=int, default=31_250)
    ap.add_argument("--sticker-precision", choices=("fp32", "fp64"), default="fp32",
                    help="arithmetic of the sticker-chain leg: the FP32 split (default) or FP64")
    ap.add_argument("--leg", choices=("served", "batched"), default=None,
                    help="run only this optional leg and print its JSON object (the main run starts each "
                         "optional leg this way, in a process of its own)")
    ap.add_argument("--leg-timeout", type=float, default=900.0, help="seconds allowed to one optional leg")
    ap.add_argument("--profile-run", action="store_true",
                    help="short run for profilers: the equilibrated workload (cached under /tmp), one forced "
                         "list build, one force evaluation and 6 steps; prints no JSON line")
    return ap.parse_args()


DT, KT, GAMMA, SKIN, SEED = 0.005, 1.0, 1.0, 0.4, 3


def workload(args, valency=None):
    valency = args.valency if valency is None else valency
    return {
        "workload": (f"uniform fluid N={args.n:,} rho={args.rho}, standard VBC(1.5,2.0,0) soft core "
                     f"E_r=20 E_a={args.E_a:g} valency {valency:g}, BAOAB dt={DT} kT={KT} gamma={GAMMA}, "
                     f"skin {SKIN}"),
        "n": args.n, "rho": args.rho, "valency": valency, "E_a": args.E_a,
        "equilibration_steps": args.equil,
        "start_state": f"the seeded uniform draw after {args.equil} untimed BAOAB steps, grid autotuning and the warm-up",
        "precision": "FP32 pair arithmetic, FP64 state and energy",
        "l2": "no flush: working set per step (~0.4 GB) > L2 (126 MB)",
    }


def max_over_ranks(v, world, device="cuda"):
    """The largest v over the ranks (the slowest rank's time): an all-reduce MAX,
    over NCCL on the GPU machine or gloo on the CPU.  v itself when world is 1."""
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps, seconds, world):
    """Timesteps per second of all replicas together: every rank advances its own
    system (weak scaling), timed by the slowest rank."""
    return steps * world / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def start_clocks(local):
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                                 "-lms", "100", "-i", str(local)], stdout=subprocess.PIPE,
                                stderr=subprocess.DEVNULL, text=True)
    except (OSError, ValueError):
        return None


def stop_clocks(proc):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        t = [x.strip() for x in line.split(",")]
        if len(t) < 9:
            continue
        try:
            sm.append(float(t[1]))
            smax.append(float(t[2]))
        except ValueError:
            continue
        for nm, v in zip(names, t[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class, n):
    """DRAM bytes per launch of one kernel class (ncu dram__bytes_read.sum +
    dram__bytes_write.sum, summed over the class's kernels) from the committed
    summary, scaled to n particles; None when the kernels changed since the
    capture."""
    try:
        with open(TRAFFIC_FILE) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    if t.get("kernel_sources_sha256_16") != kernel_hash():
        return None
    per = t.get("dram_bytes_per_particle", {}).get(kernel_class)
    return None if per is None else per * n


# Algorithmic HBM bytes per particle of each kernel class, with the per-unit
# figures of the hot-path scope table (4-byte list entries, k = mean list
# length, phi = in-window fraction).  This design moves fewer bytes than these
# figures (2-byte entries, and saturated particles read a 12-entry close list
# instead of their full row); the measured DRAM bytes are in "traffic".
def class_bytes_per_particle(k, phi):
    return {
        "count": 4.0 * k + 16.0 + 8.0,                                   # list, own position, n
        "chain": phi * (4.0 * k + 32.0),                                 # window particles only
        "force": (4.0 * k + 16.0 + 8.0 + 4.0 + 16.0)                     # pass 2: list, pos, s/n, A, F
                 + (24.0 + 24.0 + 24.0 + 24.0 + 16.0 + 16.0),            # BAOAB: x, v r/w, F read, pos write
        "rebuild": 4.0 * k + 48.0,                                       # per build
    }


# ------------------------------------------------------------------ reference arm (the oracle)
def run_oracle(args, steps, budget):
    import oracle
    from paper_2609_07842_b300 import inputs
    pos, L = inputs.uniform_positions(args.n, args.rho, seed=SEED)
    vel = inputs.maxwell_velocities(args.n, KT, seed=SEED + 1)
    p = oracle.Params(E_a=args.E_a, f=args.valency)
    t0 = time.perf_counter()
    x, v, st = oracle.baoab(pos, vel, L, p, 1, DT, KT, GAMMA, seed=SEED, mode=1)  # first step + warm caches
    t_first = time.perf_counter() - t0
    # an n-step call evaluates forces n + 1 times; size the sample to the budget
    k = int(max(1, min(steps, budget / max(t_first / 2.0, 1e-9) - 1)))
    t0 = time.perf_counter()
    x, v, st = oracle.baoab(x, v, L, p, k, DT, KT, GAMMA, seed=SEED, step=st, mode=1)
    dt = time.perf_counter() - t0
    return k / dt, k, dt, oracle.num_threads()


def reference_main(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    budget = max(10.0, min(120.0, args.cpu_budget * 3))
    value, k, secs, cores = run_oracle(args, args.steps, budget)
    sample = (f"{k} BAOAB steps of the full N={args.n:,} system with the FP64 oracle (cell-list mode, "
              f"OpenMP), {secs:.1f} s; time-bounded sample of the requested {args.steps} steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**workload(args), "precision": "FP64 oracle (cell-list mode)", "equilibration_steps": 0,
                   "start_state": ("the seeded uniform draw itself: the oracle, at about 1.5 steps/s on the full "
                                   "system, cannot run the B300 arm's 500 untimed equilibration steps inside the "
                                   "bench's time; its cost per step depends on the state only through the "
                                   "neighbour counts of its cell lists")},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ B300 arm
def profile_run(args):
    """A few launches of every kernel on the bench workload, for a profiler: the
    state after args.equil steps (cached between runs), one forced list build
    (NVTX range "build"), one force evaluation and 6 steps (NVTX range "steps"),
    so that a capture can select one kernel inside one range."""
    import torch
    from paper_2609_07842_b300 import inputs, vbc
    prm = vbc.params(E_a=args.E_a, f=args.valency)
    cache = f"/tmp/vbc_bench_state_n{args.n}_rho{args.rho}_v{args.valency:g}_e{args.equil}.npz"
    if not os.path.exists(cache):
        pos, L = inputs.uniform_positions(args.n, args.rho, seed=SEED)
        vel = inputs.maxwell_velocities(args.n, KT, seed=SEED + 1)
        with vbc.System(pos, L, prm, vel=vel, skin=SKIN, seed=SEED) as s:
            s.step(args.equil, DT, KT, GAMMA)
            p, v, _ = s.get_state()
        np.savez(cache, pos=p, vel=v, L=L)
    d = np.load(cache)
    with vbc.System(d["pos"], float(d["L"]), prm, vel=d["vel"], skin=SKIN, seed=SEED) as s:
        torch.cuda.nvtx.range_push("build")
        s.build_neighbors()
        torch.cuda.nvtx.range_pop()
        s.compute(F=np.zeros((args.n, 3)))
        torch.cuda.nvtx.range_push("steps")
        s.step(6, DT, KT, GAMMA)
        torch.cuda.nvtx.range_pop()
        st = s.stats()
    print(f"profile run: n={args.n} list mean {st.nlist_mean:.2f} unsaturated {st.unsaturated}", file=sys.stderr)
    return 0


def served_requests(args):
    """A Poisson arrival stream of simulation requests: arrival rate 20 per
    second, N log-uniform in [1k, 200k], valency uniform in {1, ..., 8}, the
    bench's pair form at density 0.5, args.served_steps steps each (seeded)."""
    rng = np.random.default_rng(20260)
    t = np.cumsum(rng.exponential(1.0 / 20.0, args.served_requests))
    n = np.exp(rng.uniform(np.log(1000), np.log(200_000), args.served_requests)).astype(int)
    v = rng.integers(1, 9, args.served_requests)
    return [(float(t[k] - t[0]), int(n[k]), float(v[k]), 100 + k) for k in range(args.served_requests)]


def run_served(args, slots):
    """Submits the request stream at its arrival times to a server with the given
    slots (150 GB budget, 1000-step chunks, state resident on the device) and
    returns latency percentiles and aggregate throughput."""
    from paper_2609_07842_b300 import inputs, vbc
    reqs = served_requests(args)
    made = [(t, inputs.uniform_positions(n, args.rho, seed=seed), v, seed) for t, n, v, seed in reqs]
    with vbc.Server(hbm_budget=150e9, slots=slots, chunk_steps=1000) as srv:
        t0 = time.perf_counter()
        ids = []
        for t, (pos, L), v, seed in made:
            dt_wait = t - (time.perf_counter() - t0)
            if dt_wait > 0:
                time.sleep(dt_wait)
            ids.append(srv.submit(pos, L, vbc.params(E_a=args.E_a, f=v), nsteps=args.served_steps, dt=DT,
                                  kT=KT, gamma=GAMMA, seed=seed))
        srv.wait()
        infos = [srv.result(i)[2] for i in ids]
    lat = np.array([x.t_done - x.t_submit for x in infos])
    span = max(x.t_done for x in infos) - min(x.t_submit for x in infos)
    steps = sum(args.served_steps for _ in infos)
    psteps = sum(args.served_steps * x.n for x in infos)
    return {"slots": slots, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "timesteps_per_s": steps / span,
            "particle_steps_per_s": psteps / span, "makespan_s": span,
            "ok": all(x.status == 0 for x in infos)}


def timed_steps(sys_, steps, dt, kT, gamma):
    """ms per step of `steps` Langevin steps (CUDA events on the library's stream)."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    ev0.record(stream)
    sys_.step(steps, dt, kT, gamma)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps


def sweep(args):
    """The single-system valency sweep (N = 100k, density 0.5, E_a = 8, FP32
    split; the cost-vs-valency curve of the paper's performance table) and the
    paper-shape point (N = 10k, density 0.05, E_a = 2, dt = 0.01, gamma = 0.1,
    f = 1..6), each after an untimed equilibration.  Prints one JSON line per
    configuration."""
    import torch
    from paper_2609_07842_b300 import inputs, vbc
    stream = torch.cuda.current_stream()
    cases = [("valency sweep", 100_000, 0.5, 8.0, float(v), DT, GAMMA, 2000, 1000) for v in (1, 2, 4, 6, 8)]
    cases += [("paper shape", 10_000, 0.05, 2.0, float(f), 0.01, 0.1, 5000, 2000) for f in range(1, 7)]
    for name, n, rho, ea, f, dt, gamma, steps, equil in cases:
        pos, L = inputs.uniform_positions(n, rho, seed=SEED)
        vel = inputs.maxwell_velocities(n, KT, seed=SEED + 1)
        with vbc.System(pos, L, vbc.params(E_a=ea, f=f), vel=vel, skin=SKIN, seed=SEED,
                        stream=stream.cuda_stream) as s:
            s.step(equil, dt, KT, gamma)
            st0 = s.stats()
            ms = timed_steps(s, steps, dt, KT, gamma)
            st1 = s.stats()
            s.compute(energy=True)  # counts the pairs within r_c
            st2 = s.stats()
        sps = 1e3 / ms
        print(json.dumps({"sweep": name, "n": n, "rho": rho, "E_a": ea, "valency": f, "dt": dt, "gamma": gamma,
                          "steps": steps, "equilibration_steps": equil, "timesteps_per_s": sps,
                          "seconds_per_1e6_steps": 1e6 / sps,
                          "pair_interactions_per_s": st2.pairs_within_rc * sps,
                          "in_window_fraction": st2.in_window / n, "unsaturated_fraction": st2.unsaturated / n,
                          "steps_per_rebuild": steps / max(st1.rebuilds - st0.rebuilds, 1),
                          "precision": "FP32 split", "data": "synthetic"}), flush=True)


def batched_systems(args):
    """Uneven independent systems: N log-uniform in [2k, 64k], valency uniform in
    {1, ..., 6}, kT uniform in [0.8, 1.5], density uniform in [0.2, 0.6] (seeded)."""
    rng = np.random.default_rng(40960)
    k = args.batched_systems
    n = np.exp(rng.uniform(np.log(2000), np.log(64_000), k)).astype(int)
    v = rng.integers(1, 7, k)
    kt = rng.uniform(0.8, 1.5, k)
    rho = rng.uniform(0.2, 0.6, k)
    return [(int(n[i]), float(rho[i]), float(v[i]), float(kt[i]), 500 + i) for i in range(k)]


def run_batched(args):
    """The uneven systems advanced by args.batched_steps steps with vbc_batch_step
    in the fused mode (one cooperative launch per iteration for all of them), in
    the graph mode (one graph launch per two steps), and one system after another
    (vbc_step_langevin each, its own graphs), after an untimed equilibration;
    aggregate timesteps/s of each (host clock, device synchronised on both sides)."""
    import torch
    from paper_2609_07842_b300 import inputs, vbc
    cfg = batched_systems(args)
    systems = []
    for n, rho, v, kt, seed in cfg:
        pos, L = inputs.uniform_positions(n, rho, seed=seed)
        vel = inputs.maxwell_velocities(n, kt, seed=seed + 1)
        systems.append(vbc.System(pos, L, vbc.params(E_a=args.E_a, f=v), vel=vel, skin=SKIN, seed=seed))
    kts = [c[3] for c in cfg]
    out = {}
    try:
        times = {}
        with vbc.Batch(systems) as b:
            b.step(200, DT, kts, GAMMA)                  # equilibration, untimed
            for name, mode in (("batched", vbc.VBC_BATCH_FUSED), ("batched_graphs", vbc.VBC_BATCH_GRAPHS)):
                b.set_mode(mode)
                b.step(4, DT, kts, GAMMA)                # untimed: captures the graphs of this mode
                torch.cuda.synchronize()
                f0 = b.fused_launches()
                t0 = time.perf_counter()
                b.step(args.batched_steps, DT, kts, GAMMA)
                torch.cuda.synchronize()
                times[name] = time.perf_counter() - t0
                out[name + "_launches"] = b.fused_launches() - f0
        t0 = time.perf_counter()
        for s, kt in zip(systems, kts):
            s.step(args.batched_steps, DT, kt, GAMMA)
        torch.cuda.synchronize()
        times["one_at_a_time"] = time.perf_counter() - t0
        nsys, ntot = len(systems), sum(c[0] for c in cfg)
        for name, t in times.items():
            out[name] = {"seconds": t, "timesteps_per_s": nsys * args.batched_steps / t,
                         "particle_steps_per_s": ntot * args.batched_steps / t}
        out["batched"]["how"] = "one cooperative launch per iteration for all systems (fused)"
        out["batched_graphs"]["how"] = "each system's two-step CUDA graph captured side by side into one graph"
        out["speedup"] = times["one_at_a_time"] / times["batched"]
        out["speedup_graphs"] = times["one_at_a_time"] / times["batched_graphs"]
        out["workload"] = (f"{nsys} systems, N log-uniform in [2k, 64k] ({ntot:,} particles), valency 1..6, "
                           f"kT 0.8..1.5, rho 0.2..0.6, E_a {args.E_a}, {args.batched_steps} steps each after 200")
    finally:
        for s in systems:
            s.close()
    return out


def stickers(args):
    """Timesteps/s of bead-spring sticker chains (Sec. 4): spacers and stickers,
    stickers attracting and counting stickers only at valency 1 (E_a 10), every
    pair with the soft core, harmonic bonds k = 100, r0 = 1; the typed path in
    the FP32 split (or FP64), after an untimed equilibration."""
    import torch
    from paper_2609_07842_b300 import inputs, vbc
    prec = vbc.VBC_FP32_SPLIT if args.sticker_precision == "fp32" else vbc.VBC_FP64
    pos, L, t, bonds = inputs.sticker_chains(args.sticker_chains, 64, 0.3, seed=SEED)
    vel = inputs.maxwell_velocities(pos.shape[0], KT, seed=SEED + 1)
    spacer, mixed, sticker = vbc.params(E_a=0.0, f=2.0), vbc.params(E_a=0.0), vbc.params(E_a=10.0, f=1.0)
    with vbc.System.typed(pos, L, t, [[spacer, mixed], [mixed, sticker]], [[0, 0], [0, 1]], bonds=bonds,
                          k_bond=100.0, r0_bond=1.0, vel=vel, skin=SKIN, seed=SEED, precision=prec) as s:
        s.step(args.equil, DT, KT, GAMMA)
        torch.cuda.synchronize()
        r0 = s.stats().rebuilds
        t0 = time.perf_counter()
        s.step(args.steps, DT, KT, GAMMA)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        st = s.stats()
    n = pos.shape[0]
    print(json.dumps({"metric": "sticker-chain timesteps/s", "value": args.steps / sec, "unit": "timesteps/s",
                      "ms_per_step": 1e3 * sec / args.steps, "particle_steps_per_s": n * args.steps / sec,
                      "steps": args.steps, "steps_per_rebuild": args.steps / max(st.rebuilds - r0, 1),
                      "dtype": "f32" if prec == vbc.VBC_FP32_SPLIT else "f64",
                      "precision": ("FP32 pair and bond arithmetic, fixed-point counts and state, FP64 energies"
                                    if prec == vbc.VBC_FP32_SPLIT else "FP64 throughout"),
                      "timing": "host clock around the steps, device synchronised on both sides",
                      "config": {"workload": (f"{args.sticker_chains:,} chains x 64 beads ({n:,} beads), bead "
                                              f"density 0.3, stickers every 4th bead (valency 1, E_a 10, count "
                                              f"stickers only), harmonic bonds k 100 r0 1, BAOAB dt {DT}"),
                                 "equilibration_steps": args.equil}}), flush=True)
    return 0


def served_leg(args):
    """The served stream through the serving loop, and the same stream one system
    at a time."""
    mix = run_served(args, args.served_slots)
    one = run_served(args, 1)
    return {"workload": (f"{args.served_requests} requests, Poisson arrivals at 20/s, N log-uniform in "
                         f"[1k, 200k], valency uniform in 1..8, rho {args.rho}, E_a {args.E_a}, "
                         f"{args.served_steps} steps each in 1000-step chunks, 150 GB admission budget"),
            **mix, "one_at_a_time": one,
            "speedup_vs_one_at_a_time": mix["timesteps_per_s"] / one["timesteps_per_s"]}


def leg_in_child(leg, argv, timeout, python=sys.executable):
    """Runs one optional leg (`bench.py --leg <leg>`) in a fresh Python process and
    returns its JSON object.  A leg that fails, faults or overruns gives
    {"error": ...} instead, so that it cannot take the main measurement with it."""
    cmd = [python, os.path.abspath(__file__), *argv, "--leg", leg]
    try:
        p = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return {"error": f"the {leg} leg did not finish within {timeout:g} s"}
    objs = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    if p.returncode != 0 or not objs:
        return {"error": f"the {leg} leg exited with status {p.returncode}",
                "stderr_tail": p.stderr[-800:]}
    return json.loads(objs[-1])


def leg_main(args):
    out = served_leg(args) if args.leg == "served" else run_batched(args)
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_main(args)
    if args.leg:
        return leg_main(args)
    if args.stickers:
        return stickers(args)
    if args.profile_run:
        return profile_run(args)
    if args.sweep:
        return sweep(args)

    import torch
    import torch.distributed as dist

    from paper_2609_07842_b300 import vbc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    main_m, sys_, L = measure(args, args.valency, rank, world, local, barrier, stream, with_clocks=True)
    ms = main_m["ms"]

    # ---- e2e: the same steps through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        chunk = max(1, min(args.e2e_chunk, args.steps))
        hp = torch.empty((args.n, 3), dtype=torch.float64).pin_memory().numpy()
        hv = torch.empty((args.n, 3), dtype=torch.float64).pin_memory().numpy()
        _, _, stp = sys_.get_state(hp, hv)
        barrier()
        t0 = time.perf_counter()
        done = 0
        while done < args.steps:
            c = min(chunk, args.steps - done)
            sys_.set_state(hp, hv, step=stp)         # h2d: positions + velocities
            sys_.step(c, DT, KT, GAMMA)
            _, _, stp = sys_.get_state(hp, hv)       # d2h: positions + velocities
            done += c
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, world)
        nchunks = -(-args.steps // chunk)
        e2e = {"value": whole_job_rate(args.steps, e2e_s, world), "unit": UNIT,
               "h2d_bytes_per_step": int(48 * args.n * nchunks / args.steps),
               "d2h_bytes_per_step": int(48 * args.n * nchunks / args.steps),
               "chunk_steps": chunk}

    # ---- valency 8 on the same system shape: the regime where the switching window and the
    # chain rule are live (most particles unsaturated), timed the same way (rank 0 reports it)
    v8 = None
    sys8 = None
    if not args.no_valency8 and args.valency != 8.0:
        m8, sys8, _ = measure(args, 8.0, rank, world, local, barrier, stream, with_clocks=True)
        v8 = {k: m8[k] for k in ("value", "unit", "ms_per_step", "roofline", "step_roofline", "kernel_ms_per_step",
                                 "rebuilds", "nlist_mean", "in_window_fraction", "steps_per_rebuild",
                                 "unsaturated_fraction", "pair_interactions_per_s", "thermo", "clocks",
                                 "gpu_launches", "tuning")}
        v8["config"] = workload(args, 8.0)

    # ---- served: a Poisson stream of uneven requests through the serving loop,
    # and the same stream one system at a time (rank 0, N = 1 only)
    # (each optional leg runs in a process of its own, while this one waits)
    served = None
    if rank == 0 and world == 1 and not args.no_served:
        served = leg_in_child("served", sys.argv[1:], args.leg_timeout)

    # ---- batched: many uneven systems in one graph against one at a time (rank 0, N = 1 only)
    batched = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = leg_in_child("batched", sys.argv[1:], args.leg_timeout)

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1 only), and the
    # error of the timed path against it at the state the timed region ended in
    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, k, secs, cores = run_oracle(args, args.steps, args.cpu_budget)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{k} BAOAB steps of the full N={args.n:,} system, FP64 oracle in cell-list mode "
                         f"(OpenMP), {secs:.1f} s"}
        parity = {f"valency_{args.valency:g}": end_state_parity(sys_, L, args.E_a, args.valency)}
        if sys8 is not None:
            parity["valency_8"] = end_state_parity(sys8, L, args.E_a, 8.0)

    if rank == 0:
        line = {
            "metric": METRIC, "value": whole_job_rate(args.steps, ms / 1e3, world), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload(args, args.valency),
            **{k: main_m[k] for k in ("pair_interactions_per_s", "pairs_within_rc", "roofline", "step_roofline",
                                      "kernel_ms_per_step", "rebuilds", "nlist_mean", "in_window_fraction",
                                      "steps_per_rebuild", "unsaturated_fraction", "capacities", "thermo",
                                      "gpu_launches", "clocks", "tuning")},
            "e2e": e2e,
            "valency_8": v8,
            "parity": parity,
            "served": served,
            "batched": batched,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    sys_.close()
    if sys8 is not None:
        sys8.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def measure(args, valency, rank, world, local, barrier, stream, with_clocks=True):
    """One N-particle system at the given valency: untimed equilibration, grid
    autotuning, W warm-up steps, then (1) K timed steps through the production
    path (CUDA graphs, inputs resident), (2) the same K steps with direct launches
    and a CUDA event pair around every kernel, for the per-class times, and (3)
    forced list builds, for the rebuild class.  Returns the measurement, the
    system (still open) and the box edge."""
    import torch

    from paper_2609_07842_b300 import inputs, vbc

    pos, L = inputs.uniform_positions(args.n, args.rho, seed=SEED + rank)
    vel = inputs.maxwell_velocities(args.n, KT, seed=SEED + 1 + rank)
    prm = vbc.params(E_a=args.E_a, f=valency)
    sys_ = vbc.System(pos, L, prm, vel=vel, skin=SKIN, seed=SEED + rank, stream=stream.cuda_stream)

    # untimed equilibration + warm-up
    sys_.step(args.equil, DT, KT, GAMMA)
    # grid settings picked by timed trials (changes no result; the trials are further equilibration)
    tuning = sys_.autotune(trial_steps=100, dt=DT, kT=KT, gamma=GAMMA)
    sys_.step(max(args.warmup, 3), DT, KT, GAMMA)
    st0 = sys_.stats()

    # ---- timed region 1: the production path (CUDA graphs with the rebuild behind a
    # device-side conditional), no per-kernel events
    launches0 = sys_.kernel_launches()
    clocks = start_clocks(local) if with_clocks else None
    time.sleep(0.3 if clocks else 0.0)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sys_.step(args.steps, DT, KT, GAMMA)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = stop_clocks(clocks)
    launches = sys_.kernel_launches() - launches0
    st1 = sys_.stats()
    th = sys_.thermo()  # FP64 reductions of the end state (outside the timed region)

    # ---- timed region 2: the same K steps with direct launches and a CUDA event pair
    # around every kernel on the library's stream, for per-kernel times (room for the
    # records of the iterations that overflows halt and their retries re-run: a system
    # still clustering can grow its capacities several times in one call)
    sys_.profile(True, max_launches=48 * (args.steps + 2) + 64)
    barrier()
    ev0.record(stream)
    sys_.step(args.steps, DT, KT, GAMMA)
    ev1.record(stream)
    barrier()
    ms_direct = ev0.elapsed_time(ev1)
    force_ms, force_n = sys_.profile_read(vbc.K_FORCE)
    count_ms, count_n = sys_.profile_read(vbc.K_COUNT)
    chain_ms, chain_n = sys_.profile_read(vbc.K_CHAIN)
    reb_ms, reb_n = sys_.profile_read(vbc.K_REBUILD)
    sys_.profile(False)
    st_d = sys_.stats()

    # ---- timed region 3: forced neighbour-list builds, one event pair each
    nb = 5
    sys_.profile(True, max_launches=4 * nb + 4)
    for _ in range(nb):
        sys_.build_neighbors()
    b_ms, b_n = sys_.profile_read(vbc.K_REBUILD)
    sys_.profile(False)
    build_ms = b_ms / max(b_n, 1)

    ms = max_over_ranks(ms, world)

    # pair interactions (unordered pairs with r < r_c) at the end configuration
    r = sys_.compute(energy=True)
    st2 = sys_.stats()
    pairs = st2.pairs_within_rc
    k_mean = st1.nlist_mean
    rebuilds = st1.rebuilds - st0.rebuilds
    rebuilds_direct = st_d.rebuilds - st1.rebuilds
    rebuild_every = args.steps / rebuilds if rebuilds > 0 else float("inf")
    phi = st2.in_window / args.n

    steps_per_s = whole_job_rate(args.steps, ms / 1e3, world)
    peak, peak_kind = hbm_peak()
    cb = class_bytes_per_particle(k_mean, phi)
    # per-launch duration of each class; the rebuild class from forced builds
    # (timed region 3), the others from timed region 2
    per_launch_ms = {"count": count_ms / max(count_n, 1), "chain": chain_ms / max(chain_n, 1),
                     "force": force_ms / max(force_n, 1), "rebuild": build_ms}
    share_ms = {"count": count_ms / args.steps, "chain": chain_ms / args.steps, "force": force_ms / args.steps,
                "rebuild": build_ms / rebuild_every if rebuilds else 0.0}  # rebuilds amortised per step
    classes = {}
    for c_, ms_ in per_launch_ms.items():
        b_ = cb[c_] * args.n
        ach = b_ / (ms_ / 1e3) / 1e9 if ms_ > 0 else 0.0
        classes[c_] = {"achieved": ach, "frac": ach / peak, "algorithmic_bytes_per_launch": b_,
                       "avg_launch_ms": ms_, "ms_per_step": share_ms[c_],
                       "traffic": ncu_traffic(c_, args.n)}
    dominant = max(share_ms, key=lambda c_: share_ms[c_])
    step_b = sum(cb[c_] for c_ in ("count", "chain", "force")) * args.n
    if rebuilds:
        step_b += cb["rebuild"] * args.n / rebuild_every
    step_gbs = step_b * (args.steps / (ms / 1e3)) / 1e9
    m = {
        "ms": ms, "value": steps_per_s, "unit": UNIT, "ms_per_step": ms / args.steps,
        "pair_interactions_per_s": pairs * steps_per_s, "pairs_within_rc": pairs,
        "roofline": {"bound": "hbm", "achieved": classes[dominant]["achieved"], "peak": peak,
                     "unit": "GB/s", "frac": classes[dominant]["frac"],
                     "traffic": classes[dominant]["traffic"], "kernel": dominant,
                     "kernels": KERNELS_OF[dominant], "peak_source": peak_kind,
                     "timing": ("CUDA events around every launch on the library stream (forced builds for "
                                "the rebuild class)"),
                     "algorithmic_bytes_per_launch": classes[dominant]["algorithmic_bytes_per_launch"],
                     "avg_launch_ms": classes[dominant]["avg_launch_ms"],
                     "dominant_by": "device time per step (rebuilds amortised)",
                     "classes": classes},
        "step_roofline": {"achieved": step_gbs, "frac": step_gbs / peak, "algorithmic_bytes_per_step": step_b,
                          "bytes_per_particle_step": step_b / args.n, "peak_source": peak_kind},
        "kernel_ms_per_step": {"rebuild": reb_ms / args.steps, "count": count_ms / args.steps,
                               "chain": chain_ms / args.steps, "force": force_ms / args.steps,
                               "build_ms": build_ms,
                               "source": "timed region 2 (direct launches, CUDA events per kernel); "
                                         "build_ms: forced builds (region 3)",
                               "ms_per_step_direct": ms_direct / args.steps,
                               "rebuilds": rebuilds_direct},
        "rebuilds": rebuilds, "nlist_mean": k_mean, "in_window_fraction": phi,
        "steps_per_rebuild": rebuild_every, "unsaturated_fraction": st2.unsaturated / args.n,
        "capacities": {"stage": st2.stage_cap, "group": st2.group_cap, "list": st2.nlist_cap, "groups": st2.groups,
                       "grows_in_timed_region": st1.capacity_grows - st0.capacity_grows},
        "thermo": {"energy_per_particle": th.U / args.n, "virial_per_particle": th.W / args.n,
                   "kinetic_temperature": 2.0 * th.KE / (3.0 * args.n), "mean_count": th.mean_n,
                   "in_window": th.in_window, "step": th.step,
                   "source": "vbc_compute_thermo at the end of timed region 1 (FP64 device reductions)"},
        "energy_per_particle": r.energy / args.n,
        "gpu_launches": launches,
        "clocks": clk,
        "tuning": {"rows_blocks_per_sm": tuning.rows_blocks_per_sm,
                   "count_blocks_per_sm": tuning.count_blocks_per_sm,
                   "rows_threads_per_block": tuning.rows_threads_per_block,
                   "threads_per_row_max": tuning.threads_per_row_max,
                   "trial_ms_per_step": tuning.ms_per_step, "note": "blocks per SM: 0 = as many as fit"},
    }
    return m, sys_, L


# Tolerances of the parity tests (tests/test_gpu_parity.py), FP32-split path.
PARITY_TOL = {"count_abs": 1e-6, "force_rel_rms": 1e-5, "energy_rel": 1e-9}


def end_state_parity(sys_, L, E_a, valency):
    """Error of the library against the FP64 oracle at the state a timed run
    ended in: counts and forces (vbc_compute_forces) and U, element by element
    over all particles, the oracle in its cell-list mode at the positions read
    back from the device."""
    import oracle
    x, _, step = sys_.get_state()
    r = sys_.compute(F=True, counts=True, energy=True)
    t0 = time.perf_counter()
    ref = oracle.evaluate(x, L, oracle.Params(E_a=E_a, f=valency), mode=1)
    secs = time.perf_counter() - t0
    rms = float(np.sqrt(np.mean(np.sum(ref.F ** 2, axis=1))))
    out = {"max_abs_dcount": float(np.max(np.abs(r.counts - ref.counts))),
           "max_abs_dF_over_rms": float(np.max(np.abs(r.F - ref.F)) / rms),
           "rel_dU": abs(r.energy - ref.U) / abs(ref.U),
           "in_window_fraction": float(np.mean(ref.ds != 0.0)), "step": step,
           "tolerances": PARITY_TOL, "oracle_seconds": secs}
    out["ok"] = (out["max_abs_dcount"] <= PARITY_TOL["count_abs"]
                 and out["max_abs_dF_over_rms"] <= PARITY_TOL["force_rel_rms"]
                 and out["rel_dU"] <= PARITY_TOL["energy_rel"])
    return out


if __name__ == "__main__":
    sys.exit(main())
