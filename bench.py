#!/usr/bin/env python3
"""Throughput benchmark of the voxel Monte Carlo photon walk on GB300 (photons/ms).

One step = one complete simulation (zero outputs, persistent walk kernel over every photon,
FP64 tally reduction) of the heterogeneous two-sphere workload: 64^3 voxels of 1 mm, two
overlapping spherical inclusions, 1e8 photons, 10 time gates of 0.5 ns, four r = 2 mm disk
detectors recording partial path lengths.  Inputs are resident in HBM when the timed region
starts; `e2e` repeats the measurement through the C ABI with host buffers (label upload and
fluence/tally/detected-record read-back inside the timed region).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU (torchrun, one rank per GPU): each rank simulates its own photon-id range of the
same size (weak scaling; photon ranges are independent, so there is no data-path
collective); the max step time over ranks gives the job throughput.  `--impl reference`
times the FP64 CPU oracle on bounded samples of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "photons/ms on one GB300"
UNIT = "photons/ms"
WORKLOAD = "c2_two_spheres_64"
WORKLOAD_DESC = ("64^3 x 1 mm label volume, background (mua 0.01, mus 10, g 0.9, n 1.37) with "
                 "spheres r=10 @ (32,32,24) and r=8 @ (20,40,30), pencil beam (32,32,0) +z, "
                 "1e8 photons, 10 gates x 0.5 ns, 4 disk detectors r=2 mm on z=0")

# Algorithmic thread-operations per event of the walk (counted from the algorithm's
# arithmetic, independent of the compiled code): every segment (face distances, event
# selection, gate, advance, absorption, run-length accumulation), a hop draw, a
# scattering event (2 uniforms, HG, azimuth, rotation, 3 reciprocals, roulette test), a
# face crossing, a Fresnel evaluation, a fluence flush, and a photon launch + finish.
OPS = {"segment": 35, "hop": 17, "scatter": 65, "face": 15, "fresnel": 25, "flush": 3,
       "photon": 60}
SM_COUNT = 152
LANES_PER_SM = 128          # 4 SM sub-partitions x 32 lanes issue per clock

# Special-function-unit operations per event of the FP32 walk: one ex2 per segment (the
# attenuation), one lg2 per hop; per scattering event the HG reciprocal, the sine from the
# deflection's cosine pair (square root), the azimuth's sine and cosine, the rotation's
# reciprocal square root and the three reciprocals of the new direction; per Fresnel
# evaluation two quotients and two square roots (incidence and refraction).
XU_OPS = {"segment": 1, "hop": 1, "scatter": 8, "fresnel": 4}

C3_WORKLOAD = "c3_layered_256x256x128"
C3_DESC = ("256x256x128 x 0.5 mm label volume, 4 planar layers 3/7/2/rest mm (mua 0.019/0.019/"
           "0.004/0.02, mus 7.8/9.4/0.01/6.6, g 0.89, n 1.37) in air, Gaussian beam w = 2 mm at "
           "the top centre +z, 1e9 photons, 50 gates x 0.1 ns, FP64 accumulation map 3.4 GB")


def algorithmic_ops(stats: dict, tally: dict) -> float:
    seg = stats["scatter"] + stats["face"] + stats["photons"]
    hop = stats["scatter"] + stats["photons"]
    return (OPS["segment"] * seg + OPS["hop"] * hop + OPS["scatter"] * stats["scatter"] +
            OPS["face"] * stats["face"] + OPS["fresnel"] * stats["fresnel"] +
            OPS["flush"] * stats["flush"] + OPS["photon"] * stats["photons"])


def xu_ops(stats: dict) -> float:
    seg = stats["scatter"] + stats["face"] + stats["photons"]
    hop = stats["scatter"] + stats["photons"]
    return (XU_OPS["segment"] * seg + XU_OPS["hop"] * hop + XU_OPS["scatter"] * stats["scatter"] +
            XU_OPS["fresnel"] * stats["fresnel"])


def measure_rates(mcx, map_bytes: dict) -> dict:
    """Measured rates (ops/s) of the resources the walk draws on (the library's
    microbenchmarks): FMA and logic issue, the special-function unit, and FP64 atomics over
    each workload's FP64 fluence map (and to hot words)."""
    r = {k: mcx.mcx_probe_rate(k) for k in ("ffma", "lop3", "lg2", "ex2", "rsqrt", "sin")}
    for name, nb in map_bytes.items():
        r[f"red_f64_{name}"] = mcx.mcx_probe_rate("red_f64", nb)
        r[f"red_f32_{name}"] = mcx.mcx_probe_rate("red_f32", nb // 2)
    r["red_f64_hot"] = mcx.mcx_probe_rate("red_f64_hot")
    return r


def co_bounds(stats: dict, n: int, ms: float, rates: dict, map_name: str, nominal_peak: float,
              traffic=None, hbm_gbs=None) -> dict:
    """The walk against each resource it draws on: photons/ms that resource alone would
    allow (rate / per-photon demand), the walk's achieved photons/ms, and the fraction.
    The atomic bound takes the rate over an L2-resident map (the best the L2 sustains);
    for a map larger than L2 the rate with addresses spread uniformly over all of it is
    reported beside it as a lower bound, not used for the binding resource, since the
    walk's deposits concentrate near the source.  With a measured DRAM traffic per launch,
    HBM bandwidth is a bound too."""
    ops, xu, fl = algorithmic_ops(stats, None) / n, xu_ops(stats) / n, stats["flush"] / n
    xu_rate = min(rates[k] for k in ("lg2", "ex2", "rsqrt", "sin"))
    at_rate = rates["red_f64_c2"]
    achieved = n / ms
    b = {"issue_nominal": {"per_photon": ops, "rate": nominal_peak * 1e12},
         "issue_measured_ffma": {"per_photon": ops, "rate": rates["ffma"]},
         "xu": {"per_photon": xu, "rate": xu_rate},
         "l2_atomics_f64": {"per_photon": fl, "rate": at_rate}}
    if traffic and hbm_gbs:
        b["hbm"] = {"per_photon": traffic / n, "rate": hbm_gbs * 1e9, "unit": "bytes"}
    for v in b.values():
        v["bound_photons_per_ms"] = v["rate"] / v["per_photon"] / 1e3
        v["frac"] = achieved / v["bound_photons_per_ms"]
    binding = min((k for k in b if k != "issue_nominal"), key=lambda k: b[k]["bound_photons_per_ms"])
    out = {"achieved_photons_per_ms": achieved, "bounds": b, "binding": binding,
           "walk_atomics_per_s": stats["flush"] / (ms * 1e-3)}
    if map_name != "c2":
        r = rates[f"red_f64_{map_name}"]
        out["atomics_spread_over_map"] = {"rate": r, "bound_photons_per_ms": r / fl / 1e3,
                                          "frac": achieved / (r / fl / 1e3)}
    return out


def peaks() -> dict:
    p = {"sm_max_mhz": 2070.0, "bf16_tflops": 1900.0, "hbm_gbs": 6800.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        p["sm_max_mhz"] = float(d.get("sm_max_mhz", 2070.0))
        p["bf16_tflops"] = float(d.get("bf16_tflops", 1900.0))
        p["hbm_gbs"] = float(d.get("hbm_gbs", 6800.0))
        p["source"] = "measured"
    return p


def walk_code_hash(path: str) -> str:
    """sha256[:16] of a source file's code: '//' comments, trailing blanks and empty lines
    removed, so that a change of comments alone keeps a capture valid."""
    lines = []
    for ln in open(path).read().splitlines():
        ln = re.sub(r"//.*", "", ln).rstrip()
        if ln.strip():
            lines.append(ln)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def walk_traffic(profile: str = "walk_kernel_c2.md", photons: int = None):
    """DRAM bytes per walk launch from the committed ncu summary, if it was taken on the
    current kernel source (matching hash); otherwise None.  A summary taken on fewer
    photons than the launch states its traffic per photon, which is scaled to `photons`
    (the map's lines are refetched at a steady per-photon rate)."""
    src = os.path.join(ROOT, "paper_1711_03244_gb300", "csrc", "walk.cu")
    prof = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(prof):
        return None
    h = walk_code_hash(src)
    text = open(prof).read()
    m_h = re.search(r"walk\.cu code sha256\[:16\][^:\n]*:\s*([0-9a-f]{16})", text)
    if not (m_h and m_h.group(1) == h):
        return None
    m_b = re.search(r"dram bytes per full launch:\s*([0-9.eE+]+)", text)
    if m_b:
        return float(m_b.group(1))
    m_p = re.search(r"dram bytes per photon:\s*([0-9.eE+]+)", text)
    if m_p and photons:
        return float(m_p.group(1)) * photons
    return None


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, wl, world, rank):
    """FP64 CPU oracle on bounded samples of the same workload (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n = args.ref_photons
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle.run(wl, n_photons=max(n // 10, 1), energy=True, n_threads=cores)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(wl, n_photons=n, photon_offset=k * n, energy=True, n_threads=cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = n / ms
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "photons_per_step": n,
                       "note": "each step is a bounded sample of the workload's photons"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} photons of {WORKLOAD} per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def study_paper(args):
    """The paper's benchmarks (60 mm cube, pencil beam, 1e8 photons; B2/B2a with the
    r = 15 mm sphere; B1 terminates at the boundary), each step timed like the main bench.
    Rows: accumulation plain FP32 / FP64 / compensated tiles (the library's counterpart of
    the paper's non-atomic B2 vs atomic B2a comparison: B2's racy adds are not built), and
    photon distribution dynamic vs the static per-thread split (the paper's Fig. 3a)."""
    import torch
    import paper_1711_03244_gb300 as mcx
    from paper_1711_03244_gb300 import build as mcx_build
    mcx_build.build()
    mcx.load()
    stream = torch.cuda.current_stream()
    rows = [("B1", 2, 0), ("B1", 0, 0), ("B1", 1, 0), ("B1", 2, 1),
            ("B2a", 2, 0), ("B2a", 0, 0), ("B2a", 1, 0), ("B2a", 2, 1)]
    for name, accum, claim in rows:
        wl = workloads.paper_b("B1" if name == "B1" else "B2", n_photons=args.photons or 100_000_000)
        with mcx.Simulation.from_workload(wl) as sim:
            def step():
                cfg = mcx.mcx_run_cfg_default(n_photons=wl.n_photons, n_gates=wl.n_gates,
                                              dt_ns=wl.dt_ns, seed=wl.seed, reflect=wl.reflect,
                                              accum_mode=accum, claim_mode=claim,
                                              cuda_stream=stream)
                mcx.mcx_run(sim.handle, cfg)
            for _ in range(args.warmup):
                step()
                mcx.mcx_sync(sim.handle, allow_cap=True)
            ms = []
            for _ in range(args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            stats = mcx.mcx_read_stats(sim.handle)
        best = min(ms)
        print(json.dumps({"study": "paper", "workload": name, "photons": wl.n_photons,
                          "accum_mode": accum, "claim_mode": claim,
                          "photons_per_ms_best": wl.n_photons / best,
                          "photons_per_ms_median": wl.n_photons / float(np.median(ms)),
                          "ms_best": best, "scatter_per_photon": stats["scatter"] / wl.n_photons,
                          "face_per_photon": stats["face"] / wl.n_photons}), flush=True)


def study_batched(args):
    """The batched workload: 256 seeded volumes (side 32..128 mm, 1-3 ellipsoids, random
    optics, 1e5..1e7 photons each, 5 gates of 1 ns) as one persistent launch recorded in a
    CUDA graph with the autotuned shape, against one mcx_run per simulation."""
    import torch
    import paper_1711_03244_gb300 as mcx
    from paper_1711_03244_gb300 import build as mcx_build
    mcx_build.build()
    mcx.load()
    stream = torch.cuda.Stream()
    sims = workloads.c4()
    total = sum(w.n_photons for w in sims)
    with mcx.Batch() as b:
        for wl in sims:
            b.add_workload(wl)
        best = b.autotune(fraction=0.05, n_gates=5, dt_ns=1.0, cuda_stream=stream)
        cfg = dict(n_gates=5, dt_ns=1.0, block_size=best["block_size"],
                   claim_chunk=best["claim_chunk"], use_graph=1, cuda_stream=stream)
        for _ in range(args.warmup):
            b.run(**cfg)
        ms = []
        for _ in range(args.steps):
            b.run(**cfg)
            ms.append(b.last_ms())
        stats = b.stats()
    # the same simulations one at a time (each a complete mcx_run: zero, walk, reduce)
    seq_ms = 0.0
    for wl in sims:
        with mcx.Simulation.from_workload(wl) as sim:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mcx.mcx_run(sim.handle, mcx.mcx_run_cfg_default(
                n_photons=wl.n_photons, n_gates=5, dt_ns=1.0, seed=wl.seed, cuda_stream=stream))
            e1.record(stream)
            e1.synchronize()
            seq_ms += e0.elapsed_time(e1)
    # the batch walk against the same issue roofline as the main bench line
    pk = peaks()
    ops = algorithmic_ops(stats, None)
    peak = SM_COUNT * LANES_PER_SM * pk["sm_max_mhz"] * 1e6 / 1e12
    achieved = ops / (min(ms) * 1e-3) / 1e12
    print(json.dumps({"study": "batched", "simulations": len(sims), "photons": total,
                      "autotuned": best, "batch_ms_best": min(ms),
                      "batch_photons_per_ms": total / min(ms),
                      "sequential_ms": seq_ms, "sequential_photons_per_ms": total / seq_ms,
                      "speedup": seq_ms / min(ms), "photons_simulated": stats["photons"],
                      "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                                   "unit": "Tthread-op/s", "frac": achieved / peak,
                                   "ops_per_photon": ops / max(stats["photons"], 1),
                                   "note": "whole graph replay (zeroing, walk, reductions)"}}),
          flush=True)


def study_denoise(args):
    """The learned denoiser: train on seeded 64 mm volumes (input: args.dn_in photons,
    target: args.dn_target photons, independent seeds), then on held-out volumes compare
    the voxel-wise log10 RMS error against args.dn_ref-photon references of the denoised
    low-photon map with plain runs along a photon ladder, and the wall time (walk kernel
    time, plus the network pass for the denoised path) at equal error.  Every training
    configuration of args.dn_configs ("steps:batch:lr", comma separated) is trained from
    the same initial weights on the same data and evaluated on the same held-out runs;
    one JSON line each."""
    import torch
    import paper_1711_03244_gb300 as mcx
    from paper_1711_03244_gb300 import build as mcx_build
    from paper_1711_03244_gb300 import denoise as dn
    mcx_build.build()
    mcx.load()
    dev = torch.device("cuda")
    shape = (64, 64, 64)
    n_aux = args.dn_aux
    configs = [tuple(c.split(":")) for c in args.dn_configs.split(",")] if args.dn_configs else \
        [(str(args.dn_steps), str(args.dn_batch), str(args.dn_lr))]
    configs = [(int(a), int(b), float(c)) for a, b, c in configs]
    train_v = workloads.c5(args.dn_train, seed=1711032450)
    test_v = workloads.c5(args.dn_test, seed=1711032451)
    n_t = len(test_v)

    # training data: network-domain pairs (a throw-away denoiser object does the encoding)
    t0 = time.time()
    phi_in = torch.empty((len(train_v),) + shape, device=dev)
    phi_tg = torch.empty_like(phi_in)
    ms_in = dn.simulate(train_v, args.dn_in, phi_in, seed_offset=0)
    ms_tg = dn.simulate(train_v, args.dn_target, phi_tg, seed_offset=1_000_003)
    gen_s = time.time() - t0
    with mcx.Denoiser(shape, max_batch=1) as enc:
        x_set, t_set = torch.empty_like(phi_in), torch.empty_like(phi_tg)
        dn.encode_set(enc, phi_in, x_set)
        dn.encode_set(enc, phi_tg, t_set)
    del phi_in, phi_tg
    aux_set = aux_t = None
    if n_aux:
        aux_set = torch.empty((len(train_v), 2) + shape, device=dev)
        dn.features(train_v, aux_set)
        aux_t = torch.empty((n_t, 2) + shape, device=dev)
        dn.features(test_v, aux_t)

    # held-out references and the plain photon ladder
    ref = torch.empty((n_t,) + shape, device=dev)
    dn.simulate(test_v, args.dn_ref, ref, seed_offset=2_000_003)
    ref_h = ref.cpu().numpy()
    ladder = [int(round(args.dn_in * f)) for f in (1, 3, 10, 30, 100, 300, 1000)]
    ladder = [n for n in ladder if n <= args.dn_ladder_max]
    plain_rms, plain_ms = [], []
    low = torch.empty_like(ref)
    for li, n in enumerate(ladder):
        ms = dn.simulate(test_v, n, low, seed_offset=3_000_017 + li)
        h = low.cpu().numpy()
        plain_rms.append(float(np.mean([dn.log_rms(h[i], ref_h[i]) for i in range(n_t)])))
        plain_ms.append(ms)
        if li == 0:
            low_in = low.clone()
            walk_in_ms = ms
    del low
    lr_, ln_, lt_ = np.log(plain_rms), np.log(ladder), np.log(plain_ms)
    # tensor-core work of one forward pass per volume (the ten 3x3x3 convolutions)
    npos = [64 ** 3, 64 ** 3, 32 ** 3, 32 ** 3, 16 ** 3, 16 ** 3, 32 ** 3, 32 ** 3, 64 ** 3, 64 ** 3]
    chans = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]
    fwd_flop = sum(2 * p * 27 * ci * co for p, (ci, co) in zip(npos, chans))
    pk = peaks()

    for steps, batch, lr in configs:
        d = mcx.Denoiser(shape, max_batch=max(batch, 16), seed=args.dn_seed, n_aux=n_aux)
        torch.cuda.synchronize()
        t1 = time.time()
        losses = dn.train(d, x_set, t_set, steps, batch, lr=lr, lr_final=lr / 10, seed=args.dn_seed,
                          log_every=max(steps // 10, 1), aux_set=aux_set)
        torch.cuda.synchronize()
        train_s = time.time() - t1
        out = torch.empty_like(ref)
        dn.denoise(d, low_in, out, aux=aux_t)      # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record()
        for _ in range(reps):
            dn.denoise(d, low_in, out, aux=aux_t)
        e1.record()
        e1.synchronize()
        d.sync()
        apply_ms = e0.elapsed_time(e1) / reps
        oh = out.cpu().numpy()
        den_rms = float(np.mean([dn.log_rms(oh[i], ref_h[i]) for i in range(n_t)]))
        # photons (and walk time) a plain run needs for the denoised error: log-log
        # interpolation along the ladder, extrapolated with the last slope past its end
        if den_rms >= plain_rms[0]:
            n_eq, t_eq, how = float(ladder[0]), plain_ms[0], "denoised no better than the input"
        else:
            j = next((j for j in range(1, len(ladder)) if plain_rms[j] <= den_rms), None)
            how = "interpolated"
            if j is None:
                j, how = len(ladder) - 1, "extrapolated"
            a = (np.log(den_rms) - lr_[j - 1]) / (lr_[j] - lr_[j - 1])
            n_eq = float(np.exp(ln_[j - 1] + a * (ln_[j] - ln_[j - 1])))
            t_eq = float(np.exp(lt_[j - 1] + a * (lt_[j] - lt_[j - 1])))
        den_ms = walk_in_ms + apply_ms
        tflops = fwd_flop * n_t / (apply_ms * 1e-3) / 1e12
        print(json.dumps({
            "study": "denoise", "volumes": "64x64x64 mm, 1-3 ellipsoids, random optics (c5)",
            "feature_channels": n_aux,
            "train_volumes": len(train_v), "test_volumes": n_t, "photons_input": args.dn_in,
            "photons_target": args.dn_target, "photons_reference": args.dn_ref,
            "data_walk_ms": ms_in + ms_tg, "data_wall_s": gen_s,
            "train_steps": steps, "train_batch": batch, "train_lr": lr, "train_s": train_s,
            "train_ms_per_step": 1e3 * train_s / max(steps, 1),
            "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-50:])),
            "ladder_photons": ladder, "ladder_rms": plain_rms, "ladder_walk_ms": plain_ms,
            "input_rms": plain_rms[0], "denoised_rms": den_rms,
            "plain_photons_for_denoised_rms": n_eq, "plain_ms_for_denoised_rms": t_eq, "equal_error": how,
            "denoised_ms": den_ms, "denoised_walk_ms": walk_in_ms, "denoiser_apply_ms": apply_ms,
            "time_fraction_of_plain": den_ms / t_eq if t_eq else None,
            "apply_tflops": tflops, "bf16_peak_tflops": pk["bf16_tflops"],
            "apply_frac_of_peak": tflops / pk["bf16_tflops"] if pk["bf16_tflops"] else None,
        }), flush=True)
        d.close()


def study_peaks(args):
    """Measured rates of the walk's resources (issue, special-function unit, FP32/FP64
    atomics over L2-resident and HBM-resident maps and to hot words), each the best of
    args.steps repetitions, against the nominal issue rate."""
    import paper_1711_03244_gb300 as mcx
    from paper_1711_03244_gb300 import build as mcx_build
    mcx_build.build()
    mcx.load()
    pk = peaks()
    maps = {"l2_10MiB": 10 << 20, "l2_21MB_c2": 64 ** 3 * 10 * 8, "hbm_3.4GB_c3": 256 * 256 * 128 * 50 * 8}
    best = {}
    for _ in range(max(args.steps, 1)):
        r = measure_rates(mcx, maps)
        for k, v in r.items():
            best[k] = max(best.get(k, 0.0), v)
    nominal = SM_COUNT * LANES_PER_SM * pk["sm_max_mhz"] * 1e6
    print(json.dumps({"study": "peaks", "rates_ops_per_s": best,
                      "nominal_issue_thread_ops_per_s": nominal,
                      "ffma_frac_of_nominal": best["ffma"] / nominal,
                      "lop3_frac_of_nominal": best["lop3"] / nominal,
                      "xu_per_sm_per_clock": {k: best[k] / SM_COUNT / (pk["sm_max_mhz"] * 1e6)
                                              for k in ("lg2", "ex2", "rsqrt", "sin")}}), flush=True)


def study_denoise_kernels(args):
    """The denoiser's kernels alone on synthetic inputs: one forward pass over 16 volumes of
    64^3 (every 3x3x3 convolution on tcgen05) and one training step of batch 4, each the
    median of args.steps timed repetitions after args.warmup untimed ones (CUDA events)."""
    import torch
    import paper_1711_03244_gb300 as mcx
    from paper_1711_03244_gb300 import build as mcx_build
    mcx_build.build()
    mcx.load()
    shape, nb = (64, 64, 64), 16
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn((nb,) + shape, device="cuda", generator=g)
    t = x + 0.1 * torch.randn((nb,) + shape, device="cuda", generator=g)
    y = torch.empty_like(x)
    npos = [64 ** 3, 64 ** 3, 32 ** 3, 32 ** 3, 16 ** 3, 16 ** 3, 32 ** 3, 32 ** 3, 64 ** 3, 64 ** 3]
    # the input layer's one channel (no medium features) is its algorithmic work, not the
    # 16 channels its padded weight gradient is computed on
    chans = [(1, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]
    fwd = sum(2 * p * 27 * ci * co for p, (ci, co) in zip(npos, chans))
    # a training step: forward, input gradients of every layer but the first, weight gradients
    dgrad = fwd - 2 * npos[0] * 27 * 1 * 16
    with mcx.Denoiser(shape, max_batch=nb, seed=1) as d:
        def timed(fn):
            for _ in range(args.warmup):
                fn()
            ms = []
            for _ in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            d.sync()
            return float(np.median(ms))
        f_ms = timed(lambda: d.forward(x, y))
        t_ms = timed(lambda: d.train_step(x[:4], t[:4], 1e-4))
    pk = peaks()
    f_tf = fwd * nb / (f_ms * 1e-3) / 1e12
    t_tf = (fwd + dgrad + fwd) * 4 / (t_ms * 1e-3) / 1e12
    print(json.dumps({"study": "denoise-kernels", "volumes": f"{nb} x 64^3 forward, 4 x 64^3 train",
                      "forward_ms": f_ms, "forward_gflop_per_volume": fwd / 1e9,
                      "forward_tflops": f_tf, "train_step_ms": t_ms, "train_tflops": t_tf,
                      "bf16_peak_tflops": pk["bf16_tflops"],
                      "forward_frac_of_peak": f_tf / pk["bf16_tflops"]}), flush=True)


def bench_c3(args, mcx, torch, stream, rates, nominal_peak):
    """The layered-tissue workload at its configured 1e9 photons (the largest single-GPU
    configuration; its 3.4 GB FP64 map lives in HBM, not L2): args.c3_warmup untimed runs,
    then args.c3_steps timed ones (CUDA events on the launching stream), the same
    e2e measurement through the C ABI with host buffers, the roofline and co-bounds with
    this workload's event counts, and the oracle on a bounded sample."""
    wl = workloads.c3(n_photons=args.c3_photons)
    n = wl.n_photons
    sim = mcx.Simulation.from_workload(wl)

    def step():
        cfg = mcx.mcx_run_cfg_default(n_photons=n, n_gates=wl.n_gates, dt_ns=wl.dt_ns,
                                      seed=wl.seed, cuda_stream=stream)
        mcx.mcx_run(sim.handle, cfg)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.c3_warmup):
        step()
        mcx.mcx_sync(sim.handle, allow_cap=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.c3_steps)]
    walk_ms = []
    with ClockSampler(int(torch.cuda.current_device())) as clk:
        torch.cuda.synchronize()
        for k in range(args.c3_steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            walk_ms.append(mcx.mcx_last_kernel_ms(sim.handle))
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    stats = mcx.mcx_read_stats(sim.handle)
    tally = mcx.mcx_read_tally(sim.handle)
    total_ms = float(sum(step_ms))
    walk_avg = float(np.mean(walk_ms))
    # e2e: labels and media in from pinned host memory, run, normalised fluence and tallies
    # back to pinned host memory, all inside the timed region
    labels_pinned = torch.from_numpy(wl.labels).pin_memory()
    flu_pinned = torch.empty((wl.n_gates,) + wl.labels.shape, dtype=torch.float32).pin_memory()
    e2e_times = []
    for k in range(args.c3_e2e_steps + 1 if args.c3_e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mcx.mcx_update_labels(sim.handle, labels_pinned.numpy())
        mcx.mcx_set_media(sim.handle, wl.media)
        step()
        mcx.mcx_sync(sim.handle, allow_cap=True)
        mcx.mcx_read_fluence(sim.handle, flu_pinned.numpy(), normalized=True)
        mcx.mcx_read_tally(sim.handle)
        dt = time.perf_counter() - t0
        if k > 0:
            e2e_times.append(dt)
    sim.close()
    del flu_pinned, labels_pinned
    e2e_ms = 1e3 * float(np.mean(e2e_times)) if e2e_times else float("nan")
    ops = algorithmic_ops(stats, tally)
    achieved = ops / (walk_avg * 1e-3) / 1e12
    out = {"workload": C3_WORKLOAD, "desc": C3_DESC, "value": n * args.c3_steps / total_ms,
           "unit": UNIT, "steps": args.c3_steps, "warmup": args.c3_warmup,
           "ms_per_step": total_ms / args.c3_steps, "photons_per_step": n,
           "l2": "inputs larger than L2 (3.4 GB FP64 map); 256 MiB write between steps",
           "accumulation": "FP64 L2 atomics per (gate, voxel) run (accum_mode 2)",
           "clocks": clk.summary(),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": nominal_peak,
                        "unit": "Tthread-op/s", "frac": achieved / nominal_peak,
                        "traffic": walk_traffic("walk_kernel_c3.md", n),
                        "ops_per_photon": ops / n, "kernel": "walk_kernel<float,false>",
                        "walk_ms": walk_avg},
           "co_bounds": co_bounds(stats, n, walk_avg, rates, "c3", nominal_peak,
                                  walk_traffic("walk_kernel_c3.md", n), peaks()["hbm_gbs"])
           if rates else None,
           "e2e": {"value": n / e2e_ms if e2e_times else None, "unit": UNIT,
                   "h2d_bytes_per_step": int(wl.labels.nbytes + wl.media.astype(np.float32).nbytes),
                   "d2h_bytes_per_step": int(wl.n_gates * wl.labels.size * 4 + 6 * 8),
                   "steps": args.c3_e2e_steps},
           "events": {k: int(v) for k, v in stats.items()},
           "energy_balance_rel": abs(tally["absorbed"] + tally["escaped"] + tally["time_exceeded"] +
                                     tally["roulette_killed"] - tally["roulette_gained"] -
                                     tally["launched"]) / max(tally["launched"], 1.0),
           "gpu_launches": 5 * args.c3_steps}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        nc = args.c3_cpu_photons
        t0 = time.perf_counter()
        oracle.run(wl, n_photons=nc, energy=True, n_threads=cores)
        cpu_ms = 1e3 * (time.perf_counter() - t0)
        out["cpu_baseline"] = {"value": nc / cpu_ms, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"first {nc} photons of {C3_WORKLOAD} (FP64 oracle, "
                                         f"{cores} OpenMP threads, {cpu_ms / 1e3:.1f} s)"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c3"],
                    help="the timed workload: c2 (two-sphere volume, the metric's configuration) "
                         "or c3 (layered tissue, 1e9 photons)")
    ap.add_argument("--photons", type=int, default=None,
                    help="photons per step (default 1e8 for c2, 1e9 for c3)")
    ap.add_argument("--ref-photons", type=int, default=200_000)
    ap.add_argument("--cpu-photons", type=int, default=1_500_000)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--c3-photons", type=int, default=1_000_000_000)
    ap.add_argument("--c3-steps", type=int, default=2)
    ap.add_argument("--c3-warmup", type=int, default=1,
                    help="untimed C3 runs (the GPU is already warm from the C2 steps)")
    ap.add_argument("--c3-e2e-steps", type=int, default=1)
    ap.add_argument("--c3-cpu-photons", type=int, default=200_000)
    ap.add_argument("--no-c3", action="store_true", help="skip the layered-tissue C3 leg")
    ap.add_argument("--no-probes", action="store_true",
                    help="skip the microbenchmarks of the issue, XU and atomic rates")
    ap.add_argument("--no-model", action="store_true",
                    help="skip the pilot runs of the linear runtime model T = a n + T0")
    ap.add_argument("--study", default=None,
                    choices=["paper", "batched", "denoise", "denoise-kernels", "peaks"],
                    help="paper: the paper's benchmarks B1/B2/B2a under each accumulation and "
                         "photon-distribution mode; batched: the 256-simulation batch in one "
                         "launch vs one launch per simulation; denoise: train the learned "
                         "denoiser and compare denoised and plain runs at equal error; "
                         "denoise-kernels: the denoiser's forward pass and training step "
                         "alone; peaks: the microbenchmarked rates of the resources the walk "
                         "draws on (one JSON line each)")
    ap.add_argument("--dn-train", type=int, default=4096, help="training volumes")
    ap.add_argument("--dn-test", type=int, default=64, help="held-out volumes")
    ap.add_argument("--dn-in", type=int, default=100_000, help="photons of an input map")
    ap.add_argument("--dn-target", type=int, default=100_000_000, help="photons of a target map")
    ap.add_argument("--dn-ref", type=int, default=1_000_000_000, help="photons of a reference map")
    ap.add_argument("--dn-ladder-max", type=int, default=100_000_000,
                    help="largest plain run of the equal-error ladder")
    ap.add_argument("--dn-steps", type=int, default=64000)
    ap.add_argument("--dn-batch", type=int, default=4)
    ap.add_argument("--dn-lr", type=float, default=1e-3)
    ap.add_argument("--dn-seed", type=int, default=7)
    ap.add_argument("--dn-configs", default="",
                    help="training configurations steps:batch:lr, comma separated (default: "
                         "--dn-steps:--dn-batch:--dn-lr)")
    ap.add_argument("--dn-aux", type=int, default=0, choices=[0, 2],
                    help="medium-feature input channels (log mua, log reduced mus)")
    args = ap.parse_args()

    world, rank, local = dist_env()
    global WORKLOAD, WORKLOAD_DESC
    if args.workload == "c3":
        wl = workloads.c3(n_photons=args.photons or 1_000_000_000)
        WORKLOAD, WORKLOAD_DESC = C3_WORKLOAD, C3_DESC
        args.no_c3 = True
    else:
        wl = workloads.c2(n_photons=args.photons or 100_000_000)
    if args.impl == "reference":
        run_reference(args, wl, world, rank)
        return
    if args.study == "paper":
        study_paper(args)
        return
    if args.study == "batched":
        study_batched(args)
        return
    if args.study == "denoise":
        study_denoise(args)
        return
    if args.study == "denoise-kernels":
        study_denoise_kernels(args)
        return
    if args.study == "peaks":
        study_peaks(args)
        return

    import torch
    import paper_1711_03244_gb300 as mcx
    from paper_1711_03244_gb300 import build as mcx_build

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(mcx.LIB_PATH):
        mcx_build.build()
    if dist is not None:
        dist.barrier()
    mcx.load()

    stream = torch.cuda.current_stream()
    sim = mcx.Simulation.from_workload(wl)
    offset, n = mcx.photon_range(rank, world, wl.n_photons)   # this rank's photon ids

    def step():
        cfg = mcx.mcx_run_cfg_default(n_photons=n, photon_offset=offset, n_gates=wl.n_gates,
                                      dt_ns=wl.dt_ns, seed=wl.seed,
                                      max_detected=wl.max_detected, cuda_stream=stream)
        mcx.mcx_run(sim.handle, cfg)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        step()
        mcx.mcx_sync(sim.handle, allow_cap=True)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    walk_ms = []
    stats = tally = None
    with ClockSampler(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()                   # L2 (129 MB) flushed between timed steps
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            walk_ms.append(mcx.mcx_last_kernel_ms(sim.handle))
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(b) for a, b in ev]
    stats = mcx.mcx_read_stats(sim.handle)
    tally = mcx.mcx_read_tally(sim.handle)
    info = mcx.mcx_launch_info(sim.handle)
    total_ms = float(sum(step_ms))
    walk_avg = float(np.mean(walk_ms))
    if dist is not None:
        t = torch.tensor([total_ms, walk_avg], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, walk_avg = float(t[0]), float(t[1])
    value = world * n * args.steps / total_ms

    # ---- e2e through the C ABI with host buffers (pinned), copies inside the timed region
    labels_pinned = torch.from_numpy(wl.labels).pin_memory()
    flu_pinned = torch.empty((wl.n_gates,) + wl.labels.shape, dtype=torch.float32).pin_memory()
    e2e_times = []
    h2d = d2h = 0
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mcx.mcx_update_labels(sim.handle, labels_pinned.numpy())
        mcx.mcx_set_media(sim.handle, wl.media)
        step()
        mcx.mcx_sync(sim.handle, allow_cap=True)
        mcx.mcx_read_fluence(sim.handle, flu_pinned.numpy(), normalized=True)
        tl = mcx.mcx_read_tally(sim.handle)
        rec, tot = mcx.mcx_read_detected(sim.handle)
        dt = time.perf_counter() - t0
        if k > 0:                             # the first pass warms the read path
            e2e_times.append(dt)
        h2d = wl.labels.nbytes + wl.media.astype(np.float32).nbytes
        d2h = flu_pinned.numel() * 4 + 6 * 8 + rec.nbytes
    e2e_ms = 1e3 * float(np.mean(e2e_times)) if e2e_times else float("nan")
    e2e_val = world * n / e2e_ms if e2e_times else None

    # ---- the paper's linear runtime model T = a n + T0 from pilot runs at 1e6 and 5e6
    # photons (device time of one complete run, and host wall time of create + run + read)
    model = None
    if not args.no_model:
        def pilot(npil):
            cfgp = mcx.mcx_run_cfg_default(n_photons=npil, photon_offset=offset,
                                           n_gates=wl.n_gates, dt_ns=wl.dt_ns, seed=wl.seed,
                                           max_detected=wl.max_detected, cuda_stream=stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with mcx.Simulation.from_workload(wl) as s2:
                s2.n_gates = wl.n_gates
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                mcx.mcx_run(s2.handle, cfgp)
                e1.record(stream)
                mcx.mcx_sync(s2.handle, allow_cap=True)
                s2.fluence()
                s2.tally()
                s2.detected()
            wall_ms = 1e3 * (time.perf_counter() - t0)
            return e0.elapsed_time(e1), wall_ms
        pilot(1_000_000)                                  # warm the path once
        d1, w1 = pilot(1_000_000)
        d2, w2 = pilot(5_000_000)
        a_dev = (d2 - d1) / 4e6
        a_wall = (w2 - w1) / 4e6
        model = {"n1": 1_000_000, "n2": 5_000_000,
                 "device": {"a_ns_per_photon": a_dev * 1e6, "T0_ms": d1 - a_dev * 1e6},
                 "wall": {"a_ns_per_photon": a_wall * 1e6, "T0_ms": w1 - a_wall * 1e6}}

    # ---- roofline of the walk kernel: algorithmic thread-ops / launch time vs issue peak
    pk = peaks()
    ops = algorithmic_ops(stats, tally)                   # per launch on this rank
    achieved = ops / (walk_avg * 1e-3) / 1e12             # T thread-op/s
    peak = SM_COUNT * LANES_PER_SM * pk["sm_max_mhz"] * 1e6 / 1e12
    c3_main = args.workload == "c3"
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tthread-op/s",
            "frac": achieved / peak,
            "traffic": walk_traffic("walk_kernel_c3.md" if c3_main else "walk_kernel_c2.md", n),
            "peak_note": f"152 SMs x 128 lanes x {pk['sm_max_mhz']:.0f} MHz ({pk['source']} max clock)",
            "ops_per_photon": ops / n,
            "kernel": "walk_kernel<float,false>" if c3_main else "walk_kernel<float,true>",
            "walk_ms": walk_avg}
    rates = None
    if not args.no_probes and rank == 0:
        rates = measure_rates(mcx, {"c2": 64 ** 3 * 10 * 8, "c3": 256 * 256 * 128 * 50 * 8})
        roof["peak_measured"] = rates["ffma"] / 1e12
        roof["frac_of_measured"] = achieved / roof["peak_measured"]
        roof["co_bounds"] = co_bounds(stats, n, walk_avg, rates, "c3" if c3_main else "c2", peak,
                                      roof["traffic"], pk["hbm_gbs"])

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "photons_per_step": n,
                       "photons_per_rank": n, "seed": wl.seed,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "accumulation": "FP64 L2 atomics per (gate, voxel) run (accum_mode 2)",
                       "launch": info, "parallelism": f"photon-id ranges x{world}"},
            "gpu_launches": 5 * args.steps,       # per mcx_run: 3 zeroing, the walk, the tally reduction
            "wall_s": wall,
            "clocks": clk.summary(),
            "roofline": roof,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps},
            "runtime_model": model,
            "events": {k: int(v) for k, v in stats.items()},
            "energy_balance_rel": abs(tally["absorbed"] + tally["escaped"] +
                                      tally["time_exceeded"] + tally["roulette_killed"] -
                                      tally["roulette_gained"] - tally["launched"]) /
            max(tally["launched"], 1.0)}

    if rank == 0 and not args.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        nc = args.cpu_photons
        t0 = time.perf_counter()
        oracle.run(wl, n_photons=nc, energy=True, n_threads=cores)
        cpu_ms = 1e3 * (time.perf_counter() - t0)
        line["cpu_baseline"] = {"value": nc / cpu_ms, "unit": UNIT, "cores": cores,
                                "kind": "oracle",
                                "sample": f"first {nc} photons of {WORKLOAD} (FP64 oracle, "
                                          f"{cores} OpenMP threads, {cpu_ms / 1e3:.1f} s)"}
        # the same oracle on one thread, over the first nc / cores of those photons
        n1 = max(nc // cores, 1000)
        t0 = time.perf_counter()
        oracle.run(wl, n_photons=n1, energy=True, n_threads=1)
        one_ms = 1e3 * (time.perf_counter() - t0)
        line["cpu_baseline"]["single_thread"] = {
            "value": n1 / one_ms, "unit": UNIT, "cores": 1,
            "sample": f"first {n1} photons of {WORKLOAD}, 1 thread, {one_ms / 1e3:.1f} s"}
    sim.close()
    if rank == 0 and world == 1 and not args.no_c3:
        line["c3"] = bench_c3(args, mcx, torch, stream, rates, peak)
    if rank == 0 and rates:
        line["measured_rates"] = rates
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
