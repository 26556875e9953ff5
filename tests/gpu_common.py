"""Helpers shared by the GPU parity tests: float32-exact inputs for both sides, running the
CUDA path through the C ABI, running the oracle, and statistical comparisons."""
from __future__ import annotations

import math

import numpy as np

import workloads

F32_RR = float(np.float32(1e-4))       # the roulette threshold both sides see


def f32(wl: workloads.Workload) -> workloads.Workload:
    """Rounds every real input through float32 so the FP64 oracle and the C ABI (float
    inputs) simulate exactly the same problem."""
    r = lambda v: float(np.float32(v))
    return wl.with_(
        voxel_mm=r(wl.voxel_mm),
        media=np.asarray(wl.media, dtype=np.float32).astype(np.float64),
        src_pos=tuple(r(v) for v in wl.src_pos),
        src_dir=tuple(r(v) for v in wl.src_dir),
        waist_mm=r(wl.waist_mm),
        detectors=np.asarray(wl.detectors, dtype=np.float32).astype(np.float64).reshape(-1, 4),
        dt_ns=r(wl.dt_ns),
    )


def gpu_run(wl, n_photons=None, seed=None, exit_log=0, precision=0, max_detected=None,
            block_size=0, grid_size=0, photon_offset=0, rr_threshold=F32_RR, rr_m=10.0,
            n_gates=None, reflect=None, max_events=0, normalized=False, claim_mode=0,
            accum_mode=2):
    """Runs the CUDA path through the C ABI; returns a dict of host outputs."""
    import paper_1711_03244_gb300 as g
    n = wl.n_photons if n_photons is None else n_photons
    G = wl.n_gates if n_gates is None else n_gates
    sim = g.Simulation.from_workload(wl)
    try:
        md = (max_detected if max_detected is not None else
              (wl.max_detected or 1_000_000)) if len(wl.detectors) else 0
        st = sim.run(n, n_gates=G, dt_ns=wl.dt_ns, seed=wl.seed if seed is None else seed,
                     exit_log=exit_log, precision=precision, max_detected=md,
                     block_size=block_size, grid_size=grid_size, photon_offset=photon_offset,
                     rr_threshold=rr_threshold, rr_m=rr_m,
                     reflect=wl.reflect if reflect is None else reflect,
                     max_events_per_photon=max_events, claim_mode=claim_mode,
                     accum_mode=accum_mode)
        out = {
            "status": st,
            "energy": sim.fluence(normalized=normalized),
            "tally": sim.tally(),
            "stats": sim.stats(),
            "exits": sim.exits(exit_log) if exit_log else None,
            "launch": sim.launch_info(),
            "kernel_ms": sim.kernel_ms(),
        }
        if len(wl.detectors):
            out["det"], out["det_total"] = sim.detected()
        return out
    finally:
        sim.close()


def balance(t: dict) -> float:
    return t["absorbed"] + t["escaped"] + t["time_exceeded"] + t["roulette_killed"] \
        - t["roulette_gained"]


def exit_match(ex_gpu, ex_orc, tol_mm=1e-3):
    """Per photon: same fate and, when escaped, exit points within tol_mm."""
    same_fate = ex_gpu["fate"] == ex_orc["fate"]
    d = np.linalg.norm(ex_gpu["pos"].astype(np.float64) - ex_orc["pos"], axis=1)
    esc = ex_orc["fate"] == 1
    ok = same_fate & (~esc | (d <= tol_mm))
    return ok, d


def welch_voxelwise(gpu_reps: np.ndarray, orc_batches: np.ndarray):
    """Welch t per voxel between two sets of replicate means (axis 0 = replicate).
    Returns (t, dof, mask of voxels with a deposit in every sample)."""
    mask = np.all(gpu_reps > 0, axis=0) & np.all(orc_batches > 0, axis=0)
    a, b = gpu_reps[:, mask], orc_batches[:, mask]
    na, nb = a.shape[0], b.shape[0]
    va, vb = a.var(axis=0, ddof=1) / na, b.var(axis=0, ddof=1) / nb
    t = (a.mean(axis=0) - b.mean(axis=0)) / np.sqrt(va + vb)
    dof = (va + vb) ** 2 / (va ** 2 / (na - 1) + vb ** 2 / (nb - 1))
    return t, dof, mask


def t_tail(dof: np.ndarray, x: float = 3.0) -> np.ndarray:
    from scipy import stats
    return 2 * stats.t.sf(x, dof)


def assert_voxelwise(gr, ob, min_vox=1000):
    """Voxel-wise Welch test of two replicate sets (axis 0): the fraction of voxels with
    |t| > 3 stays within twice the t-distribution's expectation at each voxel's Welch dof
    (plus three binomial sigmas), and the mean t^2 stays near its expectation."""
    t, dof, mask = welch_voxelwise(gr.reshape(gr.shape[0], -1), ob.reshape(ob.shape[0], -1))
    assert mask.sum() >= min_vox
    fail = np.abs(t) > 3
    expect = t_tail(dof).mean()
    chi = np.mean(t * t) / np.mean(dof / (dof - 2))
    print(f"voxels {mask.sum()}, |t|>3 {fail.mean():.4f} (t-dist {expect:.4f}), "
          f"mean t^2 / expected {chi:.3f}")
    assert fail.mean() <= 2 * expect + 3 * math.sqrt(expect / mask.sum())
    assert chi < 1.25
