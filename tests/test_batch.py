"""Batched simulations: many problems in one persistent launch.

A simulation's photon p draws the stream of (its seed, p), so each member of a batch
reproduces the same simulation run alone through mcx_run photon by photon.  The batch
walk is a separately compiled FP32 instantiation of the kernel, so rounding (FMA
contraction) can differ in the last bit and a few chaotic trajectories part ways; the
members therefore agree with their standalone runs to ~1e-6 in the tallies and ~1e-4 in
relative L2 of the map, far inside Monte Carlo noise.  The C4 batch (256 uneven volumes)
checks scale: every photon is simulated and every member's energy balances.
"""
import numpy as np
import pytest

import workloads
from gpu_common import F32_RR, assert_voxelwise, balance, exit_match, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_1711_03244_gb300 import build
    build.build()
    import paper_1711_03244_gb300 as m
    m.load()
    return m


def _members():
    sims = [f32(w) for w in workloads.c4(n_sims=6)]
    sims = [w.with_(n_photons=min(w.n_photons, 60_000)) for w in sims]
    sims.append(f32(workloads.c1(n_photons=40_000)).with_(n_gates=5, dt_ns=1.0, seed=77))
    sims.append(f32(workloads.c3(n_photons=3_000)).with_(labels=workloads.c3().labels[:40, 100:156, 100:156].copy(),
                                                      src_pos=(14.0, 14.0, 0.0), n_gates=5,
                                                      dt_ns=1.0, seed=5))
    sims.append(f32(workloads.c1(n_photons=0)).with_(n_gates=5, dt_ns=1.0, seed=9))
    return sims


def _alone(g, wl):
    with g.Simulation.from_workload(wl.with_(detectors=np.zeros((0, 4)))) as sim:
        sim.run(wl.n_photons, n_gates=5, dt_ns=1.0, seed=wl.seed, rr_threshold=F32_RR)
        return sim.fluence64(), sim.tally()


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_members_equal_standalone_runs(g, use_graph):
    sims = _members()
    with g.Batch() as b:
        for wl in sims:
            b.add_workload(wl)
        for rep in range(2):                      # the second run replays the graph
            b.run(n_gates=5, dt_ns=1.0, rr_threshold=F32_RR, use_graph=use_graph)
            stats = b.stats()
            assert stats["photons"] == sum(w.n_photons for w in sims)
            for i, wl in enumerate(sims):
                E_alone, t_alone = _alone(g, wl)
                t = b.tally(i)
                n = max(wl.n_photons, 1)
                for k in t:
                    assert abs(t[k] - t_alone[k]) <= 1e-5 * n, (i, k, t[k], t_alone[k])
                E = b.fluence(i).astype(np.float64)
                if wl.n_photons:
                    l2 = np.linalg.norm(E - E_alone) / np.linalg.norm(E_alone)
                    print(f"member {i}: map L2 vs standalone {l2:.1e}, absorbed "
                          f"{t['absorbed']:.6f} vs {t_alone['absorbed']:.6f}")
                    assert l2 < 1e-3, i
                    assert abs(balance(t) - wl.n_photons) <= 1e-6 * wl.n_photons
                else:
                    assert not E.any()


def test_batch_fp32_accumulation_and_normalisation(g):
    sims = _members()[:3]
    with g.Batch() as b:
        for wl in sims:
            b.add_workload(wl)
        b.run(n_gates=5, dt_ns=1.0, rr_threshold=F32_RR, accum_mode=0)
        for i, wl in enumerate(sims):
            E_alone, _ = _alone(g, wl)
            E = b.fluence(i).astype(np.float64)
            assert np.linalg.norm(E - E_alone) / np.linalg.norm(E_alone) < 1e-3
            Phi = b.fluence(i, normalized=True).astype(np.float64)
            mua = wl.media[:, 0].astype(np.float32).astype(np.float64)[wl.labels]
            with np.errstate(divide="ignore", invalid="ignore"):
                expect = E / (mua * wl.voxel_mm ** 3 * wl.n_photons * 1.0)
            expect[:, mua == 0] = 0
            assert np.allclose(Phi, expect, rtol=1e-5, atol=0)


def test_batch_autotune_picks_a_valid_shape(g):
    sims = [f32(w) for w in workloads.c4(n_sims=12)]
    with g.Batch() as b:
        for wl in sims:
            b.add_workload(wl, n_photons=min(wl.n_photons, 200_000))
        best = b.autotune(fraction=0.25, n_gates=5, dt_ns=1.0)
        assert best["block_size"] in (128, 256) and best["claim_chunk"] in (32, 64, 128, 256)
        assert best["ms"] > 0
        b.run(n_gates=5, dt_ns=1.0, block_size=best["block_size"], claim_chunk=best["claim_chunk"])
        for i in range(len(sims)):
            t = b.tally(i)
            assert abs(balance(t) - t["launched"]) <= 1e-6 * max(t["launched"], 1)


def test_batch_rejects_bad_input(g):
    with g.Batch() as b:
        with pytest.raises(g.McxError):
            b.run(n_gates=5, dt_ns=1.0)                          # empty batch
        wl = workloads.c1(n_photons=10)
        with pytest.raises(g.McxError):
            b.add(np.full((4, 4, 4), 5, np.uint8), 1.0, wl.media, n_photons=10)   # label 5
        b.add_workload(wl)
        with pytest.raises(g.McxError):
            b.run(n_gates=5, dt_ns=1.0, accum_mode=1)            # not in batches
        with pytest.raises(g.McxError):
            b.run(n_gates=5, dt_ns=1.0, claim_chunk=16)


def test_c4_batch_256_simulations(g):
    sims = workloads.c4()
    total = sum(w.n_photons for w in sims)
    with g.Batch() as b:
        for wl in sims:
            b.add_workload(wl)
        b.run(n_gates=5, dt_ns=1.0, use_graph=1)
        ms = b.last_ms()
        st = b.stats()
        assert st["photons"] == total
        worst = 0.0
        for i, wl in enumerate(sims):
            t = b.tally(i)
            worst = max(worst, abs(balance(t) - wl.n_photons) / wl.n_photons)
        print(f"c4: {len(sims)} simulations, {total:.3e} photons in {ms:.0f} ms "
              f"= {total / ms:.0f} photons/ms; worst energy balance {worst:.1e}")
        assert worst < 1e-5


def test_queue_order_does_not_change_results(g):
    """Longest-expected-histories-first queue order (the default) against the order of
    addition: every simulation keeps its photon streams, so tallies and maps agree to the
    FP64 summation order."""
    sims = [f32(w) for w in workloads.c4(n_sims=8)]
    sims = [w.with_(n_photons=min(w.n_photons, 50_000)) for w in sims]
    res = {}
    with g.Batch() as b:
        for wl in sims:
            b.add_workload(wl)
        for order in (0, 1):
            b.run(n_gates=5, dt_ns=1.0, order=order)
            res[order] = ([b.tally(i) for i in range(len(sims))],
                          [b.fluence(i).astype(np.float64) for i in range(len(sims))])
    for i in range(len(sims)):
        for k in res[0][0][i]:
            assert res[1][0][i][k] == pytest.approx(res[0][0][i][k], rel=1e-12, abs=1e-12)
        assert np.allclose(res[1][1][i], res[0][1][i], rtol=1e-6, atol=0)


def test_batch_members_match_the_oracle(g, orc):
    """The batched walk against the FP64 oracle, member by member.  Four C4-style members
    (sides 32, 48, 64 and 48 mm; 1-3 ellipsoids each; every medium's n between 1.33 and
    1.45 against the exterior's 1.0, so Fresnel events at every boundary) run as one batch
    that also holds eight replicates of each member under other seeds.  Per member:
      * fixed seed: the member's tallies against the oracle's on the same photon ids, to
        1e-5 of the photons launched plus two units of weight for each photon whose fate or
        exit differs (counted from a standalone run's exit log against the oracle's);
      * fluence: voxel-wise Welch t of the eight batch replicates against eight oracle
        batches of the same size (other photon ids), as in the single-simulation tests."""
    n, reps = 40_000, 8
    c4 = workloads.c4(n_sims=8)
    members = [f32(c4[i]).with_(n_photons=n) for i in (0, 4, 2, 7)]    # #7: one label has mus 0.78
    assert [w.labels.shape[0] for w in members] == [32, 48, 64, 48]
    with g.Batch() as b:
        ids = []
        for w in members:
            row = [b.add_workload(w)]
            for r in range(1, reps + 1):
                row.append(b.add_workload(w, seed=w.seed + 7919 * r))
            ids.append(row)
        b.run(n_gates=5, dt_ns=1.0, rr_threshold=F32_RR, use_graph=1)
        for m, w in enumerate(members):
            wl = w.with_(n_gates=5, dt_ns=1.0)
            o = orc.run(wl, n_photons=n, exit_cap=n, rr_threshold=F32_RR)
            with g.Simulation.from_workload(wl) as sim:
                sim.run(n, n_gates=5, dt_ns=1.0, seed=wl.seed, rr_threshold=F32_RR, exit_log=n)
                ok, _ = exit_match(sim.exits(n), o.exits)
            flips = int((~ok).sum())
            t = b.tally(ids[m][0])
            print(f"member {m} (side {wl.labels.shape[0]}): {flips} of {n} photons differ")
            assert flips <= 0.05 * n, m
            for k in ("absorbed", "escaped", "time_exceeded", "roulette_killed", "roulette_gained"):
                assert abs(t[k] - o.tally[k]) <= 1e-5 * n + 2 * flips, (m, k, t[k], o.tally[k])
            assert abs(balance(t) - n) <= 1e-6 * n
            gr = np.array([b.fluence(i).astype(np.float64) / n for i in ids[m][1:]])
            ob = np.array([orc.run(wl, n_photons=n, photon_offset=(k + 1) * n,
                                   rr_threshold=F32_RR).energy / n for k in range(reps)])
            assert_voxelwise(gr, ob, min_vox=300)
