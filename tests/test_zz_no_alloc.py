"""The allocation-free entry point, mcx_run_noalloc, against the regular mcx_run path.

mcx_run_noalloc is for callers that cannot let the library allocate device memory: an
application whose own pool or caching allocator owns the device memory, or a loop that
cannot afford the device-wide synchronisation of cudaFree.  It runs the same walk kernel
on the caller's buffers and keeps its working memory in a fixed array inside the library.

Checked here, through the C ABI: two calls in a row on caller-owned torch buffers each
reproduce the fluence and tallies of the regular entry point for the same seed (the walk
is a pure function of seed and photon ids; only the order of FP32 atomic additions may
differ), the second call does not change the device's free memory, and sizes beyond the
fixed limits are rejected.  This file is collected last on purpose."""
import numpy as np
import pytest

import workloads
from gpu_common import F32_RR, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_1711_03244_gb300 import build
    build.build()
    import paper_1711_03244_gb300 as m
    m.load()
    return m


def _regular(g, wl, n, seed):
    with g.Simulation.from_workload(wl.with_(detectors=np.zeros((0, 4)))) as sim:
        sim.run(n, n_gates=wl.n_gates, dt_ns=wl.dt_ns, seed=seed, rr_threshold=F32_RR,
                accum_mode=0)
        return sim.fluence(), sim.tally()


def _noalloc(g, torch, wl, n, seed, labels_dev, flu, tally, stream):
    cfg = g.mcx_run_cfg_default(n_photons=n, n_gates=wl.n_gates, dt_ns=wl.dt_ns, seed=seed,
                                rr_threshold=F32_RR, accum_mode=0, cuda_stream=stream)
    g.mcx_run_noalloc(labels_dev, wl.voxel_mm, wl.media, wl.src_kind, wl.src_pos, wl.src_dir,
                      wl.waist_mm, cfg, flu, tally)
    stream.synchronize()
    return flu.cpu().numpy(), dict(zip(g.TALLY_NAMES, tally.cpu().numpy().tolist()))


def test_noalloc_matches_regular_twice_in_a_row(g):
    torch = pytest.importorskip("torch")
    wl = f32(workloads.c2(n_photons=200_000))
    n, seed = 200_000, 7
    ref_flu, ref_t = _regular(g, wl, n, seed)
    labels_dev = torch.from_numpy(wl.labels).cuda()
    flu = torch.full((wl.n_gates,) + wl.labels.shape, 7.0, dtype=torch.float32, device="cuda")
    tally = torch.zeros(6, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    free = []
    for call in range(2):
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got_flu, got_t = _noalloc(g, torch, wl, n, seed, labels_dev, flu, tally, stream)
        # same photons, same trajectories: tallies to FP64 summation-order rounding,
        # fluence to FP32 atomic-order rounding
        for k in g.TALLY_NAMES:
            assert got_t[k] == pytest.approx(ref_t[k], rel=1e-9, abs=1e-9), (call, k)
        assert np.allclose(got_flu, ref_flu, rtol=1e-4, atol=1e-6), call
        assert abs(got_flu.sum(dtype=np.float64) - ref_flu.sum(dtype=np.float64)) \
            <= 1e-5 * ref_flu.sum(dtype=np.float64)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free[1]      # the second call allocated nothing


def test_noalloc_rejects_sizes_beyond_its_limits(g):
    torch = pytest.importorskip("torch")
    wl = f32(workloads.c1(n_photons=10))
    labels_dev = torch.from_numpy(wl.labels).cuda()
    flu = torch.zeros((1,) + wl.labels.shape, dtype=torch.float32, device="cuda")
    tally = torch.zeros(6, dtype=torch.float64, device="cuda")
    many = np.tile(wl.media[1], (40, 1))
    many[0] = wl.media[0]
    cfg = g.mcx_run_cfg_default(n_photons=10, dt_ns=5.0, accum_mode=0)
    with pytest.raises(g.McxError) as e:
        g.mcx_run_noalloc(labels_dev, 1.0, many, 0, wl.src_pos, wl.src_dir, 0.0, cfg, flu, tally)
    assert e.value.status == g.MCX_E_ARG and "n_media" in str(e.value)
    cfg = g.mcx_run_cfg_default(n_photons=10, dt_ns=5.0, grid_size=4096, accum_mode=0)
    with pytest.raises(g.McxError) as e:
        g.mcx_run_noalloc(labels_dev, 1.0, wl.media, 0, wl.src_pos, wl.src_dir, 0.0, cfg, flu, tally)
    assert e.value.status == g.MCX_E_ARG and "grid_size" in str(e.value)
    bad = labels_dev.clone()
    bad[0, 0, 0] = 9
    cfg = g.mcx_run_cfg_default(n_photons=10, dt_ns=5.0, accum_mode=0)
    with pytest.raises(g.McxError) as e:
        g.mcx_run_noalloc(bad, 1.0, wl.media, 0, wl.src_pos, wl.src_dir, 0.0, cfg, flu, tally)
    assert e.value.status == g.MCX_E_STATE
