"""The allocation-free entry point, mcx_run_noalloc, against the regular mcx_run path.

mcx_run_noalloc is for callers that cannot let the library allocate device memory: an
application whose own pool or caching allocator owns the device memory, or a loop that
cannot afford the device-wide synchronisation of cudaFree.  It runs the same walk kernel
on the caller's buffers and keeps its working memory in a fixed array inside the library.

Checked here, through the C ABI: two calls in a row on caller-owned torch buffers each
reproduce the fluence and tallies of the regular entry point for the same seed (the walk
is a pure function of seed and photon ids; only the order of the atomic additions may
differ), on the current stream with 256-thread blocks and FP32 accumulation, and on a
stream of the caller's with 128-thread blocks and FP64 accumulation; the second call does
not change the device's free memory; photons stopped by the per-photon event cap are
counted in the output as mcx_run counts them; sizes beyond the fixed limits, malformed
buffers, host memory and stream capture are rejected.  This file is collected last on
purpose."""
import ctypes

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


def _regular(g, wl, n, seed, accum, block, max_events=0):
    with g.Simulation.from_workload(wl.with_(detectors=np.zeros((0, 4)))) as sim:
        st = sim.run(n, n_gates=wl.n_gates, dt_ns=wl.dt_ns, seed=seed, rr_threshold=F32_RR,
                     accum_mode=accum, block_size=block, max_events_per_photon=max_events)
        flu = sim.fluence64() if accum == 2 else sim.fluence()
        return flu, sim.tally(), sim.stats(), st


def _noalloc(g, wl, n, seed, labels_dev, flu, tally, stream, accum, block, max_events=0):
    cfg = g.mcx_run_cfg_default(n_photons=n, n_gates=wl.n_gates, dt_ns=wl.dt_ns, seed=seed,
                                rr_threshold=F32_RR, accum_mode=accum, block_size=block,
                                max_events_per_photon=max_events, cuda_stream=stream)
    g.mcx_run_noalloc(labels_dev, wl.voxel_mm, wl.media, wl.src_kind, wl.src_pos, wl.src_dir,
                      wl.waist_mm, cfg, flu, tally)
    stream.synchronize()
    out = tally.cpu().numpy()
    return flu.cpu().numpy(), dict(zip(g.TALLY_NAMES, out[:6].tolist())), out[6]


@pytest.mark.parametrize("own_stream, block, accum", [(False, 256, 0), (True, 128, 2)])
def test_noalloc_matches_regular_twice_in_a_row(g, own_stream, block, accum):
    torch = pytest.importorskip("torch")
    wl = f32(workloads.c2(n_photons=200_000))
    n, seed = 200_000, 7
    ref_flu, ref_t, _, _ = _regular(g, wl, n, seed, accum, block)
    labels_dev = torch.from_numpy(wl.labels).cuda()
    dtype = torch.float64 if accum == 2 else torch.float32
    flu = torch.full((wl.n_gates,) + wl.labels.shape, 7.0, dtype=dtype, device="cuda")
    tally = torch.full((g.NOALLOC_NOUT,), 5.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream() if own_stream else torch.cuda.current_stream()
    free = []
    for call in range(2):
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got_flu, got_t, capped = _noalloc(g, wl, n, seed, labels_dev, flu, tally, stream, accum,
                                          block)
        # same photons, same trajectories: tallies to FP64 summation-order rounding,
        # fluence to the atomics' order of addition (FP32: 1e-4 relative; FP64: 1e-12)
        for k in g.TALLY_NAMES:
            assert got_t[k] == pytest.approx(ref_t[k], rel=1e-9, abs=1e-9), (call, k)
        assert capped == 0.0, call
        if accum == 2:
            assert np.allclose(got_flu, ref_flu, rtol=1e-12, atol=1e-15), call
        else:
            assert np.allclose(got_flu, ref_flu, rtol=1e-4, atol=1e-6), call
        assert abs(got_flu.sum(dtype=np.float64) - ref_flu.sum(dtype=np.float64)) \
            <= 1e-5 * ref_flu.sum(dtype=np.float64)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free[1]      # the second call allocated nothing


def test_noalloc_reports_the_event_cap(g):
    """A cap of 40 segments per photon stops most C2 photons: the count in the output's last
    word equals the regular path's capped-photon count, whose mcx_sync says MCX_E_CAP."""
    torch = pytest.importorskip("torch")
    wl = f32(workloads.c2(n_photons=4000))
    n, seed, cap = 4000, 3, 40
    ref_flu, ref_t, ref_s, st = _regular(g, wl, n, seed, 2, 256, max_events=cap)
    assert st == g.MCX_E_CAP and ref_s["capped"] > 0
    labels_dev = torch.from_numpy(wl.labels).cuda()
    flu = torch.empty((wl.n_gates,) + wl.labels.shape, dtype=torch.float64, device="cuda")
    tally = torch.zeros(g.NOALLOC_NOUT, dtype=torch.float64, device="cuda")
    got_flu, got_t, capped = _noalloc(g, wl, n, seed, labels_dev, flu, tally,
                                      torch.cuda.current_stream(), 2, 256, max_events=cap)
    assert capped == ref_s["capped"]
    assert got_t["time_exceeded"] == pytest.approx(ref_t["time_exceeded"], rel=1e-9)
    assert np.allclose(got_flu, ref_flu, rtol=1e-12, atol=1e-15)


def test_noalloc_rejects_sizes_beyond_its_limits(g):
    torch = pytest.importorskip("torch")
    wl = f32(workloads.c1(n_photons=10))
    labels_dev = torch.from_numpy(wl.labels).cuda()
    flu = torch.zeros((1,) + wl.labels.shape, dtype=torch.float32, device="cuda")
    tally = torch.zeros(g.NOALLOC_NOUT, dtype=torch.float64, device="cuda")
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
    # photon ids that wrap around, and an infinite gate width
    cfg = g.mcx_run_cfg_default(n_photons=10, photon_offset=2 ** 64 - 5, dt_ns=5.0, accum_mode=0)
    with pytest.raises(g.McxError) as e:
        g.mcx_run_noalloc(labels_dev, 1.0, wl.media, 0, wl.src_pos, wl.src_dir, 0.0, cfg, flu, tally)
    assert e.value.status == g.MCX_E_ARG and "overflows" in str(e.value)
    cfg = g.mcx_run_cfg_default(n_photons=10, dt_ns=float("inf"), accum_mode=0)
    with pytest.raises(g.McxError) as e:
        g.mcx_run_noalloc(labels_dev, 1.0, wl.media, 0, wl.src_pos, wl.src_dir, 0.0, cfg, flu, tally)
    assert e.value.status == g.MCX_E_ARG and "dt_ns" in str(e.value)


def test_noalloc_rejects_malformed_buffers(g):
    """The binding checks size, dtype, device and layout before calling the library (which
    cannot check a buffer's size); the library itself rejects host memory."""
    torch = pytest.importorskip("torch")
    wl = f32(workloads.c1(n_photons=10))
    labels_dev = torch.from_numpy(wl.labels).cuda()
    tally = torch.zeros(g.NOALLOC_NOUT, dtype=torch.float64, device="cuda")
    cfg = g.mcx_run_cfg_default(n_photons=10, n_gates=2, dt_ns=2.5, accum_mode=0)
    short = torch.zeros((1,) + wl.labels.shape, dtype=torch.float32, device="cuda")   # 1 gate of 2
    wrong_type = torch.zeros((2,) + wl.labels.shape, dtype=torch.float64, device="cuda")
    strided = torch.zeros((2,) + wl.labels.shape + (2,), dtype=torch.float32, device="cuda")[..., 0]
    for flu in (short, wrong_type, strided, np.zeros((2,) + wl.labels.shape, np.float32)):
        with pytest.raises(ValueError):
            g.mcx_run_noalloc(labels_dev, 1.0, wl.media, 0, wl.src_pos, wl.src_dir, 0.0, cfg, flu,
                              tally)
    with pytest.raises(ValueError):
        g.mcx_run_noalloc(labels_dev, 1.0, wl.media, 0, wl.src_pos, wl.src_dir, 0.0, cfg,
                          torch.zeros((2,) + wl.labels.shape, device="cuda"), tally[:6])
    with pytest.raises(ValueError):
        g.mcx_run_noalloc(wl.labels, 1.0, wl.media, 0, wl.src_pos, wl.src_dir, 0.0, cfg,
                          torch.zeros((2,) + wl.labels.shape, device="cuda"), tally)
    # pinned host memory of the right size, passed straight to the C entry point: rejected
    # by the library's pointer check (a kernel could read it, but it is not device memory)
    host = torch.zeros((2,) + wl.labels.shape, dtype=torch.float32).pin_memory()
    a = np.ascontiguousarray(wl.media, dtype=np.float32)
    p = np.ascontiguousarray(wl.src_pos, dtype=np.float32)
    d = np.ascontiguousarray(wl.src_dir, dtype=np.float32)
    nz, ny, nx = wl.labels.shape
    st = g.load().mcx_run_noalloc(ctypes.c_void_p(labels_dev.data_ptr()), nx, ny, nz, 1.0,
                                  a.shape[0], a.ctypes.data, 0, p.ctypes.data, d.ctypes.data, 0.0,
                                  ctypes.byref(cfg), ctypes.c_void_p(host.data_ptr()),
                                  ctypes.c_void_p(tally.data_ptr()))
    assert st == g.MCX_E_ARG and "device memory" in g.mcx_last_error(None)


def test_noalloc_refuses_stream_capture(g):
    """The call waits for its stream (the label check), which stream capture forbids: it
    says so instead of invalidating the capture."""
    torch = pytest.importorskip("torch")
    wl = f32(workloads.c1(n_photons=10))
    labels_dev = torch.from_numpy(wl.labels).cuda()
    flu = torch.zeros((1,) + wl.labels.shape, dtype=torch.float32, device="cuda")
    tally = torch.zeros(g.NOALLOC_NOUT, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    cfg = g.mcx_run_cfg_default(n_photons=10, dt_ns=5.0, accum_mode=0, cuda_stream=s)
    graph = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(graph, stream=s):
        try:
            g.mcx_run_noalloc(labels_dev, 1.0, wl.media, 0, wl.src_pos, wl.src_dir, 0.0, cfg,
                              flu, tally)
        except g.McxError as e:
            err = e
        flu.add_(1.0)                       # something for the capture to hold
    assert err is not None and err.status == g.MCX_E_STATE and "capture" in str(err)
    graph.replay()
    torch.cuda.synchronize()
    assert float(flu.max()) == 1.0
