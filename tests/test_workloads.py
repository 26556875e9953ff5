"""The seeded input generators (CPU): reproducibility, the configured shapes and
distributions, and disjoint training / held-out sets for the denoiser."""
import numpy as np

import workloads


def test_c5_is_seeded_and_shaped_as_configured():
    a = workloads.c5(6, seed=1711032450)
    b = workloads.c5(6, seed=1711032450)
    for x, y in zip(a, b):
        assert np.array_equal(x.labels, y.labels) and np.array_equal(x.media, y.media)
        assert x.src_pos == y.src_pos and x.seed == y.seed
    for k, wl in enumerate(a):
        assert wl.labels.shape == (64, 64, 64) and wl.voxel_mm == 1.0
        n_inc = len(wl.media) - 2                     # exterior row, background, inclusions
        assert 1 <= n_inc <= 3
        assert wl.labels.max() <= n_inc + 1 and wl.labels.min() >= 1
        m = np.asarray(wl.media)[1:]
        assert np.all((m[:, 0] >= 1e-3) & (m[:, 0] <= 0.1))
        assert np.all((m[:, 1] >= 0.5) & (m[:, 1] <= 20.0))
        assert np.all((m[:, 2] >= 0.5) & (m[:, 2] <= 0.95))
        assert np.all((m[:, 3] >= 1.33) & (m[:, 3] <= 1.45))
        assert wl.src_pos[2] == 0.0 and 0 <= wl.src_pos[0] <= 64 and 0 <= wl.src_pos[1] <= 64
        assert wl.src_dir == (0.0, 0.0, 1.0) and wl.n_gates == 1 and wl.dt_ns == 5.0
        assert wl.seed == 1711032450 + 1 + k


def test_c5_training_and_held_out_sets_differ():
    train = workloads.c5(8, seed=1711032450)
    test = workloads.c5(8, seed=1711032451)
    for x in train:
        for y in test:
            assert not (np.array_equal(x.labels, y.labels) and np.array_equal(x.media, y.media))


def test_c4_draws_the_configured_distributions():
    sims = workloads.c4()
    assert len(sims) == 256
    sides = {w.labels.shape[0] for w in sims}
    assert sides <= {32, 48, 64, 96, 128} and len(sides) == 5
    n = np.array([w.n_photons for w in sims])
    assert n.min() >= 1e5 and n.max() <= 1e7
    lg = np.log10(n)
    assert abs(lg.mean() - 6.0) < 0.15                 # log-uniform in [1e5, 1e7]
    assert all(w.n_gates == 5 and w.dt_ns == 1.0 for w in sims)


def test_paper_benchmarks_as_described():
    """B1 / B2a as the benchmark description beside Fig. 2 states them: a 60 mm cube
    (mua 0.005, mus 1.0, g 0.01, n 1.37) in air, a central r = 15 mm sphere (mua 0.002,
    mus 5.0, g 0.9, n 1.0) in B2/B2a, termination at the boundary in B1 and Snell/Fresnel
    in B2/B2a, a +z pencil beam entering at (30, 30, 0) mm, 1e8 photons."""
    import math
    b1, b2a = workloads.paper_b("B1"), workloads.paper_b("B2a")
    for wl in (b1, b2a):
        assert wl.labels.shape == (60, 60, 60) and wl.voxel_mm == 1.0
        assert tuple(wl.media[0][3:]) == (1.0,)                     # air outside
        assert tuple(wl.media[1]) == (0.005, 1.0, 0.01, 1.37)
        assert wl.src_kind == 0 and wl.src_pos == (30.0, 30.0, 0.0) and wl.src_dir == (0.0, 0.0, 1.0)
        assert wl.n_photons == 100_000_000
    assert b1.reflect == 0 and b2a.reflect == 1
    assert np.all(b1.labels == 1) and len(b1.media) == 2
    assert tuple(b2a.media[2]) == (0.002, 5.0, 0.9, 1.0)
    sphere = b2a.labels == 2
    assert abs(sphere.sum() / (4.0 / 3.0 * math.pi * 15 ** 3) - 1) < 0.02
    z, y, x = np.nonzero(sphere)
    assert np.allclose([x.mean(), y.mean(), z.mean()], 29.5)      # centred on (30, 30, 30) mm
    assert x.max() - x.min() + 1 == 30                             # 15 mm radius


def test_c1_c2_c3_as_configured():
    c1 = workloads.c1()
    assert c1.labels.shape == (64, 64, 64) and np.all(c1.labels == 1)
    assert tuple(c1.media[1]) == (0.01, 10.0, 0.9, 1.37) and c1.media[0][3] == 1.0
    assert c1.src_pos == (32.0, 32.0, 0.0) and c1.n_gates == 1 and c1.dt_ns == 5.0
    c2 = workloads.c2()
    assert c2.n_photons == 100_000_000 and c2.n_gates == 10 and c2.dt_ns == 0.5
    assert c2.labels[24, 32, 32] == 2 and c2.labels[30, 40, 20] == 3
    # the spheres overlap and the second one is painted last
    assert c2.labels[27, 37, 25] == 3 and np.sum((c2.labels == 3)) > 0
    assert np.allclose(c2.detectors[:, 3], 2.0) and np.all(c2.detectors[:, 2] == 0.0)
    assert np.allclose(np.hypot(c2.detectors[:, 0] - 32, c2.detectors[:, 1] - 32), 10.0)
    c3 = workloads.c3()
    assert c3.labels.shape == (128, 256, 256) and c3.voxel_mm == 0.5
    col = c3.labels[:, 100, 100]
    assert np.array_equal(np.flatnonzero(np.diff(col)) + 1, [6, 20, 24])   # 3, 7, 2 mm layers
    assert list(col[[0, 6, 20, 24, 127]]) == [1, 2, 3, 4, 4]
    assert c3.src_kind == 1 and c3.waist_mm == 2.0 and c3.src_pos == (64.0, 64.0, 0.0)
    assert c3.n_gates == 50 and c3.dt_ns == 0.1 and c3.n_photons == 1_000_000_000
