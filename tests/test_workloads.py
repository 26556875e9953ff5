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
