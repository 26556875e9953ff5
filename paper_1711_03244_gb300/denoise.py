"""Training data, training loop and application of the learned fluence denoiser.

The Monte Carlo maps come from the batched walk (one persistent launch per chunk of
volumes), the network runs in the library's tensor-core kernels (mcx_denoiser_*); this
module only schedules them.  Device buffers are torch CUDA tensors.  The paper has no
counterpart: the denoiser extends the method so that a low-photon run plus one network
pass stands in for a high-photon run, with a plain high-photon run as the fallback.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

from . import Batch, Denoiser

GATE_NS = 5.0          # one 0-5 ns gate: the time-integrated map of the walk's window


def features(volumes: Sequence, out):
    """medium features of each volume (mcx_denoiser_features) into out[i] (float32 CUDA
    tensor [len(volumes), 2, nz, ny, nx])"""
    import torch
    for i, wl in enumerate(volumes):
        lab = torch.from_numpy(np.ascontiguousarray(wl.labels)).to(out.device)
        Denoiser.features(lab, wl.media, out[i])


def simulate(volumes: Sequence, n_photons: int, out, seed_offset: int = 0, chunk: int = 128,
             **cfg) -> float:
    """Runs every volume with n_photons photons (seed = the volume's seed + seed_offset)
    and writes its normalised fluence (1/mm^2 per launched photon weight) into out[i]
    (a float32 CUDA tensor [len(volumes), nz, ny, nx]).  Returns the walks' summed kernel
    time in ms (batches of `chunk` volumes, one persistent launch each)."""
    total_ms = 0.0
    for c0 in range(0, len(volumes), chunk):
        part = volumes[c0:c0 + chunk]
        with Batch() as b:
            for wl in part:
                b.add_workload(wl, n_photons=n_photons, seed=wl.seed + seed_offset)
            b.run(n_gates=1, dt_ns=GATE_NS, **cfg)
            total_ms += b.last_ms()
            for i in range(len(part)):
                b.fluence(i, normalized=True, out=out[c0 + i])
    return total_ms


def encode_set(d: Denoiser, phi, x, chunk: int = 64):
    """network-domain copy of a set of fluence maps (elementwise, any count)"""
    for c0 in range(0, phi.shape[0], chunk):
        d.encode(phi[c0:c0 + chunk], x[c0:c0 + chunk])


def train(d: Denoiser, x_set, t_set, steps: int, batch: int, lr: float = 1e-3,
          lr_final: float = 1e-4, seed: int = 0, log_every: int = 0, aux_set=None) -> List[float]:
    """Adam on the mean squared error in the network domain.  Each step draws `batch`
    pairs at random with a random mirror/transpose (the same for input, features and
    target), and the learning rate decays geometrically from lr to lr_final."""
    import torch
    rng = np.random.default_rng(seed)
    n = x_set.shape[0]
    xb = torch.empty((batch,) + tuple(x_set.shape[1:]), device=x_set.device, dtype=torch.float32)
    tb = torch.empty_like(xb)
    k = d.n_aux
    ab = torch.empty((batch, k) + tuple(x_set.shape[1:]), device=x_set.device) if k else None
    aux_flat = aux_set.view((-1,) + tuple(x_set.shape[1:])) if k else None
    ab_flat = ab.view((-1,) + tuple(x_set.shape[1:])) if k else None
    square = x_set.shape[2] == x_set.shape[3]
    losses = []
    for s in range(steps):
        idx = rng.integers(0, n, size=batch).astype(np.uint64)
        flags = rng.integers(0, 8 if square else 4, size=batch).astype(np.uint32)
        d.gather(x_set, idx, flags, xb)
        d.gather(t_set, idx, flags, tb)
        if k:                                  # feature c of pair i is volume i k + c
            d.gather(aux_flat, (idx[:, None] * k + np.arange(k)).ravel(), np.repeat(flags, k), ab_flat)
        rate = lr * (lr_final / lr) ** (s / max(steps - 1, 1))
        losses.append(d.train_step(xb, tb, rate, aux=ab))
        if log_every and (s % log_every == 0 or s == steps - 1):
            print(f"step {s:5d}  lr {rate:.2e}  loss {np.mean(losses[-log_every:]):.5f}", flush=True)
    return losses


def denoise(d: Denoiser, phi_in, phi_out, chunk: Optional[int] = None, aux=None):
    """phi_out = the network's estimate of a high-photon map for each map of phi_in"""
    step = chunk or d.max_batch
    for c0 in range(0, phi_in.shape[0], step):
        d.apply(phi_in[c0:c0 + step], phi_out[c0:c0 + step],
                aux=None if aux is None else aux[c0:c0 + step])


def log_rms(phi, phi_ref, floor: float = 1e-8, rel_mask: float = 1e-6) -> float:
    """voxel-wise RMS of log10(phi + floor) - log10(phi_ref + floor) over the voxels where
    the reference exceeds rel_mask of its maximum (host arrays)"""
    a = np.asarray(phi, dtype=np.float64)
    r = np.asarray(phi_ref, dtype=np.float64)
    m = r > rel_mask * r.max()
    e = np.log10(np.maximum(a[m], 0.0) + floor) - np.log10(r[m] + floor)
    return float(math.sqrt(np.mean(e * e)))
