"""FP64 CPU oracle of the learned fluence denoiser (plain PyTorch CPU operations).

TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`: only `tests/`, `__graft_entry__`
smoke checks and the CPU legs of `bench.py` may import it; it imports nothing from the
product path and shares no code with it.

The denoiser extends the paper's method (the paper has no counterpart): a 3-level 3-D
U-Net with 16/32/64 channels and 3x3x3 convolutions that maps the log-fluence of a
low-photon run to that of a high-photon run.  The network's definition is restated here
from its description (three levels, 16/32/64 channels, 3x3x3 convolutions, BF16 weights
and activations, FP32 accumulation); its exact wiring, the parameter layout and the
fluence encoding are this project's and are documented beside the C entry points.

Every function computes in float64.  `forward(..., bf16=True)` rounds weights and stored
activations to bfloat16 at the points where the CUDA path stores BF16 (the precision the
design fixes), with straight-through gradients, so the remaining GPU-oracle difference is
the FP32 accumulation order; `bf16=False` is the exact FP64 network.

Parity status (what pins each function, tests/test_denoiser_oracle.py):
  * bf16_round: hand-checked values (ties to even, carries, signs).
  * conv3d: brute-force nested loops on tiny inputs; torch.nn.functional.conv3d.
  * avg_pool2 / upsample2: adjointness (<pool x, y> = <x, up y> / 8), constants.
  * forward: zero head returns the input; the one-layer case against brute force (with
    and without feature channels); the channel-0 pass-through network against its closed
    form x + up(up(pool(pool(relu(x))))); equivariance under shifts by 4 voxels away from
    the boundary.
  * features: hand-computed values for a two-label table and the exterior.
  * loss_and_grads: central finite differences of the exact FP64 loss; with the head's
    weights at zero, the loss and its head-bias gradient in closed form.
  * adam: the closed form of the first step (|update| = lr for non-zero gradients).
tests/test_denoiser_oracle_mutants.py plants one plausible slip at a time in a copy of
this module and checks that some pin fails on it.
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np
import torch

# (cin, cout) of the ten 3x3x3 convolutions, in parameter order
LAYERS: List[Tuple[int, int]] = [(16, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64),
                                 (96, 32), (32, 32), (48, 16), (16, 16)]
NAMES = ["e1a", "e1b", "e2a", "e2b", "ba", "bb", "d2a", "d2b", "d1a", "d1b"]


def param_count() -> int:
    return sum(27 * ci * co + co for ci, co in LAYERS) + 16 + 1


def unpack(params) -> Dict[str, torch.Tensor]:
    """Flat FP32/FP64 vector -> named float64 tensors (views, so gradients flow back to a
    flat tensor): '<name>.w' [27, cout, cin], '<name>.b' [cout], 'hw' [16], 'hb' [1].
    Layout: layer by layer, weights then bias, then the head."""
    p = params if torch.is_tensor(params) else torch.as_tensor(np.asarray(params), dtype=torch.float64)
    assert p.numel() == param_count()
    out, k = {}, 0
    for name, (ci, co) in zip(NAMES, LAYERS):
        out[name + ".w"] = p[k:k + 27 * co * ci].reshape(27, co, ci)
        k += 27 * co * ci
        out[name + ".b"] = p[k:k + co]
        k += co
    out["hw"] = p[k:k + 16]
    out["hb"] = p[k + 16:k + 17]
    return out


def bf16_round(x: torch.Tensor) -> torch.Tensor:
    """Round to the nearest bfloat16 (ties to even), returned as float64.  The value passes
    through float32 first, as the GPU's FP32 accumulators do."""
    return x.to(torch.float32).to(torch.bfloat16).to(torch.float64)


def _ste(x: torch.Tensor, on: bool) -> torch.Tensor:
    """bf16 rounding in the forward value, identity in the gradient."""
    return x + (bf16_round(x) - x).detach() if on else x


def tap_offsets():
    """tap = 9 (dz+1) + 3 (dy+1) + (dx+1) -> (dz, dy, dx)"""
    return [(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1) for t in range(27)]


def shift(x: torch.Tensor, dz: int, dy: int, dx: int) -> torch.Tensor:
    """s[n, z, y, x, c] = x[n, z+dz, y+dy, x+dx, c], zero outside the volume."""
    n, D, H, W, C = x.shape
    out = torch.zeros_like(x)
    zs, ze = max(0, -dz), min(D, D - dz)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    if zs < ze and ys < ye and xs < xe:
        out[:, zs:ze, ys:ye, xs:xe] = x[:, zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv3d(x: torch.Tensor, w: torch.Tensor, b=None) -> torch.Tensor:
    """y[n,z,y,x,o] = b[o] + sum_tap sum_c x[n, z+dz, y+dy, x+dx, c] w[tap, o, c]
    (channels last, zero padding: a 'same' 3x3x3 cross-correlation)."""
    y = None
    for t, (dz, dy, dx) in enumerate(tap_offsets()):
        term = torch.einsum("nzyxc,oc->nzyxo", shift(x, dz, dy, dx), w[t])
        y = term if y is None else y + term
    if b is not None:
        y = y + b
    return y


def avg_pool2(x: torch.Tensor) -> torch.Tensor:
    """mean over each 2x2x2 block (sizes even)"""
    n, D, H, W, C = x.shape
    return x.reshape(n, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(dim=(2, 4, 6))


def upsample2(x: torch.Tensor) -> torch.Tensor:
    """nearest-neighbour x2 in z, y, x"""
    return x.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3)


def forward(params, x, bf16: bool = True, aux=None) -> torch.Tensor:
    """x [n, nz, ny, nx] (network domain), optional medium features aux [n, k, nz, ny, nx]
    -> y [n, nz, ny, nx]; y = x + head(U-Net(x, aux)).  The input layer sees x as channel
    0 and the k features as channels 1..k of 16 (the rest zero)."""
    P = unpack(params) if not isinstance(params, dict) else params
    x = torch.as_tensor(np.asarray(x) if not torch.is_tensor(x) else x, dtype=torch.float64)
    q = lambda t: _ste(t, bf16)

    def conv(name, a):
        return q(torch.relu(conv3d(a, q(P[name + ".w"]), P[name + ".b"])))

    k = 0 if aux is None else aux.shape[1]
    feats = [q(x)[..., None]]
    if k:
        a = torch.as_tensor(np.asarray(aux), dtype=torch.float64)
        feats.append(q(a.permute(0, 2, 3, 4, 1)))
    feats.append(torch.zeros(x.shape + (15 - k,), dtype=torch.float64))
    x16 = torch.cat(feats, dim=-1)
    a0 = conv("e1a", x16)
    a1 = conv("e1b", a0)
    p1 = q(avg_pool2(a1))
    a2 = conv("e2a", p1)
    a3 = conv("e2b", a2)
    p2 = q(avg_pool2(a3))
    a4 = conv("ba", p2)
    a5 = conv("bb", a4)
    u2 = torch.cat([upsample2(a5), a3], dim=-1)
    a6 = conv("d2a", u2)
    a7 = conv("d2b", a6)
    u1 = torch.cat([upsample2(a7), a1], dim=-1)
    a8 = conv("d1a", u1)
    a9 = conv("d1b", a8)
    return x + P["hb"][0] + torch.einsum("nzyxc,c->nzyx", a9, P["hw"])


def loss_and_grads(params, x, t, bf16: bool = True, aux=None):
    """loss = mean (forward(x) - t)^2 over every voxel of the batch, and d loss / d params
    as a flat float64 vector in the parameter layout."""
    p = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    y = forward(unpack(p), x, bf16=bf16, aux=aux)
    tt = torch.as_tensor(np.asarray(t), dtype=torch.float64)
    loss = ((y - tt) ** 2).mean()
    loss.backward()
    return float(loss.detach()), p.grad.detach().numpy().copy()


def adam(params, grads, m, v, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected moments); returns (params, m, v) in float64."""
    g = np.asarray(grads, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return np.asarray(params, dtype=np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def encode(phi, floor=1e-8, mu=-4.0, sigma=2.0):
    """fluence -> network domain"""
    return (np.log10(np.maximum(np.asarray(phi, dtype=np.float64), 0) + floor) - mu) / sigma


def decode(x, floor=1e-8, mu=-4.0, sigma=2.0):
    """network domain -> fluence"""
    return np.maximum(10.0 ** (np.asarray(x, dtype=np.float64) * sigma + mu) - floor, 0)


def features(labels, media):
    """the two medium features per voxel: log10(max(mua, 1e-4)) + 2 and
    log10(max(mus (1 - g), 1e-3)); labels beyond the table count as exterior"""
    m = np.asarray(media, dtype=np.float64).reshape(-1, 4)
    f0 = np.log10(np.maximum(m[:, 0], 1e-4)) + 2.0
    f1 = np.log10(np.maximum(m[:, 1] * (1.0 - m[:, 2]), 1e-3))
    lab = np.asarray(labels).astype(np.int64)
    ok = lab < len(m)
    l = np.where(ok, lab, 0)
    return np.stack([np.where(ok, f0[l], -2.0), np.where(ok, f1[l], -3.0)])


def log_rms(phi, phi_ref, floor=1e-8, rel_mask=1e-6) -> float:
    """sqrt(mean (log10(phi + floor) - log10(phi_ref + floor))^2) over the voxels where
    phi_ref > rel_mask * max(phi_ref)."""
    a = np.asarray(phi, dtype=np.float64)
    r = np.asarray(phi_ref, dtype=np.float64)
    m = r > rel_mask * r.max()
    d = np.log10(np.maximum(a[m], 0) + floor) - np.log10(r[m] + floor)
    return float(np.sqrt(np.mean(d * d)))
