"""Python binding of the GB300 voxel Monte Carlo photon-transport library.

Argument marshalling only: every step of the photon walk, the output zeroing, the tally
reduction, the fluence normalisation and the detected-record ordering run in the CUDA
library `libmcx_gb300.so` (built in-tree for sm_103a by `build.py`).  There is no CPU
fallback: importing this package without the built library raises ImportError, and the
library itself needs a GB300 (compute capability 10.3).

The functions keep the C names of `include/mcx.h` (mcx_create_volume, mcx_set_media, ...).
Host arrays are NumPy arrays; device buffers may be torch CUDA tensors, whose data_ptr()
is passed through, and the CUDA stream may be a torch.cuda.Stream (PyTorch is used only
for device memory and streams).  `Simulation` is a small convenience wrapper.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmcx_gb300.so")

MCX_OK, MCX_E_ARG, MCX_E_STATE, MCX_E_CUDA, MCX_E_OOM, MCX_E_CAP, MCX_E_TIMEOUT = \
    0, -1, -2, -3, -4, -5, -6
FATE_NONE, FATE_ESCAPED, FATE_ROULETTE, FATE_TIME, FATE_MISSED, FATE_CAPPED = range(6)
TALLY_NAMES = ("launched", "absorbed", "escaped", "time_exceeded", "roulette_killed",
               "roulette_gained")
STAT_NAMES = ("scatter", "face", "fresnel", "flush", "roulette", "photons", "detected",
              "capped")
REC_BASE = 12


class McxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class McxRunCfg(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("n_gates", ctypes.c_uint32),
        ("n_photons", ctypes.c_uint64),
        ("photon_offset", ctypes.c_uint64),
        ("seed", ctypes.c_uint64),
        ("dt_ns", ctypes.c_float),
        ("reflect", ctypes.c_int32),
        ("rr_threshold", ctypes.c_float),
        ("rr_m", ctypes.c_float),
        ("max_detected", ctypes.c_uint64),
        ("exit_log", ctypes.c_uint64),
        ("max_events_per_photon", ctypes.c_uint64),
        ("accum_mode", ctypes.c_int32),
        ("block_size", ctypes.c_int32),
        ("grid_size", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p),
        ("tile_lo", ctypes.c_int32 * 4),
        ("tile_size", ctypes.c_int32 * 4),
        ("claim_mode", ctypes.c_int32),
        ("reserved1", ctypes.c_int32),
    ]


class McxExit(ctypes.Structure):
    _fields_ = [("fate", ctypes.c_int32), ("nscat", ctypes.c_uint32),
                ("pos", ctypes.c_float * 3), ("dir", ctypes.c_float * 3),
                ("w", ctypes.c_float), ("t", ctypes.c_float)]


EXIT_DTYPE = np.dtype([("fate", np.int32), ("nscat", np.uint32), ("pos", np.float32, 3),
                       ("dir", np.float32, 3), ("w", np.float32), ("t", np.float32)])
assert EXIT_DTYPE.itemsize == ctypes.sizeof(McxExit) == 40

class McxBatchCfg(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("n_gates", ctypes.c_uint32),
        ("dt_ns", ctypes.c_float),
        ("reflect", ctypes.c_int32),
        ("rr_threshold", ctypes.c_float),
        ("rr_m", ctypes.c_float),
        ("accum_mode", ctypes.c_int32),
        ("block_size", ctypes.c_int32),
        ("claim_chunk", ctypes.c_int32),
        ("grid_size", ctypes.c_int32),
        ("max_events_per_photon", ctypes.c_uint64),
        ("use_graph", ctypes.c_int32),
        ("order", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p),
    ]


# exported symbols and their signatures (restype, argtypes)
_P = ctypes.c_void_p
_u32, _u64, _i32, _f32, _f64 = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32,
                                 ctypes.c_float, ctypes.c_double)
SIGNATURES = {
    "mcx_abi_version": (_i32, []),
    "mcx_status_string": (ctypes.c_char_p, [_i32]),
    "mcx_run_cfg_default": (None, [ctypes.POINTER(McxRunCfg)]),
    "mcx_create_volume": (_i32, [ctypes.POINTER(_P), _u32, _u32, _u32, _f32, _P, _i32]),
    "mcx_update_labels": (_i32, [_P, _P, _i32]),
    "mcx_set_media": (_i32, [_P, _u32, _P]),
    "mcx_set_source": (_i32, [_P, _i32, _P, _P, _f32]),
    "mcx_add_detector": (_i32, [_P, _P, _f32, ctypes.POINTER(_i32)]),
    "mcx_clear_detectors": (_i32, [_P]),
    "mcx_run": (_i32, [_P, ctypes.POINTER(McxRunCfg)]),
    "mcx_sync": (_i32, [_P, _f64]),
    "mcx_last_kernel_ms": (_i32, [_P, ctypes.POINTER(_f32)]),
    "mcx_read_fluence": (_i32, [_P, _P, _u64, _i32, _i32]),
    "mcx_read_fluence64": (_i32, [_P, _P, _u64, _i32, _i32]),
    "mcx_detected_stride": (_i32, [_P]),
    "mcx_read_detected": (_i32, [_P, _P, _u64, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "mcx_read_tally": (_i32, [_P, _P]),
    "mcx_read_stats": (_i32, [_P, _P]),
    "mcx_read_exits": (_i32, [_P, _P, _u64, ctypes.POINTER(_u64)]),
    "mcx_launch_info": (_i32, [_P, _P]),
    "mcx_last_error": (ctypes.c_char_p, [_P]),
    "mcx_destroy": (None, [_P]),
    "mcx_probe_rate": (_i32, [_i32, _u64, ctypes.POINTER(_f64)]),
    "mcx_run_noalloc": (_i32, [_P, _u32, _u32, _u32, _f32, _u32, _P, _i32, _P, _P, _f32,
                               ctypes.POINTER(McxRunCfg), _P, _P]),
    "mcx_batch_cfg_default": (None, [ctypes.POINTER(McxBatchCfg)]),
    "mcx_batch_create": (_i32, [ctypes.POINTER(_P)]),
    "mcx_batch_add": (_i32, [_P, _u32, _u32, _u32, _f32, _P, _i32, _u32, _P, _i32, _P, _P, _f32,
                             _u64, _u64, ctypes.POINTER(_i32)]),
    "mcx_batch_run": (_i32, [_P, ctypes.POINTER(McxBatchCfg)]),
    "mcx_batch_sync": (_i32, [_P]),
    "mcx_batch_last_ms": (_i32, [_P, ctypes.POINTER(_f32)]),
    "mcx_batch_read_fluence": (_i32, [_P, _i32, _P, _u64, _i32, _i32]),
    "mcx_batch_read_tally": (_i32, [_P, _i32, _P]),
    "mcx_batch_read_stats": (_i32, [_P, _P]),
    "mcx_batch_autotune": (_i32, [_P, ctypes.POINTER(McxBatchCfg), _f64, ctypes.POINTER(_f32)]),
    "mcx_batch_size": (_i32, [_P]),
    "mcx_batch_last_error": (ctypes.c_char_p, [_P]),
    "mcx_batch_destroy": (None, [_P]),
    "mcx_denoiser_create": (_i32, [ctypes.POINTER(_P), _u32, _u32, _u32, _u32, _u32, _u64]),
    "mcx_denoiser_param_count": (_i32, [_P, ctypes.POINTER(_u64)]),
    "mcx_denoiser_get_params": (_i32, [_P, _P, _u64, _i32]),
    "mcx_denoiser_set_params": (_i32, [_P, _P, _u64]),
    "mcx_denoiser_set_encoding": (_i32, [_P, _f32, _f32, _f32]),
    "mcx_denoiser_forward": (_i32, [_P, _P, _P, _P, _u32, _P]),
    "mcx_denoiser_train_step": (_i32, [_P, _P, _P, _P, _u32, _f32, ctypes.POINTER(_f32), _P]),
    "mcx_denoiser_encode": (_i32, [_P, _P, _P, _u64, _P]),
    "mcx_denoiser_decode": (_i32, [_P, _P, _P, _u64, _P]),
    "mcx_denoiser_apply": (_i32, [_P, _P, _P, _P, _u32, _P]),
    "mcx_denoiser_features": (_i32, [_P, _u64, _u32, _P, _P, _P]),
    "mcx_denoiser_gather": (_i32, [_P, _P, _u64, _P, _P, _u32, _P, _P]),
    "mcx_denoiser_sync": (_i32, [_P]),
    "mcx_denoiser_destroy": (None, [_P]),
    "mcx_debug_uniforms": (_i32, [_u64, _u64, _u64, _P]),
    "mcx_debug_primitive": (_i32, [_i32, _u64, _P, _P]),
    "mcx_debug_conv3d": (_i32, [_i32, _i32, _i32, _i32, _i32, _i32, _i32, _P, _P, _P, _P, _P]),
    "mcx_debug_wait_timeout": (_i32, [_i32, _i32, ctypes.POINTER(_i32)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads the CUDA library.  Raises ImportError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1711_03244_gb300/build.py "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(sim, st: int):
    if st != MCX_OK:
        L = load()
        msg = L.mcx_last_error(sim).decode() if L.mcx_last_error(sim) else ""
        raise McxError(st, msg or L.mcx_status_string(st).decode())
    return st


def _ptr(x):
    """data pointer of a NumPy array or a torch tensor (device or host)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


def _on_device(x) -> int:
    return int(bool(getattr(x, "is_cuda", False)))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ------------------------------------------------------------------------ C-named API
def mcx_run_cfg_default(**overrides) -> McxRunCfg:
    cfg = McxRunCfg()
    load().mcx_run_cfg_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "cuda_stream":
            v = _stream_handle(v)
        if k in ("tile_lo", "tile_size"):
            v = (ctypes.c_int32 * 4)(*v)
        setattr(cfg, k, v)
    return cfg


def mcx_create_volume(labels, voxel_mm: float):
    """labels: uint8 [nz, ny, nx] NumPy array or torch tensor (host or CUDA)."""
    L = load()
    if hasattr(labels, "is_contiguous"):
        assert labels.is_contiguous() and str(labels.dtype).endswith("uint8")
        nz, ny, nx = labels.shape
    else:
        labels = np.ascontiguousarray(labels, dtype=np.uint8)
        nz, ny, nx = labels.shape
    h = ctypes.c_void_p()
    _check(None, L.mcx_create_volume(ctypes.byref(h), nx, ny, nz, float(voxel_mm), _ptr(labels),
                                     _on_device(labels)))
    return h


def mcx_update_labels(sim, labels):
    if not hasattr(labels, "is_contiguous"):
        labels = np.ascontiguousarray(labels, dtype=np.uint8)
    _check(sim, load().mcx_update_labels(sim, _ptr(labels), _on_device(labels)))


def mcx_set_media(sim, props):
    a = np.ascontiguousarray(props, dtype=np.float32).reshape(-1, 4)
    _check(sim, load().mcx_set_media(sim, a.shape[0], _ptr(a)))


def mcx_set_source(sim, kind: int, pos, direction, waist_mm: float = 0.0):
    p = np.ascontiguousarray(pos, dtype=np.float32)
    d = np.ascontiguousarray(direction, dtype=np.float32)
    _check(sim, load().mcx_set_source(sim, int(kind), _ptr(p), _ptr(d), float(waist_mm)))


def mcx_add_detector(sim, center, radius_mm: float) -> int:
    c = np.ascontiguousarray(center, dtype=np.float32)
    out = ctypes.c_int32()
    _check(sim, load().mcx_add_detector(sim, _ptr(c), float(radius_mm), ctypes.byref(out)))
    return out.value


def mcx_clear_detectors(sim):
    _check(sim, load().mcx_clear_detectors(sim))


def mcx_run(sim, cfg: McxRunCfg):
    _check(sim, load().mcx_run(sim, ctypes.byref(cfg)))


def mcx_sync(sim, timeout_s: float = -1.0, allow_cap: bool = False) -> int:
    st = load().mcx_sync(sim, float(timeout_s))
    if st == MCX_E_CAP and allow_cap:
        return st
    return _check(sim, st)


def mcx_last_kernel_ms(sim) -> float:
    ms = ctypes.c_float()
    _check(sim, load().mcx_last_kernel_ms(sim, ctypes.byref(ms)))
    return ms.value


def mcx_read_fluence(sim, dst, normalized: bool = False):
    """dst: float32 NumPy array or torch tensor of n_gates*nz*ny*nx elements."""
    n = dst.numel() if hasattr(dst, "numel") else dst.size
    _check(sim, load().mcx_read_fluence(sim, _ptr(dst), n, int(normalized), _on_device(dst)))
    return dst


def mcx_read_fluence64(sim, dst, normalized: bool = False):
    """dst: float64 NumPy array or torch tensor of n_gates*nz*ny*nx elements."""
    n = dst.numel() if hasattr(dst, "numel") else dst.size
    _check(sim, load().mcx_read_fluence64(sim, _ptr(dst), n, int(normalized), _on_device(dst)))
    return dst


def mcx_detected_stride(sim) -> int:
    return int(load().mcx_detected_stride(sim))


def mcx_read_detected(sim, cap: Optional[int] = None) -> Tuple[np.ndarray, int]:
    """Returns (records as uint32 words [n, stride], photons detected)."""
    L = load()
    stride = mcx_detected_stride(sim)
    nw, nt = ctypes.c_uint64(), ctypes.c_uint64()
    if cap is None:
        _check(sim, L.mcx_read_detected(sim, None, 0, ctypes.byref(nw), ctypes.byref(nt)))
        cap = int(nt.value)
    buf = np.zeros((max(cap, 0), stride), dtype=np.uint32)
    _check(sim, L.mcx_read_detected(sim, _ptr(buf) if cap else None, cap, ctypes.byref(nw),
                                    ctypes.byref(nt)))
    return buf[: nw.value], int(nt.value)


def mcx_read_tally(sim) -> dict:
    out = np.zeros(6, dtype=np.float64)
    _check(sim, load().mcx_read_tally(sim, _ptr(out)))
    return dict(zip(TALLY_NAMES, out.tolist()))


def mcx_read_stats(sim) -> dict:
    out = np.zeros(8, dtype=np.uint64)
    _check(sim, load().mcx_read_stats(sim, _ptr(out)))
    return dict(zip(STAT_NAMES, [int(v) for v in out]))


def mcx_read_exits(sim, cap: int) -> np.ndarray:
    buf = np.zeros(cap, dtype=EXIT_DTYPE)
    nw = ctypes.c_uint64()
    _check(sim, load().mcx_read_exits(sim, _ptr(buf) if cap else None, cap, ctypes.byref(nw)))
    return buf[: nw.value]


def mcx_launch_info(sim) -> dict:
    out = np.zeros(4, dtype=np.int32)
    _check(sim, load().mcx_launch_info(sim, _ptr(out)))
    return dict(zip(("grid", "block", "blocks_per_sm", "regs"), out.tolist()))


def mcx_last_error(sim=None) -> str:
    r = load().mcx_last_error(sim)
    return r.decode() if r else ""


def mcx_destroy(sim):
    if sim:
        load().mcx_destroy(sim)


NOALLOC_NOUT = 7        # tallies, then the count of photons stopped by the event cap


def mcx_run_noalloc(labels_dev, voxel_mm: float, media, src_kind: int, pos, direction,
                    waist_mm: float, cfg: McxRunCfg, fluence_dev, tally_dev):
    """Allocation-free run on caller-owned device tensors (see include/mcx.h): labels_dev
    uint8 [nz, ny, nx]; fluence_dev [n_gates, nz, ny, nx], float32 for accum_mode 0 and
    float64 for accum_mode 2; tally_dev float64 [7] (the six tallies, then the number of
    photons stopped by the per-photon event cap); all contiguous torch tensors on the
    current CUDA device.  Enqueued on cfg.cuda_stream.  The tensors are checked here
    before the library is called, since it cannot check a buffer's size."""
    import torch
    dev = torch.cuda.current_device()
    expect = {"labels_dev": (labels_dev, torch.uint8, None),
              "fluence_dev": (fluence_dev, torch.float64 if cfg.accum_mode == 2 else torch.float32,
                              None),
              "tally_dev": (tally_dev, torch.float64, NOALLOC_NOUT)}
    if labels_dev is not None and getattr(labels_dev, "dim", lambda: 0)() == 3:
        nz, ny, nx = labels_dev.shape
        expect["fluence_dev"] = expect["fluence_dev"][:2] + (int(cfg.n_gates) * nz * ny * nx,)
    else:
        raise ValueError("labels_dev must be a 3-D uint8 CUDA tensor [nz, ny, nx]")
    for name, (t, dtype, numel) in expect.items():
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device (cuda:{dev})")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype} (accum_mode {cfg.accum_mode}), got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"{name} must hold {numel} elements, has {t.numel()}")
    a = np.ascontiguousarray(media, dtype=np.float32).reshape(-1, 4)
    p = np.ascontiguousarray(pos, dtype=np.float32)
    d = np.ascontiguousarray(direction, dtype=np.float32)
    _check(None, load().mcx_run_noalloc(_ptr(labels_dev), nx, ny, nz, float(voxel_mm), a.shape[0],
                                        _ptr(a), int(src_kind), _ptr(p), _ptr(d), float(waist_mm),
                                        ctypes.byref(cfg), _ptr(fluence_dev), _ptr(tally_dev)))


PROBE_KINDS = ("ffma", "lop3", "lg2", "ex2", "rsqrt", "sin", "red_f32", "red_f64",
               "red_f32_hot", "red_f64_hot")


def mcx_probe_rate(kind, map_bytes: int = 0) -> float:
    """Measured rate (ops/s) of one device resource; kind is an index or a PROBE_KINDS name."""
    k = PROBE_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    r = ctypes.c_double()
    _check(None, load().mcx_probe_rate(k, int(map_bytes), ctypes.byref(r)))
    return r.value


def mcx_debug_uniforms(seed: int, photon: int, n: int) -> np.ndarray:
    """[n, 5]: per generator output, the single draw, the pair's second value and the
    three values of a triple draw."""
    out = np.zeros((n, 5), dtype=np.float32)
    _check(None, load().mcx_debug_uniforms(seed, photon, n, _ptr(out)))
    return out


def mcx_debug_primitive(kind: int, inputs: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(inputs, dtype=np.float32)
    n = a.shape[0]
    nout = {0: 2, 1: 3, 2: 1}[kind]
    out = np.zeros((n, nout), dtype=np.float32)
    _check(None, load().mcx_debug_primitive(kind, n, _ptr(a), _ptr(out)))
    return out if nout > 1 else out[:, 0]


def mcx_debug_conv3d(kind: int, x: np.ndarray, w=None, bias=None, dy=None, cout=None) -> np.ndarray:
    """One denoiser convolution on host arrays: x [n, nz, ny, nx, cin] (channels last).
    kind 0: w [27, cout, cin], bias [cout] or None -> ReLU(conv + bias), BF16-rounded
    kind 1: dy [n, nz, ny, nx, cout] -> weight gradient [27, cout, cin]"""
    xa = np.ascontiguousarray(x, dtype=np.float32)
    n, nz, ny, nx, cin = xa.shape
    if kind == 0:
        wa = np.ascontiguousarray(w, dtype=np.float32)
        cout = wa.shape[1]
        ba = None if bias is None else np.ascontiguousarray(bias, dtype=np.float32)
        out = np.zeros((n, nz, ny, nx, cout), dtype=np.float32)
        _check(None, load().mcx_debug_conv3d(kind, n, nz, ny, nx, cin, cout, _ptr(xa), _ptr(wa),
                                             _ptr(ba), None, _ptr(out)))
    else:
        da = np.ascontiguousarray(dy, dtype=np.float32)
        cout = da.shape[-1]
        out = np.zeros((27, cout, cin), dtype=np.float32)
        _check(None, load().mcx_debug_conv3d(1, n, nz, ny, nx, cin, cout, _ptr(xa), None, None,
                                             _ptr(da), _ptr(out)))
    return out


def mcx_debug_wait_timeout(arrive: bool, limit_log2: int = 16) -> bool:
    """True when the bounded mbarrier wait gave up (see include/mcx.h)."""
    out = ctypes.c_int32()
    _check(None, load().mcx_debug_wait_timeout(int(bool(arrive)), limit_log2, ctypes.byref(out)))
    return bool(out.value)


def decode_detected(rec: np.ndarray) -> dict:
    """Splits uint32 record words into named fields (see include/mcx.h)."""
    f = rec.view(np.float32)
    return {
        "id": rec[:, 0].astype(np.uint64) | (rec[:, 1].astype(np.uint64) << np.uint64(32)),
        "det": rec[:, 2].view(np.int32),
        "nscat": rec[:, 3],
        "w": f[:, 4],
        "pos": f[:, 5:8],
        "dir": f[:, 8:11],
        "nrr": rec[:, 11],
        "ppath": f[:, REC_BASE:],
    }


def photon_range(rank: int, world: int, n_per_rank: int) -> Tuple[int, int]:
    """Photon-id range [offset, offset + n) of one rank when each of `world` ranks (one per
    GPU) simulates its own n_per_rank photons.  Photons are independent and a run is a pure
    function of (seed, id range), so the ranks' results compose into one run over
    [0, world * n_per_rank) with no exchange during the walk."""
    if not (0 <= rank < world) or n_per_rank < 0:
        raise ValueError("need 0 <= rank < world and n_per_rank >= 0")
    return rank * n_per_rank, n_per_rank


# ------------------------------------------------------------------------ batches
def _bcheck(b, st: int):
    if st != MCX_OK:
        L = load()
        msg = L.mcx_batch_last_error(b) if b else L.mcx_last_error(None)
        raise McxError(st, (msg or b"").decode() or L.mcx_status_string(st).decode())
    return st


def mcx_batch_cfg_default(**overrides) -> McxBatchCfg:
    cfg = McxBatchCfg()
    load().mcx_batch_cfg_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "cuda_stream":
            v = _stream_handle(v)
        setattr(cfg, k, v)
    return cfg


class Batch:
    """Many simulations in one persistent launch (mcx_batch_* in include/mcx.h)."""

    def __init__(self):
        L = load()
        h = ctypes.c_void_p()
        _check(None, L.mcx_batch_create(ctypes.byref(h)))
        self.handle = h
        self.shapes = []
        self.n_gates = 1

    def add(self, labels, voxel_mm, media, src_kind=0, src_pos=(0, 0, 0), src_dir=(0, 0, 1),
            waist_mm=0.0, n_photons=0, seed=1) -> int:
        lab = np.ascontiguousarray(labels, dtype=np.uint8)
        nz, ny, nx = lab.shape
        a = np.ascontiguousarray(media, dtype=np.float32).reshape(-1, 4)
        p = np.ascontiguousarray(src_pos, dtype=np.float32)
        d = np.ascontiguousarray(src_dir, dtype=np.float32)
        out = ctypes.c_int32()
        _bcheck(self.handle, load().mcx_batch_add(self.handle, nx, ny, nz, float(voxel_mm),
                                                  _ptr(lab), 0, a.shape[0], _ptr(a), int(src_kind),
                                                  _ptr(p), _ptr(d), float(waist_mm), int(n_photons),
                                                  int(seed), ctypes.byref(out)))
        self.shapes.append(lab.shape)
        return out.value

    def add_workload(self, wl, n_photons=None, seed=None) -> int:
        return self.add(wl.labels, wl.voxel_mm, wl.media, wl.src_kind, wl.src_pos, wl.src_dir,
                        wl.waist_mm, wl.n_photons if n_photons is None else n_photons,
                        wl.seed if seed is None else seed)

    def run(self, wait=True, **cfg):
        c = mcx_batch_cfg_default(**cfg)
        self.n_gates = c.n_gates
        _bcheck(self.handle, load().mcx_batch_run(self.handle, ctypes.byref(c)))
        if wait:
            _bcheck(self.handle, load().mcx_batch_sync(self.handle))

    def last_ms(self) -> float:
        ms = ctypes.c_float()
        _bcheck(self.handle, load().mcx_batch_last_ms(self.handle, ctypes.byref(ms)))
        return ms.value

    def fluence(self, sim_id: int, normalized=False, out=None):
        if out is None:
            out = np.zeros((self.n_gates,) + self.shapes[sim_id], dtype=np.float32)
        n = out.numel() if hasattr(out, "numel") else out.size
        _bcheck(self.handle, load().mcx_batch_read_fluence(self.handle, sim_id, _ptr(out), n,
                                                           int(normalized), _on_device(out)))
        return out

    def tally(self, sim_id: int) -> dict:
        out = np.zeros(6, dtype=np.float64)
        _bcheck(self.handle, load().mcx_batch_read_tally(self.handle, sim_id, _ptr(out)))
        return dict(zip(TALLY_NAMES, out.tolist()))

    def stats(self) -> dict:
        out = np.zeros(8, dtype=np.uint64)
        _bcheck(self.handle, load().mcx_batch_read_stats(self.handle, _ptr(out)))
        return dict(zip(STAT_NAMES, [int(v) for v in out]))

    def autotune(self, fraction=0.05, **cfg):
        c = mcx_batch_cfg_default(**cfg)
        ms = ctypes.c_float()
        _bcheck(self.handle, load().mcx_batch_autotune(self.handle, ctypes.byref(c), float(fraction),
                                                       ctypes.byref(ms)))
        return {"block_size": c.block_size, "claim_chunk": c.claim_chunk, "ms": ms.value}

    def __len__(self):
        return int(load().mcx_batch_size(self.handle))

    def close(self):
        if self.handle:
            load().mcx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------------------ convenience
class Simulation:
    """Owns one mcx_sim handle; thin sugar over the C-named functions."""

    def __init__(self, labels, voxel_mm: float, media, src_kind: int = 0,
                 src_pos=(0.0, 0.0, 0.0), src_dir=(0.0, 0.0, 1.0), waist_mm: float = 0.0,
                 detectors=None):
        self.handle = mcx_create_volume(labels, voxel_mm)
        self.shape = tuple(labels.shape)
        mcx_set_media(self.handle, media)
        mcx_set_source(self.handle, src_kind, src_pos, src_dir, waist_mm)
        if detectors is not None:
            for d in np.asarray(detectors, dtype=np.float64).reshape(-1, 4):
                mcx_add_detector(self.handle, d[:3], d[3])
        self.n_gates = 1

    @classmethod
    def from_workload(cls, wl):
        return cls(wl.labels, wl.voxel_mm, wl.media, wl.src_kind, wl.src_pos, wl.src_dir,
                   wl.waist_mm, wl.detectors if len(wl.detectors) else None)

    def run(self, n_photons: int, n_gates: int = 1, dt_ns: float = 5.0, seed: int = 1,
            stream=None, wait: bool = True, **kw):
        cfg = mcx_run_cfg_default(n_photons=n_photons, n_gates=n_gates, dt_ns=dt_ns, seed=seed,
                                  cuda_stream=stream, **kw)
        self.n_gates = n_gates
        mcx_run(self.handle, cfg)
        if wait:
            return mcx_sync(self.handle, allow_cap=True)
        return MCX_OK

    def fluence(self, normalized: bool = False, out=None):
        if out is None:
            out = np.zeros((self.n_gates,) + self.shape, dtype=np.float32)
        return mcx_read_fluence(self.handle, out, normalized)

    def fluence64(self, normalized: bool = False, out=None):
        if out is None:
            out = np.zeros((self.n_gates,) + self.shape, dtype=np.float64)
        return mcx_read_fluence64(self.handle, out, normalized)

    def tally(self):
        return mcx_read_tally(self.handle)

    def stats(self):
        return mcx_read_stats(self.handle)

    def exits(self, cap: int):
        return mcx_read_exits(self.handle, cap)

    def detected(self, cap=None):
        rec, total = mcx_read_detected(self.handle, cap)
        return decode_detected(rec), total

    def kernel_ms(self) -> float:
        return mcx_last_kernel_ms(self.handle)

    def launch_info(self):
        return mcx_launch_info(self.handle)

    def close(self):
        if self.handle:
            mcx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Denoiser:
    """The learned fluence denoiser (mcx_denoiser_* in include/mcx.h).  Volumes are torch
    CUDA tensors of shape [n, nz, ny, nx] (float32, contiguous), medium features
    [n, n_aux, nz, ny, nx]; the stream defaults to torch's current stream."""

    def __init__(self, shape, max_batch: int = 1, seed: int = 0, n_aux: int = 0):
        nz, ny, nx = shape
        h = ctypes.c_void_p()
        _check(None, load().mcx_denoiser_create(ctypes.byref(h), nx, ny, nz, max_batch, n_aux, seed))
        self.handle = h
        self.shape = (nz, ny, nx)
        self.max_batch = max_batch
        self.n_aux = n_aux
        n = ctypes.c_uint64()
        _check(None, load().mcx_denoiser_param_count(self.handle, ctypes.byref(n)))
        self.n_params = n.value

    @staticmethod
    def _stream(stream):
        if stream is None:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(_stream_handle(stream))

    def _vol(self, t):
        if not (getattr(t, "is_cuda", False) and t.is_contiguous() and t.shape[1:] == self.shape
                and str(t.dtype) == "torch.float32"):
            raise ValueError(f"need a contiguous float32 CUDA tensor [n, {self.shape}]")
        return t.shape[0]

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(None, load().mcx_denoiser_get_params(self.handle, _ptr(out), self.n_params, 0))
        return out

    def grads(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(None, load().mcx_denoiser_get_params(self.handle, _ptr(out), self.n_params, 1))
        return out

    def set_params(self, p: np.ndarray):
        a = np.ascontiguousarray(p, dtype=np.float32)
        if a.size != self.n_params:
            raise ValueError("wrong parameter count")
        _check(None, load().mcx_denoiser_set_params(self.handle, _ptr(a), self.n_params))

    def set_encoding(self, floor: float, mu: float, sigma: float):
        _check(None, load().mcx_denoiser_set_encoding(self.handle, floor, mu, sigma))

    def _aux(self, aux, n):
        if not self.n_aux:
            return None
        if aux is None or tuple(aux.shape) != (n, self.n_aux) + self.shape or not aux.is_contiguous():
            raise ValueError(f"need medium features [n, {self.n_aux}, {self.shape}]")
        return _ptr(aux)

    def forward(self, x, y, aux=None, stream=None):
        n = self._vol(x)
        self._vol(y)
        _check(None, load().mcx_denoiser_forward(self.handle, _ptr(x), self._aux(aux, n), _ptr(y), n,
                                                 self._stream(stream)))

    def train_step(self, x, t, lr: float, aux=None, stream=None) -> float:
        n = self._vol(x)
        self._vol(t)
        loss = ctypes.c_float()
        _check(None, load().mcx_denoiser_train_step(self.handle, _ptr(x), self._aux(aux, n), _ptr(t), n, lr,
                                                    ctypes.byref(loss), self._stream(stream)))
        return loss.value

    def encode(self, phi, x, stream=None):
        _check(None, load().mcx_denoiser_encode(self.handle, _ptr(phi), _ptr(x), phi.numel(),
                                                self._stream(stream)))

    def decode(self, x, phi, stream=None):
        _check(None, load().mcx_denoiser_decode(self.handle, _ptr(x), _ptr(phi), x.numel(),
                                                self._stream(stream)))

    def apply(self, phi_in, phi_out, aux=None, stream=None):
        n = self._vol(phi_in)
        self._vol(phi_out)
        _check(None, load().mcx_denoiser_apply(self.handle, _ptr(phi_in), self._aux(aux, n), _ptr(phi_out), n,
                                               self._stream(stream)))

    @staticmethod
    def features(labels_dev, media, out, stream=None):
        """the two medium features of a label volume (torch uint8 CUDA tensor) into out
        (float32 CUDA tensor of 2 * labels.numel() values); see mcx_denoiser_features"""
        a = np.ascontiguousarray(media, dtype=np.float32).reshape(-1, 4)
        if out.numel() != 2 * labels_dev.numel():
            raise ValueError("out must hold 2 values per voxel")
        _check(None, load().mcx_denoiser_features(_ptr(labels_dev), labels_dev.numel(), a.shape[0], _ptr(a),
                                                  _ptr(out), Denoiser._stream(stream)))

    def gather(self, volumes, idx, flags, out, stream=None):
        """out[s] = transformed volumes[idx[s]] (see mcx_denoiser_gather)"""
        i = np.ascontiguousarray(idx, dtype=np.uint64)
        f = np.ascontiguousarray(flags, dtype=np.uint32)
        if i.size != f.size or out.shape[0] != i.size:
            raise ValueError("idx, flags and out must agree in length")
        self._vol(volumes)
        self._vol(out)
        _check(None, load().mcx_denoiser_gather(self.handle, _ptr(volumes), volumes.shape[0], _ptr(i),
                                                _ptr(f), i.size, _ptr(out), self._stream(stream)))

    def sync(self):
        """waits for the device and raises McxError if a tensor-core wait timed out"""
        _check(None, load().mcx_denoiser_sync(self.handle))

    def close(self):
        if self.handle:
            load().mcx_denoiser_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
