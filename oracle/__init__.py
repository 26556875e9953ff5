"""FP64 CPU oracle for the voxel Monte Carlo photon walk (Python side).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py` may import this package.  The product path (the CUDA library and its
binding) never loads it, and it loads nothing from the product path: it shares no code
with the CUDA library.  It takes its inputs from `workloads` (the seeded input
generators, which hold none of the method's arithmetic).

Parity status of each oracle function (what pins it, see tests/test_oracle_pins.py):
  * RNG (SplitMix64 seeding, xorshift128+ uniforms): SplitMix64 published test vector;
    the xorshift128+ transition's full period 2^128 - 1 (its GF(2) matrix against the
    prime factors of 2^128 - 1); the sum scrambler's nonlinearity (linear complexity of
    the top output bit); uniform moments, range and exact float
    representability; the pair and triple draws against the bit fields of the single
    draws of the same outputs.
  * orc_hg_cos: mean cosine = g, chi^2 against the HG density, isotropic limit.
  * orc_rotate: unit norm, deflection cosine, azimuth uniformity, vertical special case.
  * orc_fresnel_R: normal-incidence closed form, the independent sine/tangent form of the
    Fresnel equations, critical angle, R + T = 1 with the transmission form.
  * orc_run: Beer-Lambert column (exact), ballistic transmission through two scattering
    layers (binomial), a ray trapped by total internal reflection, a diagonal ray
    through voxel edges, the lowest-axis tie rule and a ray along x through two media
    (exact), causality of the time gates, Fresnel slab escape series
    (binomial), exact energy balance, detector weight identity, detector membership and
    tie-break, Snell refraction on a ballistic ray, Gaussian-source moments,
    diffusion-theory far field (about 10%).
  * normalise: hand-evaluated values of E / (mua h^3 N dt) (tests/golden/
    normalised_fluence.txt) and, on an oracle run of a layered purely absorbing column,
    the track-length estimate of the same fluence (the weight integrated numerically
    along the path in each voxel, over h^3 dt).
tests/test_oracle_mutants.py plants one plausible slip at a time in a copy of
mcx_oracle.c and checks that some pin fails on it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcx_oracle.c")
# MCX_ORACLE_LIB: a library compiled elsewhere from a modified copy of mcx_oracle.c (the
# mutation tests run the pins against such copies); build() then leaves it as it is
_LIB_OVERRIDE = os.environ.get("MCX_ORACLE_LIB")
_LIB = _LIB_OVERRIDE or os.path.join(_HERE, "libmcx_oracle.so")
_lock = threading.Lock()
_lib = None

FATE_NONE, FATE_ESCAPED, FATE_ROULETTE, FATE_TIME, FATE_MISSED, FATE_CAPPED = range(6)
TALLY_NAMES = ("launched", "absorbed", "escaped", "time_exceeded", "roulette_killed",
               "roulette_gained")
COUNT_NAMES = ("scatter", "face", "fresnel", "deposit_runs", "roulette", "hops", "segments",
               "detected")
C0_MM_PER_NS = 299.792458


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) next to its source."""
    if _LIB_OVERRIDE:
        return _LIB
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mcx_oracle.h"))):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIB)
        return _LIB


class OrcProblem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_uint32), ("ny", ctypes.c_uint32), ("nz", ctypes.c_uint32),
        ("h", ctypes.c_double),
        ("labels", ctypes.c_void_p),
        ("n_media", ctypes.c_uint32),
        ("props", ctypes.c_void_p),
        ("src_kind", ctypes.c_int32),
        ("src_pos", ctypes.c_double * 3),
        ("src_dir", ctypes.c_double * 3),
        ("waist", ctypes.c_double),
        ("n_det", ctypes.c_uint32),
        ("det", ctypes.c_void_p),
        ("n_photons", ctypes.c_uint64),
        ("photon_offset", ctypes.c_uint64),
        ("seed", ctypes.c_uint64),
        ("dt", ctypes.c_double),
        ("n_gates", ctypes.c_uint32),
        ("reflect", ctypes.c_int32),
        ("rr_threshold", ctypes.c_double),
        ("rr_m", ctypes.c_double),
        ("max_events", ctypes.c_uint64),
        ("n_threads", ctypes.c_int32),
    ]


class OrcExit(ctypes.Structure):
    _fields_ = [("fate", ctypes.c_int32), ("nscat", ctypes.c_uint32),
                ("pos", ctypes.c_double * 3), ("dir", ctypes.c_double * 3),
                ("w", ctypes.c_double), ("t", ctypes.c_double)]


EXIT_DTYPE = np.dtype([("fate", np.int32), ("nscat", np.uint32), ("pos", np.float64, 3),
                       ("dir", np.float64, 3), ("w", np.float64), ("t", np.float64)])
assert EXIT_DTYPE.itemsize == ctypes.sizeof(OrcExit)


class OrcResult(ctypes.Structure):
    _fields_ = [
        ("energy", ctypes.c_void_p),
        ("tally", ctypes.c_double * 6),
        ("count", ctypes.c_uint64 * 8),
        ("exits", ctypes.c_void_p),
        ("exit_cap", ctypes.c_uint64),
        ("det_rec", ctypes.c_void_p),
        ("det_cap", ctypes.c_uint64),
        ("det_n", ctypes.c_uint64),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_run.argtypes = [ctypes.POINTER(OrcProblem), ctypes.POINTER(OrcResult)]
        L.orc_run.restype = ctypes.c_int
        L.orc_splitmix64_output.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_splitmix64_output.restype = ctypes.c_uint64
        L.orc_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_void_p]
        L.orc_uniforms.restype = None
        L.orc_uniform_pairs.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_void_p]
        L.orc_uniform_pairs.restype = None
        L.orc_uniform_triples.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_void_p]
        L.orc_uniform_triples.restype = None
        L.orc_xorshift_step.argtypes = [ctypes.c_void_p]
        L.orc_xorshift_step.restype = None
        L.orc_hg_cos.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_hg_cos.restype = ctypes.c_double
        L.orc_rotate.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_void_p]
        L.orc_rotate.restype = None
        L.orc_fresnel_R.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_fresnel_R.restype = ctypes.c_double
        L.orc_rec_stride.argtypes = [ctypes.c_uint32]
        L.orc_rec_stride.restype = ctypes.c_int
        _lib = L
    return _lib


# --------------------------------------------------------------------------- primitives
def splitmix64_output(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64_output(seed, k))


def uniforms(seed: int, photon: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    lib().orc_uniforms(seed, photon, n, out.ctypes.data)
    return out


def uniform_pairs(seed: int, photon: int, n: int) -> np.ndarray:
    """n pair draws (two uniforms from one generator output each), shape [n, 2]."""
    out = np.empty(2 * n, dtype=np.float64)
    lib().orc_uniform_pairs(seed, photon, n, out.ctypes.data)
    return out.reshape(n, 2)


def uniform_triples(seed: int, photon: int, n: int) -> np.ndarray:
    """n triple draws (three uniforms from one generator output each), shape [n, 3]."""
    out = np.empty(3 * n, dtype=np.float64)
    lib().orc_uniform_triples(seed, photon, n, out.ctypes.data)
    return out.reshape(n, 3)


def xorshift_step(s0: int, s1: int):
    """the generator's state (s0, s1) after one transition"""
    st = np.array([s0, s1], dtype=np.uint64)
    lib().orc_xorshift_step(st.ctypes.data)
    return int(st[0]), int(st[1])


def hg_cos(g: float, xi: float) -> float:
    return float(lib().orc_hg_cos(g, xi))


def rotate(u, cos_t: float, phi: float) -> np.ndarray:
    a = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(3, dtype=np.float64)
    lib().orc_rotate(a.ctypes.data, cos_t, phi, out.ctypes.data)
    return out


def fresnel_R(n1: float, n2: float, cos_i: float) -> float:
    return float(lib().orc_fresnel_R(n1, n2, cos_i))


def rec_stride(n_media: int) -> int:
    return int(lib().orc_rec_stride(n_media))


# --------------------------------------------------------------------------- full runs
class OracleResult:
    def __init__(self, energy, tally, count, exits, det_rec, det_n):
        self.energy = energy          # float64 [G, nz, ny, nx] absorbed weight (or None)
        self.tally = tally            # dict of the six energy tallies
        self.count = count            # dict of event counters
        self.exits = exits            # structured array (EXIT_DTYPE) or None
        self.det_rec = det_rec        # float64 [n, stride] or None
        self.det_n = det_n


def run(wl, n_photons: Optional[int] = None, seed: Optional[int] = None,
        photon_offset: int = 0, exit_cap: int = 0, det_cap: Optional[int] = None,
        energy: bool = True, rr_threshold: float = 1e-4, rr_m: float = 10.0,
        max_events: int = 0, n_threads: int = 0, n_gates: Optional[int] = None,
        dt_ns: Optional[float] = None, reflect: Optional[int] = None) -> OracleResult:
    """Runs the oracle on a `workloads.Workload`."""
    labels = np.ascontiguousarray(wl.labels, dtype=np.uint8)
    media = np.ascontiguousarray(wl.media, dtype=np.float64)
    det = np.ascontiguousarray(wl.detectors, dtype=np.float64).reshape(-1, 4)
    nz, ny, nx = labels.shape
    P = OrcProblem()
    P.nx, P.ny, P.nz = nx, ny, nz
    P.h = wl.voxel_mm
    P.labels = labels.ctypes.data
    P.n_media = media.shape[0]
    P.props = media.ctypes.data
    P.src_kind = wl.src_kind
    P.src_pos = (ctypes.c_double * 3)(*wl.src_pos)
    P.src_dir = (ctypes.c_double * 3)(*wl.src_dir)
    P.waist = wl.waist_mm
    P.n_det = det.shape[0]
    P.det = det.ctypes.data if det.shape[0] else None
    P.n_photons = wl.n_photons if n_photons is None else n_photons
    P.photon_offset = photon_offset
    P.seed = wl.seed if seed is None else seed
    P.dt = wl.dt_ns if dt_ns is None else dt_ns
    P.n_gates = wl.n_gates if n_gates is None else n_gates
    P.reflect = wl.reflect if reflect is None else reflect
    P.rr_threshold = rr_threshold
    P.rr_m = rr_m
    P.max_events = max_events
    P.n_threads = n_threads
    G = P.n_gates
    en = np.zeros((G, nz, ny, nx), dtype=np.float64) if energy else None
    ex = np.zeros(exit_cap, dtype=EXIT_DTYPE) if exit_cap else None
    stride = rec_stride(media.shape[0])
    if det_cap is None:
        det_cap = 1_000_000 if det.shape[0] else 0
    rec = np.zeros((det_cap, stride), dtype=np.float64) if det_cap else None
    R = OrcResult()
    R.energy = en.ctypes.data if en is not None else None
    R.exits = ex.ctypes.data if ex is not None else None
    R.exit_cap = exit_cap
    R.det_rec = rec.ctypes.data if rec is not None else None
    R.det_cap = det_cap
    rc = lib().orc_run(ctypes.byref(P), ctypes.byref(R))
    if rc != 0:
        raise ValueError(f"orc_run failed with {rc}")
    tally = dict(zip(TALLY_NAMES, list(R.tally)))
    count = dict(zip(COUNT_NAMES, [int(c) for c in R.count]))
    det_n = int(R.det_n)
    if rec is not None:
        rec = rec[:min(det_n, det_cap)]
    return OracleResult(en, tally, count, ex, rec, det_n)


def normalise(energy: np.ndarray, media: np.ndarray, labels: np.ndarray, voxel_mm: float,
              n_photons: int, dt_ns: float) -> np.ndarray:
    """Fluence per launched photon (1/mm^2/ns) from absorbed weight: E / (mua h^3 N dt);
    0 where mua = 0."""
    mua = np.asarray(media)[:, 0][labels]
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = energy / (mua[None] * voxel_mm ** 3 * n_photons * dt_ns)
    phi[:, mua == 0] = 0.0
    return phi
