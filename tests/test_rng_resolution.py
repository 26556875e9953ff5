"""What the draws' finite resolution does to the results (CPU, oracle only).

The walk draws its uniforms at 21 bits (three per generator output at a scattering event)
or 23 bits (one per output elsewhere), so that one 64-bit output serves a whole scattering
event.  Here the oracle is compiled a second time with every uniform taken from its own
generator output at 53 bits (-DORC_FULL_RES_DRAWS), and the two builds are compared on
independent photons: the voxel-wise Welch test of eight 1e5-photon batches per side, in
the homogeneous volume and in the two-sphere volume with its ten gates, and the energy
tallies per launched photon within their combined Monte Carlo error.  A difference the
resolution made would show in the fluence near the source (short hops), in the deep
tail of long hops, or in the backscatter of the deflection.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads
from gpu_common import F32_RR, assert_voxelwise, f32

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

N, K = 100_000, 8

_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import oracle, workloads
from gpu_common import F32_RR, f32
name, n, k, off, path = sys.argv[2], int(sys.argv[3]), int(sys.argv[4]), int(sys.argv[5]), sys.argv[6]
wl = f32(workloads.by_name(name, n_photons=n))
maps, tallies = [], []
for i in range(k):
    o = oracle.run(wl, n_photons=n, photon_offset=off + i * n, rr_threshold=F32_RR)
    maps.append(o.energy / n)
    tallies.append([o.tally[t] / n for t in oracle.TALLY_NAMES])
np.savez(path, maps=np.array(maps), tallies=np.array(tallies))
"""


@pytest.fixture(scope="module")
def full_res_lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("fullres")
    lib = str(d / "libmcx_oracle_fullres.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-DORC_FULL_RES_DRAWS",
                    "-o", lib, os.path.join(ORACLE, "mcx_oracle.c"), "-lm"], check=True)
    return lib


def _batches(name, lib, path, off):
    env = dict(os.environ)
    if lib:
        env["MCX_ORACLE_LIB"] = lib
    else:
        env.pop("MCX_ORACLE_LIB", None)
    subprocess.run([sys.executable, "-c", _CHILD, ROOT, name, str(N), str(K), str(off), path],
                   env=env, check=True, timeout=900)
    z = np.load(path)
    return z["maps"], z["tallies"]


@pytest.mark.slow
@pytest.mark.parametrize("name", ["c1", "c2"])
def test_full_resolution_draws_agree(orc, full_res_lib, tmp_path, name):
    std_maps, std_t = _batches(name, None, str(tmp_path / "std.npz"), 0)
    full_maps, full_t = _batches(name, full_res_lib, str(tmp_path / "full.npz"), 10 * N * K)
    assert_voxelwise(std_maps, full_maps, min_vox=1000)
    # tallies per launched photon (absorbed, escaped, time_exceeded, killed, gained)
    for j in range(1, 6):
        a, b = std_t[:, j], full_t[:, j]
        se = math.sqrt(a.var(ddof=1) / K + b.var(ddof=1) / K)
        assert abs(a.mean() - b.mean()) <= 4 * se + 1e-12, (j, a.mean(), b.mean(), se)


def test_full_resolution_build_draws_53_bit_uniforms(full_res_lib):
    """The test-only build really changes the draws: its uniforms are off the 2^-24 grid of
    the single draw, and a triple draw takes three consecutive outputs (the same values as
    three single draws)."""
    code = ("import sys; sys.path.insert(0, sys.argv[1]); import oracle, json, numpy as np; "
            "u = oracle.uniforms(5, 3, 1000); t = oracle.uniform_triples(5, 3, 2); "
            "print(json.dumps([float(np.mean((u * 2**24 - 1) / 2 % 1 != 0)), u[:6].tolist(), "
            "t.ravel().tolist()]))")
    env = dict(os.environ, MCX_ORACLE_LIB=full_res_lib)
    r = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True, text=True,
                       check=True)
    off_grid, u6, t6 = json.loads(r.stdout)
    assert off_grid > 0.99
    assert u6 == t6
