"""The oracle's pins catch the slips they are there for (CPU).

Each case plants one plausible mistake -- a dropped term, a wrong sign, index or bound, a
transposed operand -- in a copy of oracle/mcx_oracle.c, compiles the copy to a library
of its own, and runs tests/test_oracle_pins.py against it (MCX_ORACLE_LIB); at least
one pin must fail (a pin that runs for more than 30 s counts as failing: some slips make
a photon loop for ever; so does a crash, which an index slip can cause).  The oracle's own source is never modified.  All cases run in
parallel subprocesses once per module.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (what the slip is, the expression, what it becomes)
MUTANTS = [
    ("hop spent in mm instead of mean free paths", "s - l * mus;", "s - l;"),
    ("time advanced at c0 instead of c0 / n", "t += l * n / ORC_C0;", "t += l / ORC_C0;"),
    ("absorption with mus instead of mua", "w * (1.0 - exp(-mua * l))", "w * (1.0 - exp(-mus * l))"),
    ("time limit distance without the index", "(t_end - t) * ORC_C0 / n;", "(t_end - t) * ORC_C0;"),
    ("gate index from t * dt", "floor(t / P->dt)", "floor(t * P->dt)"),
    ("face bounds swapped", "(dir[a] > 0.0 ? (double)(v[a] + 1) : (double)v[a]) * h",
     "(dir[a] > 0.0 ? (double)v[a] : (double)(v[a] + 1)) * h"),
    ("HG: sign of g^2 in the numerator", "c = (1.0 + g * g - f * f) / (2.0 * g);",
     "c = (1.0 - g * g - f * f) / (2.0 * g);"),
    ("rotation: sign of the azimuth term", "out[1] = sin_t * (u[1] * u[2] * cp + u[0] * sp)",
     "out[1] = sin_t * (u[1] * u[2] * cp - u[0] * sp)"),
    ("Fresnel: index ratio inverted at the face", "const double eta = na / nb;",
     "const double eta = nb / na;"),
    ("Fresnel: rp with the cosines swapped", "rp = (n1 * cos_t - n2 * cos_i)", "rp = (n1 * cos_i - n2 * cos_t)"),
    ("reflection flips the wrong component", "dir[axis] = -dir[axis];",
     "dir[(axis + 1) % 3] = -dir[(axis + 1) % 3];"),
    ("Snell: tangential components divided by eta", "if (a != axis) dir[a] *= eta;",
     "if (a != axis) dir[a] /= eta;"),
    ("roulette survivors keep their weight", "w *= P->rr_m;", "(void)0;"),
    ("detector radius compared with the squared distance", "<= dd[3] * dd[3]", "<= dd[3]"),
    ("Gaussian radius without the 1/2", "sqrt(-log(xi1) / 2.0)", "sqrt(-log(xi1))"),
    ("face ties taken on the highest axis", "if (d < d_face) { d_face = d; axis = a; bound = b; }",
     "if (d <= d_face) { d_face = d; axis = a; bound = b; }"),
    ("label lookup with x and y transposed",
     "P->labels[((uint64_t)v[2] * P->ny + (uint64_t)v[1]) * P->nx + (uint64_t)v[0]]",
     "P->labels[((uint64_t)v[2] * P->ny + (uint64_t)v[0]) * P->nx + (uint64_t)v[1]]"),
    ("deposit index with x and y transposed",
     "((uint64_t)v[2] * P->ny + (uint64_t)v[1]) * P->nx + (uint64_t)v[0];",
     "((uint64_t)v[2] * P->ny + (uint64_t)v[0]) * P->nx + (uint64_t)v[1];"),
    ("Fresnel reflectance without the 1/2", "return 0.5 * (rs * rs + rp * rp);", "return (rs * rs + rp * rp);"),
    ("roulette gain counted as m w", "(P->rr_m - 1.0) * w;", "P->rr_m * w;"),
    ("Snell: normal component reversed", "dir[axis] = dir[axis] > 0.0 ? cos_t : -cos_t;",
     "dir[axis] = dir[axis] > 0.0 ? -cos_t : cos_t;"),
    ("Gaussian azimuth over half a turn", "ph = 2.0 * ORC_PI * xi2;", "ph = ORC_PI * xi2;"),
    ("launch on a face: the voxel behind", "if (c == (double)v[a] && dir[a] < 0.0) v[a] -= 1;",
     "if (c == (double)v[a] && dir[a] > 0.0) v[a] -= 1;"),
    ("detected record: paths shifted by one medium", "r[10 + m] = L[m];", "r[10 + m] = L[m - 1];"),
    ("triple draw: third uniform from the wrong bits", "(r >> 1) & 0x1FFFFFULL", "(r >> 2) & 0x1FFFFFULL"),
    ("xorshift128+: a shift constant", "a ^= a << 23;", "a ^= a << 22;"),
    ("xorshift128+: output xor instead of sum", "const uint64_t result = a + b;", "const uint64_t result = a ^ b;"),
    ("single draw: 2k instead of 2k + 1", "return (double)(2 * k + 1) * (1.0 / 16777216.0);",
     "return (double)(2 * k) * (1.0 / 16777216.0);"),
    ("pair draw: second uniform from the wrong bits", "*u2 = (double)(2 * ((r >> 18) & 0x7FFFFFULL) + 1)",
     "*u2 = (double)(2 * ((r >> 17) & 0x7FFFFFULL) + 1)"),
]


def _run(tmp, old, new):
    src = open(os.path.join(ORACLE, "mcx_oracle.c")).read()
    if src.count(old) != 1:
        return f"the expression occurs {src.count(old)} times in mcx_oracle.c"
    os.makedirs(tmp, exist_ok=True)
    with open(os.path.join(tmp, "mcx_oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    shutil.copy(os.path.join(ORACLE, "mcx_oracle.h"), tmp)
    lib = os.path.join(tmp, "libmcx_oracle_mutant.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", lib,
                    os.path.join(tmp, "mcx_oracle.c"), "-lm"], check=True, cwd=tmp)
    env = dict(os.environ, MCX_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    # a slip can also make a photon loop for ever (a pin that never ends fails after 30 s)
    # the thread method ends the process even inside a C call that never returns
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider",
                        "--timeout", "30", "--timeout-method", "thread"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-3000:]


CONTROL = "the unmodified copy"


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = tmp_path_factory.mktemp("mutants")
    cases = [(CONTROL, "void orc_rotate(", "void orc_rotate(")] + MUTANTS
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_run, str(base / f"m{k}"), old, new)
                for k, (name, old, new) in enumerate(cases)}
        return {name: f.result() for name, f in futs.items()}


def test_the_pins_pass_on_an_unmodified_copy(outcomes):
    res = outcomes[CONTROL]
    assert not isinstance(res, str), res
    code, out = res
    assert code == 0 and " passed" in out and "failed" not in out, out


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_a_pin_fails_on(outcomes, name):
    res = outcomes[name]
    assert not isinstance(res, str), res
    code, out = res
    # a failing pin, a pin that never ends, or (an index slip reading outside the volume)
    # the process killed by a signal
    caught = (code == 1 and (" failed" in out or "Timeout" in out)) or code < 0
    assert caught, f"no pin failed (pytest exit {code}):\n{out}"


# Slips in the oracle's one Python-side arithmetic function, the fluence normalisation
# E / (mua h^3 N dt): each mutant is compiled from the function's own source with one
# expression changed, and the two normalisation pins run against it.
NORMALISE_MUTANTS = [
    ("voxel area instead of volume", "voxel_mm ** 3", "voxel_mm ** 2"),
    ("gate width dropped", "n_photons * dt_ns)", "n_photons)"),
    ("photon count dropped", "* n_photons * dt_ns", "* dt_ns"),
    ("mua of the exterior row", "np.asarray(media)[:, 0][labels]", "np.asarray(media)[0, 0] + 0 * labels"),
    ("mua = 0 voxels left undefined", "phi[:, mua == 0] = 0.0", "pass"),
]


@pytest.mark.parametrize("name, old, new", NORMALISE_MUTANTS, ids=[m[0] for m in NORMALISE_MUTANTS])
def test_a_normalisation_pin_fails_on(orc, name, old, new):
    import inspect
    import types
    import warnings
    import numpy as np
    sys.path.insert(0, os.path.dirname(PINS))
    import test_oracle_pins as pins
    src = inspect.getsource(orc.normalise)
    assert src.count(old) == 1, (name, old)
    ns = {"np": np}
    exec(src.replace(old, new), ns)
    fake = types.SimpleNamespace(**{k: getattr(orc, k) for k in dir(orc) if not k.startswith("__")})
    fake.normalise = ns["normalise"]
    failed = 0
    for pin in (pins.test_normalised_fluence_golden, pins.test_normalised_fluence_is_the_track_length_fluence):
        try:
            with warnings.catch_warnings():
                warnings.simplefilter("ignore")
                pin(fake)
        except AssertionError:
            failed += 1
    assert failed > 0, f"no normalisation pin failed on: {name}"
