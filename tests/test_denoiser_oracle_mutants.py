"""The denoiser oracle's pins catch the slips they are there for (CPU).

Each case plants one plausible mistake in a copy of oracle/denoiser.py, inside a scratch
copy of the oracle package, the input generators and the pin file, and runs
tests/test_denoiser_oracle.py there; at least one pin must fail.  The repository's own
files are never modified.  The cases run in parallel subprocesses once per module.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what the slip is, the expression, what it becomes)
MUTANTS = [
    ("taps ordered x-major instead of z-major", "(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1)",
     "(t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1)"),
    ("convolution instead of cross-correlation", "shift(x, dz, dy, dx), w[t]", "shift(x, -dz, -dy, -dx), w[t]"),
    ("bias dropped", "        y = y + b\n", "        y = y\n"),
    ("pooling sums instead of averaging", ".mean(dim=(2, 4, 6))", ".sum(dim=(2, 4, 6))"),
    ("upsampling tiles instead of repeating each voxel",
     "x.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3)",
     "x.repeat(1, 2, 2, 2, 1)"),
    ("ReLU dropped", "q(torch.relu(conv3d(a, q(P[name + \".w\"]), P[name + \".b\"])))",
     "q(conv3d(a, q(P[name + \".w\"]), P[name + \".b\"]))"),
    ("skip concatenated before the upsampled path", "torch.cat([upsample2(a7), a1], dim=-1)",
     "torch.cat([a1, upsample2(a7)], dim=-1)"),
    ("residual connection dropped", "return x + P[\"hb\"][0] + torch.einsum", "return P[\"hb\"][0] + torch.einsum"),
    ("loss summed instead of averaged", "loss = ((y - tt) ** 2).mean()", "loss = ((y - tt) ** 2).sum()"),
    ("Adam without bias correction", "mh = m / (1 - b1 ** step)", "mh = m"),
    ("Adam: eps inside the square root", "(np.sqrt(vh) + eps)", "np.sqrt(vh + eps)"),
    ("encoding: sign of the offset", "- mu) / sigma", "+ mu) / sigma"),
    ("BF16 rounding as FP16", ".to(torch.bfloat16)", ".to(torch.float16)"),
    ("feature 0 offset", "np.log10(np.maximum(m[:, 0], 1e-4)) + 2.0", "np.log10(np.maximum(m[:, 0], 1e-4)) + 1.0"),
    ("feature 1 without the anisotropy", "m[:, 1] * (1.0 - m[:, 2])", "m[:, 1]"),
]


def _run(tmp, old, new):
    src = open(os.path.join(ROOT, "oracle", "denoiser.py")).read()
    if src.count(old) != 1:
        return f"the expression occurs {src.count(old)} times in denoiser.py"
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tmp, "oracle"),
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "workloads"), os.path.join(tmp, "workloads"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(tmp, "tests"))
    for f in ("conftest.py", "test_denoiser_oracle.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(tmp, "tests", f))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp)
    with open(os.path.join(tmp, "oracle", "denoiser.py"), "w") as f:
        f.write(src.replace(old, new))
    env = dict(os.environ, OMP_NUM_THREADS="2")
    env.pop("MCX_ORACLE_LIB", None)
    # (the one pin that compares the library's metric with the oracle's needs the library
    # package, which the scratch copy leaves out)
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_denoiser_oracle.py", "-x", "-q",
                        "-k", "not study_log_rms", "-p", "no:cacheprovider",
                        "--timeout", "120", "--timeout-method", "thread"],
                       env=env, cwd=tmp, capture_output=True, text=True, timeout=900)
    return r.returncode, (r.stdout + r.stderr)[-3000:]


CONTROL = "the unmodified copy"


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = tmp_path_factory.mktemp("dn_mutants")
    cases = [(CONTROL, "def tap_offsets():", "def tap_offsets():")] + MUTANTS
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
    caught = " failed" in out or "Timeout" in out
    assert code == 1 and caught, f"no pin failed (pytest exit {code}):\n{out}"
