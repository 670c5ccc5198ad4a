"""The learned index's locator fit, on the CPU (csrc/fw_lindex_fit.h via tests/lindex_fit_check.cpp).

For interval layouts like the rule sets' (uniform, bunched, every key a start), key widths of
the address (32), port (16) and protocol (8) fields, and segment counts from 1 to 65,536, every
tested key's true interval lies within the stored error of the prediction: the device lookup's
verified window then never falls back to a full search. The stored bound is also tight enough
to matter: it is what the kernel searches.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1312_4188_gb300", "csrc")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = tmp_path_factory.mktemp("fit") / "lindex_fit_check"
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror", "-I", CSRC,
                    os.path.join(ROOT, "tests", "lindex_fit_check.cpp"), "-o", str(out)], check=True)
    return str(out)


CASES = [  # (bits, nseg, intervals, shape)
    (32, 4096, 200_000, 0), (32, 4096, 2_000, 0), (32, 1, 5_000, 0), (32, 65536, 100_000, 1),
    (32, 16, 50_000, 1), (16, 4096, 40_000, 0), (16, 65536, 60_000, 1), (16, 1, 1_000, 0),
    (16, 4096, 0, 2), (8, 256, 0, 2), (8, 4, 20, 0), (32, 4096, 0, 0),
]


@pytest.mark.parametrize("bits,nseg,intervals,shape", CASES)
@pytest.mark.parametrize("seed", [1, 2])
def test_window_holds_the_interval(exe, bits, nseg, intervals, shape, seed):
    r = subprocess.run([exe, str(seed), str(bits), str(nseg), str(intervals), str(shape)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    checked, bad, max_err, seen, m = (int(x) for x in r.stdout.split())
    assert bad == 0 and checked > 200_000 and seen <= max_err
    if shape == 2:
        assert m == 1 << bits and max_err == 0  # one interval per key: the chord is exact
