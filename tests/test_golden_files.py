"""The stored expected values (tests/golden/sigma_*.txt, written from the oracle) against facts
that hold whatever computed them: singular values positive and non-increasing, their squares
summing to at most ||X||_F^2 = sum_n cnt_n f_n^2 (sections 2.1-2.2: X's Frobenius norm counts
each f_n once per antidiagonal entry), converged residuals within the recorded tolerance, and
sampled entries of the unit singular vectors within [-1, 1]."""
import glob
import os
import re

import numpy as np
import pytest

from conftest import GOLDEN, load_golden
from paper_0911_4498_gb300 import synth

# generator and seed of each stored series (as written in the file headers)
SERIES = {"many_sines": 1, "three_sines_N5113": 7, "three_sines_N86867": 8, "damped_sines": 3}


def _series(name, N):
    if name.startswith("sigma_many_sines"):
        return synth.many_sines(N, seed=SERIES["many_sines"])
    if name.startswith("sigma_damped_sines"):
        return synth.damped_sines(N, seed=SERIES["damped_sines"])
    if name.startswith("sigma_three_sines"):
        return synth.three_sines(N, seed=SERIES[f"three_sines_N{N}"])
    raise KeyError(name)


FILES = sorted(os.path.basename(p) for p in glob.glob(os.path.join(GOLDEN, "sigma_*.txt")))


def test_golden_files_present():
    assert "sigma_many_sines_N1048576_L524288_k50.txt" in FILES


@pytest.mark.parametrize("name", FILES)
def test_golden_sigma_consistent(name):
    g = load_golden(name)
    N, L, k = int(g["N"][0]), int(g["L"][0]), int(g["k"][0])
    m = re.search(r"_N(\d+)_L(\d+)_k(\d+)\.txt$", name)
    assert (N, L, k) == tuple(int(x) for x in m.groups())
    K = N - L + 1
    s = g["sigma"]
    assert s.shape == (k,) and np.all(s > 0) and np.all(np.diff(s) <= 0)
    f = _series(name, N)
    n = np.arange(N)
    cnt = np.minimum(np.minimum(n + 1, min(L, K)), np.minimum(max(L, K), N - n))
    frob2 = float(np.sum(cnt * f * f))
    assert float(np.sum(s * s)) <= frob2 * (1 + 1e-12)
    header = open(os.path.join(GOLDEN, name)).read()
    tol = float(re.search(r"tol ([0-9.e+-]+)", header).group(1))
    assert np.all(g["resid"] <= tol * s[0] * (1 + 1e-9))
    for i in range(min(k, 8)):
        u, v = g[f"u{i}"], g[f"v{i}"]
        assert np.all(np.abs(u) <= 1.0) and np.all(np.abs(v) <= 1.0)
