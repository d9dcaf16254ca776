"""Write stored expected values for the full-size parity tests.

Calls only the CPU oracle (``oracle/``) on the seeded series of
``paper_0911_4498_gb300.synth``; nothing here touches the CUDA library.
Each output file records the generator, sizes, oracle settings and the
oracle's converged residuals beside the singular values, plus a few sampled
entries of the leading singular vectors (sign rule applied) for
element-wise checks.

  python tests/golden/make_golden.py many_sines_1M     # N = 2^20, L = 2^19, k = 50
  python tests/golden/make_golden.py realdata_shapes   # N = 5113 / 86867 stand-ins
  python tests/golden/make_golden.py damped_4M         # N = 2^22, L = 2^21, k = 100 (precision stress)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ssa  # noqa: E402
from paper_0911_4498_gb300 import synth  # noqa: E402

SAMPLE_ROWS = 16


def _write(name, header, f, L, k, out, elapsed, fft="own radix-2 FFT"):
    N = f.size
    K = N - L + 1
    rows_u = np.unique(np.linspace(0, L - 1, SAMPLE_ROWS).astype(np.int64))
    rows_v = np.unique(np.linspace(0, K - 1, SAMPLE_ROWS).astype(np.int64))
    path = os.path.join(HERE, name)
    with open(path, "w") as fh:
        fh.write("# Expected values written by tests/golden/make_golden.py from the CPU oracle\n")
        fh.write(f"# (Lanczos with FRO by MGS twice, {fft} at M = next pow2 >= 2N).\n")
        for line in header:
            fh.write("# " + line + "\n")
        fh.write(f"# oracle wall time {elapsed:.1f} s, restarts {out.get('restarts')}, matvecs {out.get('matvecs')}\n")
        fh.write(f"N: {N}\nL: {L}\nk: {k}\n")
        fh.write("sigma: " + " ".join(repr(float(x)) for x in out["sigma"]) + "\n")
        fh.write("resid: " + " ".join(repr(float(x)) for x in out["resid"]) + "\n")
        fh.write("rows_u: " + " ".join(str(int(x)) for x in rows_u) + "\n")
        fh.write("rows_v: " + " ".join(str(int(x)) for x in rows_v) + "\n")
        for i in range(min(k, 8)):
            fh.write(f"u{i}: " + " ".join(repr(float(x)) for x in out["U"][rows_u, i]) + "\n")
            fh.write(f"v{i}: " + " ".join(repr(float(x)) for x in out["V"][rows_v, i]) + "\n")
    print("wrote", path)


def many_sines_1M():
    N, L, k = 1 << 20, 1 << 19, 50
    f = synth.many_sines(N, seed=1)
    t = time.time()
    out = ssa.decompose(f, L, k, method="lanczos", tol=1e-14, seed=0)
    _write("sigma_many_sines_N1048576_L524288_k50.txt",
           ["series: synth.many_sines(N=2^20, seed=1): 20 sinusoids (periods log-uniform [5,5000],",
            "amplitudes 1/i) + trend 0.01*1.001^(1000n/N) + N(0, 0.1^2)", "tol 1e-14, seed 0"],
           f, L, k, out, time.time() - t)


def realdata_shapes():
    for N, L, k, seed in [(5113, 2556, 100, 7), (86867, 43433, 50, 8)]:
        f = synth.three_sines(N, seed=seed)
        t = time.time()
        out = ssa.decompose(f, L, k, method="lanczos", tol=1e-14, seed=0)
        _write(f"sigma_three_sines_N{N}_L{L}_k{k}.txt",
               [f"series: synth.three_sines(N={N}, seed={seed}) (shape of the section 7 real-data runs)",
                "tol 1e-14, seed 0"], f, L, k, out, time.time() - t)


def damped_4M():
    N, L, k = 1 << 22, 1 << 21, 100
    f = synth.damped_sines(N, seed=3)
    t = time.time()
    # the oracle's own radix-2 FFT takes seconds per transform at M = 2^23; numpy's FFT computes the
    # same DFT (section 4.1) and is pinned to it by tests/test_oracle_lanczos.py
    out = ssa.decompose(f, L, k, method="lanczos", tol=1e-14, seed=0, fft="library")
    _write("sigma_damped_sines_N4194304_L2097152_k100.txt",
           ["series: synth.damped_sines(N=2^22, seed=3): 20 damped cosines (rank 40, damping in",
            "[0.9999, 1], periods log-uniform [5,5000], amplitude 1) + N(0, 1e-6^2)",
            "tol 1e-14, seed 0"],
           f, L, k, out, time.time() - t, fft="numpy's FFT (fft='library')")


if __name__ == "__main__":
    for name in sys.argv[1:]:
        globals()[name]()
