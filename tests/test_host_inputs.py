"""Seeded synthetic inputs and host-side argument helpers (no GPU).

The input generators hold none of the method's arithmetic; these tests pin
their contracts: the counter-based splitmix64 against its published sequence
and against the oracle's independent implementation (the same bits reach the
GPU and the oracle), the workload recipes (sizes, window rule, ranges),
determinism by seed, and the group CSR layout the C ABI takes.
"""
import math

import numpy as np

from oracle import rng as orng
from paper_0911_4498_gb300 import synth
from paper_0911_4498_gb300._lib import groups_csr

# SplitMix64 (Steele, Lea, Flood 2014) from state 0: its first three outputs as published
# with the reference implementation.
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_published_sequence():
    g = orng.GAMMA
    assert [orng.mix(i * g & orng.MASK) for i in (1, 2, 3)] == SPLITMIX64_SEED0
    z = np.array([i * g & orng.MASK for i in (1, 2, 3)], dtype=np.uint64)
    assert [int(x) for x in synth._mix(z)] == SPLITMIX64_SEED0


def test_generators_and_oracle_draw_the_same_bits():
    for seed, stream, n in [(0, 0, 257), (7, 1, 100), (123456789, 5, 33), (2**63 + 11, 2, 64)]:
        a = 2.0 * synth.uniform(seed, stream, n) - 1.0
        b = np.array(orng.uniform_pm1(seed, stream, n))
        assert np.array_equal(a, b), (seed, stream)


def test_uniform_and_normal_moments():
    n = 200_000
    u = synth.uniform(3, 0, n)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    z = synth.normal(3, 1, n)
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2 / n)
    # offsets continue the same counter stream
    assert np.array_equal(synth.uniform(5, 2, 10, offset=7), synth.uniform(5, 2, 17)[7:])


def test_trend_reading():
    # N = 1000 keeps the literal 0.01 * 1.001^n; other N rescale n so the trend ends at the same value
    n = np.arange(1, 1001, dtype=np.float64)
    assert np.array_equal(synth.trend(n, 1000), 0.01 * 1.001 ** n)
    for N in (5113, 1 << 20, 1 << 22):
        t = synth.trend(np.array([1.0, float(N)]), N)
        assert np.all(np.isfinite(t))
        assert t[-1] == 0.01 * 1.001 ** 1000.0


def test_series_generators_are_seeded():
    for gen, N in [(synth.three_sines, 1000), (synth.many_sines, 4096), (synth.damped_sines, 4096)]:
        a, b, c = gen(N, seed=1), gen(N, seed=1), gen(N, seed=2)
        assert a.shape == (N,) and np.array_equal(a, b) and not np.array_equal(a, c)
    # amplitude bounds of the noise-free parts
    t = synth.three_sines(1000, seed=0, noise=0.0) - synth.trend(np.arange(1, 1001.0), 1000)
    assert np.max(np.abs(t)) <= 3.5
    assert np.max(np.abs(synth.damped_sines(4096, seed=3, noise=0.0))) <= 20.0
    h = sum(1.0 / i for i in range(1, 21))
    m = synth.many_sines(4096, seed=1, noise=0.0) - synth.trend(np.arange(1, 4097.0), 4096)
    assert np.max(np.abs(m)) <= h


def test_batch_workload_recipe():
    series, Ls, ks = synth.batch_workload(count=64, seed=2)
    Ns = np.array([s.size for s in series])
    assert len(series) == 64 and Ls.shape == (64,) and ks.shape == (64,)
    assert Ns.min() >= 500 and Ns.max() <= 20000
    assert np.all(Ls[0::2] == np.floor(Ns[0::2] / 3 + 0.5))   # round(N/3), ties up
    assert np.all(Ls[1::2] == Ns[1::2] // 2)
    assert ks.min() >= 4 and ks.max() <= 32
    s2, L2, k2 = synth.batch_workload(count=64, seed=2)
    assert np.array_equal(L2, Ls) and np.array_equal(k2, ks) and np.array_equal(s2[5], series[5])


def test_serving_arrivals_recipe():
    rate, dur = 2000.0, 1.0
    arr = synth.serving_arrivals(rate, dur, seed=4)
    t = np.array([a[0] for a in arr])
    N = np.array([a[1] for a in arr])
    L = np.array([a[2] for a in arr])
    k = np.array([a[3] for a in arr])
    seeds = [a[4] for a in arr]
    assert np.all(np.diff(t) > 0) and t[0] >= 0 and t[-1] < dur
    assert abs(len(arr) - rate * dur) < 5 * math.sqrt(rate * dur)       # Poisson count
    assert N.min() >= 1000 and N.max() < 1_000_000 and np.all(L == N // 2)
    assert k.min() >= 2 and k.max() <= 64
    assert len(set(seeds)) == len(seeds)
    # log-uniform sizes: half below the geometric midpoint
    frac = np.mean(N < math.sqrt(1e3 * 1e6))
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / len(arr))
    assert synth.serving_arrivals(rate, dur, seed=4) == arr


def test_groups_csr_layout():
    off, idx = groups_csr([[0, 1], [2], [3, 4, 5]])
    assert off.dtype == np.int32 and idx.dtype == np.int32
    assert off.tolist() == [0, 2, 3, 6] and idx.tolist() == [0, 1, 2, 3, 4, 5]
    off, idx = groups_csr([[4], [1, 0]])
    assert off.tolist() == [0, 1, 3] and idx.tolist() == [4, 1, 0]
    off, idx = groups_csr([])
    assert off.tolist() == [0]
