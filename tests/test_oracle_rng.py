"""Pins of the oracle's random-number building blocks (CPU only).

* Philox4x32-10 against cuRAND's host-side Philox4_32_10 generator (a library
  run on the CPU; its i-th block of four words is Philox(counter=(0,0,i,0),
  key=(seed_lo, seed_hi))).
* Poisson inversion against scipy.stats.poisson's CDF and its moments.
* Box-Muller normal against scipy.stats.norm (Kolmogorov-Smirnov).
* Reduced-precision weight rounding against torch's bfloat16 and numpy's
  float16 conversions.
"""
import ctypes
import ctypes.util
import glob
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _curand():
    cands = []
    for base in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
                 "/usr/local/cuda/targets/x86_64-linux/lib"):
        cands += sorted(glob.glob(os.path.join(base, "libcurand.so*")))
    lib = ctypes.util.find_library("curand")
    if lib:
        cands.append(lib)
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_host_philox(seed: int, n_words: int) -> np.ndarray:
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not found")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n_words)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 1000, 0x123456789ABCDEF0, 2**64 - 1, 0xDEADBEEF00000001])
def test_philox_matches_curand_host_generator(seed):
    blocks = 256
    ref = _curand_host_philox(seed, 4 * blocks).reshape(blocks, 4)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(blocks):
        got = oracle.philox((0, 0, i, 0), key)
        assert np.array_equal(got, ref[i]), (seed, i, got, ref[i])


def test_philox_counter_words_all_matter_and_outputs_uniform():
    key = (0x9E3779B9, 0x12345)
    seen = set()
    words = []
    for pos in range(4):
        for v in range(1, 2049):
            ctr = [0, 0, 0, 0]
            ctr[pos] = v
            out = oracle.philox(ctr, key)
            seen.add(tuple(out))
            words.append(out)
    assert len(seen) == 4 * 2048  # no collisions across counter words
    w = np.concatenate(words)
    # byte histogram chi-square, 255 dof
    hist = np.bincount((w & 0xFF).astype(np.int64), minlength=256)
    exp = len(w) / 256
    chi2 = float(((hist - exp) ** 2 / exp).sum())
    assert chi2 < 400, chi2
    # top bit balanced
    assert abs(float((w >> 31).mean()) - 0.5) < 0.02


@pytest.mark.parametrize("lam", [0.8, 1.28, 2.0, 2.32, 7.5, 40.0])
def test_poisson_inversion_against_scipy_cdf(lam):
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(7)
    xs = rng.integers(0, 2**32, size=4000, dtype=np.uint64)
    xs = np.concatenate([xs, np.array([0, 1, 2**32 - 1, 2**31], dtype=np.uint64)])
    for x in xs:
        k = oracle.poisson_inversion(lam, int(x))
        u = float(x) * 2.0**-32
        hi = stats.poisson.cdf(k, lam)
        lo = stats.poisson.cdf(k - 1, lam) if k > 0 else 0.0
        # inversion: F(k-1) <= u < F(k), up to rounding of the CDF evaluation
        assert lo - 1e-12 <= u < hi + 1e-12, (lam, x, k, lo, u, hi)


@pytest.mark.parametrize("lam", [0.8, 2.32])
def test_poisson_moments(lam):
    rng = np.random.default_rng(11)
    n = 200_000
    xs = rng.integers(0, 2**32, size=n, dtype=np.uint64)
    ks = np.array([oracle.poisson_inversion(lam, int(x)) for x in xs], dtype=np.float64)
    mean, var = ks.mean(), ks.var()
    assert abs(mean - lam) < 5 * np.sqrt(lam / n)
    # var of the sample variance of a Poisson ~ (lam + 2 lam^2) / n
    assert abs(var - lam) < 5 * np.sqrt((lam + 2 * lam * lam) / n)


def test_box_muller_normal_distribution():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(3)
    words = rng.integers(0, 2**32, size=(40_000, 4), dtype=np.uint64)
    z = np.array([oracle.normal_from_words(w) for w in words])
    ks = stats.kstest(z, "norm")
    assert ks.pvalue > 1e-3, ks
    # one explicit case: u1 = 1 (all-ones hi/lo give the top value) -> z = 0
    assert oracle.normal_from_words([0xFFFFFFFF, 0xFFFFFFFF, 0, 0]) == 0.0


def test_weight_rounding_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    w = np.concatenate([rng.normal(87.8, 8.78, 5000), rng.normal(-351.2, 35.1, 5000),
                        rng.uniform(0.0, 1.0, 5000), rng.normal(0.05, 0.01, 2000)]).astype(np.float32)
    ref = torch.from_numpy(w).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.round_weight(float(x), 1) for x in w], dtype=np.float32)
    assert np.array_equal(got, ref)


def test_weight_rounding_fp16_matches_numpy():
    rng = np.random.default_rng(6)
    w = np.concatenate([rng.normal(87.8, 8.78, 5000), rng.normal(-351.2, 35.1, 5000),
                        rng.uniform(-1e-6, 1e-6, 3000), rng.uniform(-7e4, 7e4, 3000),
                        rng.normal(0.05, 0.01, 2000)]).astype(np.float32)
    ref = w.astype(np.float16).astype(np.float32)
    got = np.array([oracle.round_weight(float(x), 2) for x in w], dtype=np.float32)
    assert np.array_equal(got, ref)


def test_weight_rounding_fp32_is_identity():
    for x in (87.8, -351.2, 0.05, 1e-30):
        x32 = float(np.float32(x))
        assert oracle.round_weight(x32, 0) == x32
