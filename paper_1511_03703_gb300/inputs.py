"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds no arithmetic of the method itself: it only draws the
random variables xi of the Karhunen-Loeve expansion (Sect. 4: y_i iid
uniform on [-1, 1]) and the seeded test vectors.  Both the CUDA path and the
CPU oracle receive the arrays produced here as plain inputs.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), written from its published definition as a
counter-based map: element t >= 1 of the stream seeded with `seed` is the
SplitMix64 finaliser applied to seed + t * 0x9E3779B97F4A7C15 (mod 2^64).

Sample j, KL variable k (k < 64) uses element t = 64*j + k + 1, converted to
a double u = (z >> 11) * 2^-53 in [0, 1) and xi = 2u - 1 in [-1, 1).
"""
import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB
MAX_KL_TERMS = 64


def splitmix64(seed, t):
    """Element(s) t (uint64 array, t >= 1) of the SplitMix64 stream `seed`."""
    t = np.asarray(t, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed % (1 << 64)) + t * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_MIX2)
        return z ^ (z >> np.uint64(31))


def uniform01(seed, t):
    """Doubles in [0, 1) with 53 random bits from stream elements t."""
    z = splitmix64(seed, t)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def kl_samples(seed, first_sample, num_samples, M):
    """KL random variables xi[j, k] in [-1, 1), shape (num_samples, M).

    Sample indices first_sample .. first_sample+num_samples-1 of stream
    `seed`; variable k of sample j is stream element 64*j + k + 1.
    """
    if not (0 <= M <= MAX_KL_TERMS):
        raise ValueError(f"M={M} outside [0, {MAX_KL_TERMS}]")
    j = np.arange(first_sample, first_sample + num_samples, dtype=np.uint64)
    k = np.arange(M, dtype=np.uint64)
    t = j[:, None] * np.uint64(MAX_KL_TERMS) + k[None, :] + np.uint64(1)
    return 2.0 * uniform01(seed, t) - 1.0


def ensemble_layout(xi_samples):
    """(s, M) per-sample rows -> ensemble-contiguous xi[k*s + e] (Eq. 3 ordering)."""
    xi_samples = np.ascontiguousarray(xi_samples, dtype=np.float64)
    return np.ascontiguousarray(xi_samples.T).reshape(-1)


def random_vector(seed, n, lo=-1.0, hi=1.0, stream_offset=0):
    """n seeded doubles uniform in [lo, hi); used for SpMV / dot test vectors."""
    t = np.arange(1, n + 1, dtype=np.uint64) + np.uint64(stream_offset)
    return lo + (hi - lo) * uniform01(seed, t)


# seeds used across tests and the benchmark: workload c uses seed 1000 + c
SEED_SMALL = 1001        # 8^3 mesh, M = 3, s = 4
SEED_SCALE = 1002        # 64^3 mesh, M = 10, 1024 samples
SEED_MIXED = 1003        # 128^3 mesh, M = 10, 256 samples
SEED_BATCHED = 1004      # 16^3 .. 64^3 meshes, 2048 samples
SEED_GUESS_TRAIN = 2005  # learned initial guess: training samples
SEED_GUESS_TEST = 3005   # learned initial guess: fresh test samples

# stream offsets of the learned-guess draws: far beyond every KL element
# 64*j + k + 1 used by any workload, so the streams never overlap
MLP_INIT_OFFSET = 1 << 40
POD_TEST_OFFSET = 1 << 41


def mlp_init_draws(seed, count):
    """count uniform draws in [-1, 1) for the MLP's initial parameters,
    rounded to float32 (the network's precision); both the CUDA path and the
    oracle scale the same draws."""
    return random_vector(seed, count, -1.0, 1.0, MLP_INIT_OFFSET).astype(np.float32)


def pod_test_matrix(seed, m, l):
    """m x l uniform draws in [-1, 1): the random test matrix of the POD range finder."""
    return random_vector(seed, m * l, -1.0, 1.0, POD_TEST_OFFSET).reshape(m, l)
