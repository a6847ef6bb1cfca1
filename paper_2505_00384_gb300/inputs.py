"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds random-number generation and input recipes only; none of
the discretisation's arithmetic lives here.  Both the CUDA path and the CPU
oracle receive the arrays it produces as plain inputs.

Generator: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) for uniform 64-bit words, Box-Muller for
normal deviates.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

DEFAULT_SEED = 20250501


def splitmix64(seed, n):
    """n consecutive outputs of splitmix64 started from ``seed``."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + (np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN)
        z = state
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, n):
    """Uniform deviates in the open interval (0, 1)."""
    z = splitmix64(seed, n)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed, n):
    """Standard normal deviates by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:n]


def gaussian_bump_rhs(coords, center, sigma=200.0, noise_std=1e-3, seed=DEFAULT_SEED):
    """Right-hand side of the 4x4x4 affine-box solve: a Gaussian bump at the
    DoF nodes plus independent N(0, noise_std^2) noise per DoF.

    coords: array (3, N) of physical node coordinates (supplied by the caller).
    """
    X = np.asarray(coords, dtype=np.float64)
    c = np.asarray(center, dtype=np.float64).reshape(3, 1)
    r2 = ((X - c) ** 2).sum(axis=0)
    return np.exp(-r2 / (2.0 * sigma * sigma)) + noise_std * normal(seed, X.shape[1])


def perturbed_profile(z, base, scale_height, rel_noise, seed):
    """Positive synthetic coefficient field: base * exp(-z / scale_height)
    times (1 + rel_noise * N(0,1)) per DoF (rel_noise small)."""
    z = np.asarray(z, dtype=np.float64)
    return base * np.exp(-z / scale_height) * (1.0 + rel_noise * normal(seed, z.size))


def random_field(n, seed, scale=1.0):
    """Plain N(0, scale^2) vector of length n."""
    return scale * normal(seed, n)
