"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module draws random numbers and lays out points; it holds none of the
method's arithmetic.  Random numbers come from the SplitMix64 generator
(Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) used in counter form: draw i of stream `seed` is the (i+1)-th
output of the sequence whose state starts at `seed`.  The C library's
``pinn_create`` initialises weights with the same published generator, so the
two can be compared without sharing code.

Workloads follow the paper's setup (Section 3.3: uniform random collocation
points in the interior, on the S-boundaries and at expiry) at the sizes of the
benchmark configurations.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Output number idx+1 of SplitMix64 started at state `seed` (vectorised, uint64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (np.asarray(idx, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of draws offset..offset+n-1."""
    bits = splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64)) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def xavier_params(widths, seed: int) -> np.ndarray:
    """Flat parameters [W_l (w_out x w_in, row-major), b_l] per layer: Xavier-uniform W, zero b.

    Parameter index q uses draw q of stream `seed`; W = (2u - 1) * sqrt(6 / (fan_in + fan_out)).
    """
    widths = [int(w) for w in widths]
    n = sum(widths[l] * widths[l - 1] + widths[l] for l in range(1, len(widths)))
    out = np.zeros(n)
    off = 0
    for l in range(1, len(widths)):
        wi, wo = widths[l - 1], widths[l]
        a = np.sqrt(6.0 / (wi + wo))
        u = uniform(seed, wo * wi, offset=off)
        out[off:off + wo * wi] = (2.0 * u - 1.0) * a
        off += wo * wi + wo
    return out


def collocation(seed: int, n_interior: int, n_boundary: int, n_expiry: int, Smax: float, T: float):
    """Collocation points of Section 3.3 for a 2-input (S, tau) network.

    Returns X [N, 2] (S, tau) and kind [N] int8: 0 interior (uniform in
    [0, Smax] x [0, T]), 1 on S = 0 and 2 on S = Smax (half each, tau uniform),
    3 at expiry tau = 0 (S uniform).
    """
    nb0 = n_boundary // 2
    nb1 = n_boundary - nb0
    N = n_interior + n_boundary + n_expiry
    u = uniform(seed, 2 * N)
    X = np.zeros((N, 2))
    kind = np.zeros(N, dtype=np.int8)
    i = 0
    X[i:i + n_interior, 0] = u[0:n_interior] * Smax
    X[i:i + n_interior, 1] = u[N:N + n_interior] * T
    i += n_interior
    X[i:i + nb0, 0] = 0.0
    X[i:i + nb0, 1] = u[N + i:N + i + nb0] * T
    kind[i:i + nb0] = 1
    i += nb0
    X[i:i + nb1, 0] = Smax
    X[i:i + nb1, 1] = u[N + i:N + i + nb1] * T
    kind[i:i + nb1] = 2
    i += nb1
    X[i:i + n_expiry, 0] = u[i:i + n_expiry] * Smax
    X[i:i + n_expiry, 1] = 0.0
    kind[i:i + n_expiry] = 3
    return X, kind


def collocation_parametric(seed: int, n_interior: int, n_boundary: int, n_expiry: int, smax_over_K: float,
                           T: float, K_range=(0.5, 2.0), sigma_range=(0.1, 0.5), r_range=(0.0, 0.08)):
    """Collocation points (S, tau, sigma, r, K) for a 5-input network.

    Each point draws its own K, sigma, r uniformly; S lives in [0, smax_over_K * K].
    """
    X2, kind = collocation(seed, n_interior, n_boundary, n_expiry, 1.0, T)
    N = X2.shape[0]
    u = uniform(seed + 1, 3 * N)
    K = K_range[0] + (K_range[1] - K_range[0]) * u[0:N]
    sig = sigma_range[0] + (sigma_range[1] - sigma_range[0]) * u[N:2 * N]
    r = r_range[0] + (r_range[1] - r_range[0]) * u[2 * N:3 * N]
    X = np.zeros((N, 5))
    X[:, 0] = X2[:, 0] * smax_over_K * K
    X[:, 1] = X2[:, 1]
    X[:, 2] = sig
    X[:, 3] = r
    X[:, 4] = K
    return X, kind


def batched_instances(seed: int, n: int, P: int = 64, fine_steps: int = 256, coarse_steps: int = 1,
                      Nx_choices=(256, 512, 1024, 2048, 4096), smax_over_K: float = 4.0):
    """Pricing instances of the batched workload: K~U[0.5,2], sigma~U[0.1,0.5],
    r~U[0,0.08], T~U[0.25,2], Nx uniform over Nx_choices, Smax = smax_over_K * K.

    Returns a list of dicts with keys K, sigma, r, T, Smax, Nx, P, fine_steps, coarse_steps.
    """
    u = uniform(seed, 5 * n)
    out = []
    for i in range(n):
        K = 0.5 + 1.5 * u[5 * i]
        out.append(dict(K=K, sigma=0.1 + 0.4 * u[5 * i + 1], r=0.08 * u[5 * i + 2], T=0.25 + 1.75 * u[5 * i + 3],
                        Smax=smax_over_K * K, Nx=int(Nx_choices[min(int(u[5 * i + 4] * len(Nx_choices)),
                                                                   len(Nx_choices) - 1)]),
                        P=P, fine_steps=fine_steps, coarse_steps=coarse_steps))
    return out


def random_states(seed: int, n_vec: int, Nx: int, scale: float = 1.0) -> np.ndarray:
    """n_vec x Nx test states: a smooth ramp plus uniform noise (endpoints left for the caller to set)."""
    u = uniform(seed, n_vec * Nx).reshape(n_vec, Nx)
    ramp = np.linspace(0.0, 1.0, Nx)[None, :]
    return scale * (ramp + 0.1 * (u - 0.5))
