"""Crank-Nicolson over one slice in 80-bit long double: a recomputation of
the oracle's arithmetic at higher precision, used by the tests to measure the
rounding of the FP64 oracle and of the GPU path on stress inputs.  Test
infrastructure only."""
import numpy as np


def cn_longdouble(p, n, V):
    """Crank-Nicolson slice in 80-bit long double (calibration of the oracle's rounding only)."""
    ld = np.longdouble
    Nx, M = p.Nx, p.fine_steps
    dt = ld(p.T) / (ld(p.P) * M)
    j = np.arange(Nx, dtype=ld)
    s2, r = ld(p.sigma) ** 2, ld(p.r)
    a, b, c = 0.5 * s2 * j * j - 0.5 * r * j, -s2 * j * j - r, 0.5 * s2 * j * j + 0.5 * r * j
    V = V.astype(ld).copy()
    nn = Nx - 2
    for m in range(M):
        tau = ld(p.T) * (n * M + m + 1) / (p.P * M)
        Bn = ld(p.Smax) - ld(p.K) * np.exp(-r * tau)
        d = 0.5 * dt * a[1:-1] * V[:-2] + (1 + 0.5 * dt * b[1:-1]) * V[1:-1] + 0.5 * dt * c[1:-1] * V[2:]
        d[-1] += 0.5 * dt * c[Nx - 2] * Bn
        lo, di, up = -0.5 * dt * a[1:-1], 1 - 0.5 * dt * b[1:-1], -0.5 * dt * c[1:-1]
        cp, dp = np.zeros(nn, ld), np.zeros(nn, ld)
        cp[0], dp[0] = up[0] / di[0], d[0] / di[0]
        for i in range(1, nn):
            pv = di[i] - lo[i] * cp[i - 1]
            cp[i], dp[i] = up[i] / pv, (d[i] - lo[i] * dp[i - 1]) / pv
        x = np.zeros(nn, ld)
        x[-1] = dp[-1]
        for i in range(nn - 2, -1, -1):
            x[i] = dp[i] - cp[i] * x[i + 1]
        V[1:-1], V[0], V[-1] = x, 0, Bn
    return V
