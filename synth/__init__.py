"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module holds no arithmetic of the method: it only draws nodes and data
with the shapes and distributions of the paper's experiments (Sec. VI: nodes
are a regular grid of spacing 1/P shifted by independent uniform jitters,
amplitudes are iid zero-mean unit-variance complex Gaussians) and of the
workloads derived from them (ill-conditioned clusters, log-uniform instance
sizes).  Everything is float64 / complex128 on the host (numpy PCG64).

Node convention: x_k = 2*pi*(k + u_k)/N radians; the library wraps x into
[0, 2*pi).  Draw order per generator is fixed (nodes first, then data) so a
(seed, N) pair always reproduces the same problem.
"""
import numpy as np

__all__ = [
    "rng", "jittered_nodes", "clustered_nodes", "cn01", "equispaced_nodes",
    "log_uniform_sizes", "batched_instances",
]


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def equispaced_nodes(N):
    """x_k = 2*pi*k/N (the regular grid on which the NUFFTs reduce to DFTs)."""
    return 2.0 * np.pi * np.arange(N, dtype=np.float64) / N


def jittered_nodes(N, umax, seed=None, generator=None):
    """x_k = 2*pi*(k + u_k)/N with u_k ~ U(-umax, umax) iid (Sec. VI setup,
    shifted to a symmetric interval; a common shift only rotates the
    coefficients)."""
    g = generator if generator is not None else rng(seed)
    u = g.uniform(-umax, umax, size=N)
    return 2.0 * np.pi * (np.arange(N, dtype=np.float64) + u) / N


def clustered_nodes(N, umax, frac, dmin, dmax, seed=None, generator=None):
    """Jittered nodes plus ill-conditioned clusters.

    A fraction `frac` of the even indices i (drawn without replacement, so no
    chains form) gets its node moved to within d_i grid spacings below node
    i+1: t_i = t_{i+1} - d_i/N with d_i ~ U(dmin, dmax).  Returns radians."""
    g = generator if generator is not None else rng(seed)
    u = g.uniform(-umax, umax, size=N)
    t = (np.arange(N, dtype=np.float64) + u) / N
    n_move = int(round(frac * N))
    evens = np.arange(0, N - 1, 2)
    idx = np.sort(g.choice(evens, size=min(n_move, evens.size), replace=False))
    d = g.uniform(dmin, dmax, size=idx.size)
    t[idx] = t[idx + 1] - d / N
    return 2.0 * np.pi * t


def cn01(shape, seed=None, generator=None):
    """iid circular complex Gaussian CN(0,1): Re, Im ~ N(0, 1/2)."""
    g = generator if generator is not None else rng(seed)
    re = g.normal(0.0, np.sqrt(0.5), size=shape)
    im = g.normal(0.0, np.sqrt(0.5), size=shape)
    return re + 1j * im


def log_uniform_sizes(count, nmin, nmax, seed=None, generator=None):
    """N_i = round(exp(U(ln nmin, ln nmax))) for a batch of uneven instances."""
    g = generator if generator is not None else rng(seed)
    return np.rint(np.exp(g.uniform(np.log(nmin), np.log(nmax), size=count))).astype(np.int64)


def batched_instances(count, nmin, nmax, umax, seed):
    """Uneven batch: per instance its own size and jittered nodes, plus CN(0,1)
    data.  Returns (sizes, list of node arrays, list of data arrays)."""
    g = rng(seed)
    sizes = log_uniform_sizes(count, nmin, nmax, generator=g)
    xs = [jittered_nodes(int(n), umax, generator=g) for n in sizes]
    data = [cn01(int(n), generator=g) for n in sizes]
    return sizes, xs, data
