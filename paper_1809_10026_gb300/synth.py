"""Seeded synthetic inputs (numpy PCG64).  Holds no arithmetic of the method.

Both the CUDA path and the CPU oracle consume the arrays made here; load
vectors of manufactured solutions are not made here (they need quadrature)
but from the mode parameters returned by ``smooth_modes``.
"""
import numpy as np

SEED0 = 1809100260


def rng(tag):
    """Generator for workload `tag` (an int): PCG64 seeded with 1809100260 + tag."""
    return np.random.Generator(np.random.PCG64(SEED0 + int(tag)))


def uniform(n, tag, batch=1, low=-1.0, high=1.0):
    """i.i.d. U[low, high] values, shape (batch, n) (or (n,) for batch 1)."""
    x = rng(tag).uniform(low, high, size=(batch, n))
    return x[0] if batch == 1 else x


def gaussian(n, tag, sigma=1.0, batch=1):
    """i.i.d. N(0, sigma^2) values, shape (batch, n) (or (n,) for batch 1)."""
    x = rng(tag).normal(0.0, sigma, size=(batch, n))
    return x[0] if batch == 1 else x


def smooth_modes(tag, count=8, dims=3, kmax=4):
    """Parameters of a sum of `count` separable sine modes.

    Returns (amplitudes a_m ~ N(0,1), integer wavenumbers k_{m,j} in [1, kmax])
    with shape (count,) and (count, dims).
    """
    g = rng(tag)
    return g.normal(0.0, 1.0, size=count), g.integers(1, kmax + 1, size=(count, dims))


def grid_field(sizes, tag, count=8, kmax=4, time_last=False):
    """A smooth seeded field sampled on the uniform interior grid of each direction.

    sizes = [n_1, ..., n_D] (direction 1 fastest); point i of a direction of
    size n is (i + 1) / (n + 1).  The field is sum_m a_m prod_j sin(k_mj pi x_j),
    except that with time_last=True the last direction uses sin(k pi t / 2).
    Returned flat in colexicographic order (direction 1 fastest).
    """
    a, k = smooth_modes(tag, count, len(sizes), kmax)
    axes = [(np.arange(n) + 1.0) / (n + 1.0) for n in sizes]
    out = np.zeros(tuple(sizes[::-1]))
    for m in range(count):
        term = np.ones(1)
        for j, x in enumerate(axes):
            scale = 0.5 if (time_last and j == len(sizes) - 1) else 1.0
            term = np.multiply.outer(np.sin(k[m, j] * np.pi * scale * x), term)
        out += a[m] * term.reshape(out.shape)
    return out.reshape(-1)
