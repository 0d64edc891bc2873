"""Gaussian random fields by circulant embedding.

The paper draws the Darcy permeability and the Helmholtz wavenumber from a
Gaussian random field (GRF) but prints no covariance (App. D.2).  The
workloads here use the squared-exponential covariance
    c(r) = sigma^2 * exp(-r^2 / (2 ell^2))
sampled on the node grid of the unit square (cube), spacing h = 1/(N+1).

Method: sample c on a periodic grid of side Np >= 2 (N+2) nodes, so that
every wrapped distance between two nodes of the cropped (N+2)^d block equals
the true distance; the eigenvalues of the circulant covariance are the FFT
of that sampled row; a white-noise vector filtered by their square roots has
exactly that covariance (negative eigenvalues, from truncation, are clipped
to zero).  The field is then cropped to the (N+2)^d node block.
"""
import functools

import numpy as np


def _next_smooth(n):
    """Smallest integer >= n whose only prime factors are 2, 3, 5 (FFT-friendly)."""
    m = n
    while True:
        k = m
        for p in (2, 3, 5):
            while k % p == 0:
                k //= p
        if k == 1:
            return m
        m += 1


@functools.lru_cache(maxsize=16)
def _sqrt_spectrum(npad, h, ell, sigma, ndim):
    """Square roots of the circulant covariance's eigenvalues (negative ones
    clipped to zero), for one periodic grid; a sequence of fields with the
    same grid and covariance reuses them."""
    idx = np.arange(npad)
    wrapped = np.minimum(idx, npad - idx) * h
    r2 = np.zeros((npad,) * ndim)
    for ax in range(ndim):
        shape = [1] * ndim
        shape[ax] = npad
        r2 = r2 + (wrapped ** 2).reshape(shape)
    row = sigma * sigma * np.exp(-r2 / (2.0 * ell * ell))
    lam = np.real(np.fft.fftn(row))
    root = np.sqrt(np.clip(lam, 0.0, None))
    root.setflags(write=False)
    return root


def grf_field(rng, nodes, ell, sigma=1.0, h=None, ndim=2, pad_factor=2):
    """Draw one GRF sample on a node grid.

    rng     numpy Generator (seeded by the caller)
    nodes   nodes per side, N+2 (interior N plus the two boundary nodes)
    ell     correlation length (unit-square coordinates)
    sigma   pointwise standard deviation
    h       node spacing; default 1/(nodes-1)
    ndim    2 or 3
    Returns an array of shape (nodes,)*ndim, float64.
    """
    if h is None:
        h = 1.0 / (nodes - 1)
    npad = _next_smooth(max(pad_factor * nodes, nodes + int(np.ceil(4.0 * ell / h))))
    root = _sqrt_spectrum(npad, float(h), float(ell), float(sigma), int(ndim))
    noise = rng.standard_normal((npad,) * ndim)
    field = np.real(np.fft.ifftn(root * np.fft.fftn(noise)))
    sl = tuple(slice(0, nodes) for _ in range(ndim))
    return np.ascontiguousarray(field[sl])
