"""Seeded sequences of PDE problem parameters.

Each generator returns the raw parameters of N problems of one PDE family:
coefficient fields on the node grid, scalar parameters and right-hand-side
fields.  They stand in for the paper's generated datasets (App. D.2), which
are not available; the shapes and distributions are those of the paper's
workloads (Darcy with a = exp(GRF), convection-diffusion with random nu and
beta, Helmholtz with a GRF wavenumber, Poisson with Chebyshev data), plus
batched chains of mixed grid sides and a Poisson arrival stream.
"""
import numpy as np

from .grf import grf_field


def darcy2d_sequence(nside, nsys, ell, sigma=1.0, seed=0):
    """N Darcy problems -div(a grad u) = 1 on an nside x nside interior grid.

    Returns log a at the (nside+2)^2 nodes of every problem, shape
    (nsys, nside+2, nside+2), float64.  The right-hand side is f = 1.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((nsys, nside + 2, nside + 2))
    for s in range(nsys):
        out[s] = grf_field(rng, nside + 2, ell, sigma, ndim=2)
    return out


def darcy2d_circle_sequence(nside, nsys, ell, sigma=1.0, seed=0):
    """N Darcy problems whose fields lie on a closed curve of GRF samples.

    log a(t) = cos(t) G1 + sin(t) G2 for two independent GRFs G1, G2 and
    t_i uniform on [0, 2 pi) (seeded): every field is itself a GRF sample
    with the same covariance, but neighbours along the curve are close, the
    setting in which the sort's nearest neighbours share recycle spaces.
    Returns (log a [nsys, nside+2, nside+2], t [nsys]).
    """
    rng = np.random.default_rng(seed)
    g1 = grf_field(rng, nside + 2, ell, sigma, ndim=2)
    g2 = grf_field(rng, nside + 2, ell, sigma, ndim=2)
    t = rng.uniform(0.0, 2.0 * np.pi, size=nsys)
    out = np.cos(t)[:, None, None] * g1[None] + np.sin(t)[:, None, None] * g2[None]
    return out, t


def darcy3d_sequence(nside, nsys, ell, sigma=1.0, seed=0, pad_factor=2):
    """N 3D Darcy problems on an nside^3 interior grid: log a at (nside+2)^3 nodes."""
    rng = np.random.default_rng(seed)
    out = np.empty((nsys, nside + 2, nside + 2, nside + 2))
    for s in range(nsys):
        out[s] = grf_field(rng, nside + 2, ell, sigma, ndim=3, pad_factor=pad_factor)
    return out


def convdiff2d_sequence(nside, nsys, seed=0, nu_range=(0.01, 0.1), beta_max=50.0,
                        f_ell=0.1):
    """N convection-diffusion problems -nu lap u + beta . grad u = f.

    nu ~ U[nu_range], beta = U[0, beta_max] * (cos phi, sin phi) with
    phi ~ U[0, 2 pi), f = GRF(ell = f_ell, sigma = 1) at the interior nodes.
    Returns (nu[nsys], beta[nsys, 2], f[nsys, nside*nside]).
    """
    rng = np.random.default_rng(seed)
    nu = rng.uniform(nu_range[0], nu_range[1], nsys)
    mag = rng.uniform(0.0, beta_max, nsys)
    phi = rng.uniform(0.0, 2.0 * np.pi, nsys)
    beta = np.stack([mag * np.cos(phi), mag * np.sin(phi)], axis=1)
    f = np.empty((nsys, nside * nside))
    for s in range(nsys):
        g = grf_field(rng, nside + 2, f_ell, 1.0, ndim=2)
        f[s] = g[1:-1, 1:-1].reshape(-1)
    return nu, beta, f


def convdiff_keys(nu, beta, nu_range=(0.01, 0.1), beta_max=50.0):
    """Sort / routing keys of convection-diffusion problems: (nu, beta_x,
    beta_y) z-scored by the distributions convdiff2d_sequence draws them from
    (nu uniform on nu_range; beta = U[0, beta_max] (cos phi, sin phi), whose
    components have mean 0 and standard deviation beta_max / sqrt(6)), so
    that no parameter dominates the distance by its units.  Returns [nsys, 3].
    """
    lo, hi = nu_range
    nu_mean, nu_sd = 0.5 * (lo + hi), (hi - lo) / np.sqrt(12.0)
    b_sd = beta_max / np.sqrt(6.0)
    beta = np.asarray(beta, dtype=np.float64)
    return np.stack([(np.asarray(nu, dtype=np.float64) - nu_mean) / nu_sd, beta[:, 0] / b_sd, beta[:, 1] / b_sd],
                    axis=1)


def helmholtz2d_sequence(nside, nsys, kbar, ell, sigma=1.0, spread=0.2, seed=0):
    """N Helmholtz problems -lap u - k^2 u = 1 on an nside x nside interior grid.

    The wavenumber is k = kbar * exp(spread * GRF(ell, sigma)) at the interior
    nodes (positive, log-normal around kbar).  Returns k, shape
    (nsys, nside, nside), float64; it is also the sort key.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((nsys, nside, nside))
    for s in range(nsys):
        out[s] = kbar * np.exp(spread * grf_field(rng, nside, ell, sigma, ndim=2))
    return out


def chebyshev_poisson_sequence(nside, nsys, ncoef=8, decay=0.6, seed=0):
    """N Poisson problems lap u = f with Dirichlet data from truncated Chebyshev series.

    The four boundary functions are 1D series sum_j c_j T_j(2t - 1) and f is
    the 2D series sum_ij a_ij T_i(2x - 1) T_j(2y - 1), j, i < ncoef, with
    independent normal coefficients of standard deviation decay^j
    (decay^(i+j) for f).  Returns (keys, f, g): keys (nsys, 4 ncoef + ncoef^2)
    are the coefficients (the sort keys), f (nsys, nside, nside) at the
    interior nodes, g (nsys, 4, nside) = u on x = 0, x = 1, y = 0, y = 1 at
    the interior node coordinates of that line.
    """
    from numpy.polynomial import chebyshev as C

    rng = np.random.default_rng(seed)
    t = np.arange(1, nside + 1) / (nside + 1.0)
    s = 2.0 * t - 1.0
    w1 = decay ** np.arange(ncoef)
    w2 = np.outer(w1, w1)
    keys = np.empty((nsys, 4 * ncoef + ncoef * ncoef))
    f = np.empty((nsys, nside, nside))
    g = np.empty((nsys, 4, nside))
    for q in range(nsys):
        cb = rng.standard_normal((4, ncoef)) * w1
        a = rng.standard_normal((ncoef, ncoef)) * w2
        keys[q] = np.concatenate([cb.ravel(), a.ravel()])
        for e in range(4):
            g[q, e] = C.chebval(s, cb[e])
        f[q] = C.chebgrid2d(s, s, a)
    return keys, f, g


def batched_chains(nchains, chain_len, sides=(64, 128, 192, 256, 384),
                   ell_range=(0.05, 0.3), sigma=1.0, seed=0):
    """Independent Darcy chains of mixed grid sides.

    Every chain draws its side uniformly from `sides` and its correlation
    length from U[ell_range]; each of its systems is a fresh GRF sample.
    Returns a list of (side, ell, loga[chain_len, side+2, side+2]).
    """
    rng = np.random.default_rng(seed)
    chains = []
    for _ in range(nchains):
        side = int(rng.choice(sides))
        ell = float(rng.uniform(*ell_range))
        sub = np.empty((chain_len, side + 2, side + 2))
        for s in range(chain_len):
            sub[s] = grf_field(rng, side + 2, ell, sigma, ndim=2)
        chains.append((side, ell, sub))
    return chains


def serving_stream(nreq, rate, seed=0, sides2d=(128, 256, 512, 1024),
                   sides3d=(64, 96, 128), frac3d=0.5, ell=0.1, sigma=1.0,
                   draw_fields=True):
    """A Poisson arrival stream of Darcy requests.

    Inter-arrival gaps are exponential with mean 1/rate seconds.  Each
    request is 2D (side from sides2d) or 3D (side from sides3d) with
    probability frac3d, and carries log a = GRF(ell, sigma) on its node grid.
    Returns a list of dicts {t, ndim, side, loga}.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for _ in range(nreq):
        t += rng.exponential(1.0 / rate)
        if rng.uniform() < frac3d:
            ndim, side = 3, int(rng.choice(sides3d))
        else:
            ndim, side = 2, int(rng.choice(sides2d))
        loga = grf_field(rng, side + 2, ell, sigma, ndim=ndim, pad_factor=1) if draw_fields else None
        reqs.append({"t": t, "ndim": ndim, "side": side, "loga": loga})
    return reqs


# Named workloads: grid side, number of systems, GRF length scale, solver
# settings.  Seeds 1..7.
CONFIGS = {
    "darcy32_fp64": dict(kind="darcy2d", nside=32, nsys=20, ell=0.2, sigma=1.0, seed=1,
                          m=30, k=10, precond="none", precision="fp64", tol=1e-8),
    "darcy256_mixed": dict(kind="darcy2d", nside=256, nsys=200, ell=0.1, sigma=1.0, seed=2,
                            m=40, k=20, precond="jacobi", precision="mixed", tol=1e-8),
    "convdiff512_ilu": dict(kind="convdiff2d", nside=512, nsys=500, seed=3,
                             m=40, k=20, precond="ilu0", precision="mixed", tol=1e-8),
    "batched64x50": dict(kind="batched", nchains=64, chain_len=50, seed=4,
                          m=40, k=20, precond="jacobi", precision="mixed", tol=1e-8),
    "serving": dict(kind="serving", nreq=2000, rate=200.0, seed=5,
                     m=40, k=20, precond="jacobi", precision="mixed", tol=1e-8),
    # Poisson with Chebyshev boundary data and forcing; sort keys = the coefficients
    "poisson_cheb256": dict(kind="poisson2d", nside=256, nsys=200, ncoef=8, decay=0.6, seed=7,
                             m=40, k=20, precond="jacobi", precision="mixed", tol=1e-8),
    # the paper's Helmholtz set has 10,000 unknowns (100^2)
    "helmholtz100": dict(kind="helmholtz2d", nside=100, nsys=200, kbar=10.0, ell=0.1, sigma=1.0,
                          spread=0.2, seed=6, m=40, k=20, precond="jacobi", precision="mixed", tol=1e-8),
}
