"""Seeded macroscopic initial fields (n, T, u) on an nz x ny x nx lattice (x fastest).

Every function returns float64 arrays n, T of shape (nz, ny, nx) and u of shape (3, nz, ny, nx)
(components x, y, z).  None of them evaluates the lattice Boltzmann method."""
import numpy as np


def riemann_tube(nz, T_left=1.0, T_right=0.5, ny=1, nx=1):
    """Shock tube along z (Sec. III): T_left for z < nz/2, T_right beyond, n = T^3 (so that the
    pressure n T is 1.0 | 0.0625), fluid at rest."""
    T = np.where(np.arange(nz) < nz // 2, T_left, T_right)[:, None, None] * np.ones((nz, ny, nx))
    return T ** 3, T, np.zeros((3, nz, ny, nx))


def mirrored_riemann_tube(nz=1600, T_ref=1.0, ny=1, nx=1):
    """The shock tube of Sec. III as the paper runs it: a periodic tube of nz cells holding the
    tube and its mirror image, hot (T_ref) for z < nz/4 and z >= 3nz/4, cold (T_ref / 2) between,
    n = T^3, fluid at rest.  The two discontinuities sit at nz/4 and 3nz/4; the state is symmetric
    under z -> nz - 1 - z."""
    z = np.arange(nz)
    hot = (z < nz // 4) | (z >= nz - nz // 4)
    T = np.where(hot, T_ref, 0.5 * T_ref)[:, None, None] * np.ones((nz, ny, nx))
    return T ** 3, T, np.zeros((3, nz, ny, nx))


def shear_wave(n_cells, amp=0.05, axis_len=None, ny=None, nz=None):
    """u_y = amp sin(2 pi x / nx) on uniform n = 1, T = 1 (transverse shear wave)."""
    nx = n_cells
    ny = n_cells if ny is None else ny
    nz = n_cells if nz is None else nz
    x = np.arange(nx)
    u = np.zeros((3, nz, ny, nx))
    u[1] = amp * np.sin(2 * np.pi * x / nx)[None, None, :]
    return np.ones((nz, ny, nx)), np.ones((nz, ny, nx)), u


def _band_field(shape, kmax, rng):
    """Real part of a sum of Fourier modes 0 < |k| <= kmax (integer k) with complex Gaussian
    amplitudes, evaluated on the lattice."""
    nz, ny, nx = shape
    spec = np.zeros(shape, dtype=np.complex128)
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    K2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    mask = (K2 > 0) & (K2 <= kmax * kmax)
    spec[mask] = rng.standard_normal(mask.sum()) + 1j * rng.standard_normal(mask.sum())
    return np.real(np.fft.ifftn(spec)) * spec.size


def smooth_random_fields(shape, seed=1, vmax=0.6, sigma_lnT=0.2, kmax=4, density="cube"):
    """Random-field throughput case: velocity from Fourier modes |k| <= kmax (seed), rescaled to
    max |v| = vmax; T = exp(sigma g - sigma^2/2) with g a unit-variance field of the same band
    (seed + 1), so mean T ~ 1; density "cube": n = T^3 (pressure n T = T^4), "uniform": n = 1
    (pressure T)."""
    rng = np.random.default_rng(seed)
    u = np.stack([_band_field(shape, kmax, rng) for _ in range(3)])
    vnorm = np.sqrt((u * u).sum(axis=0)).max()
    u *= vmax / vnorm if vnorm > 0 else 0.0
    g = _band_field(shape, kmax, np.random.default_rng(seed + 1))
    sd = g.std()
    g = g / sd if sd > 0 else g
    T = np.exp(sigma_lnT * g - 0.5 * sigma_lnT ** 2)
    if density == "uniform":
        return np.ones(shape), T, u
    return T ** 3, T, u
