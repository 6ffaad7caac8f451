"""FP64 CPU oracle for the long-range particle-mesh (PM) part of the PM-FMM
split (arXiv:2107.14008, Section 2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import this module.  It shares no code with the
CUDA library.

The split (Section 2): phi = phi_long + phi_short, the short-range pair force
carries T(x) = erfc(x) + (2x/sqrt(pi)) exp(-x^2), x = r/(2 r_s) (Eq. tr), so the
long-range pair force is the Newtonian force times 1 - T(x), whose potential
is -G m erf(r/(2 r_s))/r.  Its Fourier transform is -4 pi G m exp(-k^2 r_s^2)/k^2.
The paper prints the filter as exp(-k^2/4r_s^2); that is not the complement
of its own erfc(r/2r_s), and exp(-k^2 r_s^2) is taken here (the reading that
makes short + long the Newtonian force).  In a periodic box the k = 0 mode is
dropped (the mean density does not source the field).

Two functions:
  ewald_long  the exact periodic long-range acceleration, a direct sum over
              wave vectors (no mesh):
                a_i = -(4 pi G / L^3) sum_{k != 0} exp(-k^2 r_s^2)/k^2
                                   k Im(exp(i k.x_i) S(k)),  S(k) = sum_j m_j exp(-i k.x_j)
  pm_forces   the mesh method: cloud-in-cell (CIC) mass assignment on an
              N_PM^3 grid (points at g L/N_PM), FFT, Green's function
              -4 pi G exp(-k^2 r_s^2)/k^2 divided by the squared CIC window
              (optional), spectral gradient -i k (Nyquist planes zeroed),
              inverse FFT per component, CIC interpolation back to the
              particles.
"""
import numpy as np


def wrap(pos, L):
    p = np.mod(np.asarray(pos, dtype=np.float64), L)
    return np.where(p >= L, 0.0, p)


def _cic(pos, L, n):
    """Cell indices (3 x (n_p, 2)) and weights (3 x (n_p, 2)) of CIC."""
    u = wrap(pos, L) / (L / n)
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    idx = [np.stack([i0[:, a] % n, (i0[:, a] + 1) % n], axis=1) for a in range(3)]
    w = [np.stack([1.0 - f[:, a], f[:, a]], axis=1) for a in range(3)]
    return idx, w


def cic_deposit(pos, mass, L, n):
    """Density on the grid: sum_j m_j W(x_j - x_g) / Delta^3."""
    idx, w = _cic(pos, L, n)
    rho = np.zeros((n, n, n))
    m = np.asarray(mass, dtype=np.float64)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                np.add.at(rho, (idx[0][:, a], idx[1][:, b], idx[2][:, c]),
                          m * w[0][:, a] * w[1][:, b] * w[2][:, c])
    return rho / (L / n) ** 3


def cic_interp(grid, pos, L):
    """CIC interpolation of a grid field at the positions."""
    n = grid.shape[0]
    idx, w = _cic(pos, L, n)
    out = np.zeros(len(pos))
    for a in range(2):
        for b in range(2):
            for c in range(2):
                out += (w[0][:, a] * w[1][:, b] * w[2][:, c] *
                        grid[idx[0][:, a], idx[1][:, b], idx[2][:, c]])
    return out


def wavenumbers(n, L):
    """Integer and physical wave numbers of the rfftn layout (n, n, n//2+1)."""
    i0 = np.fft.fftfreq(n, d=1.0 / n)
    i2 = np.fft.rfftfreq(n, d=1.0 / n)
    I = np.meshgrid(i0, i0, i2, indexing="ij")
    return I, [2.0 * np.pi / L * v for v in I]


def green(n, L, r_s, G=1.0, deconvolve=True):
    """-4 pi G exp(-k^2 r_s^2) / k^2 [/ W_CIC(k)^2], zero at k = 0."""
    _, k = wavenumbers(n, L)
    k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(k2 > 0, -4.0 * np.pi * G * np.exp(-k2 * r_s * r_s) / k2, 0.0)
    if deconvolve:
        h = 0.5 * L / n
        for a in range(3):
            s = np.sinc(k[a] * h / np.pi)  # sin(k h) / (k h)
            g = g / s ** 4                 # assignment and interpolation windows
    return g


def pm_forces(pos, mass, L, r_s, n, G=1.0, deconvolve=True):
    """Long-range accelerations (n_p, 3) by the mesh method."""
    pos = wrap(pos, L)
    rho = cic_deposit(pos, mass, L, n)
    phi_k = green(n, L, r_s, G, deconvolve) * np.fft.rfftn(rho)
    I, k = wavenumbers(n, L)
    acc = np.zeros((len(pos), 3))
    for a in range(3):
        ak = -1j * k[a] * phi_k
        ak = np.where(np.abs(I[a]) == n // 2, 0.0, ak) if n % 2 == 0 else ak
        grid = np.fft.irfftn(ak, s=(n, n, n), axes=(0, 1, 2))
        acc[:, a] = cic_interp(grid, pos, L)
    return acc


def ewald_long(pos, mass, L, r_s, G=1.0, targets=None, tol=1e-17):
    """Exact periodic long-range accelerations (direct k-space sum) at the
    targets (indices, default all)."""
    pos = wrap(pos, L)
    m = np.asarray(mass, dtype=np.float64)
    tp = pos if targets is None else pos[np.asarray(targets)]
    kmax = np.sqrt(-np.log(tol)) / r_s
    nk = int(np.ceil(kmax * L / (2.0 * np.pi)))
    r = np.arange(-nk, nk + 1)
    I = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    I = I[np.any(I != 0, axis=1)]
    k = 2.0 * np.pi / L * I
    k2 = np.sum(k * k, axis=1)
    keep = k2 <= kmax * kmax
    k, k2 = k[keep], k2[keep]
    coef = np.exp(-k2 * r_s * r_s) / k2
    acc = np.zeros((len(tp), 3))
    for s in range(0, len(k), 4096):
        kk, cc = k[s:s + 4096], coef[s:s + 4096]
        S = np.exp(-1j * pos @ kk.T).T @ m                  # (nk,)
        im = np.imag(np.exp(1j * tp @ kk.T) * S[None, :])    # (n_t, nk)
        acc += (im * cc[None, :]) @ kk
    return -4.0 * np.pi * G / L ** 3 * acc
