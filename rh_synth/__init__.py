"""Seeded synthetic inputs shared by the oracle, the CUDA path, the tests and the bench.

This module only *describes* inputs: the model-atom description (what an atom
file would hold) and the atmosphere columns.  It contains none of the method's
arithmetic (no formal solution, no rates, no populations, no wavelength grid):
each side derives everything else from these numbers on its own.

Workloads (stand-ins for the 3D MHD snapshot and the Mg II / Ca II model atoms
of the paper, Sect. 3.3, which are not available):

* ``hydrogen_like_atom`` -- hydrogen-like atom with 5 bound levels and the
  continuum: E_n = 13.6 (1 - 1/n^2) eV, g_n = 2 n^2, all 10 bound-bound lines
  with Kramers oscillator strengths (Gaunt factor 1), 5 bound-free continua with
  Kramers threshold cross sections 7.91e-22 n m^2.  Voigt damping runs from
  1e-2 at the bottom to 1e-3 at the top (log-interpolated in depth index).
* ``chromosphere_column`` -- one column of 82 heights from 2500 km (top) to
  -100 km (bottom): T falls linearly from 6500 K at -100 km to a 4200 K minimum
  at 500 km, rises linearly to 8000 K at 2000 km and stays there above;
  n_H = 1e23 exp(-z / 150 km) m^-3; v_z = 0.
* ``chromosphere_cube`` -- nx*ny such columns: a periodic Gaussian random field
  (sigma 500 K, Gaussian correlation length 8 columns) added to T at all heights
  (T >= 3000 K), the n_H scale height jittered by U(0.8, 1.2) per column, and
  v_z = A sin(2 pi z / P + phase) with A ~ U(0, 10 km/s), P ~ U(200, 800 km),
  phase ~ U(0, 2 pi).
"""
from __future__ import annotations

import numpy as np

EV_J = 1.602176634e-19          # 1 eV in J (exact, SI 2019)
E_RYD_EV = 13.6                 # ionisation energy of the model atom, eV
AMU_H = 1.008                   # hydrogen mass, amu


def kramers_f(n_lo: int, n_up: int) -> float:
    """Kramers (semi-classical) absorption oscillator strength, Gaunt factor 1.

    f = 2^5 / (3^{3/2} pi) * 1 / (n^5 n'^3) * (1/n^2 - 1/n'^2)^-3.
    """
    return (32.0 / (3.0 * np.sqrt(3.0) * np.pi)) / (n_lo ** 5 * n_up ** 3) \
        * (1.0 / n_lo ** 2 - 1.0 / n_up ** 2) ** -3


def hydrogen_like_atom(nbound: int = 5,
                       lyman_nlambda: int = 64,
                       line_nlambda: int = 32,
                       cont_nlambda: int = 32,
                       qwing: float = 100.0,
                       cont_ratio: float = 2.5,
                       a_top: float = 1e-3,
                       a_bot: float = 1e-2,
                       nmu: int = 5,
                       T_ref: float = 5000.0,
                       metal_floor: float = 1e-4,
                       prd_lines=(),
                       prd_nlambda: int = 0) -> dict:
    """Atom description of the H-like model atom (arrays are numpy, SI units).

    Level index i = n - 1 for bound levels, the continuum is the last level.
    With the defaults the wavelength grid has 4*64 + 6*32 + 5*32 = 608 points.
    ``prd_lines``: (lower n, upper n) pairs treated in partial redistribution,
    e.g. ((1, 2), (1, 3)) for Lyman alpha and beta; ``prd_nlambda`` > 0 gives
    those lines that many wavelength points instead of their default.
    """
    nlev = nbound + 1
    E = np.array([E_RYD_EV * (1.0 - 1.0 / n ** 2) for n in range(1, nbound + 1)]
                 + [E_RYD_EV]) * EV_J
    g = np.array([2.0 * n * n for n in range(1, nbound + 1)] + [1.0])
    ll, lu, f, nl = [], [], [], []
    for n in range(1, nbound + 1):
        for m in range(n + 1, nbound + 1):
            ll.append(n - 1)
            lu.append(m - 1)
            f.append(kramers_f(n, m))
            if prd_nlambda > 0 and (n, m) in tuple(prd_lines):
                nl.append(prd_nlambda)
            else:
                nl.append(lyman_nlambda if n == 1 else line_nlambda)
    nline = len(ll)
    cont_l = list(range(nbound))
    alpha0 = [7.91e-22 * n for n in range(1, nbound + 1)]
    return dict(
        nlev=nlev, E_J=E, g=g,
        line_l=np.array(ll, np.int32), line_u=np.array(lu, np.int32),
        line_f=np.array(f), line_a_top=np.full(nline, a_top),
        line_a_bot=np.full(nline, a_bot),
        line_nlambda=np.array(nl, np.int32), line_qwing=np.full(nline, qwing),
        cont_l=np.array(cont_l, np.int32), cont_alpha0=np.array(alpha0),
        cont_nlambda=np.full(nbound, cont_nlambda, np.int32),
        cont_ratio=np.full(nbound, cont_ratio),
        mass_amu=AMU_H, T_ref=T_ref, nmu=nmu, metal_floor=metal_floor,
        line_prd=np.array([1 if (l + 1, u + 1) in tuple(prd_lines) else 0 for l, u in zip(ll, lu)], np.int32))


def small_atom(nbound: int = 3, nlambda: int = 8, cont_nlambda: int = 6,
               nmu: int = 2, **kw) -> dict:
    """A reduced H-like atom (3 bound levels + continuum) for brute-force checks."""
    return hydrogen_like_atom(nbound=nbound, lyman_nlambda=nlambda,
                              line_nlambda=nlambda, cont_nlambda=cont_nlambda,
                              nmu=nmu, **kw)


def _temperature_profile(z_km: np.ndarray) -> np.ndarray:
    T = np.empty_like(z_km)
    lo = z_km <= 500.0
    T[lo] = 6500.0 + (4200.0 - 6500.0) * (z_km[lo] + 100.0) / 600.0
    mid = (z_km > 500.0) & (z_km <= 2000.0)
    T[mid] = 4200.0 + (8000.0 - 4200.0) * (z_km[mid] - 500.0) / 1500.0
    T[z_km > 2000.0] = 8000.0
    return T


def chromosphere_column(ndep: int = 82, z_top_km: float = 2500.0,
                        z_bot_km: float = -100.0, scale_height_km: float = 150.0,
                        nH0: float = 1e23) -> dict:
    """One synthetic chromospheric column, k = 0 at the top.  Arrays [1][ndep]."""
    z_km = np.linspace(z_top_km, z_bot_km, ndep)
    T = _temperature_profile(z_km)
    nH = nH0 * np.exp(-z_km / scale_height_km)
    return dict(z=(z_km * 1e3)[None, :].copy(), T=T[None, :].copy(),
                nH=nH[None, :].copy(), vz=np.zeros((1, ndep)))


def gaussian_random_field(nx: int, ny: int, corr: float, sigma: float,
                          rng: np.random.Generator) -> np.ndarray:
    """Periodic Gaussian random field: white noise convolved with a Gaussian of
    standard deviation ``corr`` (in columns), rescaled to standard deviation ``sigma``."""
    noise = rng.standard_normal((nx, ny))
    kx = np.fft.fftfreq(nx)[:, None]
    ky = np.fft.fftfreq(ny)[None, :]
    kern = np.exp(-2.0 * (np.pi * corr) ** 2 * (kx ** 2 + ky ** 2))
    field = np.real(np.fft.ifft2(np.fft.fft2(noise) * kern))
    field -= field.mean()
    std = field.std()
    return field * (sigma / std) if std > 0 else field


def chromosphere_cube(nx: int = 256, ny: int = 256, ndep: int = 82, seed: int = 1234,
                      sigma_T: float = 500.0, corr: float = 8.0,
                      T_min: float = 3000.0, vz_max: float = 10e3,
                      period_km: tuple = (200.0, 800.0)) -> dict:
    """nx*ny perturbed columns (row-major over (x, y)); arrays [ncol][ndep]."""
    rng = np.random.default_rng(seed)
    base = chromosphere_column(ndep)
    z = base['z'][0]
    z_km = z / 1e3
    dT = gaussian_random_field(nx, ny, corr, sigma_T, rng).reshape(-1)
    ncol = nx * ny
    hscale = 150.0 * rng.uniform(0.8, 1.2, ncol)
    amp = rng.uniform(0.0, vz_max, ncol)
    per = rng.uniform(period_km[0], period_km[1], ncol)
    ph = rng.uniform(0.0, 2.0 * np.pi, ncol)
    T = np.maximum(base['T'][0][None, :] + dT[:, None], T_min)
    nH = 1e23 * np.exp(-z_km[None, :] / hscale[:, None])
    vz = amp[:, None] * np.sin(2.0 * np.pi * z_km[None, :] / per[:, None] + ph[:, None])
    return dict(z=np.ascontiguousarray(np.broadcast_to(z, (ncol, ndep))),
                T=np.ascontiguousarray(T), nH=np.ascontiguousarray(nH),
                vz=np.ascontiguousarray(vz))


def subset(cols: dict, idx) -> dict:
    """Columns ``idx`` of a column set (a copy)."""
    return {k: np.ascontiguousarray(v[idx]) for k, v in cols.items()}


def two_level_problem(ndep: int = 64, tau_min: float = 1e-6, tau_max: float = 1e4,
                      nfreq: int = 101, xmax: float = 6.0, nmu: int = 5,
                      eps: float = 1e-4, B: float = 1.0) -> dict:
    """Two-level atom, complete redistribution, isothermal: line-centre optical
    depth log-spaced from tau_min to tau_max, Doppler profile sampled at nfreq
    points over +-xmax Doppler widths, nmu Gauss-Legendre angles, constant B."""
    tau = np.logspace(np.log10(tau_min), np.log10(tau_max), ndep)
    return dict(tau=tau, nfreq=nfreq, xmax=xmax, nmu=nmu, eps=eps, B=B)
