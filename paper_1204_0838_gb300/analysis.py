"""Host-side post-processing of diagnostics (not on the GPU path).

- accelerating_phase_length: Fig. 1a of the paper plots the length of the
  accelerating phase on axis, the region inside the bubble where the
  longitudinal field is negative.  Reading used here: on the on-axis Ex
  lineout, the contiguous run of cells with Ex < 0 that contains the most
  negative Ex (the peak accelerating field at the rear of the first bucket).
- bubble_scalings: the blowout-regime estimates of Sec. 1 (energy gain at
  dephasing, Eq. (Ed); dephasing length, Eq. (Ld); critical power for
  relativistic self-focusing; accelerating-phase length, Eq. (Rb)) from the
  plasma density, the laser wavelength and the laser power.
- initial_cells: particle ids (PIC_FLAG_TRACK_IDS) encode the lab cell and
  slot a particle was loaded in (id = ((L * ny + j) * nz + k) * ppc + slot);
  decoding them gives the initial positions to cell resolution, i.e. the
  collection volume of Fig. 1b, c (initial x and radial offset of the
  electrons that reach a given energy).
"""
import numpy as np


def accelerating_phase_length(lineout, dx):
    """Length (same unit as dx) of the Ex < 0 run holding the minimum of Ex."""
    e = np.asarray(lineout, dtype=np.float64)
    if e.size == 0 or not (e.min() < 0):
        return 0.0
    i = int(np.argmin(e))
    lo = i
    while lo > 0 and e[lo - 1] < 0:
        lo -= 1
    hi = i
    while hi + 1 < e.size and e[hi + 1] < 0:
        hi += 1
    return (hi - lo + 1) * dx


def initial_cells(ids, ppc, ny, nz):
    """Decode particle ids into (lab x cell L, y cell j, z cell k, slot)."""
    ids = np.asarray(ids, dtype=np.uint64)
    slot = ids % ppc
    cell = ids // ppc
    k = cell % nz
    j = (cell // nz) % ny
    L = cell // (nz * ny)
    return L.astype(np.int64), j.astype(np.int64), k.astype(np.int64), slot.astype(np.int64)


def initial_positions(ids, ppc, grid):
    """Initial lab x and radial offset from the axis (metres) of the cell
    centres the particles were loaded in; grid: dict with nx, ny, nz, dx, dy,
    dz, x0 (metres)."""
    L, j, k, _ = initial_cells(ids, ppc, grid["ny"], grid["nz"])
    x_in = grid["x0"] + (L + 0.5) * grid["dx"]
    y = (j + 0.5 - 0.5 * grid["ny"]) * grid["dy"]
    z = (k + 0.5 - 0.5 * grid["nz"]) * grid["dz"]
    return x_in, np.hypot(y, z)


def bubble_scalings(n0_per_cm3, lambda0_m, power_W):
    """Sec. 1 estimates for a laser of power P and wavelength lambda0 in a
    plasma of density n0, with gamma_g = omega0 / omega_pe = sqrt(n_c / n0):
    E_d ~ 2.7 gamma_g^(4/3) P_TW^(1/3) MeV, L_d ~ 0.6 lambda0 gamma_g^(8/3)
    P_TW^(1/6), P_cr = 16.2 gamma_g^2 GW, L_acc ~ 0.9 lambda0 gamma_g^(2/3)
    P_TW^(1/6).  Returns SI values (m, W) and MeV."""
    c, qe, me, eps0 = 299792458.0, 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12
    omega0 = 2.0 * np.pi * c / lambda0_m
    n_c = eps0 * me * omega0 ** 2 / qe ** 2  # 1/m^3
    gamma_g = float(np.sqrt(n_c / (n0_per_cm3 * 1e6)))
    p_tw = power_W / 1e12
    return {"gamma_g": gamma_g, "n0_over_nc": n0_per_cm3 * 1e6 / n_c,
            "P_cr_W": 16.2e9 * gamma_g ** 2,
            "E_d_MeV": 2.7 * gamma_g ** (4.0 / 3.0) * p_tw ** (1.0 / 3.0),
            "L_d_m": 0.6 * lambda0_m * gamma_g ** (8.0 / 3.0) * p_tw ** (1.0 / 6.0),
            "L_acc_m": 0.9 * lambda0_m * gamma_g ** (2.0 / 3.0) * p_tw ** (1.0 / 6.0)}
