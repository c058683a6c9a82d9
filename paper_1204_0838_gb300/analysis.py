"""Host-side post-processing of diagnostics (not on the GPU path).

- accelerating_phase_length: Fig. 1a of the paper plots the length of the
  accelerating phase on axis, the region inside the bubble where the
  longitudinal field is negative.  Reading used here: on the on-axis Ex
  lineout, the contiguous run of cells with Ex < 0 that contains the most
  negative Ex (the peak accelerating field at the rear of the first bucket).
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
