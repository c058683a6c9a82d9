"""Full-size parity: the c1 workload (1536x256x256 cells, ~1.2e8 particles) in
the launch configuration bench.py times (autotuned tiles), checked against the
FP64 oracle on sampled outputs; in FP32 after the run's own first 900 steps.

For a sampled node n the outcome of one step there depends only on a small
neighbourhood: the particles whose start cell lies within [n-4, n+3] on every
axis (the only ones whose Esirkepov window reaches nodes n-1 .. n+1) and the
fields within a few cells.  The test copies a 16^3 block of the GPU's fields
around n and those particles into a periodic 16^3 oracle box, steps it once,
and compares with the GPU's full-size step: every copied particle (matched by
id), and J, E, B at n (the block is large enough that neither its periodic
wrap nor the particles left out reach n).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1204_0838_gb300 import pic, workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HALF = 8  # block = node - 8 .. node + 7


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pic.lib()


def _full(precision):
    # Both precisions: the run itself from its empty box to step 900, the state
    # bench.py times (its wake, compressed bubble walls and the particles that
    # cross cell faces there).
    pre = 900
    cfg = W.config("c1" if precision == "fp64" else "c2", start_step=0)
    g = pic.Sim(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"], cfg["lambda0"],
                x0=cfg["x0"], periodic_x=False, precision=precision, seed=cfg["seed"],
                window=cfg["window"], track_ids=True)
    g.add_species(cfg["prof_x"], cfg["prof_n"], cfg["ppc"], loading=cfg["loading"])
    g.add_laser(cfg["a0"], cfg["waist"], cfg["fwhm"], cfg["lambda0"], cfg["x_focus"], cfg["t_peak"])
    for done in range(0, pre - 3, 100):
        g.step(min(100, pre - 3 - done))
    pic.pic_autotune(g.h, 1, None)
    g.step(3)
    return g, cfg


def _block(a, n, shape):
    """16^3 block of a full-size array centred on node n (y, z wrapped)."""
    i = np.arange(n[0] - HALF, n[0] + HALF)
    j = np.arange(n[1] - HALF, n[1] + HALF) % shape[1]
    k = np.arange(n[2] - HALF, n[2] + HALF) % shape[2]
    return a[np.ix_(i, j, k)]


# FP32: offsets carry 24 bits (eps = 2^-24 of a cell), so the deposited
# S(x1) - S(x0) of a displacement d keeps a relative error of about 2 eps / d;
# the slowest drifting plasma of this state moves d ~ 1e-4 cell per step,
# hence 1e-3 for the fields.  A current value is a sum of particle
# contributions q w jc run A (|run A| <= 1) that cancel down to ~1e-4 of their
# gross size, and each one carries an absolute error of about 2 eps |q w jc|
# (the rounding of the new FP32 offset and of the running sum) whatever the
# cancellation; the particles' errors are independent, so J gets, besides
# 1e-3 of the RMS, the allowance 2 eps sqrt(sum_p (q w_p jc)^2) over the
# particles that can reach the node.  Positions: FP64 1e-10 cell; FP32 32 eps
# (2e-6) cell, the rounding of an offset in [0, 1) plus that of its move.
# FP64: the 1e-10 parity bar.
EPS32 = 2.0 ** -24


@pytest.mark.parametrize("precision,tol,xtol", [("fp64", 1e-10, 1e-10), ("fp32", 1e-3, 32 * EPS32)])
def test_c1_full_size_sampled_parity(precision, tol, xtol):
    g, cfg = _full(precision)
    shape = (cfg["nx"], cfg["ny"], cfg["nz"])
    F0 = [g.field(c) for c in range(6)]
    P0 = g.particles()
    s0 = g.info()["shifts"]
    g.step(1)
    ds = g.info()["shifts"] - s0  # the window moved: post-step state is ds cells back
    assert ds == 1
    P1 = g.particles()
    order1 = np.argsort(P1["id"])
    ids1 = P1["id"][order1]
    J1 = [g.field(c) for c in (6, 7, 8)]
    F1 = [g.field(c) for c in range(6)]
    # relative errors are normalised by max(local |ref|, RMS of the quantity over
    # the grid): a current at a node is a sum of cancelling particle terms, and
    # the oracle resolves a particle's displacement only to its position
    # rounding (absolute grid coordinates), so the local value alone is no scale
    rms = [float(np.sqrt(np.mean(a.astype(np.float64) ** 2))) for a in F1 + J1]
    cells0 = np.floor(P0["xi"]).astype(np.int64)

    rng = np.random.default_rng(20)
    # sample nodes inside the plasma, near the laser (last third of the window)
    occupied = cells0[:, rng.integers(0, cells0.shape[1], 4000)]
    cand = occupied[:, (occupied[0] > shape[0] * 2 // 3) & (occupied[0] < shape[0] - 12)]
    assert cand.shape[1] > 8
    nodes = cand[:, rng.choice(cand.shape[1], 6, replace=False)].T
    checked = 0
    for n in nodes:
        # particles whose start cell is within [n-4, n+3] on every axis (y, z periodic)
        d = cells0 - n[:, None]
        d[1] = (d[1] + shape[1] // 2) % shape[1] - shape[1] // 2
        d[2] = (d[2] + shape[2] // 2) % shape[2] - shape[2] // 2
        sel = np.all((d >= -4) & (d <= 3), axis=0)
        assert sel.sum() > 0
        o = O.Sim(16, 16, 16, cfg["dx"], cfg["dy"], cfg["dz"], cfg["lambda0"], periodic_x=True)
        for c in range(6):
            o.field(c)[...] = _block(F0[c], n, shape)
        xi_local = P0["xi"][:, sel] - (n - HALF)[:, None]
        for a in (1, 2):
            xi_local[a] = (xi_local[a] + shape[a] // 2 - HALF) % shape[a] - shape[a] // 2 + HALF
        o.set_particles(xi_local, P0["u"][:, sel], P0["w"][sel], P0["id"][sel])
        o.step(1)
        po = o.particles()
        # particles: by id against the GPU's full-size step
        pos = np.searchsorted(ids1, po["id"])
        assert np.array_equal(ids1[pos], po["id"])
        gi = order1[pos]
        u_g = P1["u"][:, gi]
        xi_g = P1["xi"][:, gi] - (n - HALF)[:, None]
        xi_g[0] += ds
        for a in (1, 2):
            xi_g[a] = (xi_g[a] + shape[a] // 2 - HALF) % shape[a] - shape[a] // 2 + HALF
        uscale = max(1.0, np.abs(po["u"]).max())
        assert np.abs(u_g - po["u"]).max() <= tol * uscale
        dxi = np.abs(xi_g - po["xi"])
        dxi = np.minimum(dxi, 16 - dxi)  # the oracle box wraps
        assert dxi.max() <= xtol, ("xi", dxi.max(), xtol)
        # J, E, B at the sampled node (post-step arrays are in the shifted frame)
        m = (n[0] - ds, n[1], n[2])
        # particles whose Esirkepov window can reach node n (start cell within n-3 .. n+2)
        near = np.all((d >= -3) & (d <= 2), axis=0)
        inf = o.info()
        jc = (1 / (inf["dt"] * inf["dy"] * inf["dz"]), 1 / (inf["dt"] * inf["dx"] * inf["dz"]),
              1 / (inf["dt"] * inf["dx"] * inf["dy"]))
        qw2 = float(np.sum(P0["w"][near].astype(np.float64) ** 2))  # |q| = 1
        for a, (c, arr) in enumerate(zip((6, 7, 8), J1)):
            ref = o.field(c)[HALF, HALF, HALF]
            scale = max(abs(ref), rms[c], 1e-300)
            j_abs = 2 * EPS32 * jc[a] * np.sqrt(qw2) if precision == "fp32" else 0.0
            assert abs(arr[m] - ref) <= tol * scale + j_abs, ("J", c, arr[m], ref, rms[c], j_abs)
        for c in range(6):
            ref = o.field(c)[HALF, HALF, HALF]
            scale = max(abs(ref), rms[c], 1e-300)
            assert abs(F1[c][m] - ref) <= tol * scale, ("F", c, F1[c][m], ref, rms[c])
        checked += 1
    assert checked == len(nodes)
    g.close()
