"""Synthetic workloads and seeded random states (inputs only, no PIC arithmetic).

The paper's runs (Sec. 3.1: lambda0 = 0.805 um, 30 fs FWHM, 70 TW, a0 = 3.27,
n0 = 6.5e18 cm^-3 with 0.5 mm ramps, dx = 0.06 lambda0, dy = dz = 0.5 lambda0,
4 macroparticles per cell, cubic splines, moving window) are physical LWFA
simulations, not datasets.  These recipes stand in for them with the same
kind of laser, plasma, grid anisotropy and particle loading at sizes that fit
one GPU (and, for the small ones, a CPU oracle).

Every value here is a set-up parameter in SI units (densities in n_c) or a
seeded random number; both the CUDA library and the CPU oracle consume them.
"""
import numpy as np

LAMBDA0 = 0.8e-6
C0 = 299792458.0
DEFAULT_SEED = 12040838


def config(name, crop=None, start_step=0):
    """Workload recipe by name.

    c0: 128x32x32, dx = lambda0/8, dy = dz = lambda0/2, uniform n = 0.02 n_c,
        1 ppc random in cell, a0 = 2, waist 4 lambda0, FWHM 4 lambda0/c, laser
        entering at x = 0 through the boundary source, no window, 100 steps, FP64.
    c1: 1536x256x256, dx = lambda0/24, dy = dz = lambda0/3, n = 0.004 n_c after a
        50 um linear up-ramp from x = 0, 2 ppc jittered lattice, a0 = 4, 30 fs,
        waist 16 um, window at c, 1000 steps, FP64.
    c2: c1 in FP32.
    c4: 2048x256x256, dx = lambda0/32, 4 ppc, 5000 steps, FP32, injected-charge and
        electron-spectrum diagnostics every 250 steps.
    inj: a dense window in which the wake traps electrons early: the c1
        spacings on 384x96x96 cells, n = 0.03 n_c after a 10 um linear
        up-ramp, a0 = 5, waist 4 um, 15 fs, 2 ppc lattice, window at c, FP64;
        by step 5000 a few nC sit above gamma 20 (the injected charge of
        Table 1 needs such a state; c1/c2 at 1000 steps have none).
    crop=(nx, ny, nz) keeps the spacings and physics on a smaller box.
    start_step=S places the window (and the laser with it) where it is after S
    steps of the run, with the plasma that has entered by then loaded cold.
    """
    lam = LAMBDA0
    if name == "c0":
        nx, ny, nz = 128, 32, 32
        cfg = dict(nx=nx, ny=ny, nz=nz, dx=lam / 8, dy=lam / 2, dz=lam / 2, lambda0=lam, x0=0.0,
                   periodic_x=False, precision="fp64", seed=DEFAULT_SEED, window=None,
                   prof_x=[-1.0, 1.0], prof_n=[0.02, 0.02], ppc=1, loading="random",
                   a0=2.0, waist=4 * lam, fwhm=4 * lam / C0, x_focus=0.0, t_peak=8 * lam / C0,
                   steps=100)
    elif name in ("c1", "c2", "c4"):
        if name == "c4":
            nx, ny, nz, dx, ppc, steps = 2048, 256, 256, lam / 32, 4, 5000
        else:
            nx, ny, nz, dx, ppc, steps = 1536, 256, 256, lam / 24, 2, 1000
        fwhm = 30e-15
        cfg = dict(nx=nx, ny=ny, nz=nz, dx=dx, dy=lam / 3, dz=lam / 3, lambda0=lam,
                   x0=-nx * dx, periodic_x=False,
                   precision="fp64" if name == "c1" else "fp32", seed=DEFAULT_SEED,
                   window=(1.0, 0.0), prof_x=[0.0, 50e-6, 1.0], prof_n=[0.0, 0.004, 0.004],
                   ppc=ppc, loading="lattice", a0=4.0, waist=16e-6, fwhm=fwhm, x_focus=0.0,
                   t_peak=2 * fwhm, steps=steps)
        if name == "c4":
            cfg["diag_every"] = 250  # injected charge and electron spectrum
    elif name == "inj":
        nx, ny, nz, dx = 384, 96, 96, lam / 24
        fwhm = 15e-15
        cfg = dict(nx=nx, ny=ny, nz=nz, dx=dx, dy=lam / 3, dz=lam / 3, lambda0=lam, x0=-nx * dx,
                   periodic_x=False, precision="fp64", seed=DEFAULT_SEED, window=(1.0, 0.0),
                   prof_x=[0.0, 10e-6, 1.0], prof_n=[0.0, 0.03, 0.03], ppc=2, loading="lattice",
                   a0=5.0, waist=4e-6, fwhm=fwhm, x_focus=0.0, t_peak=2 * fwhm, steps=5000)
    else:
        raise KeyError(name)
    if crop is not None:
        cfg["nx"], cfg["ny"], cfg["nz"] = crop
        if cfg["window"] is not None:
            cfg["x0"] = -cfg["nx"] * cfg["dx"]
    if start_step:
        # c dt = dx: the window moves one cell per step
        cfg["x0"] += start_step * cfg["dx"]
        cfg["t_peak"] -= start_step * cfg["dx"] / C0
    cfg["name"] = name
    return cfg


def batch_configs(n=32, seed=DEFAULT_SEED):
    """Batched scan: a0 ~ U[2,5], n ~ U[0.003, 0.02] n_c, waist ~ U[10,20] um,
    nx in {256..768}, ny = nz in {64, 96, 128}, dx = lambda0/16, dy = dz =
    lambda0/3, 1-2 ppc, window at c, FP32."""
    rng = np.random.default_rng(seed)
    lam = LAMBDA0
    out = []
    for i in range(n):
        nx = int(rng.choice([256, 384, 512, 640, 768]))
        nt = int(rng.choice([64, 96, 128]))
        dx = lam / 16
        fwhm = 30e-15
        dens = float(rng.uniform(0.003, 0.02))
        out.append(dict(nx=nx, ny=nt, nz=nt, dx=dx, dy=lam / 3, dz=lam / 3, lambda0=lam,
                        x0=-nx * dx, periodic_x=False, precision="fp32", seed=seed + i,
                        window=(1.0, 0.0), prof_x=[0.0, 20e-6, 1.0], prof_n=[0.0, dens, dens],
                        ppc=int(rng.choice([1, 2])), loading="lattice",
                        a0=float(rng.uniform(2, 5)), waist=float(rng.uniform(10e-6, 20e-6)),
                        fwhm=fwhm, x_focus=0.0, t_peak=2 * fwhm, steps=500, name="c3.%d" % i))
    return out


def random_state(shape, n_particles, seed, umax=2.0, periodic_x=True, field_scale=0.1,
                 weight=0.01, dV=1.0, yz_margin=0):
    """Seeded random fields (9, nx, ny, nz) and particles (grid-unit positions
    inside the allowed range, momenta in [-umax, umax], positive weights);
    yz_margin keeps y and z inside [margin, n - margin) (absorbing layers)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    fields = rng.standard_normal((9, nx, ny, nz)) * field_scale
    fields[6:] = 0.0
    lo, hi = (0.0, nx) if periodic_x else (3.0, nx - 5.0)
    m = float(yz_margin)
    xi = np.stack([rng.uniform(lo, hi, n_particles), rng.uniform(m, ny - m, n_particles),
                   rng.uniform(m, nz - m, n_particles)])
    u = rng.uniform(-umax, umax, (3, n_particles))
    w = rng.uniform(0.5, 1.5, n_particles) * weight * dV
    ids = np.arange(n_particles, dtype=np.uint32)
    return fields, xi, u, w, ids
