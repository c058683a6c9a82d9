"""Build the same simulation on the GPU library and on the CPU oracle."""
import numpy as np

from oracle import oracle as O
from paper_1204_0838_gb300 import pic


def make_gpu(cfg, track_ids=True, precision=None, laser=True, species=True, max_particles=0):
    g = pic.Sim(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"], cfg["lambda0"],
                x0=cfg["x0"], periodic_x=cfg["periodic_x"], precision=precision or cfg["precision"],
                seed=cfg["seed"], window=cfg["window"], track_ids=track_ids,
                max_particles=max_particles, pml=cfg.get("pml", 0))
    if species:
        g.add_species(cfg["prof_x"], cfg["prof_n"], cfg["ppc"], loading=cfg["loading"])
    if laser:
        g.add_laser(cfg["a0"], cfg["waist"], cfg["fwhm"], cfg["lambda0"], cfg["x_focus"], cfg["t_peak"])
    return g


def make_oracle(cfg, laser=True, species=True):
    o = O.Sim(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"], cfg["lambda0"],
              x0=cfg["x0"], periodic_x=cfg["periodic_x"], seed=cfg["seed"], window=cfg["window"],
              pml=cfg.get("pml", 0))
    if species:
        o.add_species(cfg["prof_x"], cfg["prof_n"], cfg["ppc"], loading=cfg["loading"])
    if laser:
        o.add_laser(cfg["a0"], cfg["waist"], cfg["fwhm"], cfg["lambda0"], cfg["x_focus"], cfg["t_peak"])
    return o


def by_id(p):
    order = np.argsort(p["id"], kind="stable")
    return {k: (v[:, order] if v.ndim == 2 else v[order]) for k, v in p.items()}


def rel_err(got, ref):
    """max |got - ref| normalised by max(|ref|max, RMS of ref) (never zero)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(np.abs(ref).max() if ref.size else 0.0, np.sqrt(np.mean(ref ** 2)) if ref.size else 0.0)
    if scale == 0.0:
        return np.abs(got).max() if got.size else 0.0
    return np.abs(got - ref).max() / scale


def compare_particles(pg, po, tol):
    """Particles matched by id: positions to tol cells (absolute), momenta and
    weights to tol relative (rel_err)."""
    pg, po = by_id(pg), by_id(po)
    assert pg["id"].size == po["id"].size, (pg["id"].size, po["id"].size)
    assert np.array_equal(pg["id"], po["id"])
    errs = {}
    # positions in absolute cells: the offsets live in [0, 1) of a cell whatever the grid size
    errs["xi"] = np.abs(pg["xi"] - po["xi"]).max() if po["id"].size else 0
    errs["u"] = rel_err(pg["u"], po["u"])
    errs["w"] = rel_err(pg["w"], po["w"])
    for k, v in errs.items():
        assert v <= tol, (k, v, tol)
    return errs


def compare_fields(g, o, tol, comps=range(9)):
    errs = {}
    for c in comps:
        errs[pic.COMPONENTS[c]] = rel_err(g.field(c), o.field(c))
    bad = {k: v for k, v in errs.items() if v > tol}
    assert not bad, (bad, tol)
    return errs
