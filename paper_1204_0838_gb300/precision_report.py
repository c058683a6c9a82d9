"""FP32 against FP64 on the same workload: the error of each diagnostic.

Runs the c1 workload in FP64 and its FP32 twin (c2: fields, momenta, offsets
and currents in FP32; window accumulator and reductions in FP64) from the same
seeded state for the same steps, then compares the on-axis Ex lineout (L2
relative), the field energy, the charge above a gamma threshold and the
electron spectrum (L1 relative).  Diagnostics are computed on the GPU in FP64.

    python -m paper_1204_0838_gb300.precision_report [--steps 1000] [--start-step 0]
        [--crop nx,ny,nz] [--every 100]

Prints one JSON object per checkpoint and a final summary line.
"""
import argparse
import json
import time

import numpy as np

from . import pic, workloads as W


def _make(cfg, precision):
    g = pic.Sim(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"], cfg["lambda0"],
                x0=cfg["x0"], periodic_x=cfg["periodic_x"], precision=precision, seed=cfg["seed"],
                window=cfg["window"])
    g.add_species(cfg["prof_x"], cfg["prof_n"], cfg["ppc"], loading=cfg["loading"])
    g.add_laser(cfg["a0"], cfg["waist"], cfg["fwhm"], cfg["lambda0"], cfg["x_focus"], cfg["t_peak"])
    return g


def _diags(g, nx, gamma_min, e_max):
    return {"lineout": g.diag("ex_lineout", nx), "energy": g.diag("field_energy")[0],
            "charge": g.diag("charge", 1, gamma_min)[0], "charge_all": g.diag("charge", 1, 0.0)[0],
            "charge_g2": g.diag("charge", 1, 2.0)[0], "spectrum": g.diag("spectrum", 200, 0.0, e_max)}


def compare(d64, d32):
    def rel(a, b):
        return abs(a - b) / abs(b) if b != 0 else (0.0 if a == 0 else float("inf"))
    l64, l32 = d64["lineout"], d32["lineout"]
    s64, s32 = d64["spectrum"], d32["spectrum"]
    return {"lineout_l2_rel": float(np.linalg.norm(l32 - l64) / max(np.linalg.norm(l64), 1e-300)),
            "energy_rel": rel(d32["energy"], d64["energy"]),
            "charge_rel": rel(d32["charge"], d64["charge"]),
            "charge_all_rel": rel(d32["charge_all"], d64["charge_all"]),
            "charge_gamma2_rel": rel(d32["charge_g2"], d64["charge_g2"]),
            "spectrum_l1_rel": float(np.abs(s32 - s64).sum() / max(s64.sum(), 1e-300)),
            "charge_fp64_C": d64["charge"], "charge_gamma2_fp64_C": d64["charge_g2"],
            "energy_fp64_J": d64["energy"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--start-step", type=int, default=0)
    ap.add_argument("--every", type=int, default=250)
    ap.add_argument("--crop", default="")
    ap.add_argument("--gamma-min", type=float, default=20.0)
    ap.add_argument("--e-max", type=float, default=50.0)
    args = ap.parse_args()
    crop = tuple(int(v) for v in args.crop.split(",")) if args.crop else None
    cfg = W.config("c1", crop=crop, start_step=args.start_step)
    t0 = time.time()
    g64, g32 = _make(cfg, "fp64"), _make(cfg, "fp32")
    done = 0
    out = None
    while done < args.steps:
        n = min(args.every, args.steps - done)
        g64.step(n)
        g32.step(n)
        done += n
        out = compare(_diags(g64, cfg["nx"], args.gamma_min, args.e_max),
                      _diags(g32, cfg["nx"], args.gamma_min, args.e_max))
        out.update({"step": args.start_step + done, "particles_fp64": g64.info()["np"],
                    "particles_fp32": g32.info()["np"], "elapsed_s": time.time() - t0})
        print(json.dumps(out), flush=True)
    summary = {"workload": "c1/c2 %dx%dx%d, steps %d..%d" % (cfg["nx"], cfg["ny"], cfg["nz"],
                                                             args.start_step, args.start_step + done),
               "lineout_l2_rel": out["lineout_l2_rel"], "charge_rel": out["charge_rel"],
               "gamma_min": args.gamma_min, "pass_lineout_1pct": out["lineout_l2_rel"] <= 0.01,
               "pass_charge_2pct": out["charge_rel"] <= 0.02 if out["charge_fp64_C"] > 0 else None}
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    main()
