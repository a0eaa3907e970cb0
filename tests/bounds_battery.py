"""Runs every instrumented kernel of liblf2 on small cases and saves the results (helper of
test_gpu_debug_bounds.py; run as a script, not collected by pytest).

    python tests/bounds_battery.py <library path> <output .npz>

Prints one JSON line with the index violations the library counted (null for a library built
without the checks)."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main(lib_path, out_path):
    import torch
    from paper_1508_05610_gb300 import inputs, lf2
    lf2.load(lib_path)
    out = {}
    kw = dict(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.05)
    p = lf2.params(**kw)
    tb = lf2.LF2_KERNEL_TBLOCK
    cases = [
        # shape, ncomp, precision, kernel configurations
        ((40, 16, 9), 1, "f32k", [dict(kernel=lf2.LF2_KERNEL_SITE), dict(kernel=lf2.LF2_KERNEL_STREAM),
                                  dict(kernel=tb, depth=4, cx=2, tile_x=16, tile_y=8),
                                  dict(kernel=tb, depth=3, cx=1, tile_x=12, tile_y=6, zchunk=4),
                                  dict(kernel=tb, depth=4, cx=2, tile_x=24, tile_y=8, cluster=2)]),
        ((34, 8, 6), 2, "f64", [dict(kernel=lf2.LF2_KERNEL_STREAM), dict(kernel=tb, depth=2, cx=1, tile_x=8, tile_y=4)]),
        ((32, 12, 7), 2, "f32", [dict(kernel=tb, depth=4, cx=2, tile_x=24, tile_y=8),
                                 dict(kernel=tb, depth=3, cx=2, tile_x=24, tile_y=10, cluster=4, zchunk=3)]),
        ((24, 12, 7), 4, "f32k", [dict(kernel=tb, depth=3, cx=1, tile_x=10, tile_y=8)]),
        ((33, 10, 6), 6, "f32", [dict(kernel=tb, depth=2, cx=1, tile_x=12, tile_y=8), dict(kernel=lf2.LF2_KERNEL_SITE)]),
        ((24, 8, 8), 3, "f64", [dict(kernel=lf2.LF2_KERNEL_STREAM)]),
    ]
    for ci, (shape, ncomp, prec, cfgs) in enumerate(cases):
        nx, ny, nz = shape
        phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.4, seed=300 + ci)
        pi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.1, seed=400 + ci)
        for j, cfg in enumerate(cfgs):
            with lf2.System(shape, ncomp, prec) as s:
                s.upload(phi0, pi0)
                lf2.lf2_leapfrog_init(s.phi, s.pi, p)
                lf2.lf2_leapfrog_ex(s.phi, s.pi, p, 7, **cfg)
                phi, pi = s.download()
                e = lf2.lf2_energy(s.phi, s.pi, p, ncomp=ncomp)
                # the same reduction on the library's fixed scratch array
                e_fixed = lf2.lf2_energy_noalloc(s.phi, s.pi, p, ncomp=ncomp)
            out[f"c{ci}_{j}_phi"], out[f"c{ci}_{j}_pi"] = phi, pi
            out[f"c{ci}_{j}_energy"] = np.array([e["total"]])
            out[f"c{ci}_{j}_energy_noalloc"] = np.array([e_fixed["total"], e_fixed["kinetic"], e_fixed["gradient"]])
    # fused step + energy: one launch per step (larger lattice) and all steps in one launch
    for ci, (shape, ncomp, prec) in enumerate([((16, 16, 16), 1, "f64"), ((80, 64, 48), 2, "f32k")]):
        nx, ny, nz = shape
        phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.4, seed=500 + ci)
        rec = torch.zeros((5, 16), dtype=torch.float64, device="cuda")
        with lf2.System(shape, ncomp, prec) as s:
            s.upload(phi0, np.zeros_like(phi0))
            lf2.lf2_leapfrog_init(s.phi, s.pi, p)
            lf2.lf2_leapfrog_energy(s.phi, s.pi, p, 5, rec.data_ptr())
            torch.cuda.synchronize()
            out[f"fused{ci}_phi"] = s.download()[0]
        out[f"fused{ci}_rec"] = rec.cpu().numpy()
    # an ensemble of three lattices
    shapes = [(24, 16, 12), (40, 24, 10), (16, 16, 16)]
    systems = [lf2.System(sh, 1, "f32k") for sh in shapes]
    try:
        for i, s in enumerate(systems):
            phi0 = inputs.gaussian_field(*shapes[i], 1, sigma=0.4, seed=600 + i)
            s.upload(phi0, np.zeros_like(phi0))
        e = lf2.lf2_ensemble_create([s.phi for s in systems], [s.pi for s in systems], [p] * 3)
        try:
            lf2.lf2_ensemble_set_config(e, depth=3, cx=2, tile_x=12, tile_y=8)
            lf2.lf2_ensemble_run(e, 7)
            torch.cuda.synchronize()
        finally:
            lf2.lf2_ensemble_destroy(e)
        for i, s in enumerate(systems):
            out[f"ens{i}_phi"] = s.download()[0]
    finally:
        for s in systems:
            s.close()
    np.savez(out_path, **out)
    try:
        violations = lf2.lf2_debug_bounds()
    except lf2.LF2Error as err:
        if err.status != lf2.LF2_ERR_UNSUPPORTED:
            raise
        violations = None
    print(json.dumps({"violations": violations, "arrays": len(out)}))


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
