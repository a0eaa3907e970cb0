"""Stated error of the FP32 paths against FP64 on full-size lattices (one JSON line).

    python -m paper_1508_05610_gb300.errorstudy --n 1024 --ncomp 1 --init grf --steps 2000 \\
        --compare-at 10 100 2000
    python -m paper_1508_05610_gb300.errorstudy --n 1536 --ncomp 2 --init gauss --steps 200 \\
        --compare-at 50 --energy-every 10

Three GPU runs from one seeded initial field phi0 (pi0 = 0), all through the C ABI:
  * FP64 reference from phi0 (one-step kernel), with FP64 snapshots of phi (and pi when memory
    allows) at the comparison steps and its energy every `--energy-every` steps;
  * FP32 (compensated drift by default, tuned kernel plan) from float32(phi0), compared with
    the snapshots;
  * control: FP64 from float64(float32(phi0)) -- the FP32 rounding of the initial data alone --
    compared with the snapshots.  The FP32 error divided by the control error says how much of
    the FP32 error is the dynamics amplifying the input rounding (about 1) and how much is
    arithmetic (well above 1).
Runs are staged so that at most one field state plus the snapshots is resident.  Errors are
max-norm and 2-norm relative errors, reduced in FP64 on the device by lf2_field_compare.
"""
from __future__ import annotations

import argparse
import json
import math
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--ncomp", type=int, default=1)
    ap.add_argument("--init", default="gauss", choices=["gauss", "grf"])
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--compare-at", type=int, nargs="+", default=[10, 100])
    ap.add_argument("--energy-every", type=int, default=0)
    ap.add_argument("--prec", default="f32k", choices=["f32k", "f32"])
    ap.add_argument("--dt", type=float, default=0.05)
    ap.add_argument("--lam", type=float, default=1.0)
    ap.add_argument("--eta", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=None)
    args = ap.parse_args(argv)

    import torch

    from . import build, inputs, lf2
    build.build()
    lf2.load()
    seed = inputs.BASE_SEED if args.seed is None else args.seed
    n, c = args.n, args.ncomp
    p = lf2.params(dx=1.0, dt=args.dt, lam=args.lam, eta=args.eta)
    stream = torch.cuda.current_stream()
    compare = sorted(set(k for k in args.compare_at if k <= args.steps))
    state_bytes64 = n ** 3 * c * 8
    free = torch.cuda.mem_get_info()[0]
    snap_pi = free > 3 * state_bytes64 + 2 * len(compare) * state_bytes64 + (8 << 30)

    def phi0_fp64():
        if args.init == "grf":
            if c != 1:
                raise SystemExit("the Gaussian random field initial condition is for real fields")
            return inputs.grf_field_device(n, sigma=0.1, seed=seed)
        return inputs.gaussian_field_device(n, n, n, c, sigma=0.1, seed=seed)

    class Run:
        """phi / pi with every buffer a torch tensor borrowed by the library."""

        def __init__(self, prec, phi0, tblock):
            # one-step kernels need phi, its back buffer and pi; temporal blocking also needs
            # back buffers of pi and of the compensation
            self.prec = lf2.PRECISIONS[prec]
            self.bufs = [phi0, torch.empty_like(phi0)]
            if self.prec == lf2.LF2_F32_KAHAN:
                self.bufs += [torch.zeros_like(phi0)] + ([torch.zeros_like(phi0)] if tblock else [])
            self.pis = [torch.zeros_like(phi0)] + ([torch.empty_like(phi0)] if tblock else [])
            self.lat = lf2.lf2_lattice_create((n, n, n))
            self.fphi = lf2.lf2_field_wrap(self.lat, c, self.prec, [t.data_ptr() for t in self.bufs])
            self.fpi = lf2.lf2_field_wrap(self.lat, c, self.prec, [t.data_ptr() for t in self.pis])

        def phi(self):
            ptr = lf2.lf2_field_buffer(self.fphi, 0)
            return next(t for t in self.bufs if t.data_ptr() == ptr)

        def pi(self):
            ptr = lf2.lf2_field_buffer(self.fpi, 0)
            return next(t for t in self.pis if t.data_ptr() == ptr)

        def close(self):
            lf2.lf2_field_free(self.fphi)
            lf2.lf2_field_free(self.fpi)
            lf2.lf2_lattice_destroy(self.lat)
            self.bufs = self.pis = None

    def errors(field, ref):
        """(max |f - ref| / max |ref|, ||f - ref|| / ||ref||) of the field's current values
        against an FP64 device snapshot, reduced in FP64 by the library (lf2_field_compare)."""
        d = lf2.lf2_field_compare(field, ref.data_ptr(), lf2.LF2_F64, 0, stream)
        return d["relmax"], d["rel_l2"]

    def evolve(run, cfg, snapshots=None, compare_with=None, energy_every=0, until=None):
        """Runs to `until` steps; records energies, snapshots, or errors against snapshots."""
        out = {"energy": {}, "errors": {}}
        lf2.lf2_leapfrog_init(run.fphi, run.fpi, p, stream)
        marks = set(compare)
        if energy_every:
            marks |= set(range(0, until + 1, energy_every))
        marks = sorted(k for k in marks if k <= until)
        done = 0
        t_run = 0.0
        for k in marks:
            if k > done:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                lf2.lf2_leapfrog_ex(run.fphi, run.fpi, p, k - done, stream=stream, **cfg)
                torch.cuda.synchronize()
                t_run += time.perf_counter() - t0
                done = k
            if energy_every and k % energy_every == 0 or k in compare:
                out["energy"][k] = lf2.lf2_energy(run.fphi, run.fpi, p, stream, ncomp=c)["total"]
            if k in compare and snapshots is not None:
                snapshots[k] = (run.phi().clone(), run.pi().clone() if snap_pi else None, out["energy"][k])
            if k in compare and compare_with is not None:
                ref_phi, ref_pi, ref_e = compare_with[k]
                e_phi = errors(run.fphi, ref_phi)
                row = {"phi_relmax": e_phi[0], "phi_rel_l2": e_phi[1],
                       "energy_rel": abs(out["energy"][k] - ref_e) / abs(ref_e)}
                if ref_pi is not None:
                    e_pi = errors(run.fpi, ref_pi)
                    row.update({"pi_relmax": e_pi[0], "pi_rel_l2": e_pi[1]})
                out["errors"][k] = row
        out["seconds"] = t_run
        out["gsu_per_s"] = n ** 3 * until / t_run / 1e9 if t_run > 0 else None
        return out

    def drift(energies):
        e0 = energies[0]
        return max(abs(e - e0) / abs(e0) for e in energies.values())

    one_step = {"kernel": lf2.LF2_KERNEL_STREAM}
    result = {"lattice": [n, n, n], "ncomp": c, "init": args.init, "steps": args.steps, "compare_at": compare,
              "prec": args.prec, "dt": args.dt, "snapshots_of_pi": snap_pi}

    # 1. FP64 reference
    snaps = {}
    run = Run("f64", phi0_fp64(), tblock=False)
    ref = evolve(run, one_step, snapshots=snaps, energy_every=args.energy_every, until=args.steps)
    run.close()
    del run
    torch.cuda.empty_cache()
    result["fp64"] = {"gsu_per_s": ref["gsu_per_s"], "energy_drift_max": drift(ref["energy"])
                      if args.energy_every else None}

    # 2. FP32 path from float32(phi0), tuned plan
    phi32 = phi0_fp64().float()
    torch.cuda.empty_cache()
    run = Run(args.prec, phi32, tblock=True)
    plan = {k: v for k, v in lf2.lf2_tune(run.fphi, run.fpi, p, stream=stream).items() if v}
    low = evolve(run, plan, compare_with=snaps, energy_every=args.energy_every, until=args.steps)
    run.close()
    del run, phi32
    torch.cuda.empty_cache()
    result["fp32"] = {"plan": plan, "gsu_per_s": low["gsu_per_s"], "errors": low["errors"],
                      "energy_drift_max": drift(low["energy"]) if args.energy_every else None}

    # 3. control: FP64 from float64(float32(phi0))
    phic = phi0_fp64().float().double()
    torch.cuda.empty_cache()
    run = Run("f64", phic, tblock=False)
    ctl = evolve(run, one_step, compare_with=snaps, until=max(compare))
    run.close()
    del run, phic
    result["control_fp64_from_fp32_rounded_phi0"] = {"errors": ctl["errors"]}
    result["fp32_over_control_phi_relmax"] = {
        k: (low["errors"][k]["phi_relmax"] / ctl["errors"][k]["phi_relmax"]) if ctl["errors"][k]["phi_relmax"] > 0
        else None for k in compare}
    print(json.dumps(result))


if __name__ == "__main__":
    main()
