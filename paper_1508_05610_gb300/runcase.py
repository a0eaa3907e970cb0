"""Run one kernel configuration on one lattice and print its throughput (one JSON line).

    python -m paper_1508_05610_gb300.runcase --n 256 --ncomp 2 --prec f32k \\
        --kernel tblock --depth 3 --cx 1 --tile 10x24 --steps 24

``--kernel tune`` lets lf2_tune choose.  The fields hold seeded Gaussian data generated on the
device; the timed region is `--steps` steps between CUDA events after `--warmup` steps.
Used to compare configurations and as the command line of the committed ncu summaries.
"""
from __future__ import annotations

import argparse
import json

KERNELS = {"auto": 0, "site": 1, "stream": 2, "tblock": 3}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[256], help="side, or nx ny nz")
    ap.add_argument("--ncomp", type=int, default=1)
    ap.add_argument("--prec", default="f32k", choices=["f64", "f32k", "f32"])
    ap.add_argument("--kernel", default="auto", choices=list(KERNELS) + ["tune"])
    ap.add_argument("--depth", type=int, default=0)
    ap.add_argument("--cx", type=int, default=0)
    ap.add_argument("--tile", default="0x0", help="tile_x x tile_y (tile_y alone matters for stream)")
    ap.add_argument("--zchunk", type=int, default=0)
    ap.add_argument("--cluster", type=int, default=0, help="CTAs per tile (thread-block cluster), tblock only")
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--op", default="leapfrog",
                    choices=["leapfrog", "derivative", "energy", "step_energy", "ensemble"],
                    help="derivative: time lf2_field_derivative along --dim; energy: time lf2_energy_device; "
                         "step_energy: time lf2_leapfrog_energy (a step with its energy record per launch); "
                         "ensemble: the 64-lattice FP32+Kahan ensemble (sides 64..192, lambda in [0.5, 2]), "
                         "--steps per graph launch, --kernel tune or tblock with --depth/--cx/--tile")
    ap.add_argument("--dim", type=int, default=0)
    ap.add_argument("--serial", action="store_true",
                    help="with --op ensemble: run the members one after another with lf2_leapfrog and "
                         "their own tuned plans instead of as one ensemble")
    args = ap.parse_args(argv)

    import torch

    from . import build, inputs, lf2
    build.build()
    lf2.load()
    if args.op == "ensemble":
        run_ensemble(args, torch, lf2, inputs)
        return
    nx, ny, nz = (args.n * 3)[:3] if len(args.n) == 1 else args.n
    stream = torch.cuda.current_stream()
    p = lf2.params(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    tx, ty = (int(v) for v in args.tile.split("x"))
    dtype = torch.float64 if args.prec == "f64" else torch.float32
    prec = lf2.PRECISIONS[args.prec]
    # every buffer the kernels use is a torch tensor borrowed through lf2_field_wrap
    phi = inputs.gaussian_field_device(nx, ny, nz, args.ncomp, sigma=0.1, dtype=dtype)
    bufs = [phi, torch.empty_like(phi)]
    if prec == lf2.LF2_F32_KAHAN:
        bufs += [torch.zeros_like(phi), torch.zeros_like(phi)]
    pis = [torch.zeros_like(phi), torch.empty_like(phi)]
    lat = lf2.lf2_lattice_create((nx, ny, nz))
    fphi = lf2.lf2_field_wrap(lat, args.ncomp, prec, [t.data_ptr() for t in bufs])
    fpi = lf2.lf2_field_wrap(lat, args.ncomp, prec, [t.data_ptr() for t in pis])
    if args.op == "derivative":
        out = torch.empty_like(phi)
        fout = lf2.lf2_field_wrap(lat, args.ncomp, prec, [out.data_ptr()])
        try:
            for _ in range(args.warmup):
                lf2.lf2_field_derivative(fphi, fout, args.dim, 1.0, stream)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.steps):
                lf2.lf2_field_derivative(fphi, fout, args.dim, 1.0, stream)
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3 / args.steps
        finally:
            for f in (fout, fphi, fpi):
                lf2.lf2_field_free(f)
            lf2.lf2_lattice_destroy(lat)
        nbytes = 2 * phi.numel() * phi.element_size()  # read src once, write dst once
        print(json.dumps({"op": "derivative", "lattice": [nx, ny, nz], "ncomp": args.ncomp, "prec": args.prec,
                          "dim": args.dim, "seconds_per_call": t, "algorithmic_GBps": nbytes / t / 1e9}))
        return
    if args.op in ("energy", "step_energy"):
        rec = torch.zeros((max(args.steps, args.warmup, 1), 16), dtype=torch.float64, device=phi.device)
        try:
            lf2.lf2_leapfrog_init(fphi, fpi, p, stream)

            def run(count):
                if args.op == "energy":
                    for j in range(count):
                        lf2.lf2_energy_device(fphi, fpi, p, rec[j].data_ptr(), stream)
                else:
                    lf2.lf2_leapfrog_energy(fphi, fpi, p, count, rec.data_ptr(), stream)
            run(args.warmup)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run(args.steps)
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3 / args.steps
        finally:
            lf2.lf2_field_free(fphi)
            lf2.lf2_field_free(fpi)
            lf2.lf2_lattice_destroy(lat)
        print(json.dumps({"op": args.op, "lattice": [nx, ny, nz], "ncomp": args.ncomp, "prec": args.prec,
                          "seconds_per_call": t, "gsu_per_s": nx * ny * nz / t / 1e9}))
        return
    try:
        lf2.lf2_leapfrog_init(fphi, fpi, p, stream)
        if args.kernel == "tune":
            cfg = {k: v for k, v in lf2.lf2_tune(fphi, fpi, p, stream=stream).items() if v}
        else:
            cfg = {"kernel": KERNELS[args.kernel], "depth": args.depth, "cx": args.cx, "tile_x": tx, "tile_y": ty,
                   "zchunk": args.zchunk, "cluster": args.cluster}
        lf2.lf2_leapfrog_ex(fphi, fpi, p, args.warmup, stream=stream, **cfg)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lf2.lf2_leapfrog_ex(fphi, fpi, p, args.steps, stream=stream, **cfg)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
    finally:
        lf2.lf2_field_free(fphi)
        lf2.lf2_field_free(fpi)
        lf2.lf2_lattice_destroy(lat)
    sites = nx * ny * nz
    print(json.dumps({"lattice": [nx, ny, nz], "ncomp": args.ncomp, "prec": args.prec, "config": cfg,
                      "steps": args.steps, "seconds": t, "gsu_per_s": sites * args.steps / t / 1e9}))


def run_ensemble(args, torch, lf2, inputs):
    """The batched ensemble: 64 real lattices with sides drawn from {64, 96, 128, 160, 192} and
    lambda uniform in [0.5, 2] (seeded), FP32 + Kahan, dt = 0.05, one graph launch per run."""
    stream = torch.cuda.current_stream()
    members = inputs.ensemble_members()
    keep, fields, plist, sites = [], [], [], 0
    for side, lam, seed in members:
        phi = inputs.gaussian_field_device(side, side, side, 1, sigma=0.1, seed=seed, dtype=torch.float32)
        pi = torch.zeros_like(phi)
        lat = lf2.lf2_lattice_create((side, side, side))
        fields.append((lat, lf2.lf2_field_wrap(lat, 1, lf2.LF2_F32_KAHAN, [phi.data_ptr()]),
                       lf2.lf2_field_wrap(lat, 1, lf2.LF2_F32_KAHAN, [pi.data_ptr()])))
        keep += [phi, pi]
        sites += side ** 3
        plist.append(lf2.params(dx=1.0, dt=0.05, lam=lam, eta=1.0))
        lf2.lf2_leapfrog_init(fields[-1][1], fields[-1][2], plist[-1], stream)
    if args.serial:
        try:
            for (lat, fphi, fpi), p in zip(fields, plist):
                lf2.lf2_tune(fphi, fpi, p, stream=stream)
                lf2.lf2_leapfrog(fphi, fpi, p, 4, stream)  # warm-up with the plan
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for (lat, fphi, fpi), p in zip(fields, plist):
                lf2.lf2_leapfrog(fphi, fpi, p, args.steps, stream)
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3
        finally:
            for lat, fphi, fpi in fields:
                lf2.lf2_field_free(fphi)
                lf2.lf2_field_free(fpi)
                lf2.lf2_lattice_destroy(lat)
        print(json.dumps({"op": "ensemble", "serial": True, "members": len(members), "sites": sites,
                          "steps": args.steps, "seconds": t, "gsu_per_s": sites * args.steps / t / 1e9}))
        return
    e = lf2.lf2_ensemble_create([f[1] for f in fields], [f[2] for f in fields], plist)
    try:
        if args.kernel in ("tune", "auto"):
            cfg = lf2.lf2_ensemble_tune(e, stream=stream)
        else:
            tx, ty = (int(v) for v in args.tile.split("x"))
            cfg = {"kernel": KERNELS[args.kernel], "depth": args.depth, "cx": args.cx, "tile_x": tx, "tile_y": ty}
            lf2.lf2_ensemble_set_config(e, **cfg)
        lf2.lf2_ensemble_run(e, args.steps, stream)  # capture + warm-up
        torch.cuda.synchronize()
        best = None
        for _ in range(3):  # best of three timed runs
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lf2.lf2_ensemble_run(e, args.steps, stream)
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3
            best = t if best is None else min(best, t)
    finally:
        lf2.lf2_ensemble_destroy(e)
        for lat, fphi, fpi in fields:
            lf2.lf2_field_free(fphi)
            lf2.lf2_field_free(fpi)
            lf2.lf2_lattice_destroy(lat)
    print(json.dumps({"op": "ensemble", "members": len(members), "sites": sites, "config": cfg,
                      "steps": args.steps, "seconds": best, "gsu_per_s": sites * args.steps / best / 1e9}))


if __name__ == "__main__":
    main()
