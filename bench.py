"""Benchmark of the leapfrog lattice-field hot path on GB300.

Workload (one GPU, or N independent replicas under torchrun): a 256^3 complex (two real
components) phi^4 field, V = lambda/4 (|phi|^2 - eta^2)^2 with lambda = eta = 1, dx = 1,
dt = 0.05, phi0 components i.i.d. N(0, 0.1^2) (seeded), pi0 = 0.  A "step" is one leapfrog
step of the whole lattice: force (7-point Laplacian + potential), kick and drift.

The headline line times the FP64 path with the plain one-step-per-pass kernel (no temporal
blocking).  The same line carries the FP32 path with the Kahan-compensated drift on the same
lattice and initial data: its throughput, roofline fraction, speedup over FP64 and its error
against the FP64 run.  The lattice state (805 MB FP64, 402 MB FP32+Kahan) is larger than the
129 MB L2, so no flush is needed between steps.

Metric: GSite-updates/s = sites x steps / seconds, with inputs resident in HBM.  The roofline
counts compulsory HBM bytes per site-update: FP64 complex 64 B (read phi, read+write pi, write
phi'), FP32+Kahan complex 48 B (plus read+write of the compensation).

``--impl reference`` times the FP64 CPU oracle on the host cores instead (a bounded slab of the
same lattice per step).
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GSite-updates/s per leapfrog step and % of HBM roofline, FP32 vs FP64 at stated error"
UNIT = "GSite-updates/s"
N = 256
NCOMP = 2
KW = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
WORKLOAD = "phi4 complex 256^3 periodic lattice, dt=0.05, lambda=eta=1, sigma=0.1 Gaussian init"
BYTES_PER_SITE = {"f64": 8 * NCOMP * 4, "f32k": 4 * NCOMP * 6, "f32": 4 * NCOMP * 4}
FALLBACK_HBM_GBS = 6800.0
# FP64 is bound by the FP64 pipe on GB300: the nominal 1.25 TFLOP/s FP64 rate is 2 DFMA per SM
# per clock x 152 SMs x 2.07 GHz = 629 G DP instructions/s.  The FP64 step issues 10 DP
# instructions per real site and 19 per complex site (lf2_internal.cuh, update_f64).
FP64_PEAK_GINST = 2 * 152 * 2.07
DP_INSTR_PER_SITE = {1: 10, 2: 19}
CSRC = os.path.join(ROOT, "paper_1508_05610_gb300", "csrc")


def traffic_key(prec, cfg):
    if cfg.get("kernel") == 3:
        return (f"k_tblock_{prec}_c{NCOMP}_{N}_d{cfg.get('depth')}_cx{cfg.get('cx')}_"
                f"{cfg.get('tile_x')}x{cfg.get('tile_y')}")
    return f"k_stream_{prec}_c{NCOMP}_{N}"


def measured_traffic(key):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            entry = json.load(f)[key]
        h = hashlib.sha256()
        for name in entry["sources"]:
            with open(os.path.join(CSRC, name), "rb") as f:
                h.update(f.read())
        return entry["bytes"] if h.hexdigest()[:16] == entry["src_sha"] else None
    except (OSError, ValueError, KeyError):
        return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for key in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
            if key in d:
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        if shutil.which("nvidia-smi"):
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.tmp:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------- multi-rank helpers
def rank_info():
    """(rank, world size, local rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(t, dist, device):
    """Slowest rank's time: replicas are timed independently and the job takes the maximum."""
    if dist is None:
        return t
    import torch
    x = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def replica_seed(rank):
    """Each replica evolves its own lattice: seeds differ per rank."""
    from paper_1508_05610_gb300 import inputs
    return inputs.BASE_SEED + rank


def aggregate_gsu(sites, world, steps, seconds):
    """Whole-job throughput: every rank's site-updates over the slowest rank's time."""
    return sites * world * steps / seconds / 1e9


# ------------------------------------------------------------------- GPU arm helpers
class WrappedPair:
    """phi and pi (and their back buffers) as torch device tensors, borrowed by the library
    through lf2_field_wrap, so every buffer the kernels touch is visible as a tensor."""

    def __init__(self, torch, lf2, prec, phi0):
        self.torch, self.lf2, self.prec = torch, lf2, lf2.PRECISIONS[prec]
        dtype = torch.float64 if prec == "f64" else torch.float32
        self.phi = phi0.to(dtype=dtype, copy=True).contiguous()
        self.tensors = [self.phi, torch.empty_like(self.phi)]
        ptrs = [t.data_ptr() for t in self.tensors]
        if self.prec == lf2.LF2_F32_KAHAN:
            comp = [torch.zeros_like(self.phi), torch.zeros_like(self.phi)]
            self.tensors += comp
            ptrs += [t.data_ptr() for t in comp]
        pis = [torch.zeros_like(self.phi), torch.empty_like(self.phi)]
        self.tensors += pis
        self.lat = lf2.lf2_lattice_create((N, N, N))
        self.fphi = lf2.lf2_field_wrap(self.lat, NCOMP, self.prec, ptrs)
        self.fpi = lf2.lf2_field_wrap(self.lat, NCOMP, self.prec, [t.data_ptr() for t in pis])

    def _tensor(self, ptr):
        return next(t for t in self.tensors if t.data_ptr() == ptr)

    def front(self):
        return self._tensor(self.lf2.lf2_field_buffer(self.fphi, 0))

    def pi_front(self):
        return self._tensor(self.lf2.lf2_field_buffer(self.fpi, 0))

    def close(self):
        self.lf2.lf2_field_free(self.fphi)
        self.lf2.lf2_field_free(self.fpi)
        self.lf2.lf2_lattice_destroy(self.lat)


def time_steps(torch, lf2, pair, p, steps, warmup, stream, cfg):
    """Warm-up, then EXACTLY `steps` leapfrog steps between CUDA events on the launch stream.
    With a one-step kernel each step is one launch; with temporal blocking the steps go in
    passes of `depth` (one launch each) plus single steps for the remainder."""
    lf2.lf2_leapfrog_init(pair.fphi, pair.fpi, p, stream)
    depth = cfg.get("depth", 0) if cfg.get("kernel") == lf2.LF2_KERNEL_TBLOCK else 1
    for _ in range(warmup):
        lf2.lf2_leapfrog_ex(pair.fphi, pair.fpi, p, depth, stream=stream, **cfg)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    done = 0
    while done < steps:
        n = min(depth, steps - done)
        lf2.lf2_leapfrog_ex(pair.fphi, pair.fpi, p, n, stream=stream, **cfg)
        done += n
    stop.record(stream)
    torch.cuda.synchronize()
    launches = steps // depth + steps % depth
    return start.elapsed_time(stop) / 1e3, launches


def run_gpu(args):
    import torch

    from paper_1508_05610_gb300 import build, inputs, lf2

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    lf2.load()
    stream = torch.cuda.current_stream()
    sites = N ** 3
    p = lf2.params(**KW)
    hbm_peak, peak_src = peaks()

    phi0 = inputs.gaussian_field_device(N, N, N, NCOMP, sigma=0.1, seed=replica_seed(rank))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()


    # kernel configurations: FP64 on the plain one-step streaming kernel; FP32+Kahan tuned
    # (the tuner times candidates on a copy of the lattice before the timed region)
    cfgs = {"f64": {"kernel": lf2.LF2_KERNEL_STREAM}}
    tune_pair = WrappedPair(torch, lf2, "f32k", phi0)
    cfgs["f32k"] = {k: v for k, v in lf2.lf2_tune(tune_pair.fphi, tune_pair.fpi, p, stream=stream).items() if v}
    tune_pair.close()
    del tune_pair

    results, launches = {}, {}
    with ClockSampler(local) as clocks:
        for prec in ("f64", "f32k"):
            pair = WrappedPair(torch, lf2, prec, phi0)
            barrier()
            t, nl = time_steps(torch, lf2, pair, p, args.steps, args.warmup, stream, cfgs[prec])
            results[prec], launches[prec] = max_over_ranks(t, dist, "cuda"), nl
            pair.close()
            del pair
            torch.cuda.empty_cache()
    clk = clocks.summary()

    # error of the FP32+Kahan path against FP64 after 10 and 100 steps from the same data
    err = {}
    pairs = {prec: WrappedPair(torch, lf2, prec, phi0) for prec in ("f64", "f32k")}
    done = 0
    for prec in pairs:
        lf2.lf2_leapfrog_init(pairs[prec].fphi, pairs[prec].fpi, p, stream)
    e0 = {prec: lf2.lf2_energy(pairs[prec].fphi, pairs[prec].fpi, p, stream)["total"] for prec in pairs}
    drift = {prec: 0.0 for prec in pairs}
    for n in (10, 100):
        for prec in pairs:
            lf2.lf2_leapfrog_ex(pairs[prec].fphi, pairs[prec].fpi, p, n - done, stream=stream, **cfgs[prec])
        done = n
        e64 = lf2.lf2_energy(pairs["f64"].fphi, pairs["f64"].fpi, p, stream)
        e32 = lf2.lf2_energy(pairs["f32k"].fphi, pairs["f32k"].fpi, p, stream)
        for prec, e in (("f64", e64), ("f32k", e32)):
            drift[prec] = max(drift[prec], abs(e["total"] - e0[prec]) / abs(e0[prec]))
        # FP64 error norms on the device (lf2_field_compare) against the FP64 run's buffers
        cphi = lf2.lf2_field_compare(pairs["f32k"].fphi, pairs["f64"].front().data_ptr(), lf2.LF2_F64, 0, stream)
        cpi = lf2.lf2_field_compare(pairs["f32k"].fpi, pairs["f64"].pi_front().data_ptr(), lf2.LF2_F64, 0, stream)
        err[str(n)] = {"phi_relmax": cphi["relmax"], "phi_rel_l2": cphi["rel_l2"],
                       "pi_relmax": cpi["relmax"], "pi_rel_l2": cpi["rel_l2"],
                       "energy_rel": abs(e32["total"] - e64["total"]) / abs(e64["total"])}
    for pair in pairs.values():
        pair.close()
    del pairs
    torch.cuda.empty_cache()

    # end to end through the public C API with host buffers: upload from pinned host memory,
    # init, K steps, energy read-back, download of phi and pi.
    host_phi = torch.empty((N, N, N, NCOMP), dtype=torch.float64, pin_memory=True)
    host_phi.copy_(phi0)
    host_pi = torch.zeros_like(host_phi).pin_memory()
    out_phi = torch.empty_like(host_phi).pin_memory()
    out_pi = torch.empty_like(host_phi).pin_memory()
    import ctypes
    dptr = ctypes.POINTER(ctypes.c_double)
    with lf2.System((N, N, N), NCOMP, "f64") as s:
        lib = lf2.load()
        def e2e_once(nsteps):
            lib.lf2_field_upload(s.phi, ctypes.cast(host_phi.data_ptr(), dptr), stream.cuda_stream)
            lib.lf2_field_upload(s.pi, ctypes.cast(host_pi.data_ptr(), dptr), stream.cuda_stream)
            lf2.lf2_leapfrog_init(s.phi, s.pi, p, stream)
            lf2.lf2_leapfrog(s.phi, s.pi, p, nsteps, stream)
            lf2.lf2_energy(s.phi, s.pi, p, stream)
            lib.lf2_field_download(s.phi, ctypes.cast(out_phi.data_ptr(), dptr), stream.cuda_stream)
            lib.lf2_field_download(s.pi, ctypes.cast(out_pi.data_ptr(), dptr), stream.cuda_stream)
        e2e_once(args.warmup)
        barrier()
        t0 = time.perf_counter()
        e2e_once(args.steps)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    state_bytes = N ** 3 * NCOMP * 8 * 2

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    def gsu(t):
        return aggregate_gsu(sites, world, args.steps, t)

    def roof(prec, t, traffic_key):
        # one launch = one pass over HBM = `depth` steps; algorithmic bytes of a pass are the
        # one-step compulsory bytes (read phi, pi, comp; write them once)
        depth = cfgs[prec].get("depth", 1) if cfgs[prec].get("kernel") == lf2.LF2_KERNEL_TBLOCK else 1
        per_step = t / args.steps
        achieved = BYTES_PER_SITE[prec] * sites / (per_step * depth) / 1e9
        hbm = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
               "frac": round(achieved / hbm_peak, 4), "traffic": measured_traffic(traffic_key),
               "peak_source": f"{peak_src} HBM copy bandwidth",
               "bytes_per_site_update": BYTES_PER_SITE[prec], "steps_per_launch": depth,
               "effective_frac": round(BYTES_PER_SITE[prec] * sites / per_step / 1e9 / hbm_peak, 4)}
        if hbm["traffic"] is not None:
            # ncu DRAM bytes of one launch per site-update it performs
            hbm["dram_bytes_per_site_update"] = round(hbm["traffic"] / (sites * depth), 2)
        if depth > 1:
            # sites each stage computes per output site in the x-y plane: the tile plus its halo
            # (depth rows, depth columns rounded up to whole thread groups), over whole tiles
            c = cfgs[prec]
            tp = -(-depth // c["cx"]) * c["cx"]
            ntx, nty = -(-N // c["tile_x"]), -(-N // c["tile_y"])
            hbm["halo_redundancy_xy"] = round(
                ntx * nty * (c["tile_x"] + 2 * tp) * (c["tile_y"] + 2 * depth) / (N * N), 3)
        if prec != "f64":
            return hbm
        ginst = DP_INSTR_PER_SITE[NCOMP] * sites / per_step / 1e9
        return {"bound": "alu", "achieved": round(ginst, 1), "peak": round(FP64_PEAK_GINST, 1),
                "unit": "G FP64 instr/s", "frac": round(ginst / FP64_PEAK_GINST, 4),
                "traffic": hbm["traffic"], "peak_source": "nominal FP64 rate 1.25 TFLOP/s = 2 DFMA/clk/SM x 152 SMs x 2.07 GHz",
                "dp_instr_per_site_update": DP_INSTR_PER_SITE[NCOMP], "hbm": {k: hbm[k] for k in ("achieved", "peak", "frac", "dram_bytes_per_site_update") if k in hbm}}

    t64, t32 = results["f64"], results["f32k"]
    line = {
        "metric": METRIC, "value": round(gsu(t64), 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t64 / args.steps * 1e3, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Gaussian phi0)",
        "config": {"workload": WORKLOAD + ", FP64, one step per HBM pass (plain path)", "lattice": [N, N, N],
                   "ncomp": NCOMP, "sites": sites, "precision": "f64", "parallelism": f"replicas x{world}",
                   "l2_policy": "state 805 MB > 129 MB L2; no flush needed",
                   "seed": replica_seed(0), "seed_rule": "rank r uses seed + r"},
        "roofline": roof("f64", t64, "k_stream_f64_c2_256"),
        "kernel": "k_stream (one step per launch)",
        "fp32_kahan": {"value": round(gsu(t32), 3), "unit": UNIT, "ms_per_step": round(t32 / args.steps * 1e3, 5),
                       "roofline": roof("f32k", t32, traffic_key("f32k", cfgs["f32k"])),
                       "plan": cfgs["f32k"], "launches": launches["f32k"], "speedup_vs_fp64": round(t64 / t32, 3),
                       "error_vs_fp64": err,
                       "energy_drift_max_100_steps": {k: float(f"{v:.3e}") for k, v in drift.items()}},
        "e2e": {"value": round(aggregate_gsu(sites, world, args.steps, t_e2e), 3), "unit": UNIT,
                "h2d_bytes_per_step": state_bytes / args.steps, "d2h_bytes_per_step": (state_bytes + 64) / args.steps,
                "note": "upload phi,pi from pinned host + half-kick + K steps + energy + download, per step"},
        "gpu_launches": launches["f64"],
        "clocks": clk,
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ CPU baseline arm
def oracle_rate(nz_slab, steps, threads):
    """FP64 CPU oracle on a 256 x 256 x nz_slab periodic slab of the workload."""
    from oracle import oracle
    from paper_1508_05610_gb300 import inputs
    phi0 = inputs.gaussian_field(N, N, nz_slab, NCOMP, sigma=0.1, seed=inputs.BASE_SEED)
    pi0 = phi0 * 0.0
    phi, pi = oracle.evolve(phi0, pi0, 0, half_kick=True, threads=threads, **KW)
    t0 = time.perf_counter()
    oracle.evolve(phi, pi, steps, threads=threads, **KW)
    dt = time.perf_counter() - t0
    return N * N * nz_slab * steps / dt / 1e9, dt


def cpu_baseline():
    threads = os.cpu_count() or 1
    # 250 steps of the full lattice: about 11 s on 16 Grace cores
    nz_slab, steps = 256, 250
    v, dt = oracle_rate(nz_slab, steps, threads)
    return {"value": round(v, 5), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"FP64 oracle, {steps} steps of the 256x256x{nz_slab} complex lattice "
                      f"(OpenMP over z-planes), {dt:.1f} s"}


def oracle_table():
    """The CPU oracle on the workloads of the baseline plan, on this host's cores (one JSON
    line): the 32^3 real lattice (dt 0.1, 100 steps) on one thread and on all threads, the
    256^3 complex lattice for 10 steps and the 1024^3 real lattice for 2 steps on all threads.
    The threaded runs are bitwise equal to single-thread ones (OpenMP over z-planes)."""
    from oracle import oracle
    from paper_1508_05610_gb300 import inputs
    threads = os.cpu_count() or 1
    rows = []
    for n, c, dt, steps, th in ((32, 1, 0.1, 100, 1), (32, 1, 0.1, 100, threads), (256, 2, 0.05, 10, threads),
                                (1024, 1, 0.05, 2, threads)):
        kw = dict(dx=1.0, dt=dt, lam=1.0, eta=1.0, m2=0.0)
        phi0 = inputs.gaussian_field(n, n, n, c, sigma=0.1, seed=inputs.BASE_SEED)
        phi, pi = oracle.evolve(phi0, phi0 * 0.0, 0, half_kick=True, threads=th, **kw)
        del phi0
        t0 = time.perf_counter()
        oracle.evolve(phi, pi, steps, threads=th, **kw)
        sec = time.perf_counter() - t0
        del phi, pi
        rows.append({"lattice": [n, n, n], "ncomp": c, "steps": steps, "threads": th, "seconds": round(sec, 3),
                     "gsu_per_s": round(n ** 3 * steps / sec / 1e9, 5)})
    print(json.dumps({"oracle_table": rows, "cores": threads, "unit": UNIT}))


def run_reference(args):
    rank = rank_info()[0]
    if rank != 0:  # the CPU reference runs once, on rank 0
        return
    threads = os.cpu_count() or 1
    nz_slab = 64  # several z-planes per host thread
    from oracle import oracle
    from paper_1508_05610_gb300 import inputs
    phi0 = inputs.gaussian_field(N, N, nz_slab, NCOMP, sigma=0.1, seed=inputs.BASE_SEED)
    phi, pi = oracle.evolve(phi0, phi0 * 0.0, 0, half_kick=True, threads=threads, **KW)
    phi, pi = oracle.evolve(phi, pi, args.warmup, threads=threads, **KW)
    # the K timed steps run in the oracle's own loop (one call), so per-call array conversion
    # is not counted as stepping time
    t0 = time.perf_counter()
    phi, pi = oracle.evolve(phi, pi, args.steps, threads=threads, **KW)
    dt = time.perf_counter() - t0
    sites = N * N * nz_slab
    v = sites * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian phi0)",
            "config": {"workload": WORKLOAD + ", FP64 CPU oracle", "lattice": [N, N, nz_slab], "ncomp": NCOMP},
            "cpu_baseline": {"value": round(v, 5), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step: one leapfrog step of a 256x256x{nz_slab} periodic slab"},
            "e2e": {"value": round(v, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lf2", choices=["lf2", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--oracle-table", action="store_true",
                    help="time the CPU oracle on the baseline plan's workloads (host only) and exit")
    args = ap.parse_args()
    if args.oracle_table:
        oracle_table()
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
