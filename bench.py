"""Benchmark of the leapfrog lattice-field hot path on GB300.

Workload (one GPU, or N independent replicas under torchrun): a 1536^3 complex (two real
components) phi^4 field, V = lambda/4 (|phi|^2 - eta^2)^2 with lambda = eta = 1, dx = 1,
dt = 0.05, phi0 components i.i.d. N(0, 0.1^2) (seeded), pi0 = 0, stored in FP32 with the
Kahan-compensated drift (FP64 energy reductions) and advanced by temporal-blocking passes whose
depth (1 to 8) and tiles the library's tuner picks before the timed region.  A "step" is one
leapfrog step of the whole lattice: force (7-point Laplacian + potential), kick and drift.

The line's `value` is that FP32 + Kahan path.  The same line carries the plain FP64 GPU path on
the same lattice and initial data (one step per pass, the comparison path): its throughput, its
FP64-pipe roofline and the speedup of the FP32 path over it; the FP32 path's error against the
FP64 run at step 50 (with a control: FP64 from the FP32-rounded initial data); and the energy
drift of both over 50 steps.

Metric: GSite-updates/s = sites x steps / seconds with inputs resident in HBM: the median of
five timed regions of K steps, each between CUDA events on the launch stream with a device
synchronisation on both sides.  The lattice state (174 GB) is far larger than the 129 MB L2, so
no flush is needed between steps.  The roofline counts compulsory HBM bytes per site-update of
one pass: FP32 + Kahan complex 48 B (read phi, read+write pi and the compensation, write phi'),
which a temporal-blocking pass of depth T moves once for T steps.

``--impl reference`` times the FP64 CPU oracle on the host cores instead, on a bounded slab of
the same lattice per step.
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
N_DEFAULT = 1536
NCOMP = 2
KW = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
WORKLOAD = ("phi4 complex {n}^3 periodic lattice, dt=0.05, lambda=eta=1, sigma=0.1 Gaussian phi0, pi0=0; "
            "FP32 storage with Kahan-compensated drift, FP64 energy reductions, temporal-blocking depth "
            "tuned over 1-8")
# compulsory bytes per site-update of one HBM pass (complex): phi read, phi' write, pi and the
# Kahan compensation read + write
BYTES_PER_SITE = {"f64": 8 * NCOMP * 4, "f32k": 4 * NCOMP * 6, "f32": 4 * NCOMP * 4}
FALLBACK_HBM_GBS = 6800.0
# The FP64 step issues 10 DP instructions per real site and 19 per complex site (the folded
# update of lf2_arith.cuh); the FP64 pipe issues 2 DFMA per SM per clock.
DP_INSTR_PER_SITE = {1: 10, 2: 19}
ERROR_STEP = 50        # error against FP64 and energy drift are taken at this step
ENERGY_EVERY = 10
TIMED_REGIONS = 5      # the headline is the median of this many timed regions
CPU_SLAB_Z = 16        # the CPU oracle's sample: a 1536 x 1536 x 16 periodic slab
CPU_BASELINE_STEPS = 100
CSRC = os.path.join(ROOT, "paper_1508_05610_gb300", "csrc")


def traffic_key(prec, cfg, n):
    if cfg.get("kernel") == 3:
        cl = cfg.get("cluster") or 1
        return (f"k_tblock{'_cluster' if cl > 1 else ''}_{prec}_c{NCOMP}_{n}_d{cfg.get('depth')}_cx{cfg.get('cx')}_"
                f"{cfg.get('tile_x')}x{cfg.get('tile_y')}" + (f"_cl{cl}" if cl > 1 else ""))
    return f"k_stream_{prec}_c{NCOMP}_{n}"


def measured_traffic(key):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged
    (and the note on how it was taken)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            entry = json.load(f)[key]
        h = hashlib.sha256()
        for name in entry["sources"]:
            with open(os.path.join(CSRC, name), "rb") as f:
                h.update(f.read())
        if h.hexdigest()[:16] != entry["src_sha"]:
            return None, None
        return entry["bytes"], entry.get("note")
    except (OSError, ValueError, KeyError):
        return None, None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for key in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
            if key in d:
                return float(d[key]), "measured", d.get("sm_max_mhz")
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback", None


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
    through lf2_field_wrap, so every buffer the kernels touch is visible as a tensor.  Takes
    ownership of `phi` (already in the storage type).  Temporal blocking needs back buffers of
    pi and of the compensation; the FP64 one-step path needs only phi's."""

    def __init__(self, torch, lf2, prec, phi, tblock):
        self.torch, self.lf2, self.prec = torch, lf2, lf2.PRECISIONS[prec]
        n = phi.shape[0]
        self.tensors = [phi, torch.empty_like(phi)]
        ptrs = [t.data_ptr() for t in self.tensors]
        if self.prec == lf2.LF2_F32_KAHAN:
            comp = [torch.zeros_like(phi)] + ([torch.zeros_like(phi)] if tblock else [])
            self.tensors += comp
            ptrs += [t.data_ptr() for t in comp]
        pis = [torch.zeros_like(phi)] + ([torch.empty_like(phi)] if tblock else [])
        self.tensors += pis
        self.lat = lf2.lf2_lattice_create((n, n, n))
        self.fphi = lf2.lf2_field_wrap(self.lat, NCOMP, self.prec, ptrs)
        self.fpi = lf2.lf2_field_wrap(self.lat, NCOMP, self.prec, [t.data_ptr() for t in pis])

    def _tensor(self, ptr):
        return next(t for t in self.tensors if t.data_ptr() == ptr)

    def front(self):
        return self._tensor(self.lf2.lf2_field_buffer(self.fphi, 0))

    def pi_front(self):
        return self._tensor(self.lf2.lf2_field_buffer(self.fpi, 0))

    def close(self, keep=()):
        """Frees the handles and every tensor not in `keep` (returned in that order)."""
        self.lf2.lf2_field_free(self.fphi)
        self.lf2.lf2_field_free(self.fpi)
        self.lf2.lf2_lattice_destroy(self.lat)
        self.tensors = None
        return keep


def time_regions(torch, lf2, pair, p, steps, warmup, stream, cfg, regions):
    """Half-kick, `warmup` untimed steps, then `regions` timed regions of EXACTLY `steps` leapfrog
    steps, each between CUDA events on the launch stream with a synchronisation on both sides.
    A step pass is one launch (`depth` steps under temporal blocking, one otherwise); remainder
    steps run as single-step launches.  Each pass launch is also bracketed by its own events, so
    the dominant kernel's average launch duration is measured live.  Returns (region seconds,
    average seconds of one full pass, passes per region, launches per region)."""
    lf2.lf2_leapfrog_init(pair.fphi, pair.fpi, p, stream)
    depth = cfg.get("depth", 0) if cfg.get("kernel") == lf2.LF2_KERNEL_TBLOCK else 1
    lf2.lf2_leapfrog_ex(pair.fphi, pair.fpi, p, warmup, stream=stream, **cfg)
    torch.cuda.synchronize()
    times, pass_events = [], []
    for _ in range(regions):
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(stream)
        done = 0
        while done < steps:
            k = min(depth, steps - done)
            if k == depth:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lf2.lf2_leapfrog_ex(pair.fphi, pair.fpi, p, k, stream=stream, **cfg)
                b.record(stream)
                pass_events.append((a, b))
            else:
                lf2.lf2_leapfrog_ex(pair.fphi, pair.fpi, p, k, stream=stream, **cfg)
            done += k
        stop.record(stream)
        torch.cuda.synchronize()
        times.append(start.elapsed_time(stop) / 1e3)
    per_pass = statistics.mean(a.elapsed_time(b) / 1e3 for a, b in pass_events) if pass_events else None
    passes = steps // depth
    return times, per_pass, passes, passes + steps % depth


def error_block(torch, lf2, inputs, n, p, plan32, stream, seed):
    """FP32 + Kahan against FP64 at ERROR_STEP, staged so that at most 232 GB is resident:
      1. FP32 + Kahan from float32(phi0) with the tuned plan, energies every ENERGY_EVERY steps;
         its phi and pi are kept;
      2. FP64 from phi0 on the one-step kernel, energies likewise; phi and pi errors of run 1 are
         reduced in FP64 on the device against this run's buffers (lf2_field_compare);
      3. control: FP64 from float64(float32(phi0)), its phi error against run 2's phi -- the
         error that rounding the initial data alone causes."""
    marks = list(range(0, ERROR_STEP + 1, ENERGY_EVERY))

    def evolve(pair, cfg):
        lf2.lf2_leapfrog_init(pair.fphi, pair.fpi, p, stream)
        energies, done = {}, 0
        for k in marks:
            if k > done:
                lf2.lf2_leapfrog_ex(pair.fphi, pair.fpi, p, k - done, stream=stream, **cfg)
                done = k
            energies[k] = lf2.lf2_energy(pair.fphi, pair.fpi, p, stream)["total"]
        return energies

    def drift(en):
        return max(abs(e - en[0]) / abs(en[0]) for e in en.values())

    one_step = {"kernel": lf2.LF2_KERNEL_STREAM}
    pair = WrappedPair(torch, lf2, "f32k", inputs.gaussian_field_device(n, n, n, NCOMP, sigma=0.1, seed=seed,
                                                                        dtype=torch.float32), tblock=True)
    e32 = evolve(pair, plan32)
    phi32, pi32 = pair.close(keep=(pair.front(), pair.pi_front()))
    del pair
    torch.cuda.empty_cache()

    pair = WrappedPair(torch, lf2, "f64", inputs.gaussian_field_device(n, n, n, NCOMP, sigma=0.1, seed=seed),
                       tblock=False)
    e64 = evolve(pair, one_step)
    lat = lf2.lf2_lattice_create((n, n, n))
    f32 = lf2.lf2_field_wrap(lat, NCOMP, lf2.LF2_F32_KAHAN, [phi32.data_ptr()])
    g32 = lf2.lf2_field_wrap(lat, NCOMP, lf2.LF2_F32_KAHAN, [pi32.data_ptr()])
    cphi = lf2.lf2_field_compare(f32, pair.front().data_ptr(), lf2.LF2_F64, 0, stream)
    cpi = lf2.lf2_field_compare(g32, pair.pi_front().data_ptr(), lf2.LF2_F64, 0, stream)
    lf2.lf2_field_free(f32)
    lf2.lf2_field_free(g32)
    (phi64,) = pair.close(keep=(pair.front(),))
    del pair, phi32, pi32
    torch.cuda.empty_cache()

    ctl0 = inputs.gaussian_field_device(n, n, n, NCOMP, sigma=0.1, seed=seed, dtype=torch.float32).double()
    torch.cuda.empty_cache()
    pair = WrappedPair(torch, lf2, "f64", ctl0, tblock=False)
    lf2.lf2_leapfrog_init(pair.fphi, pair.fpi, p, stream)
    lf2.lf2_leapfrog_ex(pair.fphi, pair.fpi, p, ERROR_STEP, stream=stream, **one_step)
    cctl = lf2.lf2_field_compare(pair.fphi, phi64.data_ptr(), lf2.LF2_F64, 0, stream)
    pair.close()
    lf2.lf2_lattice_destroy(lat)
    del pair, phi64, ctl0
    torch.cuda.empty_cache()
    k = ERROR_STEP
    return {
        "step": k,
        "phi_relmax": cphi["relmax"], "phi_rel_l2": cphi["rel_l2"],
        "pi_relmax": cpi["relmax"], "pi_rel_l2": cpi["rel_l2"],
        "energy_rel": abs(e32[k] - e64[k]) / abs(e64[k]),
        "control_phi_relmax": cctl["relmax"],
        "phi_relmax_over_control": cphi["relmax"] / cctl["relmax"] if cctl["relmax"] > 0 else None,
        "energy_drift_max": {"f32k": float(f"{drift(e32):.3e}"), "f64": float(f"{drift(e64):.3e}")},
        "energy_every": ENERGY_EVERY,
    }


def pin_host(torch, arr):
    """Page-locks a numpy array in place (exact size, no allocator rounding)."""
    rt = torch.cuda.cudart()
    err = rt.cudaHostRegister(arr.ctypes.data, arr.nbytes, 0)
    code = err.value if hasattr(err, "value") else int(err)
    if code != 0:
        raise RuntimeError(f"cudaHostRegister failed ({code})")


def unpin_host(torch, arr):
    torch.cuda.cudart().cudaHostUnregister(arr.ctypes.data)


def e2e_run(torch, lf2, inputs, n, p, steps, warmup, stream, seed, dist, world):
    """End to end through the public C API with host buffers: upload phi and pi (FP64 host arrays,
    the API's host format, converted to FP32 on the device) from page-locked memory, half-kick,
    `steps` steps with the tuned plan, the energy read-back, download of phi and pi.  The
    downloads reuse the upload buffers (2 x 58 GB of page-locked host memory)."""
    import numpy as np
    need = 2 * n ** 3 * NCOMP * 8
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = None
    local_ranks = int(os.environ.get("LOCAL_WORLD_SIZE", "1"))
    if avail is not None and avail < need * local_ranks + (16 << 30):
        return None, f"host memory: {avail / 2**30:.0f} GiB free, {need * local_ranks / 2**30:.0f} GiB needed"
    host_phi = np.empty((n, n, n, NCOMP), dtype=np.float64)
    host_pi = np.zeros_like(host_phi)
    dev = inputs.gaussian_field_device(n, n, n, NCOMP, sigma=0.1, seed=seed)
    torch.from_numpy(host_phi).copy_(dev)
    del dev
    torch.cuda.empty_cache()
    pin_host(torch, host_phi)
    pin_host(torch, host_pi)
    shape = host_phi.shape
    try:
        with lf2.System((n, n, n), NCOMP, "f32k") as s:
            def once(nsteps):
                lf2.lf2_field_upload(s.phi, host_phi, stream)
                lf2.lf2_field_upload(s.pi, host_pi, stream)
                lf2.lf2_leapfrog_init(s.phi, s.pi, p, stream)
                lf2.lf2_leapfrog(s.phi, s.pi, p, nsteps, stream)
                lf2.lf2_energy(s.phi, s.pi, p, stream)
                lf2.lf2_field_download(s.phi, shape, stream, out=host_phi)
                lf2.lf2_field_download(s.pi, shape, stream, out=host_pi)
            once(warmup)
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            once(steps)
            torch.cuda.synchronize()
            t = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    finally:
        unpin_host(torch, host_phi)
        unpin_host(torch, host_pi)
    state = n ** 3 * NCOMP * 8 * 2
    return {"value": round(aggregate_gsu(n ** 3, world, steps, t), 3), "unit": UNIT,
            "h2d_bytes_per_step": state / steps, "d2h_bytes_per_step": (state + 8 * 16) / steps,
            "seconds": round(t, 3),
            "note": "per run: upload phi, pi (FP64 host arrays from page-locked memory, converted to FP32 on the "
                    "device) + half-kick + K steps (tuned plan) + energy read-back + download of phi, pi into "
                    "the same host arrays"}, None


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
    n = args.lattice
    sites = n ** 3
    p = lf2.params(**KW)
    hbm_peak, peak_src, peaks_sm_mhz = peaks()
    seed = replica_seed(rank)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # FP32 + Kahan: the tuner times candidates on a proxy copy of the lattice's first planes
    # before any timed region; the FP64 comparison path runs the one-step streaming kernel
    pair = WrappedPair(torch, lf2, "f32k", inputs.gaussian_field_device(n, n, n, NCOMP, sigma=0.1, seed=seed,
                                                                        dtype=torch.float32), tblock=True)
    t_tune = time.perf_counter()
    plan32 = {k: v for k, v in lf2.lf2_tune(pair.fphi, pair.fpi, p, stream=stream).items() if v}
    t_tune = time.perf_counter() - t_tune
    cfgs = {"f32k": plan32, "f64": {"kernel": lf2.LF2_KERNEL_STREAM}}

    res = {}
    with ClockSampler(local) as clocks:
        barrier()
        res["f32k"] = time_regions(torch, lf2, pair, p, args.steps, args.warmup, stream, plan32, TIMED_REGIONS)
        pair.close()
        del pair
        torch.cuda.empty_cache()
        pair = WrappedPair(torch, lf2, "f64", inputs.gaussian_field_device(n, n, n, NCOMP, sigma=0.1, seed=seed),
                           tblock=False)
        barrier()
        res["f64"] = time_regions(torch, lf2, pair, p, args.steps, args.warmup, stream, cfgs["f64"], TIMED_REGIONS)
        pair.close()
        del pair
        torch.cuda.empty_cache()
    clk = clocks.summary()
    med = {prec: max_over_ranks(statistics.median(r[0]), dist, "cuda") for prec, r in res.items()}

    err = error_block(torch, lf2, inputs, n, p, plan32, stream, seed) if not args.no_error else None
    e2e, e2e_skip = (None, "skipped (--no-e2e)")
    if not args.no_e2e:
        e2e, e2e_skip = e2e_run(torch, lf2, inputs, n, p, args.steps, args.warmup, stream, seed, dist, world)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    def gsu(t):
        return aggregate_gsu(sites, world, args.steps, t)

    # roofline of the dominant kernel: a temporal-blocking pass of `depth` steps moves the
    # compulsory bytes of one step once (B1 x sites); achieved = those bytes / the pass's
    # average duration (CUDA events around each pass launch in the timed regions)
    times32, pass32, passes32, launches32 = res["f32k"]
    depth = plan32.get("depth", 1) if plan32.get("kernel") == lf2.LF2_KERNEL_TBLOCK else 1
    b1 = BYTES_PER_SITE["f32k"]
    achieved = b1 * sites / pass32 / 1e9
    tkey = traffic_key("f32k", plan32, n)
    traffic, traffic_note = measured_traffic(tkey)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
                "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "kernel": ("k_tblock_cluster" if (plan32.get("cluster") or 1) > 1 else "k_tblock") if depth > 1
                else "k_stream",
                "bytes_per_site_update_one_pass": b1, "steps_per_launch": depth,
                "algorithmic_bytes_per_launch": b1 * sites, "launch_seconds_avg": pass32,
                "one_pass_equivalent": round(b1 * gsu(statistics.median(times32)) / hbm_peak, 4),
                "one_pass_equivalent_note": "GSU/s x B1 / peak: the bandwidth a one-pass-per-step code would need "
                                            "for the same throughput; not the roofline fraction"}
    if traffic is not None:
        roofline["traffic_note"] = traffic_note
        roofline["dram_bytes_per_site_update"] = round(traffic / (sites * depth), 2)
    if depth > 1:
        # sites each stage computes per output site in the x-y plane: the tile plus its halo
        # (depth rows, depth columns rounded up to whole thread groups), over whole tiles
        tp = -(-depth // plan32["cx"]) * plan32["cx"]
        ntx, nty = -(-n // plan32["tile_x"]), -(-n // plan32["tile_y"])
        roofline["halo_redundancy_xy"] = round(
            ntx * nty * (plan32["tile_x"] + 2 * tp) * (plan32["tile_y"] + 2 * depth) / (n * n), 3)

    times64, pass64, _, launches64 = res["f64"]
    sm_mhz = clk.get("sm_mhz") or peaks_sm_mhz or 2070.0
    max_mhz = clk.get("sm_max_mhz") or peaks_sm_mhz or 2070.0
    fp64_peak = 2 * sms * max_mhz / 1e3  # G DP instructions/s
    ginst = DP_INSTR_PER_SITE[NCOMP] * sites / pass64 / 1e9
    hbm64 = BYTES_PER_SITE["f64"] * sites / pass64 / 1e9
    t64 = med["f64"]
    t32 = med["f32k"]
    fp64 = {"value": round(gsu(t64), 3), "unit": UNIT, "ms_per_step": round(t64 / args.steps * 1e3, 4),
            "kernel": "k_stream (one step per launch)",
            "region_seconds": [round(x, 5) for x in times64],
            "roofline": {"bound": "alu", "achieved": round(ginst, 1), "peak": round(fp64_peak, 1),
                         "unit": "G FP64 instr/s", "frac": round(ginst / fp64_peak, 4),
                         "frac_at_sampled_clock": round(ginst / (2 * sms * sm_mhz / 1e3), 4),
                         "peak_source": f"2 DFMA/clk/SM x {sms} SMs x {max_mhz:.0f} MHz (device SM count, max SM clock)",
                         "dp_instr_per_site_update": DP_INSTR_PER_SITE[NCOMP],
                         "hbm": {"achieved": round(hbm64, 1), "peak": hbm_peak, "frac": round(hbm64 / hbm_peak, 4)}},
            "launches_per_region": launches64}
    line = {
        "metric": METRIC, "value": round(gsu(t32), 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t32 / args.steps * 1e3, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Gaussian phi0, pi0 = 0)",
        "config": {"workload": WORKLOAD.format(n=n), "lattice": [n, n, n], "ncomp": NCOMP, "sites": sites,
                   "precision": "f32 + Kahan-compensated drift (FP64 energy)", "plan": plan32,
                   "parallelism": f"replicas x{world}",
                   "l2_policy": "state 174 GB > 129 MB L2; no flush needed",
                   "timing": f"median of {TIMED_REGIONS} timed regions of K steps",
                   "seed": replica_seed(0), "seed_rule": "rank r uses seed + r"},
        "region_seconds": [round(x, 5) for x in times32],
        "region_spread": round((max(times32) - min(times32)) / statistics.median(times32), 4),
        "roofline": roofline,
        "kernel": (f"k_tblock{'_cluster' if (plan32.get('cluster') or 1) > 1 else ''} (depth {depth}, "
                   f"{plan32.get('tile_x')}x{plan32.get('tile_y')} tiles, cx {plan32.get('cx')}, "
                   f"{plan32.get('cluster') or 1} CTA per tile)") if depth > 1 else "k_stream",
        "tune_seconds": round(t_tune, 2),
        "fp64": fp64,
        "speedup_vs_fp64": round(t64 / t32, 3),
        "error_vs_fp64": err,
        "e2e": e2e if e2e is not None else {"value": None, "unit": UNIT, "h2d_bytes_per_step": None,
                                            "d2h_bytes_per_step": None, "skipped": e2e_skip},
        "gpu_launches": launches32,
        "gpu_launches_note": f"launches of liblf2 kernels in one timed region of K steps ({TIMED_REGIONS} regions timed)",
        "clocks": clk,
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ CPU baseline arm
def oracle_slab(n, steps, warmup, threads):
    """FP64 CPU oracle on an n x n x CPU_SLAB_Z periodic slab of the workload: `warmup` untimed
    steps after the half-kick, then `steps` timed steps in one call of the oracle's own loop.
    Returns (GSite-updates/s, seconds)."""
    from oracle import oracle
    from paper_1508_05610_gb300 import inputs
    phi0 = inputs.gaussian_field(n, n, CPU_SLAB_Z, NCOMP, sigma=0.1, seed=inputs.BASE_SEED)
    phi, pi = oracle.evolve(phi0, phi0 * 0.0, warmup, half_kick=True, threads=threads, **KW)
    t0 = time.perf_counter()
    oracle.evolve(phi, pi, steps, threads=threads, **KW)
    dt = time.perf_counter() - t0
    return n * n * CPU_SLAB_Z * steps / dt / 1e9, dt


def cpu_baseline(n):
    threads = os.cpu_count() or 1
    v, dt = oracle_slab(n, CPU_BASELINE_STEPS, 0, threads)
    return {"value": round(v, 5), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"FP64 oracle, {CPU_BASELINE_STEPS} steps of a {n}x{n}x{CPU_SLAB_Z} periodic slab of the "
                      f"workload (OpenMP over z-planes, {threads} threads), {dt:.1f} s"}


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
    n = args.lattice
    threads = os.cpu_count() or 1
    v, dt = oracle_slab(n, args.steps, args.warmup, threads)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian phi0, pi0 = 0)",
            "config": {"workload": WORKLOAD.format(n=n), "lattice": [n, n, n], "ncomp": NCOMP,
                       "sample_lattice": [n, n, CPU_SLAB_Z],
                       "note": "FP64 CPU oracle; each step is one leapfrog step of a periodic slab of the lattice"},
            "cpu_baseline": {"value": round(v, 5), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step: one leapfrog step of a {n}x{n}x{CPU_SLAB_Z} periodic slab "
                                       f"(OpenMP over z-planes, {threads} threads); the timed steps run in one "
                                       "oracle call"},
            "e2e": {"value": round(v, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lf2", choices=["lf2", "reference"])
    ap.add_argument("--lattice", type=int, default=N_DEFAULT, help="lattice side (the workload is 1536)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-error", action="store_true", help="skip the error-vs-FP64 block")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end run through host buffers")
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
