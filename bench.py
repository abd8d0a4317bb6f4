"""Benchmark: rays/s of GB300 inverse ray-shooting on the paper-shaped mid-size
workload (kappa_* = 0.45, kappa_s = 0, gamma = 0.45, 1e5 Salpeter lenses in
0.1-1 rescaled to kappa_*, 2000^2 map over 20 x 20 theta_E, 100 rays per
unlensed pixel: 1.12e10 rays per map).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--method interp|brute]
                  [--impl ours|reference]

One step = one magnification map through irs_make_map (INTERP: mass sum, cell
lists, far field, ray pass, binning, magnification).  The plain brute-force map of the
same workload costs ~1e15 pair terms (minutes), so it is timed on a band of
lattice rows through irs_make_map_rows and reported per ray, with the same
band made by the interpolated method as the accuracy check (per-pixel
magnification relative RMS over pixels with >= 100 rays).

Multi-GPU: maps are independent problems, so by default each rank makes its
own map (weak scaling, no collective on the data path); value = all ranks'
rays / the slowest rank's time.  --shard strips makes ONE map over all ranks
(strong scaling): each rank shoots a strip of whole cell rows and the count
maps are summed (one all-reduce per map, inside the timed step).

The default run (one GPU, paper-mid interp) adds three sub-records to its
line, measured after the timed steps: "high_res" (the 1e6-lens, 10000^2,
9.6e10-ray workload: whole-map rays/s, ray-pass roofline, error and speed-up
against a brute-force band), "learned" (the learned far field's workload:
learned and series forms against a brute-force band) and "batched" (256
uneven maps in one captured graph against one call per map).  --no-extra
skips them.

--study accuracy | planes | border replays the paper's accuracy-vs-rays slope,
its rectangular vs circular lens plane comparison and its protective-border
deflection distribution (one GPU; one JSON line each).

--impl reference times the FP64 CPU oracle (the plain definition the GPU path
is checked against) on a bounded sample of the same workload on the host
cores.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="paper-mid: kappa*=0.45 kappa_s=0 gamma=0.45, 1e5 Salpeter lenses, "
                     "2000^2 px over 20x20 thetaE, 100 rays/px",
                kappa_star=0.45, kappa_s=0.0, gamma=0.45, S=20.0, npix=2000, nav=100.0,
                n_star=100000, shape="salpeter", seed=2)
# high resolution: 1e6 lenses, 1e8-pixel map (count map larger than L2)
WORKLOAD_HIGHRES = dict(name="high-res: kappa*=0.35 kappa_s=0.15 gamma=0.4, 1e6 uniform lenses 0.1-1, "
                             "10000^2 px over 25x25 thetaE, 40 rays/px",
                        kappa_star=0.35, kappa_s=0.15, gamma=0.4, S=25.0, npix=10000, nav=40.0,
                        n_star=1000000, shape="uniform", seed=3)
# the learned far field's workload
WORKLOAD_LEARNED = dict(name="learned: kappa*=0.4 kappa_s=0.1 gamma=0.35, 2e5 equal-mass lenses, "
                             "4000^2 px over 20x20 thetaE, 64 rays/px",
                        kappa_star=0.4, kappa_s=0.1, gamma=0.35, S=20.0, npix=4000, nav=64.0,
                        n_star=200000, shape="equal", seed=5)
BRUTE_ROWS = 256            # band of lattice rows for the brute-force timing
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # the timed region starts once the sampler is producing lines
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
            self.lines.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def slowest_rank_ms(my_ms, dist, device):
    """Max over ranks of this rank's timed milliseconds (the job ends with the slowest)."""
    import torch
    t = torch.tensor([float(my_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rays_per_s(rays_per_step_per_rank, world, ms_per_step):
    """Weak scaling: every rank makes its own map, so the job shoots world x the rays."""
    return rays_per_step_per_rank * world / (ms_per_step * 1e-3)


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_params(irs, method, w=WORKLOAD):
    S = w["S"]
    m = {"interp": irs.IRS_INTERP, "brute": irs.IRS_BRUTE, "mlp": irs.IRS_MLP}[method]
    return irs.make_params(w["kappa_star"], w["kappa_s"], w["gamma"], (-S / 2, S / 2, -S / 2, S / 2),
                           w["npix"], w["nav"], n_star=w["n_star"], method=m)


def lens_field(lensgen, box, seed, w=WORKLOAD):
    area = (box[1] - box[0]) * (box[3] - box[2])
    return lensgen.lens_field(w["n_star"], box, shape=w["shape"], seed=seed,
                              total_mass=w["kappa_star"] * area / np.pi)


# ------------------------------------------------------------------ ours
# Per-ray work of the interpolated ray pass, in flops: 10 per near pair (the
# same pair arithmetic as the brute force), 8 per complex multiply-add of the
# level-2 Horner (K2 - 1 of them for K2 series terms), and 20 for the smooth
# terms, sub-cell index and pixel.
IP_VARIANT_K2 = [6, 7, 6, 6, 6, 6, 6, 6, 6, 8, 6, 5, 5, 5, 5, 5, 4]  # series terms K2 of ray-pass variants 0..16
IP_FLOPS_OTHER = 20


def ip_flops_fixed(variant):
    return 8 * (IP_VARIANT_K2[variant] - 1) + IP_FLOPS_OTHER


# DRAM bytes per launch of the ray pass (ncu dram__bytes_read.sum +
# dram__bytes_write.sum), valid only for the kernel build, workload and cell
# size they were captured on: (workload, cell multiplier, variant) -> bytes.
# Source: profiles/k_ip_ray_paper-mid-full.md.
IP_TRAFFIC = {("paper-mid", 0.57, 11): 106.890752e6 + 3.025408e6,
              ("paper-mid", 0.57, 13): 107.035136e6 + 3.787776e6,
              ("paper-mid", 0.57, 14): 106.874368e6 + 3.572224e6,
              ("paper-mid", 0.57, 16): 106.763776e6 + 4.427264e6}


def mean_near_lenses(info, xy):
    """Mean over rays of the lenses in a ray's 3x3 block of level-1 cells."""
    h = info.cell_x
    ncx, ncy = info.ncell_x, info.ncell_y
    gx0 = info.lens_x0 - 0.0  # rectangular plane: grid origin = plane corner
    gy0 = info.lens_y0
    cx = np.clip(np.floor((xy[:, 0] - gx0) / h).astype(np.int64), 0, ncx - 1)
    cy = np.clip(np.floor((xy[:, 1] - gy0) / h).astype(np.int64), 0, ncy - 1)
    cnt = np.zeros((ncy + 2, ncx + 2))
    np.add.at(cnt, (cy + 1, cx + 1), 1.0)
    blk = sum(cnt[1 + dy:1 + dy + ncy, 1 + dx:1 + dx + ncx] for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    k = info.rays_per_cell_x
    wx = np.full(ncx, k, dtype=np.float64)
    wx[-1] = info.n_rays_x - k * (ncx - 1)
    wy = np.full(ncy, k, dtype=np.float64)
    wy[-1] = info.n_rays_y - k * (ncy - 1)
    w = wy[:, None] * wx[None, :]
    return float((blk * w).sum() / w.sum())


def run_ours(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_init()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2204_10871_gb300 import build as libbuild
    libbuild.build()
    from paper_2204_10871_gb300 import irs, lensgen

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(local)
    n_sms = props.multi_processor_count
    named = {"paper-mid": WORKLOAD, "high-res": WORKLOAD_HIGHRES, "learned": WORKLOAD_LEARNED}
    w = dict(named[args.workload] if args.workload else
             (WORKLOAD_LEARNED if args.method == "mlp" else WORKLOAD))
    if args.n_star:
        w["n_star"] = args.n_star
    if args.npix:
        w["npix"] = args.npix
    if args.nav:
        w["nav"] = args.nav
    full = args.method != "brute"

    params = workload_params(irs, args.method, w)
    probe = irs.Plan(params)  # the lens plane does not depend on the tuning
    box = (probe.info.lens_x0, probe.info.lens_x1, probe.info.lens_y0, probe.info.lens_y1)
    probe.close()
    sharded = args.shard == "strips" and full
    # replicas: a map per rank (own lens field); strips: one map over all ranks
    xy, m = lens_field(lensgen, box, w["seed"] + (0 if sharded else 1000 * rank), w)
    dxy = torch.from_numpy(xy).to(dev)
    dm = torch.from_numpy(m).to(dev)
    torch.cuda.synchronize()
    t_cold0 = time.perf_counter()  # cold start: tuning (cache miss), plan, first map
    tune = None
    if args.variant >= 0:
        params.kernel_variant = args.variant
        if args.cell_mult > 0:
            params.cell_mult = args.cell_mult
    elif args.method == "interp" and not args.no_tune:  # untimed: pick cell size and ray-pass variant
        t0 = time.perf_counter()
        params, res = irs.irs_autotune(params, dxy, dm)
        tune = {"cell_mult": res.cell_mult, "kernel_variant": res.kernel_variant,
                "candidates": res.candidates, "est_ms_tuned": res.ms_per_map,
                "est_ms_default": res.ms_default, "from_cache": bool(res.from_cache),
                "tuning_s": time.perf_counter() - t0}
    plan = irs.Plan(params)
    info = plan.info
    learned = None
    if args.method == "mlp":  # untimed: train the network on this lens field
        rep = irs.irs_mlp_train(plan.handle, dxy, dm, seed=11)
        learned = {"samples": rep.samples, "steps": rep.steps, "loss_first": rep.loss_first,
                   "loss_final": rep.loss_final, "heldout_rel_rms": rep.valid_rel_rms,
                   "target_rms_thetaE": rep.target_rms, "ms_samples": rep.ms_samples,
                   "ms_train": rep.ms_train}
    shape = (w["npix"], w["npix"])
    counts = torch.zeros(shape, dtype=torch.uint32, device=dev)
    mag = torch.zeros(shape, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    irs.irs_plan_set_timing(plan.handle, True)
    band_rows = args.band_rows or BRUTE_ROWS
    r0 = (info.n_rays_y // 2 // 64) * 64  # whole brute tiles (64 rows)
    band = (r0, min(info.n_rays_y, r0 + band_rows))

    from paper_2204_10871_gb300 import shard

    def step():
        if sharded:  # this rank's strip of rows, then the sum of the count maps
            shard.make_map_sharded(plan, dxy, dm, counts, world, rank, mag=mag)
        elif full:
            irs.irs_make_map(plan.handle, dxy, dm, counts, mag)
        else:
            counts.zero_()
            irs.irs_make_map_rows(plan.handle, dxy, dm, band[0], band[1], counts)

    rays_per_step = info.n_rays if full else (band[1] - band[0]) * info.n_rays_x
    my_rays = rays_per_step  # rays this rank shoots per step
    if sharded:
        s0, s1 = shard.strip_rows(int(info.n_rays_y), world, rank, shard.row_align(plan))
        my_rays = (s1 - s0) * info.n_rays_x
    step()  # the first map of this workload: the end of its cold start
    plan.sync()
    cold_start_s = time.perf_counter() - t_cold0
    for _ in range(args.warmup - 1):
        step()
    plan.sync()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    ray_ms, tot_ms, launches = [], [], 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))  # evict L2 between timed steps
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            t = irs.irs_plan_timings(plan.handle)  # events of this map (syncs on them)
            ray_ms.append(t.ms_raypass)
            tot_ms.append(t.ms_total)
            launches += t.launches
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
    plan.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    my_ms = float(np.sum(step_ms))
    if world > 1:
        my_ms = slowest_rank_ms(my_ms, dist, dev)
        dist.barrier()
    ms_per_step = my_ms / args.steps
    value = (rays_per_step / (ms_per_step * 1e-3) if sharded
             else whole_job_rays_per_s(rays_per_step, world, ms_per_step))

    # ---- end to end through the public API with host buffers
    h_xy = torch.from_numpy(xy).pin_memory()
    h_m = torch.from_numpy(m).pin_memory()
    h_counts = torch.empty(shape, dtype=torch.uint32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        dxy.copy_(h_xy, non_blocking=True)
        dm.copy_(h_m, non_blocking=True)
        step()
        h_counts.copy_(counts, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    if world > 1:
        e2e_ms = slowest_rank_ms(e2e_ms, dist, dev)
    e2e_value = (rays_per_step / (e2e_ms * 1e-3) if sharded
                 else whole_job_rays_per_s(rays_per_step, world, e2e_ms))
    h2d = xy.nbytes + m.nbytes
    d2h = h_counts.numel() * 4
    clocks = clk.summary()

    # ---- roofline of the dominant kernel (the ray pass): FP32 ALU bound
    pk = peaks() or {}
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    peak_tflops = n_sms * 128 * 2 * sm_max * 1e6 / 1e12
    ray_ms_mean = float(np.mean(ray_ms))
    traffic = None
    if full:
        n_near = mean_near_lenses(info, xy)
        variant = int(params.kernel_variant)
        flops_per_ray = 10.0 * n_near + ip_flops_fixed(variant)
        kname = f"k_ip_ray variant {variant} (near pair sum + level-2 Horner, FP32 pipe + MUFU)"
        key = (w["name"].split(":")[0], round(float(params.cell_mult or 1.0), 2), variant)
        if key in IP_TRAFFIC:
            traffic = IP_TRAFFIC[key]
    else:
        n_near = None
        flops_per_ray = 10.0 * w["n_star"]
        kname = "k_brute (pair sum, FP32 pipe + MUFU)"
    achieved = flops_per_ray * my_rays / (ray_ms_mean * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                "peak_basis": f"{n_sms} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                              "(max SM clock of MEASURED_PEAKS.json)",
                "flops_per_ray": flops_per_ray}
    if n_near is not None:
        roofline["mean_near_lenses"] = n_near
    if clocks.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = achieved / (n_sms * 256 * clocks["sm_mhz"] * 1e6 / 1e12)

    # ---- brute force on a band of the same lattice: rays/s and the accuracy reference
    brute = None
    if full and not args.no_brute and rank == 0:
        brute = brute_band(irs, torch, w, xy, m, dxy, dm, band, plan, n_sms, peak_tflops, value)
    if learned is not None and rank == 0:
        # the series form on the same workload, and its error on the same band
        pi = irs.Plan(workload_params(irs, "interp", w))
        irs.irs_plan_set_timing(pi.handle, True)
        ms = []
        for k in range(3):
            irs.irs_make_map(pi.handle, dxy, dm, counts, mag)
            t = irs.irs_plan_timings(pi.handle)
            if k:
                ms.append(t.ms_total)
        learned["interp_rays_per_s"] = info.n_rays / (float(np.mean(ms)) * 1e-3)
        if brute is not None:
            learned["interp_map_rel_rms_vs_brute"] = band_rel_rms(irs, torch, pi, dxy, dm, band, shape)
        pi.close()

    # ---- the other workloads of the hot path, one GPU: high resolution, the
    # batched persistent launch, the learned far field (sub-records)
    extra = {}
    if world == 1 and args.method == "interp" and not args.no_extra and not (args.n_star or args.npix or args.nav):
        extra["high_res"] = high_res_record(irs, torch, lensgen, n_sms, peak_tflops, flush)
        torch.cuda.empty_cache()
        extra["learned"] = learned_record(irs, torch, lensgen, flush)
        torch.cuda.empty_cache()
        extra["batched"] = batched_measure(torch, irs, lensgen, 256, 1, 3)
        torch.cuda.empty_cache()

    if rank == 0:
        cpu = cpu_baseline(xy, m, w) if (world == 1 and not args.no_cpu) else None
        line = {
            "metric": "rays/s per GB300 (" + args.method + ")",
            "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None,
            "dtype": "f32 (pairs), f64 (far field, setup)",
            "data": "synthetic (seeded lens fields; the paper's lens catalogues are not public)",
            "config": {"workload": w["name"] if not (args.n_star or args.npix or args.nav)
                       else "reduced case for profiling", "method": args.method,
                       "rays_per_step": rays_per_step, "n_star": w["n_star"], "npix": w["npix"],
                       "rays_per_pixel": w["nav"],
                       "band_rows": None if full else [int(band[0]), int(band[1])],
                       "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"{'strips' if sharded else 'replicas'} x{world}"},
            "e2e": {"value": e2e_value, "unit": "rays/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "autotune": tune,
            "cold_start": {"s": cold_start_s,
                           "includes": "autotuning (no cache), plan creation, first map, wall clock; "
                                       "lens field already on the device"},
            "learned": learned if learned is not None else extra.get("learned"),
            "high_res": extra.get("high_res"),
            "batched": extra.get("batched"),
            "roofline": roofline,
            "clocks": clocks,
            "stage_ms": {"raypass_mean": ray_ms_mean, "map_total_mean": float(np.mean(tot_ms)),
                         "wall_s": wall},
            "brute": brute,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


BRUTE_BAND_MAP = {}


def band_rel_rms(irs, torch, plan, dxy, dm, band, shape):
    """Per-pixel magnification rel RMS of `plan` against the last brute band map."""
    a = BRUTE_BAND_MAP["counts"]
    c = torch.zeros(shape, dtype=torch.uint32, device=dxy.device)
    irs.irs_make_map_rows(plan.handle, dxy, dm, band[0], band[1], c)
    plan.sync()
    b = c.cpu().numpy().astype(np.float64)
    sel = a >= 100
    r = (b[sel] - a[sel]) / a[sel]
    return float(np.sqrt(np.mean(r * r))) if sel.any() else None


def brute_band(irs, torch, w, xy, m, dxy, dm, band, plan_fast, n_sms, peak_tflops, fast_value):
    """Brute force over `band` rows: rays/s, its kernel's FP32 fraction, and the
    per-pixel magnification relative RMS of the fast method on the same rays
    (pixels with >= 100 rays)."""
    dev = dxy.device
    shape = (w["npix"], w["npix"])
    pb = irs.Plan(workload_params(irs, "brute", w))
    irs.irs_plan_set_timing(pb.handle, True)
    cb = torch.zeros(shape, dtype=torch.uint32, device=dev)
    ms = []
    for k in range(3):
        cb.zero_()
        irs.irs_make_map_rows(pb.handle, dxy, dm, band[0], band[1], cb)
        t = irs.irs_plan_timings(pb.handle)
        if k:
            ms.append((t.ms_total, t.ms_raypass))
    pb.sync()
    rays = (band[1] - band[0]) * pb.info.n_rays_x
    tot = float(np.mean([a for a, _ in ms]))
    ray = float(np.mean([b for _, b in ms]))
    ach = 10.0 * len(m) * rays / (ray * 1e-3) / 1e12
    cf = torch.zeros(shape, dtype=torch.uint32, device=dev)
    irs.irs_make_map_rows(plan_fast.handle, dxy, dm, band[0], band[1], cf)
    plan_fast.sync()
    a = cb.cpu().numpy().astype(np.float64)
    b = cf.cpu().numpy().astype(np.float64)
    sel = a >= 100
    rel = (b[sel] - a[sel]) / a[sel]
    pb.close()
    value = rays / (tot * 1e-3)
    BRUTE_BAND_MAP["counts"] = a
    return {"value": value, "unit": "rays/s", "band_rows": [int(band[0]), int(band[1])],
            "rays": int(rays), "ms_per_band": tot,
            "roofline": {"bound": "alu", "kernel": "k_brute", "achieved": ach, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": ach / peak_tflops},
            "speedup_of_fast_method": fast_value / value,
            "map_rel_rms_vs_brute": float(np.sqrt(np.mean(rel * rel))) if sel.any() else None,
            "pixels_compared": int(sel.sum()), "min_rays_per_pixel": 100}


def timed_maps(irs, torch, plan, dxy, dm, counts, mag, flush, reps=3):
    """Mean CUDA-event time (ms) of a whole map and of its ray pass over `reps`
    maps after one warm-up map, with L2 flushed before each."""
    irs.irs_plan_set_timing(plan.handle, True)
    irs.irs_make_map(plan.handle, dxy, dm, counts, mag)
    plan.sync()
    tot, ray = [], []
    for k in range(reps):
        flush.fill_(float(k))
        irs.irs_make_map(plan.handle, dxy, dm, counts, mag)
        t = irs.irs_plan_timings(plan.handle)
        tot.append(t.ms_total)
        ray.append(t.ms_raypass)
    plan.sync()
    return float(np.mean(tot)), float(np.mean(ray))


def band_pair(irs, torch, w, dxy, dm, band, plans_fast):
    """The brute force over lattice rows `band` (timed once, CUDA events) and
    the same rows made by each plan of `plans_fast`: brute rays/s and each
    fast map's per-pixel magnification rel RMS against the brute force over
    pixels with >= 100 rays."""
    shape = (w["npix"], w["npix"])
    pb = irs.Plan(workload_params(irs, "brute", w))
    irs.irs_plan_set_timing(pb.handle, True)
    cb = torch.zeros(shape, dtype=torch.uint32, device=dxy.device)
    irs.irs_make_map_rows(pb.handle, dxy, dm, band[0], band[1], cb)
    t = irs.irs_plan_timings(pb.handle)
    pb.sync()
    rays = (band[1] - band[0]) * pb.info.n_rays_x
    pb.close()
    a = cb.cpu().numpy().astype(np.float64)
    del cb
    sel = a >= 100
    rels = []
    for pf in plans_fast:
        c = torch.zeros(shape, dtype=torch.uint32, device=dxy.device)
        irs.irs_make_map_rows(pf.handle, dxy, dm, band[0], band[1], c)
        pf.sync()
        b = c.cpu().numpy().astype(np.float64)
        del c
        r = (b[sel] - a[sel]) / a[sel]
        rels.append(float(np.sqrt(np.mean(r * r))) if sel.any() else None)
    return {"rays_per_s": rays / (t.ms_total * 1e-3), "band_rows": [int(band[0]), int(band[1])],
            "rays": int(rays), "ms": float(t.ms_total), "ms_raypass": float(t.ms_raypass),
            "pixels_compared": int(sel.sum())}, rels


def high_res_record(irs, torch, lensgen, n_sms, peak_tflops, flush):
    """The high-resolution workload (1e6 lenses, 10000^2 map, 40 rays/px,
    9.6e10 rays; the 400 MB count map is larger than L2), autotuned: whole-map
    rays/s, the ray pass's FP32 roofline, and the per-pixel magnification rel
    RMS against the brute force on a 64-row band (one brute-force tile row)."""
    w = WORKLOAD_HIGHRES
    dev = torch.device("cuda", torch.cuda.current_device())
    params = workload_params(irs, "interp", w)
    with irs.Plan(params) as probe:
        box = (probe.info.lens_x0, probe.info.lens_x1, probe.info.lens_y0, probe.info.lens_y1)
    xy, m = lens_field(lensgen, box, w["seed"], w)
    dxy, dm = torch.from_numpy(xy).to(dev), torch.from_numpy(m).to(dev)
    t0 = time.perf_counter()
    params, res = irs.irs_autotune(params, dxy, dm)
    tune_s = time.perf_counter() - t0
    plan = irs.Plan(params)
    info = plan.info
    shape = (w["npix"], w["npix"])
    counts = torch.zeros(shape, dtype=torch.uint32, device=dev)
    mag = torch.zeros(shape, dtype=torch.float32, device=dev)
    ms_map, ms_ray = timed_maps(irs, torch, plan, dxy, dm, counts, mag, flush)
    del counts, mag
    variant = int(params.kernel_variant)
    n_near = mean_near_lenses(info, xy)
    flops = 10.0 * n_near + ip_flops_fixed(variant)
    ach = flops * info.n_rays / (ms_ray * 1e-3) / 1e12
    r0 = (info.n_rays_y // 2 // 64) * 64
    brute, (rel,) = band_pair(irs, torch, w, dxy, dm, (r0, r0 + 64), [plan])
    plan.close()
    value = info.n_rays / (ms_map * 1e-3)
    brute_ach = 10.0 * w["n_star"] * brute["rays"] / (brute["ms_raypass"] * 1e-3) / 1e12
    return {"workload": w["name"], "value": value, "unit": "rays/s", "n_rays": int(info.n_rays),
            "ms_per_map": ms_map, "ms_raypass": ms_ray,
            "autotune": {"cell_mult": res.cell_mult, "kernel_variant": res.kernel_variant,
                         "candidates": res.candidates, "tuning_s": tune_s},
            "roofline": {"bound": "alu", "kernel": f"k_ip_ray variant {variant}", "achieved": ach,
                         "peak": peak_tflops, "unit": "TFLOP/s", "frac": ach / peak_tflops,
                         "flops_per_ray": flops, "mean_near_lenses": n_near},
            "brute": dict(brute, roofline_frac=brute_ach / peak_tflops),
            "speedup_over_brute": value / brute["rays_per_s"],
            "map_rel_rms_vs_brute": rel, "min_rays_per_pixel": 100}


def learned_record(irs, torch, lensgen, flush):
    """The learned far field's workload (2e5 equal-mass lenses, 4000^2 map, 64
    rays/px): the network trained on this lens field (untimed), whole-map
    rays/s of the learned and of the series form, and each one's per-pixel
    magnification rel RMS against the brute force on a 256-row band."""
    w = WORKLOAD_LEARNED
    dev = torch.device("cuda", torch.cuda.current_device())
    pm = workload_params(irs, "mlp", w)
    plan = irs.Plan(pm)
    info = plan.info
    box = (info.lens_x0, info.lens_x1, info.lens_y0, info.lens_y1)
    xy, m = lens_field(lensgen, box, w["seed"], w)
    dxy, dm = torch.from_numpy(xy).to(dev), torch.from_numpy(m).to(dev)
    rep = irs.irs_mlp_train(plan.handle, dxy, dm, seed=11)
    pi = irs.Plan(workload_params(irs, "interp", w))
    shape = (w["npix"], w["npix"])
    counts = torch.zeros(shape, dtype=torch.uint32, device=dev)
    mag = torch.zeros(shape, dtype=torch.float32, device=dev)
    ms_mlp, _ = timed_maps(irs, torch, plan, dxy, dm, counts, mag, flush)
    ms_int, _ = timed_maps(irs, torch, pi, dxy, dm, counts, mag, flush)
    del counts, mag
    r0 = (info.n_rays_y // 2 // 64) * 64
    brute, (rel_mlp, rel_int) = band_pair(irs, torch, w, dxy, dm, (r0, r0 + 256), [plan, pi])
    plan.close()
    pi.close()
    v_mlp, v_int = info.n_rays / (ms_mlp * 1e-3), info.n_rays / (ms_int * 1e-3)
    return {"workload": w["name"], "n_rays": int(info.n_rays),
            "network": {"samples": rep.samples, "steps": rep.steps, "heldout_rel_rms": rep.valid_rel_rms,
                        "target_rms_thetaE": rep.target_rms, "loss_first": rep.loss_first,
                        "loss_final": rep.loss_final, "ms_samples": rep.ms_samples, "ms_train": rep.ms_train},
            "learned": {"value": v_mlp, "unit": "rays/s", "ms_per_map": ms_mlp,
                        "map_rel_rms_vs_brute": rel_mlp, "speedup_over_brute": v_mlp / brute["rays_per_s"]},
            "interp": {"value": v_int, "unit": "rays/s", "ms_per_map": ms_int,
                       "map_rel_rms_vs_brute": rel_int, "speedup_over_brute": v_int / brute["rays_per_s"]},
            "brute": brute, "bar_rel_rms": 1e-3, "min_rays_per_pixel": 100}


def cpu_baseline(xy, m, w, target_s=15.0):
    """The FP64 oracle timed on this host's cores on a bounded band of the same
    lattice (all lenses, a few thousand rays)."""
    import oracle
    S = w["S"]
    po = oracle.make_params(w["kappa_star"], w["kappa_s"], w["gamma"], (-S / 2, S / 2, -S / 2, S / 2),
                            w["npix"], w["nav"])
    qo = oracle.size(po)
    cores = os.cpu_count() or 1
    r0 = qo.nry // 2
    rows = cores
    t0 = time.perf_counter()
    probe = 64
    oracle.make_map(po, qo, xy, m, rows=(r0, r0 + rows), cols=(0, probe), threads=cores)
    dt = time.perf_counter() - t0
    cols = int(max(probe, min(qo.nrx, probe * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.make_map(po, qo, xy, m, rows=(r0, r0 + rows), cols=(0, cols), threads=cores)
    dt = time.perf_counter() - t0
    rays = rows * cols
    return {"value": rays / dt, "unit": "rays/s", "cores": cores, "kind": "oracle",
            "sample": f"{rows} lattice rows x {cols} rays ({rays} rays, all {len(m)} lenses, "
                      f"FP64 brute force) in {dt:.1f} s"}


# ------------------------------------------------------------------ studies
# Measurements the paper reports beside its speed figures, replayed on
# synthetic lens fields: the accuracy-vs-rays slope (Sec. 3.3, fig. Accuracy),
# the rectangular vs the circular lens plane (Sec. 2.2) and the deflection
# perturbation behind the protective border (Sec. 2.3, fig. Proscale).

def log_binned_rms(n, err, nbins=300, n_max=None, min_count=30):
    """RMS of `err` in logarithmic bins of the per-pixel ray count `n` (n >= 1).
    Returns (bin centres, rms, pixels per bin) for bins with >= min_count pixels."""
    n = np.asarray(n, dtype=np.float64)
    err = np.asarray(err, dtype=np.float64)
    keep = n >= 1
    n, err = n[keep], err[keep]
    top = float(n_max if n_max else n.max())
    edges = np.logspace(0.0, np.log10(top) + 1e-9, nbins + 1)
    idx = np.clip(np.searchsorted(edges, n, side="right") - 1, 0, nbins - 1)
    cnt = np.bincount(idx, minlength=nbins)
    sq = np.bincount(idx, weights=err * err, minlength=nbins)
    sn = np.bincount(idx, weights=n, minlength=nbins)
    ok = cnt >= min_count
    return sn[ok] / cnt[ok], np.sqrt(sq[ok] / cnt[ok]), cnt[ok]


def loglog_slope(x, y, w=None):
    """Least-squares slope of log10 y against log10 x (weights w)."""
    lx, ly = np.log10(np.asarray(x, float)), np.log10(np.asarray(y, float))
    w = np.ones_like(lx) if w is None else np.asarray(w, float)
    mx, my = np.average(lx, weights=w), np.average(ly, weights=w)
    return float(np.sum(w * (lx - mx) * (ly - my)) / np.sum(w * (lx - mx) ** 2))


def katz_density(u, n_lens, c=1.454, npts=20001):
    """Density per unit area of the deflection perturbation in units of
    phi_0 = sqrt(kappa_*): Katz et al.'s Eq. 13 with numerator c (3.05 in
    Katz; 1.454 in the paper's modified form, Sec. 2.3):
        rho(u) = (1/2pi) int_0^x* x J0(x u) exp[-(x^2/2) ln(c sqrt(N)/x)] dx.
    The form is asymptotic: the exponent is most negative at
    x* = c sqrt(N) e^-1/2 (where it equals -x*^2/4) and rises beyond, so the
    integral stops there, or earlier where the integrand is below e^-60."""
    from scipy.special import j0
    xs = c * np.sqrt(n_lens) * np.exp(-0.5)
    # end where the integrand is below e^-60, if that comes before x*
    xg = np.linspace(1e-6, xs, 100001)
    past = np.nonzero(0.5 * xg * xg * np.log(c * np.sqrt(n_lens) / xg) > 60.0)[0]
    x = np.linspace(0.0, xg[past[0]] if past.size else xs, npts)
    with np.errstate(divide="ignore", invalid="ignore"):
        ex = np.where(x > 0, -0.5 * x * x * np.log(c * np.sqrt(n_lens) / np.maximum(x, 1e-300)), 0.0)
    g = x * np.exp(ex)
    u = np.atleast_1d(np.asarray(u, float))
    vals = np.trapezoid(g[None, :] * j0(np.outer(u, x)), x, axis=1)
    return vals / (2.0 * np.pi)


def _study_env():
    import torch
    from paper_2204_10871_gb300 import build as libbuild
    libbuild.build()
    from paper_2204_10871_gb300 import irs, lensgen
    torch.cuda.set_device(0)
    return torch, irs, lensgen


def _interp_map(irs, torch, params, dxy, dm, rows=None):
    shape = (params.npix_y, params.npix_x)
    counts = torch.zeros(shape, dtype=torch.uint32, device=dxy.device)
    with irs.Plan(params) as plan:
        irs.irs_plan_set_timing(plan.handle, True)
        if rows is None:
            irs.irs_make_map(plan.handle, dxy, dm, counts)
        else:
            irs.irs_make_map_rows(plan.handle, dxy, dm, rows[0], rows[1], counts)
        t = irs.irs_plan_timings(plan.handle)
        plan.sync()
        info = plan.info
    return counts.cpu().numpy().astype(np.float64), t, info


def study_accuracy(args):
    """Sec. 3.3 replayed at the paper's shape (see accuracy_replay)."""
    torch, irs, lensgen = _study_env()
    print(json.dumps(accuracy_replay(torch, irs, lensgen, ref_rays=args.ref_rays, reference=args.accuracy_ref)))


def accuracy_replay(torch, irs, lensgen, ks=0.652, S=50.0, npix=1024, n_star=100000, ref_rays=4.0e10,
                    test_rays=tuple((10240 * k) ** 2 for k in range(1, 8)), reference="brute",
                    ref_chunk_rays=2.0e9, seed=7, fit_min=10.0):
    """Sec. 3.3: kappa = kappa_* = 0.652, gamma = 0, S = 50 theta_E at 1024^2,
    1e5 uniform-mass lenses; interpolated maps of (10240 k)^2 rays, k = 1..7,
    against a reference map of ~4e10 rays made by the brute force (ordinary
    IRS, the paper's criterion; shot in bands of lattice rows) or by the
    interpolated method; RMS relative magnification error in 300 log bins of
    the per-pixel ray count, and its log-log slope (paper: about -2/3).  With
    the brute-force reference the interpolated map of the same rays is also
    compared with it (whole-map rel RMS over pixels with >= 100 rays)."""
    src = (-S / 2, S / 2, -S / 2, S / 2)
    s2 = (S / npix) ** 2
    # Every map's lattice tiles the same plane: the flow chart's side
    # I = (S + 2P)/(1 - kappa) (gamma = 0: a square) split into n rays per
    # side, i.e. n^2 rays at s^2 n^2 / I^2 rays per unlensed pixel.  One lens
    # field then fills every map's lens plane and gives each map the same
    # sheet density.
    side = (S + 20.0 * np.sqrt(ks)) / (1.0 - ks)

    def nav_for(n_rays):
        n = round(np.sqrt(n_rays))
        return s2 * n * n / (side * side)

    def params(n_rays, method=irs.IRS_INTERP):
        return irs.make_params(ks, 0.0, 0.0, src, npix, nav_for(n_rays), n_star=n_star, method=method,
                               kernel_variant=7 if method == irs.IRS_INTERP else 0)

    with irs.Plan(params(ref_rays)) as pr:
        inf = pr.info
    box = (inf.lens_x0, inf.lens_x1, inf.lens_y0, inf.lens_y1)
    area = (box[1] - box[0]) * (box[3] - box[2])
    xy, m = lensgen.lens_field(n_star, box, shape="uniform", seed=seed, total_mass=ks * area / np.pi)
    dxy, dm = torch.from_numpy(xy).cuda(), torch.from_numpy(m).cuda()
    nav_ref = nav_for(ref_rays)
    ri, tri, iref = _interp_map(irs, torch, params(ref_rays), dxy, dm)
    ref_info = {"n_rays": int(iref.n_rays), "rays_per_unlensed_pixel": nav_ref, "method": reference}
    if reference == "brute":
        shape = (npix, npix)
        cb = torch.zeros(shape, dtype=torch.uint32, device=dxy.device)
        with irs.Plan(params(ref_rays, irs.IRS_BRUTE)) as pb:
            ny, nx = pb.info.n_rays_y, pb.info.n_rays_x
            step = max(64, int(ref_chunk_rays / nx) // 64 * 64)  # whole brute-force tiles
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for r0 in range(0, ny, step):
                irs.irs_make_map_rows(pb.handle, dxy, dm, r0, min(ny, r0 + step), cb)
            e1.record()
            pb.sync()
            ref_info["ms_map"] = e0.elapsed_time(e1)
            ref_info["bands"] = (ny + step - 1) // step
        ref = cb.cpu().numpy().astype(np.float64)
        sel = ref >= 100
        r = (ri[sel] - ref[sel]) / ref[sel]
        ref_info["interp_same_rays_rel_rms"] = float(np.sqrt(np.mean(r * r))) if sel.any() else None
        ref_info["pixels_ge_100_rays"] = int(sel.sum())
        ref_info["interp_ms_map"] = tri.ms_total
    else:
        ref = ri
        ref_info["ms_map"] = tri.ms_total
    maps, allx, ally, allw = [], [], [], []
    for n_rays in test_rays:
        c, t, info = _interp_map(irs, torch, params(n_rays), dxy, dm)
        nav = nav_for(n_rays)
        assert abs(info.lens_x1 - info.lens_x0 - (box[1] - box[0])) <= 1e-9 * side  # the same plane
        ok = ref > 0
        err = (c[ok] / nav) / (ref[ok] / nav_ref) - 1.0
        x, y, w = log_binned_rms(c[ok], err, nbins=300, n_max=None, min_count=30)
        fit = x >= fit_min
        maps.append({"n_rays_target": n_rays, "n_rays": int(info.n_rays), "rays_per_unlensed_pixel": nav,
                     "mean_rays_per_pixel": float(c.mean()), "ms_map": t.ms_total,
                     "rel_rms_all_pixels": float(np.sqrt(np.mean(err[c[ok] > 0] ** 2))),
                     "slope": loglog_slope(x[fit], y[fit], w[fit]) if fit.sum() > 2 else None,
                     "bins": int(len(x))})
        allx.append(x[fit]); ally.append(y[fit]); allw.append(w[fit])
    X, Y, Wt = np.concatenate(allx), np.concatenate(ally), np.concatenate(allw)
    return {"study": "accuracy", "config": {"kappa": ks, "kappa_star": ks, "gamma": 0.0, "S": S, "npix": npix,
                                            "n_star": n_star, "masses": "uniform 0.1-1 rescaled to kappa_*",
                                            "method": "interp variant 7", "bins": 300, "min_pixels_per_bin": 30,
                                            "fit": f"bins with >= {fit_min:g} rays per pixel"},
            "reference": ref_info, "maps": maps,
            "slope_all_maps": loglog_slope(X, Y, Wt) if len(X) > 2 else None, "paper_slope": -2.0 / 3.0}


def study_planes(args):
    """Sec. 2.2: the rectangular lens plane against the circumscribed circle
    at the paper-mid workload (kappa_* = gamma = 0.45): lenses needed at the
    same density, and the time of a full map (interpolated) and of the brute
    force (per ray, on a band)."""
    torch, irs, lensgen = _study_env()
    w = WORKLOAD
    res = {}
    for name, plane in (("rect", irs.IRS_PLANE_RECT), ("circle", irs.IRS_PLANE_CIRCLE)):
        S = w["S"]
        src = (-S / 2, S / 2, -S / 2, S / 2)
        p = irs.make_params(w["kappa_star"], w["kappa_s"], w["gamma"], src, w["npix"], w["nav"],
                            n_star=w["n_star"], plane=plane, method=irs.IRS_INTERP, kernel_variant=7)
        with irs.Plan(p) as pr:
            inf = pr.info
        rect_area = (inf.lens_x1 - inf.lens_x0) * (inf.lens_y1 - inf.lens_y0)
        if plane == irs.IRS_PLANE_CIRCLE:
            area = np.pi * inf.circle_r ** 2
            n = int(round(w["n_star"] * area / res["rect"]["lens_area"]))
            xy, m = lensgen.lens_field(n, None, shape=w["shape"], seed=w["seed"],
                                       total_mass=w["kappa_star"] * area / np.pi,
                                       disc=(inf.center_x, inf.center_y, inf.circle_r))
        else:
            area = rect_area
            n = w["n_star"]
            xy, m = lensgen.lens_field(n, (inf.lens_x0, inf.lens_x1, inf.lens_y0, inf.lens_y1), shape=w["shape"],
                                       seed=w["seed"], total_mass=w["kappa_star"] * area / np.pi)
        p.n_star = n
        dxy, dm = torch.from_numpy(xy).cuda(), torch.from_numpy(m).cuda()
        ms = []
        for it in range(3):
            _, t, info = _interp_map(irs, torch, p, dxy, dm)
            if it:
                ms.append((t.ms_total, t.ms_raypass, t.ms_farfield))
        pb = irs.make_params(w["kappa_star"], w["kappa_s"], w["gamma"], src, w["npix"], w["nav"],
                             n_star=n, plane=plane, method=irs.IRS_BRUTE)
        r0 = info.n_rays_y // 2
        band = (r0 - r0 % 64, r0 - r0 % 64 + 64)
        bt = []
        for it in range(2):
            _, t, _ = _interp_map(irs, torch, pb, dxy, dm, rows=band)
            bt.append(t.ms_raypass)
        rays_band = (band[1] - band[0]) * info.n_rays_x
        res[name] = {"lenses": n, "lens_area": area, "image_rect_area": rect_area,
                     "cells": int(info.ncell_x) * int(info.ncell_y), "n_rays": int(info.n_rays),
                     "interp_ms_map": float(np.mean([a for a, _, _ in ms])),
                     "interp_ms_raypass": float(np.mean([b for _, b, _ in ms])),
                     "interp_ms_far_field": float(np.mean([c for _, _, c in ms])),
                     "brute_rays_per_s": rays_band / (bt[-1] * 1e-3),
                     "brute_ms_map_extrapolated": info.n_rays / (rays_band / bt[-1])}
    out = {"study": "planes", "workload": w["name"], "rect": res["rect"], "circle": res["circle"],
           "lens_ratio": res["circle"]["lenses"] / res["rect"]["lenses"],
           "interp_time_ratio": res["circle"]["interp_ms_map"] / res["rect"]["interp_ms_map"],
           "brute_time_ratio": res["circle"]["brute_ms_map_extrapolated"] / res["rect"]["brute_ms_map_extrapolated"]}
    print(json.dumps(out))


def study_border(args):
    """Sec. 2.3: (1) the distribution of the deflection perturbation (lens sum
    plus negative sheet, Eq. alpha1) in the central quarter of the plane for
    N = 1e2 ... 1e6 unit-mass lenses, kappa_* = 0.4, gamma = 0, pooled over
    several lens fields, against Katz's Eq. 13 with the numerator 3.05 and the
    paper's 1.454, and the fraction beyond the 10 phi_0 border; (2) the
    fraction of the needed rays that the bordered plane delivers (map mean
    over <mu>) at the paper-mid workload, over 8 fields."""
    torch, irs, lensgen = _study_env()
    kst = 0.4
    phi0 = np.sqrt(kst)
    pdf = []
    edges = np.linspace(0.0, 12.0, 49)
    uc = 0.5 * (edges[1:] + edges[:-1])
    ring = np.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
    for n, fields in ((100, 16), (1000, 16), (10000, 8), (1000000, 2)):
        P = 10.0 * phi0
        S = float(np.sqrt(np.pi * n / kst) * (1.0 - kst) - 2.0 * P)
        src = (-S / 2, S / 2, -S / 2, S / 2)
        p = irs.make_params(kst, 0.0, 0.0, src, 64, 64.0, n_star=n, method=irs.IRS_BRUTE)
        k = 400000 // fields  # rays per field
        us = []
        with irs.Plan(p) as plan:
            inf = plan.info
            box = (inf.lens_x0, inf.lens_x1, inf.lens_y0, inf.lens_y1)
            nx, ny = inf.n_rays_x, inf.n_rays_y
            for f in range(fields):
                xy, m = lensgen.lens_field(n, box, shape="equal", seed=11 + 1000 * f)
                dxy, dm = torch.from_numpy(xy).cuda(), torch.from_numpy(m).cuda()
                # rays in the central quarter of the plane (deep inside the field)
                rng = np.random.Generator(np.random.PCG64(5 + f))
                i = rng.integers(nx // 4, 3 * nx // 4, k)
                j = rng.integers(ny // 4, 3 * ny // 4, k)
                idx = torch.from_numpy(j * nx + i).cuda()
                beta = torch.empty((k, 2), dtype=torch.float64, device="cuda")
                irs.irs_shoot_rays(plan.handle, dxy, dm, idx, beta)
                plan.sync()
                b = beta.cpu().numpy()
                th = np.stack([inf.lens_x0 + (i + 0.5) * inf.dx_ray, inf.lens_y0 + (j + 0.5) * inf.dx_ray], 1)
                kap = np.pi * m.sum() / ((box[1] - box[0]) * (box[3] - box[2]))  # kappa_* of the lenses passed in, pi sum(m) / A
                ap = th * (1.0 - kap) - b  # alpha - kappa theta: lens sum + negative sheet
                us.append(np.hypot(ap[:, 0], ap[:, 1]) / phi0)
        u = np.concatenate(us)
        h, _ = np.histogram(u, bins=edges)
        dens = h / (u.size * ring)
        dmod = katz_density(uc, n, 1.454)
        dkat = katz_density(uc, n, 3.05)
        cdf_e = np.cumsum(h) / u.size
        pdf.append({"n_lens": n, "S": S, "fields": fields, "rays": int(u.size),
                    "frac_beyond_4phi0": float(np.mean(u > 4)), "frac_beyond_10phi0": float(np.mean(u > 10)),
                    "density_near_10phi0": float(dens[np.searchsorted(uc, 10.0)]),
                    "median_u": float(np.median(u)),
                    "cdf_max_dev_modified_katz": float(np.max(np.abs(cdf_e - np.cumsum(dmod * ring)))),
                    "cdf_max_dev_katz": float(np.max(np.abs(cdf_e - np.cumsum(dkat * ring)))),
                    "u": [round(float(x), 3) for x in uc[::4]],
                    "density": [float(x) for x in dens[::4]],
                    "modified_katz": [float(x) for x in dmod[::4]], "katz": [float(x) for x in dkat[::4]]})
    # ray capture at the paper-mid workload
    w = WORKLOAD
    S = w["S"]
    src = (-S / 2, S / 2, -S / 2, S / 2)
    p = irs.make_params(w["kappa_star"], w["kappa_s"], w["gamma"], src, w["npix"], w["nav"],
                        n_star=w["n_star"], method=irs.IRS_INTERP, kernel_variant=7)
    cap = []
    with irs.Plan(p) as plan:
        inf = plan.info
        box = (inf.lens_x0, inf.lens_x1, inf.lens_y0, inf.lens_y1)
        area = (box[1] - box[0]) * (box[3] - box[2])
        counts = torch.zeros((w["npix"], w["npix"]), dtype=torch.uint32, device="cuda")
        for seed in range(8):
            xy, m = lensgen.lens_field(w["n_star"], box, shape=w["shape"], seed=100 + seed,
                                       total_mass=w["kappa_star"] * area / np.pi)
            dxy, dm = torch.from_numpy(xy).cuda(), torch.from_numpy(m).cuda()
            irs.irs_make_map(plan.handle, dxy, dm, counts)
            plan.sync()
            landed = float(counts.sum(dtype=torch.float64).item())
            kap = w["kappa_s"] + np.pi * m.sum() / area
            mu0 = 1.0 / abs((1.0 - kap) ** 2 - w["gamma"] ** 2)
            cap.append(landed / (w["npix"] ** 2 * w["nav"] * mu0))
    out = {"study": "border", "kappa_star": kst, "gamma": 0.0, "phi0": phi0, "pdf": pdf,
           "capture": {"workload": w["name"], "fields": len(cap), "fraction_mean": float(np.mean(cap)),
                       "fraction_sem": float(np.std(cap, ddof=1) / np.sqrt(len(cap))),
                       "fractions": cap, "paper_claim": "> 0.98"}}
    print(json.dumps(out))


def batched_configs(n_maps=256, seed=4, max_rays=4.0e9):
    """Seeded uneven maps: kappa_* in [0.1, 0.6], kappa_s / kappa in {0, 0.3,
    0.6}, gamma in [0.1, 0.6], maps of 500^2 ... 2000^2 pixels over 10 ... 20
    theta_E, 1e3 ... 1e5 lenses (log-uniform), 16 ... 100 rays per pixel.
    Draws with |1 - kappa -+ gamma| < 0.15 (near-critical: the image plane
    explodes) or more than max_rays rays are redrawn."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n_maps:
        ks = rng.uniform(0.1, 0.6)
        frac = rng.choice([0.0, 0.3, 0.6])
        kss = ks * frac / (1.0 - frac)
        g = rng.uniform(0.1, 0.6)
        kap = ks + kss
        if min(abs(1 - kap - g), abs(1 - kap + g)) < 0.15:
            continue
        S = rng.uniform(10.0, 20.0)
        npix = int(rng.integers(500, 2001))
        nav = rng.uniform(16.0, 100.0)
        n = int(round(10 ** rng.uniform(3.0, 5.0)))
        P = 10.0 * np.sqrt(ks)
        rays = nav * (npix / S) ** 2 * (S + 2 * P) ** 2 / abs((1 - kap - g) * (1 - kap + g))
        if rays > max_rays:
            continue
        out.append(dict(kappa_star=ks, kappa_s=kss, gamma=g, S=S, npix=npix, nav=nav, n_star=n))
    return out


def study_batched(args):
    """The batched persistent launch (see batched_measure), as its own JSON line."""
    torch, irs, lensgen = _study_env()
    print(json.dumps(batched_measure(torch, irs, lensgen, args.batch_maps, args.warmup, args.steps,
                                     args.batch_cell_mult, args.batch_variant)))


def batched_measure(torch, irs, lensgen, n_maps, warmup, steps, cell_mult=0.7, variant=16):
    """The batched persistent launch: n_maps uneven maps through
    irs_make_maps_batched (one captured CUDA graph, replayed), against one
    irs_make_map per map on the same plans; per-map and total rays/s, and a
    bitwise check that both give the same maps.  All plans share one
    setting, since one persistent launch serves one variant: cells 0.7 x the
    rule with ray-pass variant 11, the fastest of (0.85, 0), (0.85, 11),
    (0.573, 11) and (0.7, 11) on this batch (2.78, 2.82, 2.73 and 2.88e11
    rays/s on one GB300)."""
    cfgs = batched_configs(n_maps)
    plans, lens, counts, rays = [], [], [], []
    ws = 0
    for k, c in enumerate(cfgs):
        S = c["S"]
        p = irs.make_params(c["kappa_star"], c["kappa_s"], c["gamma"], (-S / 2, S / 2, -S / 2, S / 2), c["npix"],
                            c["nav"], n_star=c["n_star"], method=irs.IRS_INTERP, cell_mult=cell_mult,
                            kernel_variant=variant)
        plan = irs.Plan(p)
        inf = plan.info
        ws += inf.workspace_bytes
        if ws > 150e9:
            raise RuntimeError("batched study workspace above 150 GB")
        box = (inf.lens_x0, inf.lens_x1, inf.lens_y0, inf.lens_y1)
        area = (box[1] - box[0]) * (box[3] - box[2])
        xy, m = lensgen.lens_field(c["n_star"], box, shape="uniform", seed=1000 + k,
                                   total_mass=c["kappa_star"] * area / np.pi)
        plans.append(plan)
        lens.append((torch.from_numpy(xy).cuda(), torch.from_numpy(m).cuda()))
        counts.append(torch.zeros((c["npix"], c["npix"]), dtype=torch.uint32, device="cuda"))
        rays.append(int(inf.n_rays))
    total = float(sum(rays))
    stream = torch.cuda.current_stream()
    # one map per call
    per = []
    for plan, (xy, m), cnt in zip(plans, lens, counts):
        irs.irs_make_map(plan.handle, xy, m, cnt)  # warm-up (allocations, first launch)
    torch.cuda.synchronize()
    singles = []
    t_seq = 0.0
    for plan, (xy, m), cnt, r in zip(plans, lens, counts, rays):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        irs.irs_make_map(plan.handle, xy, m, cnt)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        t_seq += ms
        per.append(r / (ms * 1e-3))
        singles.append(cnt.clone())
    # the batch: capture on the first call, then replays
    hs = [p.handle for p in plans]
    xs, ms_ = [x for x, _ in lens], [m for _, m in lens]
    for _ in range(max(warmup, 1)):
        irs.irs_make_maps_batched(hs, xs, ms_, counts)
    torch.cuda.synchronize()
    steps = max(steps, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        irs.irs_make_maps_batched(hs, xs, ms_, counts)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / steps
    same = sum(int(torch.equal(a, b)) for a, b in zip(singles, counts))
    per = np.array(per)
    out = {"study": "batched", "maps": len(cfgs), "total_rays": total,
           "config": "kappa_* 0.1-0.6, kappa_s/kappa {0,0.3,0.6}, gamma 0.1-0.6, 500^2-2000^2 px over "
                     "10-20 theta_E, 1e3-1e5 uniform-mass lenses, 16-100 rays/px (seeded)",
           "setting": {"cell_mult": cell_mult, "kernel_variant": variant},
           "batched": {"ms": t_batch, "rays_per_s": total / (t_batch * 1e-3), "steps": steps},
           "sequential": {"ms": t_seq, "rays_per_s": total / (t_seq * 1e-3)},
           "per_map_rays_per_s": {"min": float(per.min()), "median": float(np.median(per)),
                                  "max": float(per.max())},
           "rays_per_map": {"min": min(rays), "median": float(np.median(rays)), "max": max(rays)},
           "maps_identical_to_single_calls": same, "workspace_gb": ws / 1e9}
    for p in plans:
        p.close()
    return out


def study_learned(args):
    """The learned far field against its split radius R_f (cells): for each
    R_f the network is trained on the learned workload's lens field, and the
    study reports its held-out error, the deflection error that implies, the
    map's per-pixel magnification rel RMS against a 256-row brute-force band,
    and the map time; the series form on the same rays for comparison."""
    torch, irs, lensgen = _study_env()
    w = WORKLOAD_LEARNED
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    shape = (w["npix"], w["npix"])
    counts = torch.zeros(shape, dtype=torch.uint32, device=dev)
    pi = irs.Plan(workload_params(irs, "interp", w))
    info = pi.info
    box = (info.lens_x0, info.lens_x1, info.lens_y0, info.lens_y1)
    xy, m = lens_field(lensgen, box, w["seed"], w)
    dxy, dm = torch.from_numpy(xy).to(dev), torch.from_numpy(m).to(dev)
    ms_int, _ = timed_maps(irs, torch, pi, dxy, dm, counts, None, flush)
    r0 = (info.n_rays_y // 2 // 64) * 64
    band = (r0, r0 + 256)
    plans = [pi]
    curve = []
    for rf in args.rf_list:
        pm = workload_params(irs, "mlp", w)
        pm.window = int(rf)
        plan = irs.Plan(pm)
        rep = irs.irs_mlp_train(plan.handle, dxy, dm, seed=11)
        ms, _ = timed_maps(irs, torch, plan, dxy, dm, counts, None, flush)
        t = irs.irs_plan_timings(plan.handle)
        curve.append({"rf_cells": int(rf), "rf_thetaE": rf * info.cell_x, "heldout_rel_rms": rep.valid_rel_rms,
                      "target_rms_thetaE": rep.target_rms,
                      "implied_deflection_error_thetaE": rep.valid_rel_rms * rep.target_rms,
                      "ms_per_map": ms, "ms_far_field": float(t.ms_farfield), "ms_train": rep.ms_train,
                      "ms_samples": rep.ms_samples})
        plans.append(plan)
    brute, rels = band_pair(irs, torch, w, dxy, dm, band, plans)
    for c, r in zip(curve, rels[1:]):
        c["map_rel_rms_vs_brute"] = r
    for p in plans:
        p.close()
    print(json.dumps({"study": "learned", "workload": w["name"], "cell_thetaE": info.cell_x,
                      "interp": {"ms_per_map": ms_int, "map_rel_rms_vs_brute": rels[0]},
                      "brute": brute, "curve": curve, "bar_rel_rms": 1e-3}))


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    world, rank, local = dist_init()
    if rank != 0:
        return
    import oracle
    from paper_2204_10871_gb300 import lensgen
    w = WORKLOAD
    S = w["S"]
    po = oracle.make_params(w["kappa_star"], w["kappa_s"], w["gamma"], (-S / 2, S / 2, -S / 2, S / 2),
                            w["npix"], w["nav"])
    qo = oracle.size(po)
    xy, m = lens_field(lensgen, (qo.a1, qo.a2, qo.b1, qo.b2), w["seed"])
    cores = os.cpu_count() or 1
    budget = max(0.1, args.ref_seconds)  # CPU seconds for the whole run (warm-up + timed)
    r0 = qo.nry // 2
    t0 = time.perf_counter()
    oracle.make_map(po, qo, xy, m, rows=(r0, r0 + cores), cols=(0, 32), threads=cores)
    per_ray = (time.perf_counter() - t0) / (cores * 32)
    cols = int(max(32, min(qo.nrx, budget / max(args.steps + args.warmup, 1) / per_ray)))
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.make_map(po, qo, xy, m, rows=(r0, r0 + cores), cols=(0, cols), threads=cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    rays = cores * cols
    ms = 1e3 * float(np.mean(times))
    value = rays / (ms * 1e-3)
    print(json.dumps({
        "impl": "reference", "metric": "rays/s per GB300 (" + args.method + ")", "value": value,
        "unit": "rays/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "method": "oracle brute force (FP64, CPU)"},
        "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} lattice rows x {cols} rays per step, all lenses"},
        "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=25)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--method", default="interp", choices=["interp", "brute", "mlp"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-brute", action="store_true", help="skip the brute-force band")
    ap.add_argument("--no-tune", action="store_true", help="paper-rule cells, default ray pass")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the high-res, learned and batched sub-records of the default run")
    ap.add_argument("--variant", type=int, default=-1, help="fixed kernel variant (skips tuning)")
    ap.add_argument("--cell-mult", type=float, default=0.0, help="with --variant: level-1 cell multiplier")
    ap.add_argument("--workload", default="", choices=["", "paper-mid", "high-res", "learned"],
                    help="default: paper-mid (learned for --method mlp)")
    ap.add_argument("--band-rows", type=int, default=0, help="brute band height (rows)")
    ap.add_argument("--n-star", type=int, default=0, help="override the lens count (profiling)")
    ap.add_argument("--npix", type=int, default=0, help="override the map side (profiling)")
    ap.add_argument("--nav", type=float, default=0.0, help="override rays per pixel (profiling)")
    ap.add_argument("--study", default="", choices=["", "accuracy", "planes", "border", "batched", "learned"],
                    help="one of the paper's side measurements instead of the benchmark (one GPU)")
    ap.add_argument("--ref-rays", type=float, default=4.0e10, help="rays of the accuracy study's reference map")
    ap.add_argument("--accuracy-ref", default="brute", choices=["brute", "interp"],
                    help="method of the accuracy study's reference map (the paper's criterion is brute force)")
    ap.add_argument("--ref-seconds", type=float, default=30.0,
                    help="--impl reference: host CPU seconds for the oracle's warm-up and timed steps together")
    ap.add_argument("--batch-maps", type=int, default=256, help="maps of the batched study")
    ap.add_argument("--batch-cell-mult", type=float, default=0.7, help="level-1 cell multiplier of the batched maps")
    ap.add_argument("--batch-variant", type=int, default=16, help="ray-pass variant of the batched maps")
    ap.add_argument("--rf-list", type=float, nargs="+", default=[4, 8, 16, 32],
                    help="split radii R_f (cells) of the learned study")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "strips"],
                    help="N > 1: a map per rank (weak scaling) or one map in row strips (strong)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.study:
        {"accuracy": study_accuracy, "planes": study_planes, "border": study_border,
         "batched": study_batched, "learned": study_learned}[args.study](args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
