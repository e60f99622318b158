"""Benchmark of the DIC hot path on GB300: converged POI/s.

One step = one pass of the whole hot path over one image pair: bind the pair
(precompute kernel: gradients of f, float copy and BF16 tap quads of g),
brute-force ZNCC integer search (BF16 tensor-core form), IC-GN sub-pixel
refinement with the FP64 6x6 solve.  Workload ``affine1024``: one 1024x1024
speckle pair (40000 speckles, affine exx=0.5 %, eyy=-0.2 %, 1 deg,
t=(7.3, 4.1) px, noise sigma 2), subset 31x31, grid step 5 (36100 POIs),
search +-20 px, tol 1e-3, at most 50 iterations.  Synthetic, seeded inputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs one replica per GPU (launched by torchrun; each rank processes
its own pair, no collective on the data path) and reports the aggregate.
``--impl reference`` times the FP64 CPU oracle on a bounded POI sample of the
same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "affine1024"
SUBSET, STEP, RADIUS, TOL, MAX_ITER = 31, 5, 20, 1e-3, 50
METRIC = "converged POI/s"
UNIT = "POI/s"
L2_FLUSH_BYTES = 256 << 20     # > 129 MB L2
FP32_LANES_PER_SM = 128


# FP32 operations per interpolated sample of the sub-pixel refinement
# (IC-GN): warp 8, Keys weights 2 x 17, 4x4 convolution 35, residual and
# right-hand-side sums 16, the cross sum of Eq. 1 3.
FLOP_PER_SAMPLE = 96
# per sample of a POI's first pass, at the integer start: the samples are
# pixels (no warp, weights or convolution), only the sums remain
FLOP_PER_PIXEL_SAMPLE = 19
# per reference point of the IC-GN precompute, once per POI (Section 2.2:
# the quantities IC-GN computes once): sum f 1, f - fbar and its square 3,
# the SD products gx dx, gx dy, gy dx, gy dy 4, the 21 entries of the
# Hessian sum SD^T SD 42, sum SD 6, sum SD (f - fbar) 12
FLOP_PER_SETUP_POINT = 68
# algorithmic bytes per pixel of the precompute kernel: f and g read (1 + 1),
# gradient (8), float g (4) and BF16 tap quads (8) written
PRECOMPUTE_BYTES_PER_PX = 22
# kernels launched per step: precompute, then the integer search (phase
# images, template bank, box-sum maps of f and g in one launch, tile,
# reduce; or one FP32 search kernel), then the sub-pixel kernel
LAUNCHES_TC = 1 + 5 + 1
LAUNCHES_PLAIN = 1 + 1 + 1


def traffic_of(name: str):
    """DRAM bytes per launch from a committed ncu summary, only while every
    source it was taken on is unchanged (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name)
    try:
        meta = json.load(open(path))
        for rel, digest in meta["sources"].items():
            if hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest() != digest:
                return None
        return meta.get("bytes_per_launch")
    except (OSError, ValueError, KeyError):
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--solve-bits", type=int, default=64,
                    help="6x6 solve precision of the chosen form (the precision form: FP64)")
    ap.add_argument("--form", default="tc", choices=["tc", "fp32"],
                    help="integer-search form of the chosen configuration")
    ap.add_argument("--cpu-sample", type=int, default=36100,
                    help="POIs in the oracle's CPU sample (default: the whole pair)")
    ap.add_argument("--workload", default="affine1024",
                    choices=["affine1024", "sine2048x64", "mixed32", "affine1024x8",
                             "tensile1024x16"],
                    help="affine1024 is the headline; the others measure the batched form "
                         "and the adjoint")
    ap.add_argument("--pairs", type=int, default=0, help="limit the number of pairs (0 = all)")
    ap.add_argument("--sub-records", default="all", choices=["all", "none"],
                    help="add the batched (sine2048x64, mixed32) and adjoint (affine1024x8) "
                         "records to the default line (1 GPU only)")
    ap.add_argument("--sub-steps", type=int, default=5)
    ap.add_argument("--sub-warmup", type=int, default=3)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard(n_units: int, rank: int, world: int) -> list[int]:
    """Units (image pairs) of one rank: round-robin, no data exchange."""
    return list(range(rank, n_units, world))


def reduce_over_ranks(ms: float, units: float, device) -> tuple[float, float]:
    """Whole-job timing of the replicas: the largest timed milliseconds and
    the summed units (converged POIs) over all ranks.  Only these two
    numbers cross ranks; the data path exchanges nothing."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(ms), float(units)
    t_ms = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    t_units = torch.tensor([float(units)], dtype=torch.float64, device=device)
    tdist.all_reduce(t_ms, op=tdist.ReduceOp.MAX)
    tdist.all_reduce(t_units, op=tdist.ReduceOp.SUM)
    return float(t_ms.item()), float(t_units.item())


def config_dict(world: int) -> dict:
    return {"workload": WORKLOAD, "image": "1024x1024 u8", "pairs_per_gpu": 1,
            "subset": SUBSET, "grid_step": STEP, "search_radius": RADIUS, "pois_per_pair": 36100,
            "method": "IC-GN", "conv_tol": TOL, "max_iter": MAX_ITER,
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"replicas x{world}"}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling during the timed region (read-only)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout_s: float = 3.0):
        """Block until the first sample has arrived (nvidia-smi starts slowly)."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.01)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    import paper_1905_06228_gb300 as dic
    from workloads import configs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dic.build()
    pairs = shard(world, rank, world)          # one pair per rank (weak scaling)
    pair = configs.affine1024(pair=pairs[0])
    ref_d = torch.from_numpy(pair.ref).to(dev)
    def_d = torch.from_numpy(pair.defm).to(dev)
    stream = torch.cuda.Stream(dev)
    props = torch.cuda.get_device_properties(dev)

    def make(solve_bits, form):
        d = dic.DIC(SUBSET, STEP, RADIUS, TOL, MAX_ITER, solve_bits=solve_bits, stream=stream)
        if form == "tc":
            dic.dic_set_form(d.h, dic.DIC_FORM_BF16TC)
        return d

    d = make(args.solve_bits, args.form)
    n, nx, ny = d.set_pair(ref_d, def_d)
    with torch.cuda.stream(stream):
        s_out = d.integer_search()
        p_out = d.subpixel(s_out)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(dd, events=None, method=dic.DIC_ICGN):
        # events: (before search, after search, after sub-pixel), on the
        # stream the kernels are launched on
        dic.dic_set_pair(dd.h, ref_d, def_d)
        if events:
            events[0].record(stream)
        dic.dic_integer_search(dd.h, s_out["u0"], s_out["v0"], s_out["zncc0"], s_out["status0"])
        if events:
            events[1].record(stream)
        dic.dic_subpixel(dd.h, method, s_out["u0"], s_out["v0"], s_out["status0"],
                         p_out["u"], p_out["v"], p_out["ux"], p_out["uy"], p_out["vx"],
                         p_out["vy"], p_out["zncc"], p_out["iters"], p_out["status"])
        if events:
            events[2].record(stream)

    # bounded device waits that gave up in a timed loop (each kernel's wait
    # records it in the handle's flag; a number taken then is not valid)
    gave_up = []

    def check_waits(dd, where):
        try:
            dic.dic_check(dd.h)
        except dic.DICError as ex:
            gave_up.append(f"{where}: {ex}")

    def timed_loop(dd, steps, warmup, sampler=None, method=dic.DIC_ICGN):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                flush.zero_()
                step(dd, method=method)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
        starts = [ev() for _ in range(steps)]
        ends = [ev() for _ in range(steps)]
        sev = [(ev(), ev(), ev()) for _ in range(steps)]
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(steps):
                flush.zero_()
                starts[i].record(stream)
                step(dd, sev[i], method=method)
                ends[i].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        clocks = sampler.stop() if sampler else None
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        search_ms = [a.elapsed_time(b) for a, b, _ in sev]
        sub_ms = [b.elapsed_time(c) for _, b, c in sev]
        conv = int((p_out["status"] == 0).sum().item())
        check_waits(dd, "timed loop")
        return step_ms, (search_ms, sub_ms), conv, wall, clocks

    # clocks: sampled from just before the headline's timed loop to the end of
    # the last timed loop of this line (forms and e2e), every 10 ms
    sampler = ClockSampler(local)
    sampler.start()
    sampler.wait_first()
    step_ms, (search_ms, sub_ms), conv, wall, _ = timed_loop(d, args.steps, args.warmup)
    total_ms, conv_all = reduce_over_ranks(sum(step_ms), conv, dev)
    ms_per_step = total_ms / args.steps
    value = conv_all * args.steps / (total_ms / 1e3)

    # plain form (FP32 search, FP32 6x6 solve) on the same input, same rules
    d32 = make(32, "fp32")
    d32.set_pair(ref_d, def_d)
    st32, se32, conv32, _, _ = timed_loop(d32, max(10, args.steps // 4), 3)
    plain_value = conv32 * len(st32) / (sum(st32) / 1e3)
    plain_search_ms = statistics.mean(se32[0])
    d32.close()
    # the chosen search with the other 6x6 solve precision
    other_bits = 32 if args.solve_bits == 64 else 64
    dob = make(other_bits, args.form)
    dob.set_pair(ref_d, def_d)
    sto, seo, convo, _, _ = timed_loop(dob, max(10, args.steps // 4), 3)
    other_value = convo * len(sto) / (sum(sto) / 1e3)
    other_sub_ms = statistics.mean(seo[1])
    dob.close()
    # the chosen form with forward-additive Newton-Raphson (Gauss-Newton
    # form) in place of IC-GN
    dnr = make(args.solve_bits, args.form)
    dnr.set_pair(ref_d, def_d)
    stn, sen, convn, _, _ = timed_loop(dnr, max(10, args.steps // 4), 3, method=dic.DIC_FANR)
    fanr_value = convn * len(stn) / (sum(stn) / 1e3)
    fanr_sub_ms = statistics.mean(sen[1])
    dnr.close()
    # the chosen form with the bilinear interpolation of Eq. 5
    dbl = make(args.solve_bits, args.form)
    dic.dic_set_interpolation(dbl.h, dic.DIC_INTERP_BILINEAR)
    dbl.set_pair(ref_d, def_d)
    stb, seb, convb, _, _ = timed_loop(dbl, max(10, args.steps // 4), 3)
    bil_value = convb * len(stb) / (sum(stb) / 1e3)
    bil_sub_ms = statistics.mean(seb[1])
    dbl.close()

    # the second-order (12-parameter) shape function, IC-GN, same search and
    # solve precision, same rules
    h2 = dic.dic_create(SUBSET, STEP, RADIUS, 2, TOL, MAX_ITER)
    dic.dic_set_solve_precision(h2, args.solve_bits)
    if args.form == "tc":
        dic.dic_set_form(h2, dic.DIC_FORM_BF16TC)
    dic.dic_set_stream(h2, stream)
    p12 = torch.empty((n, 12), dtype=torch.float32, device=dev)
    o2 = {k: torch.empty(n, dtype=dt, device=dev) for k, dt in
          (("zncc", torch.float32), ("iters", torch.int32), ("status", torch.uint8))}

    def step2():
        dic.dic_set_pair(h2, ref_d, def_d)
        dic.dic_integer_search(h2, s_out["u0"], s_out["v0"], s_out["zncc0"], s_out["status0"])
        dic.dic_subpixel2(h2, dic.DIC_ICGN, s_out["u0"], s_out["v0"], s_out["status0"], p12,
                          o2["zncc"], o2["iters"], o2["status"])
    k2 = max(5, args.steps // 4)
    with torch.cuda.stream(stream):
        for _ in range(3):
            flush.zero_()
            step2()
        ev2 = [(ev(), ev()) for _ in range(k2)]
        for a_, b_ in ev2:
            flush.zero_()
            a_.record(stream)
            step2()
            b_.record(stream)
    torch.cuda.synchronize(dev)
    ms2 = statistics.mean(a_.elapsed_time(b_) for a_, b_ in ev2)
    conv2 = int((o2["status"] == 0).sum().item())
    second_order = {"shape": "second order (12 parameters)", "method": "IC-GN",
                    "solve": f"fp{args.solve_bits}", "ms_per_step": ms2,
                    "value": conv2 / (ms2 / 1e3), "converged_fraction": conv2 / n}
    dic.dic_destroy(h2)

    # the particle swarm integer searches (Section 2.1, Eqs. 2-4; the modified
    # swarm with the star search) timed beside the dense search on the same
    # pair, with their agreement with its exact argmax
    from workloads import swarm
    rand = torch.from_numpy(swarm.uniforms(1, n)).to(dev)
    pso = {}
    ds = make(args.solve_bits, args.form)
    ds.set_pair(ref_d, def_d)
    po = {k: torch.empty(n, dtype=dt, device=dev) for k, dt in
          (("u0", torch.int32), ("v0", torch.int32), ("zncc", torch.float32),
           ("status", torch.uint8), ("gens", torch.int32), ("evals", torch.int32))}
    for modified in (False, True):
        ev_a, ev_b = ev(), ev()
        reps = max(3, args.steps // 4)
        with torch.cuda.stream(stream):
            for _ in range(2):
                dic.dic_pso_search(ds.h, rand, po["u0"], po["v0"], po["zncc"], po["status"],
                                   po["gens"], po["evals"], modified=modified)
            ev_a.record(stream)
            for _ in range(reps):
                dic.dic_pso_search(ds.h, rand, po["u0"], po["v0"], po["zncc"], po["status"],
                                   po["gens"], po["evals"], modified=modified)
            ev_b.record(stream)
        torch.cuda.synchronize(dev)
        ms = ev_a.elapsed_time(ev_b) / reps
        agree = ((po["u0"] == s_out["u0"]) & (po["v0"] == s_out["v0"])).float().mean().item()
        pso["modified_swarm" if modified else "standard_swarm"] = {
            "ms": ms, "pois_per_s": n / (ms / 1e3), "agrees_with_dense_argmax": agree,
            "mean_evaluations": po["evals"].float().mean().item(),
            "mean_generations": po["gens"].float().mean().item(),
            "dense_search_ms": statistics.mean(search_ms)}
    ds.close()
    del rand

    # e2e through the public calls with host buffers: H2D of both images,
    # the three kernels, D2H of every per-POI output, all inside the events.
    # The two images travel as one pinned (2, H, W) buffer and the thirteen
    # per-POI outputs live in one device buffer (each a view at a 16-byte
    # aligned offset), so each direction is one copy.
    h_img = torch.stack([torch.from_numpy(pair.ref), torch.from_numpy(pair.defm)]).pin_memory()
    img_d = torch.empty_like(h_img, device=dev)
    o_specs = [(k, v.dtype) for k, v in s_out.items()] + [(k, v.dtype) for k, v in p_out.items()]
    o_offs, o_total = [], 0
    for _, dt in o_specs:
        o_offs.append(o_total)
        o_total += (n * torch.empty((), dtype=dt).element_size() + 15) // 16 * 16
    flat_d = torch.empty(o_total, dtype=torch.uint8, device=dev)
    flat_h = torch.empty(o_total, dtype=torch.uint8).pin_memory()

    def views(buf):
        out = {}
        for (k, dt), off in zip(o_specs, o_offs):
            nb = n * torch.empty((), dtype=dt).element_size()
            out[k] = buf[off:off + nb].view(dt)
        return out

    e_d, e_h = views(flat_d), views(flat_h)
    ek = max(10, args.steps // 4)
    e_starts = [ev() for _ in range(ek)]
    e_ends = [ev() for _ in range(ek)]
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for i in range(ek):
            flush.zero_()
            e_starts[i].record(stream)
            img_d.copy_(h_img, non_blocking=True)
            dic.dic_set_pair(d.h, img_d[0], img_d[1])
            dic.dic_integer_search(d.h, e_d["u0"], e_d["v0"], e_d["zncc0"], e_d["status0"])
            dic.dic_subpixel(d.h, dic.DIC_ICGN, e_d["u0"], e_d["v0"], e_d["status0"], e_d["u"],
                             e_d["v"], e_d["ux"], e_d["uy"], e_d["vx"], e_d["vy"], e_d["zncc"],
                             e_d["iters"], e_d["status"])
            flat_h.copy_(flat_d, non_blocking=True)
            e_ends[i].record(stream)
    torch.cuda.synchronize(dev)
    check_waits(d, "e2e loop")
    # one more step of the chosen form into the device outputs (the rooflines
    # below count its samples); the e2e host copies hold the same results
    with torch.cuda.stream(stream):
        step(d)
    torch.cuda.synchronize(dev)
    for k, v in list(s_out.items()) + list(p_out.items()):
        assert torch.equal(e_h[k], v.cpu()), ("e2e output differs", k)
    clocks = sampler.stop()
    clocks["window"] = "headline, forms and e2e timed loops"
    e_ms, e_conv = reduce_over_ranks(sum(s.elapsed_time(e) for s, e in zip(e_starts, e_ends)) / ek,
                                     int((e_h["status"] == 0).sum().item()), dev)
    e2e = {"value": e_conv / (e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(h_img.numel()),
           "d2h_bytes_per_step": int(flat_h.numel()),
           "copies_per_step": {"h2d": 1, "d2h": 1}}

    # rooflines.  Dominant kernel: the sub-pixel refinement (one launch per
    # step), bound by FP32 issue; algorithmic work = FLOP_PER_SAMPLE per
    # interpolated subset sample, N samples per pass.
    peak_mhz = 2070.0
    fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * peak_mhz * 1e6 / 1e12
    fp32_basis = (f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                  f"x {peak_mhz:.0f} MHz (nominal max clock)")
    # passes per POI: one per iteration (the first at the integer start reads
    # pixels), plus one interpolating pass at the returned shape for POIs
    # that did not converge
    its = p_out["iters"].to(torch.int64)
    ran = (s_out["status0"] == 0) & (its >= 1)
    extra = (p_out["status"] != 0).to(torch.int64)
    pixel_samples = int(ran.sum().item()) * SUBSET * SUBSET
    samples = int(((its - 1) + extra)[ran].sum().item()) * SUBSET * SUBSET
    setup_points = int((s_out["status0"] == 0).sum().item()) * SUBSET * SUBSET
    sub_flop = (FLOP_PER_SAMPLE * samples + FLOP_PER_PIXEL_SAMPLE * pixel_samples +
                FLOP_PER_SETUP_POINT * setup_points)
    sub_avg_s = statistics.mean(sub_ms) / 1e3
    sub_achieved = sub_flop / sub_avg_s / 1e12
    roofline = {"bound": "alu", "achieved": sub_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": sub_achieved / fp32_peak,
                "traffic": traffic_of("subpixel_affine1024_traffic.json"),
                "kernel": f"subpixel_kernel<IC-GN, fp{args.solve_bits} solve>",
                "peak_basis": fp32_basis, "ms": sub_avg_s * 1e3,
                "work": (f"{FLOP_PER_SAMPLE} flop x {samples} interpolated samples + "
                         f"{FLOP_PER_PIXEL_SAMPLE} flop x {pixel_samples} first-pass pixel "
                         f"samples + {FLOP_PER_SETUP_POINT} flop x {setup_points} set-up "
                         f"points per launch")}
    # the integer search: algorithmic flops 2 N (2R+1)^2 per POI (padded and
    # wasted MACs not counted)
    search_avg_s = statistics.mean(search_ms) / 1e3
    flops = 2.0 * SUBSET * SUBSET * (2 * RADIUS + 1) ** 2 * n
    if args.form == "tc":
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        peak = float(peaks.get("bf16_tflops", 1900.0))
        bound, kernel = "tensor", ("integer search, tensor-core form (phase + bank + box-map + "
                                   "tile + reduce kernels)")
        basis = ("measured dense BF16 (cuBLAS burst) " + ("of measured" if peaks else "of fallback"))
        prof = "search_tc_affine1024_traffic.json"
    else:
        peak = fp32_peak
        bound, kernel = "alu", "search_kernel (FP32 FMA correlation)"
        basis = fp32_basis
        prof = "search_affine1024_traffic.json"
    achieved = flops / search_avg_s / 1e12
    roofline_search = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak, "traffic": traffic_of(prof), "kernel": kernel,
                       "peak_basis": basis, "ms": search_avg_s * 1e3,
                       "plain_fp32_search": {"ms": plain_search_ms,
                                             "achieved_tflops": flops / (plain_search_ms / 1e3)
                                             / 1e12,
                                             "frac_of_fp32_peak": flops / (plain_search_ms / 1e3)
                                             / 1e12 / fp32_peak}}

    # whole-path roofline: each step at its own bound (search flops at the
    # search's peak, sub-pixel flops at the FP32 peak, precompute bytes at
    # HBM), summed, against the measured step time
    peaks_all = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks_all.get("hbm_gbs", 6800.0)) * 1e9
    pre_bytes = PRECOMPUTE_BYTES_PER_PX * pair.ref.size
    t_roof = flops / (peak * 1e12) + sub_flop / (fp32_peak * 1e12) + pre_bytes / hbm
    roofline_path = {"roofline_ms": t_roof * 1e3, "measured_ms": ms_per_step,
                     "frac": t_roof * 1e3 / ms_per_step,
                     "terms": {"search_ms": flops / (peak * 1e12) * 1e3,
                               "subpixel_ms": sub_flop / (fp32_peak * 1e12) * 1e3,
                               "precompute_ms": pre_bytes / hbm * 1e3},
                     "hbm_basis": "measured" if peaks_all else "fallback"}

    # measured FP32 FMA throughput beside the nominal peak the fraction uses
    fp32_meas = dic.dic_measure_peak(dic.DIC_PEAK_FP32_FMA, stream) / 1e12
    roofline["measured_fma_peak"] = fp32_meas
    roofline["frac_of_measured_fma"] = sub_achieved / fp32_meas
    sub_records = None
    if world == 1 and args.sub_records == "all":
        d.close()
        for dd in (d32, dob, dnr, dbl):
            dd.close()
        del flush
        torch.cuda.empty_cache()
        t_sub = time.perf_counter()
        atomic_peak = dic.dic_measure_peak(dic.DIC_PEAK_SMEM_ATOMIC_F32, stream)
        sub_records = {
            "batch_sine2048x64": batch_record("sine2048x64", dev, args.sub_steps,
                                              args.sub_warmup, solve_bits=args.solve_bits,
                                              fp32_peak=fp32_peak),
            "batch_mixed32": batch_record("mixed32", dev, args.sub_steps, args.sub_warmup,
                                          solve_bits=args.solve_bits, fp32_peak=fp32_peak),
            "adjoint_affine1024x8": adjoint_record(dev, args.sub_steps, args.sub_warmup,
                                                   fp32_peak=fp32_peak,
                                                   atomic_peak=atomic_peak),
            "stream_tensile1024x16": stream_record(dev, args.sub_steps, args.sub_warmup,
                                                   solve_bits=args.solve_bits,
                                                   fp32_peak=fp32_peak),
            "measured_peaks": {"fp32_fma_tflops": fp32_meas,
                               "smem_atomic_f32_per_s": atomic_peak},
            "wall_s": None}
        sub_records["wall_s"] = time.perf_counter() - t_sub

    cpu = None
    if rank == 0:
        cpu = cpu_baseline(pair, args.cpu_sample, single=True)
    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16+f32" if args.form == "tc" else "f32",
                "data": "synthetic (seeded speckle renders)",
                "config": config_dict(world), "e2e": e2e,
                "gpu_launches": (LAUNCHES_TC if args.form == "tc" else LAUNCHES_PLAIN)
                * args.steps,
                "roofline": roofline, "roofline_search": roofline_search,
                "roofline_path": roofline_path,
                "cpu_baseline": cpu, "clocks": clocks,
                "forms": {"chosen": {"search": "bf16-tensor-core-exact" if args.form == "tc"
                                     else "fp32-exact", "solve": f"fp{args.solve_bits}",
                                     "value": value},
                          "chosen_fp%d_solve" % other_bits: {
                              "search": "bf16-tensor-core-exact" if args.form == "tc"
                              else "fp32-exact", "solve": f"fp{other_bits}",
                              "value": other_value, "subpixel_ms": other_sub_ms},
                          "chosen_fanr": {"method": "FA-NR (Gauss-Newton form)",
                                          "solve": f"fp{args.solve_bits}",
                                          "value": fanr_value, "subpixel_ms": fanr_sub_ms},
                          "chosen_bilinear": {"interpolation": "bilinear (Eq. 5)",
                                              "solve": f"fp{args.solve_bits}",
                                              "value": bil_value, "subpixel_ms": bil_sub_ms},
                          "plain_fp32": {"search": "fp32-exact", "solve": "fp32",
                                         "value": plain_value},
                          "swarm_searches": pso,
                          "second_order_shape": second_order},
                "converged_fraction": conv / n, "wall_s_timed": wall,
                "device_waits_gave_up": gave_up,
                "sub_records": sub_records}
        print(json.dumps(line))
    d.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------- CPU oracle arm
def cpu_sample_idx(n: int, k: int):
    import numpy as np
    k = min(k, n)
    return np.unique(np.linspace(0, n - 1, k).round().astype(np.int64))


def cpu_baseline(pair, sample: int, single: bool = False) -> dict:
    """The FP64 oracle, as it stands, on an evenly spaced POI sample of the
    same pair, on every host core."""
    import numpy as np

    import oracle
    nx, ny = oracle.grid(pair.ref.shape[1], pair.ref.shape[0], SUBSET, STEP, RADIUS)
    idx = cpu_sample_idx(nx * ny, sample)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.integer_search(pair.ref, pair.defm, SUBSET, STEP, RADIUS, poi_idx=idx,
                              threads=threads)
    s = oracle.subpixel(pair.ref, pair.defm, SUBSET, STEP, RADIUS, r["u0"], r["v0"],
                        r["status"], tol=TOL, max_iter=MAX_ITER, poi_idx=idx, threads=threads)
    dt = time.perf_counter() - t0
    conv = int((s["status"] == 0).sum())
    out = {"value": conv / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{len(idx)} evenly spaced POIs of {WORKLOAD} (search + IC-GN), {dt:.1f} s"}
    if single:
        # the same oracle on one host core, on a smaller evenly spaced sample
        idx1 = cpu_sample_idx(nx * ny, 256)
        t0 = time.perf_counter()
        r = oracle.integer_search(pair.ref, pair.defm, SUBSET, STEP, RADIUS, poi_idx=idx1,
                                  threads=1)
        s = oracle.subpixel(pair.ref, pair.defm, SUBSET, STEP, RADIUS, r["u0"], r["v0"],
                            r["status"], tol=TOL, max_iter=MAX_ITER, poi_idx=idx1, threads=1)
        dt1 = time.perf_counter() - t0
        out["single_thread"] = {"value": int((s["status"] == 0).sum()) / dt1, "unit": UNIT,
                                "cores": 1, "sample": f"{len(idx1)} evenly spaced POIs, "
                                                      f"{dt1:.1f} s"}
        out["cpu_model"] = cpu_model()
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from workloads import configs
    pair = configs.affine1024(pair=0)
    for _ in range(args.warmup):
        cpu_baseline(pair, 64)
    # POIs per step: sized from a calibration sample so that all timed steps
    # together take about 90 s of host time (at least 64 POIs per step)
    rate = cpu_baseline(pair, 512)["value"]
    sample = int(min(args.cpu_sample, max(64, 90.0 / max(1, args.steps) * rate)))
    vals, secs = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(pair, sample)
        secs.append(time.perf_counter() - t0)
        vals.append(cb["value"])
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded speckle renders)", "config": config_dict(world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count() or 1,
                             "kind": "oracle",
                             "sample": f"{sample} evenly spaced POIs of {WORKLOAD} per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------- batched / adjoint forms
def cpu_model() -> str:
    """Host CPU model (lscpu's model name, else /proc/cpuinfo, else the
    machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_sample(pairs, pair_ids, pois_per_pair: int, threads: int) -> dict:
    """The FP64 oracle (integer search + IC-GN), as it stands, on evenly
    spaced POIs of the chosen pairs; converged POIs per second."""
    import numpy as np

    import oracle
    conv, n, dt = 0, 0, 0.0
    for k in pair_ids:
        p = pairs[k]
        nx, ny = oracle.grid(p.ref.shape[1], p.ref.shape[0], p.subset, p.step, p.radius)
        idx = cpu_sample_idx(nx * ny, pois_per_pair)
        t0 = time.perf_counter()
        r = oracle.integer_search(p.ref, p.defm, p.subset, p.step, p.radius, poi_idx=idx,
                                  threads=threads)
        s = oracle.subpixel(p.ref, p.defm, p.subset, p.step, p.radius, r["u0"], r["v0"],
                            r["status"], tol=TOL, max_iter=MAX_ITER, poi_idx=idx,
                            threads=threads)
        dt += time.perf_counter() - t0
        conv += int((s["status"] == 0).sum())
        n += len(idx)
    return {"value": conv / dt, "seconds": dt, "pois": n}


def subpixel_work(iters, status, status0, subset: int) -> tuple[int, int, int]:
    """Interpolated and first-pass pixel samples of one sub-pixel launch: one
    pass per solve (the first at the integer start reads pixels) plus one
    interpolating pass at the returned shape for POIs that did not
    converge; N = subset^2 samples per pass; and the set-up points (N per
    POI that entered the refinement)."""
    import torch
    its = iters.to(torch.int64)
    ran = (status0 == 0) & (its >= 1)
    extra = (status != 0).to(torch.int64)
    n = subset * subset
    return (int(((its - 1) + extra)[ran].sum().item()) * n, int(ran.sum().item()) * n,
            int((status0 == 0).sum().item()) * n)


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def batch_record(workload: str, dev, steps: int, warmup: int, form: int = 1,
                 solve_bits: int = 64, n_pairs: int = 0, cpu_pairs: int = 4,
                 cpu_pois: int = 1024, plain_steps: int = 1, fp32_peak: float | None = None,
                 clocks: bool = True) -> dict:
    """Many pairs in one CUDA graph (sine2048x64, mixed32): converged POI/s of
    the batch (autotuned launch shape), the same pairs through the
    single-pair calls (per-kernel times and rooflines from CUDA events on the
    launching stream), the plain FP32-search batch, and the oracle on a
    sample of the same pairs."""
    import torch

    import paper_1905_06228_gb300 as dic
    from workloads import configs
    if workload == "sine2048x64":
        n_pairs = n_pairs or 64
        pairs = [configs.sine2048(k) for k in range(n_pairs)]
    else:
        n_pairs = n_pairs or 32
        pairs = [configs.mixed(k) for k in range(n_pairs)]
    props = torch.cuda.get_device_properties(dev)
    if fp32_peak is None:
        fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * 2070.0 * 1e6 / 1e12
    peaks = load_peaks()
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0)) * 1e9
    h = dic.dic_create(21, 5, 10, 1, TOL, MAX_ITER)
    dic.dic_set_solve_precision(h, solve_bits)
    stream = torch.cuda.Stream(dev)
    dic.dic_set_stream(h, stream)
    tens = [(torch.from_numpy(p.ref).to(dev), torch.from_numpy(p.defm).to(dev),
             p.subset, p.step, p.radius) for p in pairs]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    dic.dic_set_form(h, form)
    dic.dic_set_pairs(h, tens)
    total, offs = dic.dic_batch_pois(h, len(tens))
    out = dic.batch_outputs(total, dev)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        chosen = dic.dic_autotune(h, dic.DIC_ICGN, out)
        for _ in range(warmup):
            dic.dic_run_batch(h, dic.DIC_ICGN, out)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(dev.index or 0) if clocks else None
    if sampler:
        sampler.start()
        sampler.wait_first()
    starts = [ev() for _ in range(steps)]
    ends = [ev() for _ in range(steps)]
    with torch.cuda.stream(stream):
        for i in range(steps):
            starts[i].record(stream)
            dic.dic_run_batch(h, dic.DIC_ICGN, out)
            ends[i].record(stream)
    torch.cuda.synchronize(dev)
    clk = sampler.stop() if sampler else None
    ms = statistics.mean(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    conv = int((out["status"] == 0).sum())
    # work of the step: search flops 2 N (2R+1)^2 per POI, sub-pixel samples
    # from the batch's own outputs, precompute bytes per pixel
    search_flop = sub_flop = 0.0
    pre_bytes = 0
    for k, p in enumerate(pairs):
        a, b = offs[k], offs[k + 1]
        search_flop += 2.0 * p.subset ** 2 * (2 * p.radius + 1) ** 2 * (b - a)
        si, sp, su = subpixel_work(out["iters"][a:b], out["status"][a:b],
                                   out["status0"][a:b], p.subset)
        sub_flop += FLOP_PER_SAMPLE * si + FLOP_PER_PIXEL_SAMPLE * sp + FLOP_PER_SETUP_POINT * su
        pre_bytes += PRECOMPUTE_BYTES_PER_PX * p.ref.size
    t_roof = search_flop / (bf16_peak * 1e12) + sub_flop / (fp32_peak * 1e12) + pre_bytes / hbm
    # the same pairs through the single-pair calls, one after the other, with
    # events around each pair's search and sub-pixel launch
    singles = []
    for (f8, g8, s_, st_, r_) in tens:
        hh = dic.dic_create(s_, st_, r_, 1, TOL, MAX_ITER)
        dic.dic_set_solve_precision(hh, solve_bits)
        dic.dic_set_form(hh, form)
        dic.dic_set_stream(hh, stream)
        singles.append(hh)
    n_each = []
    with torch.cuda.stream(stream):
        for hh, (f8, g8, *_r) in zip(singles, tens):
            dic.dic_set_pair(hh, f8, g8)
            n_each.append(dic.dic_num_pois(hh)[0])
    bufs = [dic.batch_outputs(n, dev) for n in n_each]
    pev = [(ev(), ev(), ev()) for _ in tens]

    def one_by_one(record=False):
        for j, (hh, (f8, g8, *_r), o) in enumerate(zip(singles, tens, bufs)):
            dic.dic_set_pair(hh, f8, g8)
            if record:
                pev[j][0].record(stream)
            dic.dic_integer_search(hh, o["u0"], o["v0"], o["zncc0"], o["status0"])
            if record:
                pev[j][1].record(stream)
            dic.dic_subpixel(hh, dic.DIC_ICGN, o["u0"], o["v0"], o["status0"], o["u"], o["v"],
                             o["ux"], o["uy"], o["vx"], o["vy"], o["zncc"], o["iters"],
                             o["status"])
            if record:
                pev[j][2].record(stream)
    with torch.cuda.stream(stream):
        one_by_one()
        torch.cuda.synchronize(dev)
        a_, e_ = ev(), ev()
        a_.record(stream)
        one_by_one(record=True)
        e_.record(stream)
    torch.cuda.synchronize(dev)
    ms_single = a_.elapsed_time(e_)
    search_ms = sum(x.elapsed_time(y) for x, y, _ in pev)
    sub_ms = sum(y.elapsed_time(z) for _, y, z in pev)
    for hh in singles:
        dic.dic_destroy(hh)
    del bufs
    # the plain form of the same batch: FP32 integer search (persistent
    # kernels per template width); pairs whose FP32 window does not fit
    # shared memory are left out of this comparison and named
    plain = None
    skipped = []
    if form == 1 and plain_steps > 0:
        keep = list(range(len(tens)))
        hp = None
        while keep:
            hp = dic.dic_create(21, 5, 10, 1, TOL, MAX_ITER)
            dic.dic_set_solve_precision(hp, 32)
            dic.dic_set_stream(hp, stream)
            dic.dic_set_pairs(hp, [tens[k] for k in keep])
            tp, _ = dic.dic_batch_pois(hp, len(keep))
            op = dic.batch_outputs(tp, dev)
            try:
                with torch.cuda.stream(stream):
                    dic.dic_run_batch(hp, dic.DIC_ICGN, op)
                break
            except dic.DICError:
                msg = dic.dic_last_error(hp)
                dic.dic_destroy(hp)
                hp = None
                bad = int(msg.split("pair ")[1].split(":")[0])
                skipped.append(keep.pop(bad))
        if hp is not None:
            torch.cuda.synchronize(dev)
            with torch.cuda.stream(stream):
                a_, e_ = ev(), ev()
                a_.record(stream)
                for _ in range(plain_steps):
                    dic.dic_run_batch(hp, dic.DIC_ICGN, op)
                e_.record(stream)
            torch.cuda.synchronize(dev)
            ms_plain = a_.elapsed_time(e_) / plain_steps
            conv_plain = int((op["status"] == 0).sum())
            plain = {"search": "fp32-exact", "solve": "fp32", "pairs": len(keep),
                     "pairs_left_out": skipped, "ms_per_step": ms_plain,
                     "value": conv_plain / (ms_plain / 1e3)}
            dic.dic_destroy(hp)
    dic.dic_destroy(h)
    threads = os.cpu_count() or 1
    ids = sorted(set(round(i * (len(pairs) - 1) / max(1, cpu_pairs - 1))
                     for i in range(cpu_pairs)))
    cs = oracle_sample(pairs, ids, cpu_pois, threads)
    shape = tuple(chosen)
    return {
        "workload": workload, "pairs": len(tens), "pois": int(total),
        "ms_per_step": ms, "value": conv / (ms / 1e3), "unit": UNIT,
        "pairs_per_s": len(tens) / (ms / 1e3), "converged_fraction": conv / max(1, int(total)),
        "form": ("one CUDA graph: " + ("tensor-core search pair by pair, " if form == 1 else
                                       "persistent FP32 search per template width, ") +
                 ("per-pair sub-pixel launches on a second stream, each overlapping the next "
                  "pairs' searches" if shape == (0, 0) else "one persistent sub-pixel kernel")),
        "autotuned": {"warps_per_cta": chosen[0], "grid_mult": chosen[1]},
        "solve": f"fp{solve_bits}", "steps": steps, "warmup": warmup,
        "roofline_path": {"roofline_ms": t_roof * 1e3, "measured_ms": ms,
                          "frac": t_roof * 1e3 / ms,
                          "terms_ms": {"search": search_flop / (bf16_peak * 1e12) * 1e3,
                                       "subpixel": sub_flop / (fp32_peak * 1e12) * 1e3,
                                       "precompute": pre_bytes / hbm * 1e3}},
        "roofline_search": {"bound": "tensor", "achieved": search_flop / (search_ms / 1e3) / 1e12,
                            "peak": bf16_peak, "unit": "TFLOP/s",
                            "frac": search_flop / (search_ms / 1e3) / 1e12 / bf16_peak,
                            "ms": search_ms,
                            "basis": "per-pair search launches, events; measured BF16 peak"},
        "roofline_subpixel": {"bound": "alu", "achieved": sub_flop / (sub_ms / 1e3) / 1e12,
                              "peak": fp32_peak, "unit": "TFLOP/s",
                              "frac": sub_flop / (sub_ms / 1e3) / 1e12 / fp32_peak,
                              "ms": sub_ms,
                              "basis": "per-pair sub-pixel launches, events; nominal FP32"},
        "per_pair_launches": {"ms_per_step": ms_single, "value": conv / (ms_single / 1e3),
                              "batch_gain": ms_single / ms},
        "plain_fp32_batch": plain,
        "cpu_baseline": {"value": cs["value"], "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": (f"{cs['pois']} POIs: {cpu_pois} evenly spaced POIs of each "
                                    f"of pairs {ids} (search + IC-GN), {cs['seconds']:.1f} s; "
                                    "a rate on the sample, not extrapolated")},
        "l2": "inputs and scratch larger than L2",
        "clocks": clk}


# FP32 operations per subset sample of the ZNSSD forward (dic_znssd) and
# backward (dic_backward) launches, counted from the kernel: each launch
# samples g twice (value pass: warp 12, Keys weights 34, 4x4 convolution 35,
# sums 6 = 87; value-and-gradient pass: warp 12, value and derivative weights
# 62, convolutions 77, loss 7 = 158); the backward launch adds the adjoint
# (weight 5, dL/dp 12, Keys weights 34, 16 scatter products 20 = 71).
ADJ_FLOP_FWD = 87 + 158
ADJ_FLOP_BWD = 87 + 158 + 71
ADJ_SCATTER_PER_SAMPLE = 16


def adjoint_record(dev, steps: int, warmup: int, n_pairs: int = 8,
                   fp32_peak: float | None = None, atomic_peak: float | None = None,
                   cpu_pois: int = 4096) -> dict:
    """ZNSSD forward + backward at the imposed shapes over the affine1024x8
    differentiation set (8 pairs, subset 31, step 8: 14161 POIs each)."""
    import numpy as np
    import torch

    import oracle
    import paper_1905_06228_gb300 as dic
    from workloads import configs
    pairs = [configs.affine1024x8(k) for k in range(n_pairs)]
    stream = torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    total_ms, n_poi, samples = 0.0, 0, 0
    shapes = []
    for p in pairs:
        s_, st_, r_ = p.subset, p.step, p.radius
        nx = (1024 - 1 - 2 * (s_ // 2 + r_ + 2)) // st_ + 1
        n = nx * nx
        b = s_ // 2 + r_ + 2
        kk = np.arange(n)
        x0 = (b + (kk % nx) * st_).astype(np.float64)
        y0 = (b + (kk // nx) * st_).astype(np.float64)
        shp = np.stack(p.deformation.displacement(x0, y0), 1).astype(np.float32)
        shapes.append(shp)
        f = torch.from_numpy(p.ref).to(dev).float().contiguous()
        g = torch.from_numpy(p.defm).to(dev).float().contiguous()
        sh = torch.from_numpy(shp).to(dev).contiguous()
        hh = dic.dic_create(s_, st_, r_)
        dic.dic_set_stream(hh, stream)
        dg = torch.empty_like(g)
        dp = torch.empty_like(sh)
        tot = torch.empty((), dtype=torch.float32, device=dev)
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            dic.dic_set_pair_f32(hh, f, g)
            for _ in range(warmup):
                dic.dic_znssd(hh, sh, None, tot)
                dic.dic_backward(hh, sh, None, 1.0, dg, dp)
            a, e = ev(), ev()
            a.record(stream)
            for _ in range(steps):
                dic.dic_znssd(hh, sh, None, tot)
                dic.dic_backward(hh, sh, None, 1.0, dg, dp)
            e.record(stream)
        torch.cuda.synchronize(dev)
        total_ms += a.elapsed_time(e) / steps
        n_poi += n
        samples += n * s_ * s_
        dic.dic_destroy(hh)
    rate = samples / (total_ms / 1e3)
    flops = (ADJ_FLOP_FWD + ADJ_FLOP_BWD) * rate / 1e12
    adds = ADJ_SCATTER_PER_SAMPLE * rate
    # the oracle's FP64 ZNSSD + adjoint (single-threaded, as it stands) on a
    # POI sample of the first pair
    p = pairs[0]
    idx = cpu_sample_idx(len(shapes[0]), cpu_pois)
    t0 = time.perf_counter()
    oracle.znssd(p.ref, p.defm, p.subset, p.step, p.radius, shapes[0][idx].astype(np.float64),
                 poi_idx=idx)
    dt = time.perf_counter() - t0
    rec = {"workload": "affine1024x8", "pairs": n_pairs, "pois": n_poi, "subset": 31,
           "grid_step": 8, "metric": "adjoint POI/s (ZNSSD forward + backward)",
           "value": n_poi / (total_ms / 1e3), "unit": "POI/s", "ms_per_step": total_ms,
           "steps": steps, "warmup": warmup, "samples_per_s": rate,
           "scatter_atomics_per_s": adds,
           "roofline": {"bound": "alu", "achieved": flops, "peak": fp32_peak,
                        "unit": "TFLOP/s", "frac": flops / fp32_peak if fp32_peak else None,
                        "work": (f"{ADJ_FLOP_FWD} + {ADJ_FLOP_BWD} flop per subset sample "
                                 "(forward + backward launch)")},
           "roofline_atomic": {"bound": "smem atomics", "achieved": adds / 1e9,
                               "peak": atomic_peak / 1e9 if atomic_peak else None,
                               "unit": "G adds/s",
                               "frac": adds / atomic_peak if atomic_peak else None,
                               "peak_basis": "measured (dic_measure_peak, shared-memory float "
                                             "atomic adds)"},
           "cpu_baseline": {"value": len(idx) / dt, "unit": "POI/s", "cores": 1,
                            "kind": "oracle",
                            "sample": f"{len(idx)} evenly spaced POIs of pair 0, ZNSSD + FP64 "
                                      f"adjoint, single thread, {dt:.1f} s"}}
    return rec


def stream_record(dev, steps: int, warmup: int, solve_bits: int = 64,
                  fp32_peak: float | None = None, cpu_pois: int = 8192) -> dict:
    """The tensile1024x16 frame sequence (17 frames, reference updated every
    frame) through dic_stream_push: converged POI/s over its 16 consecutive
    pairs with the frames resident, the same pairs through the single-pair
    calls, and end to end with every frame copied from pinned host memory
    inside the timed region (one frame per pair)."""
    import torch

    import paper_1905_06228_gb300 as dic
    from workloads import configs
    seq = configs.tensile_sequence()
    fr, S, st, R = seq["frames"], seq["subset"], seq["step"], seq["radius"]
    peaks = load_peaks()
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0)) * 1e9
    stream = torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    frames = [torch.from_numpy(f).to(dev) for f in fr]
    h = dic.dic_create(S, st, R, 1, TOL, MAX_ITER)
    dic.dic_set_form(h, dic.DIC_FORM_BF16TC)
    dic.dic_set_solve_precision(h, solve_bits)
    dic.dic_set_stream(h, stream)
    with torch.cuda.stream(stream):
        dic.dic_stream_push(h, frames[0], dic.DIC_ICGN)
    n, _, _ = dic.dic_num_pois(h)
    outs = [dic.batch_outputs(n, dev) for _ in range(len(fr) - 1)]

    def run_seq():
        dic.dic_stream_reset(h)
        dic.dic_stream_push(h, frames[0], dic.DIC_ICGN)
        for k in range(1, len(fr)):
            dic.dic_stream_push(h, frames[k], dic.DIC_ICGN, outs[k - 1])
        dic.dic_stream_flush(h)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            run_seq()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    sampler.wait_first()
    a, e = ev(), ev()
    with torch.cuda.stream(stream):
        a.record(stream)
        for _ in range(steps):
            run_seq()
        e.record(stream)
    torch.cuda.synchronize(dev)
    clk = sampler.stop()
    ms = a.elapsed_time(e) / steps
    conv = sum(int((o["status"] == 0).sum()) for o in outs)
    pairs = len(fr) - 1
    search_flop = 2.0 * S * S * (2 * R + 1) ** 2 * n * pairs
    sub_flop = 0.0
    for o in outs:
        si, sp, su = subpixel_work(o["iters"], o["status"], o["status0"], S)
        sub_flop += FLOP_PER_SAMPLE * si + FLOP_PER_PIXEL_SAMPLE * sp + FLOP_PER_SETUP_POINT * su
    if fp32_peak is None:
        props = torch.cuda.get_device_properties(dev)
        fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * 2070.0 * 1e6 / 1e12
    pre_bytes = PRECOMPUTE_BYTES_PER_PX * fr[0].size * pairs
    t_roof = search_flop / (bf16_peak * 1e12) + sub_flop / (fp32_peak * 1e12) + pre_bytes / hbm
    # the same pairs through the single-pair calls
    hs = dic.dic_create(S, st, R, 1, TOL, MAX_ITER)
    dic.dic_set_form(hs, dic.DIC_FORM_BF16TC)
    dic.dic_set_solve_precision(hs, solve_bits)
    dic.dic_set_stream(hs, stream)
    so = dic.batch_outputs(n, dev)

    def run_pairs():
        for k in range(1, len(fr)):
            dic.dic_set_pair(hs, frames[k - 1], frames[k])
            dic.dic_integer_search(hs, so["u0"], so["v0"], so["zncc0"], so["status0"])
            dic.dic_subpixel(hs, dic.DIC_ICGN, so["u0"], so["v0"], so["status0"], so["u"],
                             so["v"], so["ux"], so["uy"], so["vx"], so["vy"], so["zncc"],
                             so["iters"], so["status"])
    with torch.cuda.stream(stream):
        run_pairs()
        torch.cuda.synchronize(dev)
        a, e = ev(), ev()
        a.record(stream)
        for _ in range(steps):
            run_pairs()
        e.record(stream)
    torch.cuda.synchronize(dev)
    ms_pairs = a.elapsed_time(e) / steps
    dic.dic_destroy(hs)
    # end to end: each frame from pinned host memory into one device buffer,
    # pushed, every pair's outputs read back, all inside the events
    hfr = [torch.from_numpy(f).pin_memory() for f in fr]
    hout = [{k: torch.empty_like(v, device="cpu").pin_memory() for k, v in o.items()}
            for o in outs]
    dbuf = torch.empty_like(frames[0])
    with torch.cuda.stream(stream):
        a, e = ev(), ev()
        a.record(stream)
        dic.dic_stream_reset(h)
        dbuf.copy_(hfr[0], non_blocking=True)
        dic.dic_stream_push(h, dbuf, dic.DIC_ICGN)
        for k in range(1, len(fr)):
            dbuf.copy_(hfr[k], non_blocking=True)
            dic.dic_stream_push(h, dbuf, dic.DIC_ICGN, outs[k - 1])
            if k >= 2:  # the previous pair's outputs are complete on this stream now
                for key in hout[k - 2]:
                    hout[k - 2][key].copy_(outs[k - 2][key], non_blocking=True)
        dic.dic_stream_flush(h)
        for key in hout[-1]:
            hout[-1][key].copy_(outs[-1][key], non_blocking=True)
        e.record(stream)
    torch.cuda.synchronize(dev)
    e_ms = a.elapsed_time(e)
    e_conv = sum(int((o["status"] == 0).sum()) for o in hout)
    dic.dic_destroy(h)

    class _P:
        pass
    pl = []
    for k in (1, pairs // 2, pairs):
        q = _P()
        q.ref, q.defm, q.subset, q.step, q.radius = fr[k - 1], fr[k], S, st, R
        pl.append(q)
    threads = os.cpu_count() or 1
    cs = oracle_sample(pl, range(len(pl)), cpu_pois, threads)
    return {"workload": "tensile1024x16", "frames": len(fr), "pairs": pairs, "pois_per_pair": n,
            "subset": S, "grid_step": st, "search_radius": R,
            "form": "dic_stream_push: tensor-core search on the handle's stream, sub-pixel "
                    "(IC-GN) on a second stream overlapping the next pair's search",
            "solve": f"fp{solve_bits}", "ms_per_step": ms, "value": conv / (ms / 1e3),
            "unit": UNIT, "frames_per_s": pairs / (ms / 1e3), "steps": steps, "warmup": warmup,
            "converged_fraction": conv / (n * pairs),
            "single_pair_calls": {"ms_per_step": ms_pairs, "value": conv / (ms_pairs / 1e3),
                                  "stream_gain": ms_pairs / ms},
            "e2e": {"value": e_conv / (e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(f.size for f in fr)),
                    "d2h_bytes_per_step": int(sum(v.numel() * v.element_size()
                                                  for o in hout for v in o.values()))},
            "roofline_path": {"roofline_ms": t_roof * 1e3, "measured_ms": ms,
                              "frac": t_roof * 1e3 / ms},
            "cpu_baseline": {"value": cs["value"], "unit": UNIT, "cores": threads,
                             "kind": "oracle",
                             "sample": (f"{cs['pois']} POIs: {cpu_pois} evenly spaced POIs of "
                                        f"pairs 1, {pairs // 2}, {pairs}, {cs['seconds']:.1f} s")},
            "clocks": clk}


def run_batch_workload(args):
    """One record of the batched forms (sine2048x64, mixed32) or of the
    adjoint (affine1024x8), printed as its own JSON line."""
    import torch

    import paper_1905_06228_gb300 as dic
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    dic.build()
    fp32_peak = dic.dic_measure_peak(dic.DIC_PEAK_FP32_FMA) / 1e12
    if args.workload == "tensile1024x16":
        rec = stream_record(dev, args.steps, args.warmup, solve_bits=args.solve_bits,
                            fp32_peak=fp32_peak)
    elif args.workload == "affine1024x8":
        rec = adjoint_record(dev, args.steps, args.warmup, n_pairs=args.pairs or 8,
                             fp32_peak=fp32_peak,
                             atomic_peak=dic.dic_measure_peak(dic.DIC_PEAK_SMEM_ATOMIC_F32))
    else:
        rec = batch_record(args.workload, dev, args.steps, args.warmup,
                           form=1 if args.form == "tc" else 0, solve_bits=args.solve_bits,
                           n_pairs=args.pairs)
    rec.update({"metric": rec.get("metric", METRIC), "n_gpus": 1, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "data": "synthetic (seeded speckle renders)",
                "fp32_fma_measured_tflops": fp32_peak})
    print(json.dumps(rec))


def traffic_record(csv_path: str, kernel_regex: str, sources: list[str], out: str,
                   command: str, workload: str) -> dict:
    """DRAM bytes per launch of the kernels matching kernel_regex in an ncu
    CSV (--metrics dram__bytes_read.sum,dram__bytes_write.sum --csv), with
    the SHA-256 of the given sources as they are when this runs -- run it in
    the same command as the capture, so the hashes are those of the code
    that was captured."""
    import csv
    import hashlib
    import re
    per_id: dict[str, float] = {}
    names: dict[str, str] = {}
    with open(csv_path, newline="") as fh:
        rows = [ln for ln in fh if ln.startswith('"')]
    for row in csv.DictReader(rows):
        name = row.get("Kernel Name", "")
        metric = row.get("Metric Name", "")
        if not re.search(kernel_regex, name) or metric not in ("dram__bytes_read.sum",
                                                               "dram__bytes_write.sum"):
            continue
        unit = row.get("Metric Unit", "byte").lower()
        scale = {"byte": 1, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9}.get(unit, 1)
        val = float(row["Metric Value"].replace(",", "")) * scale
        per_id[row["ID"]] = per_id.get(row["ID"], 0.0) + val
        names[row["ID"]] = name
    if not per_id:
        raise SystemExit(f"no launch of {kernel_regex} in {csv_path}")
    rec = {"kernel": sorted(set(names.values()))[0][:160], "workload": workload,
           "launches": len(per_id),
           "bytes_per_launch": int(round(statistics.mean(per_id.values()))),
           "counters": "dram__bytes_read.sum + dram__bytes_write.sum",
           "command": command,
           "sources": {rel: hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read())
                       .hexdigest() for rel in sources}}
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=1)
    return rec


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--traffic-record":
        ap = argparse.ArgumentParser()
        ap.add_argument("--traffic-record", required=True, help="ncu CSV")
        ap.add_argument("--kernel", required=True)
        ap.add_argument("--sources", required=True, help="comma-separated repo paths")
        ap.add_argument("--out", required=True)
        ap.add_argument("--command", required=True)
        ap.add_argument("--workload", default=WORKLOAD)
        a = ap.parse_args()
        print(json.dumps(traffic_record(a.traffic_record, a.kernel, a.sources.split(","), a.out,
                                        a.command, a.workload)))
        return
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "affine1024":
        run_batch_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
