"""Throughput benchmark: 3-level multiscale denoise of 12 MP frames.

Workload (default): 8 frames of 4032x3024 RGB, FP16 storage / FP32
arithmetic, camera-like noise (variance 0.01 x + (10/255)^2 with a smooth
gain field in [0.5, 2]), 3 pyramid levels, 7x7 fine + 7x7 coarse per-channel
filters (D = 98), 216 buckets per level, FP16 banks resident in shared memory.
One step = pyramid (2 launches) + level-1 filter + level-0 filter, all through
the C ABI, inputs resident in HBM (585 MB per step, larger than L2).

Metric: Mpix/s of finest-level input pixels (whole job, all ranks).
`--impl reference` times the FP64 CPU oracle on the host cores instead.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H, W, LEVELS = 3024, 4032, 3
METRIC = "Mpix/s 3-level denoise at 12MP"
# DRAM bytes (read + write) of one level-0 k_level3 launch per 4032x3024 FP16
# frame, from the ncu capture in profiles/k_level3_12mp_level0_fp16.md; set to
# None whenever that kernel changes until it is captured again.
LEVEL0_TRAFFIC_PER_FRAME = (91.645184 + 38.008576) * 1e6


def _gen_frame(seed):
    import synth
    return synth.noisy_pair(H, W, seed, model="camera")[0]


def make_frames(n, seed0):
    """n distinct seeded frames, generated in a spawn pool (before any CUDA use)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=min(n, os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        return np.stack(list(ex.map(_gen_frame, [seed0 + i for i in range(n)])))


def random_banks(seed, D=98, K=216, nb=LEVELS - 1):
    """Random FP16 banks with taps summing to ~1 (values keep the output in range)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nb):
        b = rng.standard_normal((K, 3, D)).astype(np.float32) * 0.03
        b += (1.0 - b.sum(axis=2, keepdims=True)) / D
        out.append(b)
    return out


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- multi-rank

def max_over_ranks(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank time over all ranks (rank 0 reports it)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(pixels_per_rank_step: int, steps: int, world: int, ms_max: float) -> float:
    """Weak scaling: every rank denoises its own batch; Mpix/s of the job."""
    return pixels_per_rank_step * steps * world / (ms_max * 1e-3) / 1e6


# ---------------------------------------------------------------- CPU oracle

def cpu_oracle_run(steps, warmup, sample_hw=(768, 1024), threads=None):
    """Times the FP64 oracle (as it stands) on 3-level denoises of crops of the
    benchmark frame, on all host threads or on `threads`; returns Mpix/s,
    seconds, sample description, threads used."""
    import oracle as O
    import synth
    h, w = sample_hw
    all_threads = O.max_threads()
    O.set_threads(threads or all_threads)
    used = O.max_threads()
    z = synth.noisy_pair(h, w, 40000, model="camera")[0]
    z16 = O.round_storage(z, "f16")
    geom = O.Geometry(3, 3)
    banks = [b.astype(np.float64) for b in random_banks(7)]
    for _ in range(warmup):
        O.denoise_multiscale(z16, banks, geom, storage="f16")
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        O.denoise_multiscale(z16, banks, geom, storage="f16")
        times.append(time.perf_counter() - t0)
    O.set_threads(all_threads)
    tot = sum(times)
    mpix = h * w * steps / 1e6
    return (mpix / tot, tot, f"{steps} x 3-level denoise of a {w}x{h} crop (FP16-rounded input, FP64 arithmetic)",
            used)


def cpu_baseline_block(steps, warmup):
    """cpu_baseline: all host threads on the bounded sample, plus one thread
    on a single crop."""
    v, _, sample, used = cpu_oracle_run(steps, warmup)
    v1, _, sample1, _ = cpu_oracle_run(1, 0, threads=1)
    return {"value": round(v, 3), "unit": "Mpix/s", "cores": used, "kind": "oracle", "sample": sample,
            "single_thread": {"value": round(v1, 3), "unit": "Mpix/s", "cores": 1, "sample": sample1}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    v, tot, sample, used = cpu_oracle_run(args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * tot / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "3-level denoise, 7x7+7x7 per-channel YCbCr filters, 216 buckets, "
                                   "FP16 inputs, crop of a 4032x3024 camera-noise frame"},
            "cpu_baseline": {"value": round(v, 3), "unit": "Mpix/s", "cores": used, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 3), "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- accuracy

def _dilate(mask, r):
    """Binary dilation by a (2r+1)^2 square (bookkeeping for the band rule)."""
    if r <= 0:
        return mask.copy()
    h, w = mask.shape
    out = np.zeros_like(mask)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            ys, xs = slice(max(dy, 0), h + min(dy, 0)), slice(max(dx, 0), w + min(dx, 0))
            yd, xd = slice(max(-dy, 0), h + min(-dy, 0)), slice(max(-dx, 0), w + min(-dx, 0))
            out[yd, xd] |= mask[ys, xs]
    return out


def _affected(mism, r_coarse, shapes):
    """Finest-level pixels whose output depends on a bucket that differs from
    the oracle's (own bucket, or the coarser output within r_coarse)."""
    aff = mism[-1].copy()
    for l in range(len(mism) - 2, -1, -1):
        h, w = shapes[l]
        up = np.repeat(np.repeat(_dilate(aff, max(r_coarse, 0)), 2, 0), 2, 1)[:h, :w]
        aff = mism[l] | up
    return aff


def accuracy_headline(mdn, frame, banks32, dev, crop=128, margin=64):
    """Headline path (3 levels, 4032x3024) against the FP64 oracle on crops of
    one benchmark frame: max-abs error per path at pixels whose buckets (and
    coarser dependencies) agree with the oracle's, plus the threshold-band and
    mismatch counts.  The oracle gets the banks unrounded (the FP32 values the
    FP16 device banks were rounded from) and, separately, FP16-rounded (the
    kernel's arithmetic alone)."""
    import torch
    import oracle as O
    Hf, Wf = frame.shape[1:]
    geom_o, geom = O.Geometry(3, 3), mdn.Geometry(3, 3)
    bps = [mdn.default_bparams(0), mdn.default_bparams(1)]
    banks64 = [b.astype(np.float64) for b in banks32]
    banks16 = [O.round_storage(b, "f16") for b in banks64]
    dbanks = {"f16": [torch.tensor(b, dtype=torch.float16, device=dev) for b in banks32],
              "f32": [torch.tensor(b, dtype=torch.float32, device=dev) for b in banks32]}
    crops = [(0, 0), (0, Wf - crop), (Hf - crop, 0), (Hf - crop, Wf - crop), (1504, 2000), (752, 3136)]
    out = {"crops": f"{len(crops)} crops of {crop}x{crop} (corners and interior) of frame 0, oracle run on the "
                    f"crop plus a {margin}-pixel margin; errors at pixels not affected by a bucket that differs "
                    "from the oracle's (those differ only in the 1e-5 threshold band)", "paths": {}}
    for storage, tdt, bank_dt in [("f16", torch.float16, "f16"), ("f32", torch.float32, "f16"),
                                  ("f32", torch.float32, "f32")]:
        z = O.round_storage(frame.astype(np.float64), storage)
        zt = torch.tensor(z, dtype=tdt, device=dev)[None]
        maps = [torch.empty((1, Hf, Wf), dtype=torch.uint8, device=dev),
                torch.empty((1, (Hf + 1) // 2, (Wf + 1) // 2), dtype=torch.uint8, device=dev)]
        y = mdn.denoise_multiscale(zt, dbanks[bank_dt], geom, bps, bucket_maps=maps)[0].float().cpu().numpy()
        gmaps = [m[0].cpu().numpy() for m in maps]
        pairs = [("unrounded", banks64), ("f16_rounded", banks16)] if bank_dt == "f16" else [("unrounded", banks64)]
        for bank_name, bo in pairs:
            worst, band, aff_n, mism_out, npx = 0.0, 0, 0, 0, 0
            for (y0, x0) in crops:
                cy0, cx0 = max(y0 - margin, 0), max(x0 - margin, 0)
                cy1, cx1 = min(y0 + crop + margin, Hf), min(x0 + crop + margin, Wf)
                ref = O.denoise_multiscale(z[:, cy0:cy1, cx0:cx1], bo, geom_o, storage=storage, mirror32=True)
                mism = []
                for l in range(2):
                    s_ = 2 ** l
                    g = gmaps[l][cy0 // s_: cy0 // s_ + ref.buckets[l].shape[0],
                                 cx0 // s_: cx0 // s_ + ref.buckets[l].shape[1]]
                    m = g != ref.buckets[l]
                    inner = np.zeros_like(m)
                    b_ = 16 // s_
                    inner[b_ if cy0 else 0: m.shape[0] - (b_ if cy1 < Hf else 0),
                          b_ if cx0 else 0: m.shape[1] - (b_ if cx1 < Wf else 0)] = True
                    mism_out += int((m & ~ref.bands[l] & inner).sum())
                    band += int((ref.bands[l] & inner).sum())
                    mism.append(m & inner)
                aff = _affected(mism, 3, [r.shape[1:] for r in ref.pyramid])
                ry, rx = y0 - cy0, x0 - cx0
                keep = ~aff[ry:ry + crop, rx:rx + crop]
                d = np.abs(y[:, y0:y0 + crop, x0:x0 + crop] - ref.out[:, ry:ry + crop, rx:rx + crop]).max(axis=0)
                worst = max(worst, float(d[keep].max()) if keep.any() else 0.0)
                aff_n += int((~keep).sum())
                npx += crop * crop
            bar = 2e-3 if storage == "f16" else 1e-4
            rec = {"max_abs": float(f"{worst:.3g}"), "bar": bar, "within_bar": worst <= bar, "pixels": npx,
                   "pixels_excluded_affected": aff_n, "band_pixels": band, "bucket_mismatches_outside_band": mism_out}
            if storage == "f32" and bank_dt == "f16" and bank_name == "unrounded":
                rec["note"] = ("FP16 bank rounding alone exceeds the FP32 path's 1e-4 bar: the FP32 path is held to it "
                               "with FP32 banks (next entry) or against the FP16-rounded banks")
            out["paths"][f"{storage}_storage_{bank_dt}_banks_vs_oracle_{bank_name}_banks"] = rec
    return out


def accuracy_training(mdn, dev, n=4, size=1024):
    """Config-3 training precisions against the FP64 oracle on a subset of n
    of the benchmark's pairs: Gram and bank relative Frobenius (whole bank and
    per bucket with n_k >= 10 D), and the denoised-output max-abs error of each
    precision's bank on a held-out 1024x1024 image (single-level cross-channel
    7x7x3 filter) at pixels whose bucket agrees with the oracle's."""
    import torch
    import oracle as O
    import synth
    geom_o, geom = O.Geometry(3, -1, cross=1), mdn.Geometry(3, -1, 1)
    bp_o, bp = O.default_bparams(0), mdn.default_bparams(0)
    pairs = [synth.noisy_pair(size, size, 30000 + i) for i in range(n)]
    t0 = time.perf_counter()
    gram = counts = None
    for z, u in pairs:
        b, _, _ = O.select(z, bp_o, mirror32=True)
        gram, counts = O.gram_accumulate(z, None, u, b, 216, geom_o, gram, counts)
    bank_o = O.solve_bank(gram, counts, geom_o, 1e-3)
    t_oracle = time.perf_counter() - t0
    zt, ut = synth.noisy_pair(size, size, 39999)
    bt, band_t, _ = O.select(zt, bp_o, mirror32=True)
    ref_out = O.filter_level(zt, None, bt, bank_o, geom_o)
    Z = torch.tensor(np.stack([p[0] for p in pairs]), device=dev)
    U = torch.tensor(np.stack([p[1] for p in pairs]), device=dev)
    xt = torch.tensor(zt, dtype=torch.float32, device=dev)[None]
    D = geom_o.D()
    big = np.nonzero(counts >= 10 * D)[0]
    res = {"subset": f"{n} of the 256 config-3 pairs ({n * size * size} patches); oracle Gram + solve "
                     f"{t_oracle:.1f} s on the host", "buckets_compared": int(len(big)), "precisions": {}}
    for prec, name in [(0, "fp32_simt"), (1, "tf32"), (2, "bf16"), (3, "split_bf16")]:
        g, c, bank = mdn.train_level_filters(Z, None, U, geom, bp, prec, lam=1e-3)
        m = torch.empty((1, size, size), dtype=torch.uint8, device=dev)
        y = mdn.filter_level(xt, None, bank, geom, bp, buckets_out=m)
        torch.cuda.synchronize()
        gn, cn, bn = g.cpu().numpy(), c.cpu().numpy(), bank.cpu().numpy().astype(np.float64)
        per = [np.linalg.norm(bn[k] - bank_o[k]) / np.linalg.norm(bank_o[k]) for k in big]
        keep = m[0].cpu().numpy() == bt
        d = np.abs(y[0].cpu().numpy().astype(np.float64) - ref_out).max(axis=0)
        res["precisions"][name] = {
            "gram_rel": float(f"{np.linalg.norm(gn - gram) / np.linalg.norm(gram):.3g}"),
            "bank_rel": float(f"{np.linalg.norm(bn - bank_o) / np.linalg.norm(bank_o):.3g}"),
            "bank_rel_per_bucket_median": float(f"{np.median(per):.3g}"),
            "bank_rel_per_bucket_max": float(f"{np.max(per):.3g}"),
            "bank_bar": 1e-3, "bank_within_bar": bool(np.max(per) <= 1e-3),
            "counts_equal": bool(np.array_equal(cn, counts)),
            "output_max_abs": float(f"{d[keep].max():.3g}"), "output_pixels_excluded": int((~keep).sum())}
    return res


# ---------------------------------------------------------------- GPU arm

def run_variants(mdn, x, geom, dev, stream, reps=10):
    """The rest of the 12 MP metric run, timing only (same frames, denoise via
    mdn_denoise_multiscale with preallocated output and workspace, L2 flushed
    before every timed call, median): FP16 and FP32 storage, batch 1 and 8,
    the 4-level pipeline of the 12 MP batch, FP32 banks, and the paper's own
    16 x 16 x 16 grid with 7x7 + 5x5 taps (4096 buckets).  Banks too large for
    shared memory (the 4096-bucket grid, FP32 banks of 7x7 + 7x7 taps) run
    plain (tile kernel, taps through L2) and prepared (mdn_prepare_bank_rows:
    the fused kernel reading row slots through L2)."""
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    res = {}
    paper_geom = mdn.Geometry(3, 2)
    f16, f32 = torch.float16, torch.float32
    grid = "f16_batch1_3level_grid16x16x16_7x7+5x5"
    for name, xv, levels, bank_dt, prepared in [
            ("f16_batch1_3level", x[:1], 3, f16, False), ("f32_batch1_3level", x[:1].float(), 3, f16, False),
            ("f32_batch8_3level", x.float(), 3, f16, False), ("f16_batch8_4level", x, 4, f16, False),
            ("f32_batch1_3level_f32bank", x[:1].float(), 3, f32, False),
            ("f32_batch1_3level_f32bank_prepared", x[:1].float(), 3, f32, True),
            (grid, x[:1], 3, f16, False), (grid + "_prepared", x[:1], 3, f16, True),
            (grid.replace("batch1", "batch8") + "_prepared", x, 3, f16, True)]:
        paper = "grid16" in name
        g = paper_geom if paper else geom
        banks = [torch.tensor(b, dtype=bank_dt, device=dev)
                 for b in (random_banks(7, D=74, K=4096, nb=levels - 1) if paper else random_banks(7, nb=levels - 1))]
        if prepared:
            banks = [mdn.prepare_bank(b, g) for b in banks]
        bps = [(mdn.paper_grid_bparams if paper else mdn.default_bparams)(l) for l in range(levels - 1)]
        nv = xv.shape[0]
        dt = mdn.F16 if xv.dtype == torch.float16 else mdn.F32
        ws = torch.empty(mdn.denoise_workspace_bytes(nv, H, W, levels, dt), dtype=torch.uint8, device=dev)
        out = torch.empty_like(xv)
        for _ in range(2):
            mdn.denoise_multiscale(xv, banks, g, bps, out=out, ws=ws)
        times = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mdn.denoise_multiscale(xv, banks, g, bps, out=out, ws=ws)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        ms = statistics.median(times)
        res[name] = {"ms": round(ms, 4), "mpix_s": round(nv * H * W / ms / 1e3, 1)}
        del xv, out, ws
    return res


def run_gpu(args, rank, world, frames):
    import torch
    import paper_1802_06130_gb300 as mdn

    torch.cuda.set_device(args.local_rank)
    dev = torch.device("cuda", args.local_rank)
    mdn.build()
    L = mdn.lib()
    n = frames.shape[0]
    geom = mdn.Geometry(3, 3)
    bps = [mdn.default_bparams(0), mdn.default_bparams(1)]
    banks = [torch.tensor(b, dtype=torch.float16, device=dev) for b in random_banks(7)]
    x = torch.tensor(frames, dtype=torch.float16, device=dev)
    hl = [H, (H + 1) // 2, (H + 3) // 4]
    wl = [W, (W + 1) // 2, (W + 3) // 4]
    z1 = torch.empty((n, 3, hl[1], wl[1]), dtype=torch.float16, device=dev)
    z2 = torch.empty((n, 3, hl[2], wl[2]), dtype=torch.float16, device=dev)
    u1 = torch.empty_like(z1)
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    import ctypes as C
    sp = C.c_void_p(stream.cuda_stream)
    lv = (C.c_void_p * 2)(z1.data_ptr(), z2.data_ptr())

    ev = None

    def step(record):
        if record:
            ev[0].record(stream)
        mdn._check(L.mdn_build_pyramid(C.c_void_p(x.data_ptr()), mdn.F16, n, H, W, LEVELS, lv, sp))
        if record:
            ev[1].record(stream)
        mdn._check(L.mdn_filter_level(C.c_void_p(z1.data_ptr()), C.c_void_p(z2.data_ptr()), mdn.F16, n, hl[1],
                                      wl[1], C.c_void_p(banks[1].data_ptr()), mdn.F16, C.byref(geom),
                                      C.byref(bps[1]), C.c_void_p(u1.data_ptr()), None, sp))
        if record:
            ev[2].record(stream)
        mdn._check(L.mdn_filter_level(C.c_void_p(x.data_ptr()), C.c_void_p(u1.data_ptr()), mdn.F16, n, H, W,
                                      C.c_void_p(banks[0].data_ptr()), mdn.F16, C.byref(geom), C.byref(bps[0]),
                                      C.c_void_p(out.data_ptr()), None, sp))
        if record:
            ev[3].record(stream)

    # the level-wise sequence is exactly what mdn_denoise_multiscale launches
    ref = mdn.denoise_multiscale(x, banks, geom, bps)
    step(False)
    torch.cuda.synchronize()
    assert torch.equal(ref, out), "level-wise step differs from mdn_denoise_multiscale"

    for _ in range(args.warmup):
        step(False)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(args.local_rank) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            ev = evs[k]
            step(True)
        t1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    if dist is not None:
        dist.barrier()
    pyr = [e[0].elapsed_time(e[1]) for e in evs]
    lv1 = [e[1].elapsed_time(e[2]) for e in evs]
    lv0 = [e[2].elapsed_time(e[3]) for e in evs]

    # ---- end to end: pinned host frames -> device -> denoise -> host, through
    # mdn_denoise_multiscale_pipelined (chunks of e2e_chunk frames: uploads,
    # kernels and downloads of consecutive chunks overlap; two compute streams).
    # Consecutive steps alternate between two sets of device buffers and
    # streams (double buffering), so one step's last download overlaps the
    # next step's first upload; every step still copies its whole batch in and
    # its whole result out inside the timed region.
    host_in = torch.empty((n, 3, H, W), dtype=torch.float16, pin_memory=True)
    host_in.copy_(torch.from_numpy(frames.astype(np.float16)))
    chunk = max(1, min(args.e2e_chunk, n))
    per = (mdn.denoise_workspace_bytes(chunk, H, W, LEVELS, mdn.F16) + 255) // 256 * 256
    sets = []
    for k in range(2):
        comp = stream if k == 0 else torch.cuda.Stream(device=dev)
        sets.append({"host_out": torch.empty_like(host_in, pin_memory=True), "xin": torch.empty_like(x),
                     "dout": torch.empty_like(x), "ws": torch.empty(2 * per, dtype=torch.uint8, device=dev),
                     "streams": (torch.cuda.Stream(device=dev), comp, torch.cuda.Stream(device=dev),
                                 torch.cuda.Stream(device=dev))})

    def e2e_step(k):
        st_ = sets[k % 2]
        mdn.denoise_multiscale_pipelined(host_in, banks, geom, bps, st_["host_out"], chunk=chunk, dev_in=st_["xin"],
                                         dev_out=st_["dout"], ws=st_["ws"], streams=st_["streams"])

    e2e_step(0)
    e2e_step(1)
    torch.cuda.synchronize()
    assert torch.equal(sets[0]["host_out"], ref.cpu()) and torch.equal(sets[1]["host_out"], ref.cpu()), \
        "pipelined host path differs from the device path"
    for k in range(max(2, args.warmup)):
        e2e_step(k)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sets[1]["streams"][1].wait_event(e0)
    e2e_steps = max(2, args.steps // 2)
    for k in range(e2e_steps):
        e2e_step(k)
    join = torch.cuda.Event()
    join.record(sets[1]["streams"][1])
    stream.wait_event(join)
    e1.record(stream)
    torch.cuda.synchronize()
    ems = max_over_ranks(e0.elapsed_time(e1), world, dev)

    if rank != 0:
        return
    variants = run_variants(mdn, x, geom, dev, stream) if args.variants else None
    pix = n * H * W
    value = whole_job_rate(pix, args.steps, world, ms)
    e2e_value = whole_job_rate(pix, e2e_steps, world, ems)
    # roofline of the dominant kernel (level-0 fused select + filter).  Its
    # binding roof is the FP32 ALU: algorithmic FLOPs per filtered pixel =
    # 3 x 98 x 2 = 588 (filter) + 180 (structure tensor, features, colour
    # conversions) = 768; peak = 152 SMs x 128 FP32 lanes x 2 FLOP x the SM
    # clock.  The HBM roof is reported beside it: algorithmic bytes per launch =
    # read z^0 (6 B/px) + read u^1 (1.5 B per finest px) + write u^0 (6 B/px)
    # = 13.5 B per finest pixel, against the measured copy bandwidth.
    t_lv0 = statistics.mean(lv0) * 1e-3
    bytes_lv0 = 13.5 * pix
    achieved = bytes_lv0 / t_lv0 / 1e9
    peak, peak_kind = measured_peaks()
    clk_summary = clk.summary()
    flop_rate = 768.0 * pix / t_lv0 / 1e12
    sm_mhz = clk_summary["sm_mhz"] or 2070.0
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "3-level denoise of 8 x 4032x3024 RGB frames per GPU, FP16 storage, FP32 "
                               "arithmetic, 7x7+7x7 per-channel YCbCr filters, 216 buckets/level, FP16 banks",
                   "batch_per_gpu": n, "h": H, "w": W, "levels": LEVELS, "storage": "f16",
                   "l2": "inputs larger than L2 (585 MB per step)", "parallelism": f"replicas x{world}"},
        "gpu_launches": 4 * args.steps,
        "kernel_ms": {"pyramid": round(statistics.mean(pyr), 4), "level1": round(statistics.mean(lv1), 4),
                      "level0": round(statistics.mean(lv0), 4)},
        "roofline": {"bound": "alu", "kernel": "k_level3 (level 0)", "achieved": round(flop_rate, 2),
                     "peak": round(alu_peak, 1), "unit": "TFLOP/s", "frac": round(flop_rate / alu_peak, 4),
                     "traffic": (round(LEVEL0_TRAFFIC_PER_FRAME * n) if LEVEL0_TRAFFIC_PER_FRAME else None),
                     "traffic_note": "ncu DRAM read+write of a one-frame capture, scaled by frames",
                     "flop_per_pixel": 768, "peak_source":
                         "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x median SM clock (FMA throughput probe on "
                         "this part: 72-76 TFLOP/s at 2.07 GHz)",
                     "hbm": {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(achieved / peak, 4),
                             "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"},
                     "note": "bound on chip by shared-memory wavefronts and issue (see profiles/); at 768 FLOP per "
                             "13.5 B the kernel's HBM roof is about 5x its FP32 ALU roof"},
        "e2e": {"value": round(e2e_value, 2), "unit": "Mpix/s", "h2d_bytes_per_step": int(pix * 3 * 2),
                "d2h_bytes_per_step": int(pix * 3 * 2), "api": "mdn_denoise_multiscale_pipelined",
                "chunk_frames": chunk, "compute_streams": 2, "buffer_sets": 2,
                "ms_per_step": round(ems / e2e_steps, 4)},
        "clocks": {"sm_mhz": clk_summary["sm_mhz"], "sm_max_mhz": clk_summary["sm_max_mhz"],
                   "reasons": clk_summary["reasons"]},
    }
    if variants is not None:
        line["variants"] = variants
    if args.train and world == 1:
        line["training"] = run_training(args, dev)
    if args.serve and world == 1:
        line["serving"] = serving_subprocess(args)
    if args.accuracy and world == 1:
        line["accuracy"] = {"headline": accuracy_headline(mdn, frames[0], random_banks(7), dev)}
        if args.train:
            line["accuracy"]["training_vs_oracle"] = accuracy_training(mdn, dev)
    if args.autotune and world == 1:
        line["autotune"] = run_autotune(mdn)
    if args.cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_block(12, 1)
    print(json.dumps(line), flush=True)


def run_autotune(mdn):
    """The level-kernel autotuner on the metric's configurations (after every
    timed section; the table is emptied again so that nothing above depends
    on it): ms per call of each applicable variant and the chosen one, per
    (geometry, storage, bank type, buckets, size)."""
    out = []
    g33, g32 = mdn.Geometry(3, 3), mdn.Geometry(3, 2)
    for name, geom, bp, dt, bdt, n, h, w in [
            ("7x7+7x7 216 f16/f16 12MP", g33, mdn.default_bparams(0), mdn.F16, mdn.F16, 1, H, W),
            ("7x7+7x7 216 f16/f16 1080p", g33, mdn.default_bparams(0), mdn.F16, mdn.F16, 1, 1080, 1920),
            ("7x7+7x7 216 f16/f16 2016x1512 (level 1)", g33, mdn.default_bparams(1), mdn.F16, mdn.F16, 1,
             (H + 1) // 2, (W + 1) // 2),
            ("7x7+7x7 216 f32/f32 12MP", g33, mdn.default_bparams(0), mdn.F32, mdn.F32, 1, H, W),
            ("7x7+7x7 216 f32/f32-prepared 12MP", g33, mdn.default_bparams(0), mdn.F32, mdn.F32_ROWS, 1, H, W),
            ("7x7+5x5 4096 f16/f16 12MP", g32, mdn.paper_grid_bparams(0), mdn.F16, mdn.F16, 1, H, W),
            ("7x7+5x5 4096 f16/f16-prepared 12MP", g32, mdn.paper_grid_bparams(0), mdn.F16, mdn.F16_ROWS, 1, H, W)]:
        best, ms = mdn.autotune_level(geom, bp, dt, bdt, n, h, w)
        out.append({"config": name, "chosen": mdn.LEVEL_VARIANTS[best], "ms": ms})
    mdn.autotune_clear()
    return out


# ---------------------------------------------------------------- serving

SERVE_SIZES = [(480, 640), (720, 1280), (1080, 1920), (3024, 4032)]
SERVE_SIGMAS = [15, 25, 50]


def _serve_stream(mdn, srv, sets, geom, frames, out_pool, pick, arr, dev):
    """One Poisson request stream through the server, then through the plain
    per-image path (one mdn_denoise_multiscale per request, in arrival order,
    torch copies in and out); latency percentiles and Mpix/s of both."""
    import threading
    import torch
    nreq = len(pick)
    sizes = list(out_pool)
    pix = sum(hw[0] * hw[1] for hw, _, _ in pick)
    # server: submissions at the arrival times, a poller thread (blocking
    # poll, GIL released in the C call) timestamps completions.  Output
    # buffers: a LIFO pool of 8 per size (the most recently released host
    # buffer is reused first; past 8 in flight of one size buffers are shared
    # round-robin, the bench does not read outputs).
    lat, inflight, spill = [], {}, {hw: 0 for hw in sizes}
    free = {hw: list(range(len(out_pool[hw]) - 1, -1, -1)) for hw in sizes}
    internal, by_size = [], {hw: [] for hw in sizes}
    lock = threading.Lock()
    stop = [False]

    def poller():
        got = 0
        while got < nreq and not stop[0]:
            for r in srv.poll(64, 50):
                t = time.perf_counter() - t0
                with lock:
                    a, hw_, bi = inflight.pop(r["id"])
                    if bi not in free[hw_]:
                        free[hw_].append(bi)
                    lat.append((t - a) * 1e3)
                    by_size[hw_].append((t - a) * 1e3)
                    internal.append(r["done_ms"] - r["submit_ms"])
                got += 1

    t0 = time.perf_counter()
    th = threading.Thread(target=poller)
    th.start()
    for i in range(nreq):
        wait = arr[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        hw, si, f = pick[i]
        with lock:
            if free[hw]:
                bi = free[hw].pop()
            else:
                bi = spill[hw] % len(out_pool[hw])
                spill[hw] += 1
            rid = srv.submit(frames[hw][f], out_pool[hw][bi], si)
            inflight[rid] = (arr[i], hw, bi)
    th.join(timeout=120)
    stop[0] = True
    span = time.perf_counter() - t0
    pct = lambda v, q: round(float(np.percentile(v, q)), 3)
    srv_line = {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mpix_s": round(pix / span / 1e6, 1),
                "internal_p50_ms": pct(internal, 50), "internal_p99_ms": pct(internal, 99),
                "by_size_p50_p99_ms": {f"{w}x{h}": [pct(v, 50), pct(v, 99)] for (h, w), v in by_size.items() if v}}
    # plain per-image path, same stream of requests
    lat_b = []
    stream = torch.cuda.current_stream()
    xin = {hw: torch.empty((1, 3, *hw), dtype=torch.float16, device=dev) for hw in sizes}
    t0 = time.perf_counter()
    for k in range(nreq):
        wait = arr[k] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        hw, si, f = pick[k]
        banks, bps = sets[si]
        xin[hw][0].copy_(frames[hw][f], non_blocking=True)
        y = mdn.denoise_multiscale(xin[hw], banks, geom, bps)
        out_pool[hw][0].copy_(y[0], non_blocking=True)
        stream.synchronize()
        lat_b.append((time.perf_counter() - t0 - arr[k]) * 1e3)
    span_b = time.perf_counter() - t0
    return srv_line, {"p50_ms": pct(lat_b, 50), "p99_ms": pct(lat_b, 99), "mpix_s": round(pix / span_b / 1e6, 1)}


def run_serving(args, dev):
    """Poisson request streams (mixed sizes, sigma and level count) through
    the continuous-batching server and through the plain per-image path;
    p50/p99 latency and Mpix/s for both at every rate.  Then the paper's
    16 x 16 x 16 grid (4096 buckets, 7x7 + 5x5 taps) served the same way at
    one rate (the server reads its prepared banks through L2; the per-image
    path is given the banks prepared too)."""
    import torch
    import paper_1802_06130_gb300 as mdn
    import synth
    rng = np.random.default_rng(50000)
    # bank sets: one per (sigma, levels in {3, 4}); random FP16 banks
    sets, set_of = [], {}
    for si, sg in enumerate(SERVE_SIGMAS):
        for L in (3, 4):
            banks = [torch.tensor(b, dtype=torch.float16, device=dev) for b in random_banks(100 + 10 * si + L, nb=L - 1)]
            set_of[(sg, L)] = len(sets)
            sets.append((banks, [mdn.default_bparams(l) for l in range(L - 1)]))
    # two distinct pinned input frames per size
    frames = {(h, w): [torch.tensor(synth.noisy_pair(h, w, 50100 + i + h)[0], dtype=torch.float16).pin_memory()
                       for i in range(2)] for (h, w) in SERVE_SIZES}
    nreq = args.serve_requests
    out_pool = {hw: [torch.empty((3, *hw), dtype=torch.float16).pin_memory() for _ in range(8)] for hw in SERVE_SIZES}
    geom = mdn.Geometry(3, 3)
    results = []
    srv = mdn.Server(sets, budget_bytes=80 << 30, max_active=64, autotune=True)
    tune = srv.stats()
    try:
        for rate in args.serve_rates:
            arr = np.cumsum(rng.exponential(1.0 / rate, nreq))
            pick = []
            for _ in range(nreq):
                hw, sg, L = SERVE_SIZES[rng.integers(4)], SERVE_SIGMAS[rng.integers(3)], int(rng.integers(3, 5))
                pick.append((hw, set_of[(sg, L)], int(rng.integers(2))))
            srv_line, img_line = _serve_stream(mdn, srv, sets, geom, frames, out_pool, pick, arr, dev)
            results.append({"rate_rps": rate, "requests": nreq,
                            "label": "saturation sweep (offered load above capacity)" if rate >= 1000 else "offered load",
                            "server": srv_line, "per_image": img_line})
        st = srv.stats()
    finally:
        srv.close()
    # the paper's grid: 4096 buckets, 7x7 + 5x5 per channel, 3 levels
    pg = mdn.Geometry(3, 2)
    pbanks = [torch.tensor(b, dtype=torch.float16, device=dev) for b in random_banks(900, D=74, K=4096, nb=2)]
    pbps = [mdn.paper_grid_bparams(l) for l in range(2)]
    psrv = mdn.Server([(pbanks, pbps)], budget_bytes=40 << 30, max_active=64, autotune=True, geom=pg)
    try:
        rate, n = args.paper_grid_rate, max(nreq // 2, 1)
        arr = np.cumsum(rng.exponential(1.0 / rate, n))
        pick = [(SERVE_SIZES[rng.integers(4)], 0, int(rng.integers(2))) for _ in range(n)]
        srv_line, img_line = _serve_stream(mdn, psrv, [([mdn.prepare_bank(b, pg) for b in pbanks], pbps)], pg,
                                           frames, out_pool, pick, arr, dev)
        paper = {"workload": "the paper's 16x16x16 grid (4096 buckets), 7x7 + 5x5 taps, 3 levels; sizes as above",
                 "rate_rps": rate, "requests": n, "server": srv_line, "per_image": img_line,
                 "tile_variant": psrv.stats()["tile_variant"]}
    finally:
        psrv.close()
    return {"workload": "Poisson arrivals; sizes uniform over 640x480, 1280x720, 1920x1080, 4032x3024 FP16; "
                        "sigma in {15,25,50}/255 and 3 or 4 levels per request (one bank set each); 80 GB budget; "
                        "64 slots; host transfers by SM copy kernels (pinned, aligned buffers)",
            "rates": results, "tile_variant": tune["tile_variant"],
            "autotune_ms": [round(v, 3) for v in tune["variant_ms"]],
            "mean_stages_per_tick": round(st["tick_items"] / max(st["ticks"], 1), 2),
            "large_ticks": st["ticks_large"], "paper_grid": paper}


# ---------------------------------------------------------------- training

def _gen_pair_1mp(seed):
    import synth
    return synth.noisy_pair(1024, 1024, seed)


def run_training(args, dev):
    """Bucketed Gram accumulation (sort + Gram + FP64 reduce) on config-3 data:
    n x 1024x1024 pairs (n = 256 by default: 268,435,456 patches), sigma
    25/255, cross-channel 7x7x3 regressors (D = 147) + 3 targets; every Gram
    precision.  Algorithmic FLOPs per patch = Dp (Dp + 1) with Dp = 150 (the
    upper triangle of the symmetric Gram).  Each tensor-core precision's Gram
    and solved bank are compared with the FP32 CUDA-core path on the same
    patches (relative Frobenius; per bucket for n_k >= 10 D)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import torch
    import paper_1802_06130_gb300 as mdn
    n = args.train_images
    Z = torch.empty((n, 3, 1024, 1024), dtype=torch.float32, device=dev)
    U = torch.empty_like(Z)
    with cf.ProcessPoolExecutor(max_workers=min(n, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        for i, (z, u) in enumerate(ex.map(_gen_pair_1mp, [30000 + i for i in range(n)])):
            Z[i].copy_(torch.from_numpy(z))
            U[i].copy_(torch.from_numpy(u))
    geom = mdn.Geometry(3, -1, 1)
    bp = mdn.default_bparams(0)
    npatch = n * 1024 * 1024
    alg = npatch * 150 * 151
    peaks = measured_tensor_peaks()
    out = {"workload": f"{n} x 1024x1024 pairs, cross-channel 7x7x3 (D=147) + 3 targets, 216 buckets",
           "patches": npatch, "precisions": {}}
    ref = None
    for prec, name in [(0, "fp32_simt"), (1, "tf32"), (2, "bf16"), (3, "split_bf16")]:
        ws = None
        times = []
        for rep in range(3):
            s_, e_ = torch.cuda.Event(True), torch.cuda.Event(True)
            s_.record()
            g, c, _ = mdn.train_level_filters(Z, None, U, geom, bp, prec, lam=1e-3, solve=False, ws=ws)
            e_.record()
            torch.cuda.synchronize()
            times.append(s_.elapsed_time(e_))
        ms = min(times[1:])
        d = {"ms": round(ms, 3), "mpatch_s": round(npatch / ms / 1e3, 1), "alg_tflops": round(alg / ms / 1e9, 2)}
        if prec in (1, 2, 3):
            mult = 3 if prec == 3 else 1
            peak = peaks["tf32"] if prec == 1 else peaks["bf16"]
            d["tensor_frac_of_peak"] = round(mult * alg / ms / 1e9 / peak, 4)
            d["peak_tflops"] = round(peak, 1)
        bank, status = mdn.solve_bank(g, c, geom, 1e-3)
        gn, bn, cn = g.cpu().numpy(), bank.cpu().numpy().astype(np.float64), c.cpu().numpy()
        if ref is None:
            ref = (gn, bn, cn)
        else:
            big = np.nonzero(cn >= 10 * 147)[0]
            per = [np.linalg.norm(bn[k] - ref[1][k]) / np.linalg.norm(ref[1][k]) for k in big]
            d["vs_fp32_simt"] = {"gram_rel": float(f"{np.linalg.norm(gn - ref[0]) / np.linalg.norm(ref[0]):.3g}"),
                                 "bank_rel": float(f"{np.linalg.norm(bn - ref[1]) / np.linalg.norm(ref[1]):.3g}"),
                                 "bank_rel_per_bucket_median": float(f"{np.median(per):.3g}"),
                                 "bank_rel_per_bucket_max": float(f"{np.max(per):.3g}"),
                                 "buckets_compared": int(len(big)), "counts_equal": bool(np.array_equal(cn, ref[2]))}
        d["solve_status"] = int(status.item())
        out["precisions"][name] = d
        del g, c, bank
    out["peak_source"] = peaks["source"]
    # the paper's own selector grid and footprint on the same pairs: 16 x 16 x 16
    # = 4096 buckets, 7x7 fine + 5x5 coarse per channel (D = 74, three Gram
    # groups of Dp = 75), the coarse input z^1 of each pair; TF32
    pg = mdn.Geometry(3, 2)
    Zc = mdn.build_pyramid(Z, 2)[0]
    times = []
    for rep in range(3):
        s_, e_ = torch.cuda.Event(True), torch.cuda.Event(True)
        s_.record()
        g, c, _ = mdn.train_level_filters(Z, Zc, U, pg, mdn.paper_grid_bparams(0), mdn.GRAM_TF32, lam=1e-3,
                                          solve=False)
        e_.record()
        torch.cuda.synchronize()
        times.append(s_.elapsed_time(e_))
    ms = min(times[1:])
    alg16 = npatch * 3 * 75 * 76
    out["grid16x16x16_7x7+5x5_tf32"] = {
        "ms": round(ms, 3), "mpatch_s": round(npatch / ms / 1e3, 1), "alg_tflops": round(alg16 / ms / 1e9, 2),
        "counts_total_ok": bool(int(c.sum().item()) == npatch), "buckets_hit": int((c > 0).sum().item())}
    del g, c, Zc
    return out


def _gen_pair(args_):
    import synth
    h, w, seed, sigma = args_
    return synth.noisy_pair(h, w, seed, sigma=sigma)


def run_quality(args, dev):
    """Whole-pipeline sanity check on synthetic data (the paper's test images
    and training set are not available): banks trained on the GPU, then
    denoising of held-out frames, PSNR = 10 log10(1 / MSE) against the clean
    frame.  Config 1: 8 pairs of 256x256, sigma 25/255, 5x5 single-level
    filters, with and without the dihedral augmentation.  Config 2: 1920x1080,
    3 levels, 7x7 + 7x7 filters, one bank set per sigma in {15, 25, 50}/255
    trained on args.quality_pairs pairs; held-out frames are denoised with the
    bank set of the nearest estimated noise level."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import torch
    import paper_1802_06130_gb300 as mdn

    def psnr(a, b):
        return float(10 * np.log10(1.0 / np.mean((a.astype(np.float64) - b) ** 2)))

    sig = [15 / 255, 25 / 255, 50 / 255]
    npair = args.quality_pairs
    jobs = [(256, 256, 1000 + i, 25 / 255) for i in range(8)] + [(256, 256, 2000, 25 / 255)]
    train_at, test_at = [], []
    for si, s_ in enumerate(sig):
        train_at.append(len(jobs))
        jobs += [(1080, 1920, 10000 + 1000 * si + i, s_) for i in range(npair)]
        test_at.append(len(jobs))
        jobs += [(1080, 1920, 20000 + 1000 * si + i, s_) for i in range(4)]
    with cf.ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        data = list(ex.map(_gen_pair, jobs))
    out = {}
    # config 1
    tr, te = data[:8], data[8]
    Z = torch.tensor(np.stack([p[0] for p in tr]), device=dev)
    U = torch.tensor(np.stack([p[1] for p in tr]), device=dev)
    g1 = mdn.Geometry(2, -1)
    xt = torch.tensor(te[0], device=dev)[None]
    c1 = {"psnr_noisy_db": round(psnr(te[0], te[1]), 2)}
    for aug in (False, True):
        banks, _ = mdn.train_cascade(Z, U, g1, 1, augment=aug)
        y = mdn.denoise_multiscale(xt, banks, g1, [mdn.default_bparams(0)])
        c1["psnr_denoised_augmented_db" if aug else "psnr_denoised_db"] = round(psnr(_np_(y[0]), te[1]), 2)
    out["config1_256x256_single_level_5x5"] = c1
    # config 2
    g2 = mdn.Geometry(3, 3)
    bsets = []
    for si in range(3):
        tr = data[train_at[si]:train_at[si] + npair]
        Z = torch.tensor(np.stack([p[0] for p in tr]), device=dev)
        U = torch.tensor(np.stack([p[1] for p in tr]), device=dev)
        banks, _ = mdn.train_cascade(Z, U, g2, 3, chunk=4)
        bsets.append(banks)
        del Z, U
    c2 = {"training_pairs_per_sigma": npair, "per_sigma": []}
    for si in range(3):
        rows = []
        for k in range(4):
            z, u = data[test_at[si] + k]
            x = torch.tensor(z, device=dev)[None]
            est = float(mdn.estimate_noise(x)[0])
            pick = mdn.nearest_level(est, sig)
            y = mdn.denoise_multiscale(x, bsets[pick], g2, [mdn.default_bparams(l) for l in range(2)])
            rows.append((psnr(z, u), psnr(_np_(y[0]), u), est * 255, pick == si))
        r = np.array(rows, dtype=np.float64)
        c2["per_sigma"].append({"sigma_255": round(sig[si] * 255), "psnr_noisy_db": round(r[:, 0].mean(), 2),
                                "psnr_denoised_db": round(r[:, 1].mean(), 2),
                                "sigma_estimate_255": round(r[:, 2].mean(), 2),
                                "bank_set_chosen_correctly": int(r[:, 3].sum())})
    out["config2_1080p_3level_7x7_7x7"] = c2
    return out


def _np_(t):
    return t.detach().float().cpu().numpy()


def measured_tensor_peaks():
    """Dense tensor peaks: measured BF16 (burst) and TF32 = BF16 x the nominal
    ratio 1.1 / 2.25."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    bf16, src = 1900.0, "fallback"
    if os.path.exists(p):
        with open(p) as f:
            bf16, src = json.load(f).get("bf16_tflops", 1900.0), "measured"
    return {"bf16": bf16, "tf32": bf16 * 1.1 / 2.25, "source": src + " (TF32 = BF16 x 1.1/2.25 nominal)"}


def serving_subprocess(args):
    """The serving measurement runs in a fresh process (its own CUDA context and
    host memory) so that the throughput benchmark's allocations do not colour
    its latencies."""
    cmd = [sys.executable, os.path.abspath(__file__), "--serve-only", "--serve-requests", str(args.serve_requests),
           "--serve-rates", *[str(r) for r in args.serve_rates], "--paper-grid-rate", str(args.paper_grid_rate)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=1800)
    for ln in r.stdout.splitlines()[::-1]:
        if ln.startswith("{"):
            return json.loads(ln)
    return {"error": (r.stderr or r.stdout)[-500:]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--e2e-chunk", type=int, default=1, help="frames per chunk of the pipelined end-to-end path")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-serve", dest="serve", action="store_false")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[50, 100, 200, 400, 1600])
    ap.add_argument("--paper-grid-rate", type=float, default=200, help="request rate of the 4096-bucket serving run")
    ap.add_argument("--serve-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-train", dest="train", action="store_false")
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--no-accuracy", dest="accuracy", action="store_false")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--train-images", type=int, default=256)
    ap.add_argument("--train-only", action="store_true", help="only the training section (profiling driver)")
    ap.add_argument("--quality", action="store_true", help="whole-pipeline PSNR sanity check (configs 1 and 2), then exit")
    ap.add_argument("--quality-pairs", type=int, default=16, help="training pairs per sigma for --quality config 2")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    args.local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.train_only:
        import torch
        import paper_1802_06130_gb300 as mdn
        mdn.build()
        print(json.dumps(run_training(args, torch.device("cuda", args.local_rank))), flush=True)
        return
    if args.quality:
        import torch
        import paper_1802_06130_gb300 as mdn
        mdn.build()
        print(json.dumps(run_quality(args, torch.device("cuda", args.local_rank))), flush=True)
        return
    if args.serve_only:
        import torch
        import paper_1802_06130_gb300 as mdn
        mdn.build()
        print(json.dumps(run_serving(args, torch.device("cuda", args.local_rank))), flush=True)
        return
    # frames first: the spawn pool runs before this process touches CUDA
    frames = make_frames(args.batch, 40000 + 100 * rank)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(args.local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", args.local_rank))
    try:
        run_gpu(args, rank, world, frames)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
