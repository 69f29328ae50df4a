#!/usr/bin/env python
"""Benchmark: isosurfaces of a block-compressed 512^3 volume on one GB300.

Workload (a stand-in for the paper's Plasma 512^3, Table "mc_benchmark_data"):
512^3 float32 six-octave gradient noise (seed 1), compressed at 8 bits per
value in 4^3 blocks (128 MiB), isovalues -1, -0.5, 0, 0.5, 1 extracted one
after another.  One step = drop the decoded-block cache, then extract the
five surfaces in order (the first decodes every active block, the later
ones reuse what the cache holds, as in the paper's sweep benchmarks).

Metric: triangles/s (whole step, all five surfaces), with voxels/s
(5 * 512^3 per step) and the p50/p99 latency of one isovalue change.

  value    device-resident volume; each surface written into a
           preallocated device buffer (iso_extract_into); CUDA events on
           the library's stream around each step; L2 flushed between steps
  e2e      the same step through the public API from host memory: upload
           the compressed volume and ranges from pinned host buffers
           (iso_load_volume), five iso_extract calls (library-allocated
           meshes), read back the counts, release; volumes are streamed
           with double buffering (the next volume's upload overlaps this
           volume's surfaces), and the one-at-a-time figure is reported
           beside it as e2e.serial
  roofline one whole extraction from an empty cache (every kernel, the
           count readback): the bytes the method must move per surface,
           n_new * (8R + 256) + 48T, over its CUDA-event duration, against
           the measured HBM copy peak; the dominant kernel's own figure
           (algorithmic bytes per launch over its duration) nested in it
  serving  the request loop on the serving volume at a quarter of its x
           and y extent (2560 x 1920 x 1536 channel flow, 2 bits/value,
           4 GB cache budget): Poisson isovalue requests served by the
           batched server (max_batch 2 and 8) and by the plain per-request
           path, and both under overload; p50/p99 latency and triangles/s;
           a warm single request both ways (--workload serve runs the full
           size)
  configs  sphere64 and channel2k extracted whole, cold and warm
  cpu_baseline  the plain CPU oracle on a bounded window of the same field
  parity   the library on that window against the oracle's surfaces:
           triangle counts, order and block ids exact, and the largest
           float32-vs-float64 position difference
  packed_vertices / indexed_mesh  the same steps writing the compact
           8-byte vertices / the within-block indexed mesh
  render   the isovalue-0 surface drawn at 1920x1080 (iso_render) as the
           float4 soup, the compact soup and the indexed mesh

--impl reference times the CPU oracle alone (the reference arm: there is no
other implementation of this method to run).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (512, 512, 512)
RATE = 8
SEED = 1
ISOS = (-1.0, -0.5, 0.0, 0.5, 1.0)
METRIC = "triangles/s and voxels/s per isosurface on 1 GB300; p50/p99 isovalue-change latency"
WORKLOAD = ("noise512: 512^3 float32 6-octave gradient noise (seed 1), fixed rate 8 bits/value in 4^3 blocks, "
            "isovalues -1,-0.5,0,0.5,1 extracted in sequence from a cold decoded-block cache")
CPU_WINDOW = (512, 512, 128)      # oracle sample: a window of the same field (about 11 s on one core)
CPU_ORIGIN = (0, 0, 192)
REF_WINDOW = (128, 128, 64)       # per-step sample of the reference arm
L2_FLUSH_BYTES = 512 << 20
CTL_BYTES = 168                   # control block (struct Ctl): iso_extract reads it back after the scan and after the emission
KERNELS_PER_SURFACE = 8           # prep, cull, lru_a, lru_b (list append), decode, count, scan, emit
KERNELS_PER_RESET = 2
KERNELS = ("cull", "cache_update", "decode", "count", "scan", "emit")
KERNEL_OF = {"cull": ("cull_kernel", "extract.cu"), "cache_update": ("lru_a_kernel+lru_b_kernel", "extract.cu"),
             "decode": ("decode_new_kernel", "extract.cu"), "count": ("mc_count_kernel", "mc.cu"),
             "scan": ("mc_scan_kernel", "mc.cu"), "emit": ("mc_emit_kernel", "mc.cu")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-volume batch comparison")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg of the default run")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other single-volume configurations (sphere64, channel2k) of the default run")
    ap.add_argument("--workload", default="noise512", choices=["noise512", "serve"],
                    help="serve: the request loop on the 10240x7680x1536 channel volume")
    ap.add_argument("--serve-scale", type=float, default=1.0,
                    help="fraction of the serving volume's x and y extent (1 = full size)")
    ap.add_argument("--requests", type=int, default=1000,
                    help="requests of --workload serve (the default run's serving leg takes 200)")
    ap.add_argument("--dims", type=int, default=512,
                    help="cube edge of the noise volume (default 512; smaller sizes are for profiling captures)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_over_ranks(seconds, units, device):
    """Whole-job figures of independent replicas: the slowest rank's time and
    the units all ranks processed (the process group must be initialised)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(n)
    return float(t.item()), float(n.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampled every 100 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[4:8]) if v.lower() == "active"})
        busy = sorted(sm)[len(sm) // 4:] if len(sm) > 4 else sm     # drop idle samples at the edges
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- helpers

def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


PROFILE_SOURCES = ("extract.cu", "mc.cu", "codec.cuh", "common.cuh", "kernels.cuh", "launch.cuh", "tile_scan.cuh")


def profile_sources_sha():
    h = hashlib.sha256()
    for f in PROFILE_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2009_03254_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profile_line(key):
    """A figure of the committed launch list of the benchmark's cold
    extractions (profiles/extraction_cold_noise512.md), if it was taken on
    the current kernel sources (else None)."""
    try:
        text = open(os.path.join(ROOT, "profiles", "extraction_cold_noise512.md")).read()
        sha = profile_sources_sha()
    except OSError:
        return None
    for line in text.splitlines():
        parts = line.split()
        if len(parts) >= 4 and parts[0] == key + ":" and parts[2] == "sources_sha256_16:" and parts[3] == sha:
            return float(parts[1])
    return None


def profile_traffic(kernel_file, kernel):
    """DRAM bytes per launch of `kernel` over the benchmark's cold extractions."""
    return profile_line(f"traffic_per_launch_bytes[{kernel}]")


def extraction_traffic():
    """DRAM bytes of one cold extraction (all its kernels, mean over the five
    isovalues) from the committed launch list."""
    return profile_line("traffic_per_extraction_bytes")


def stage_bytes(stats, rate, nb):
    """Algorithmic bytes each kernel must move for one surface."""
    na, nn, nc, T = stats["n_active"], stats["n_new"], stats["n_candidates"], stats["num_triangles"]
    no = stats["n_occupied"]
    return {
        "cull": 8 * nb + nb / 8 + 4 * na + 4 * nn + 8 * na + 4 * nc,   # hulls, mask, I_active, I_new, +group hulls, I_cand
        "cache_update": 0.0,
        "decode": nn * (8 * rate + 256 + 8),                           # compressed in, decoded out, I_new + slot
        "count": nc * (256 + 4 + 4 + 64),                              # decoded tiles in, id in, count and cases out
        "scan": nc * (4 + 8) + 4 * no,                                 # counts in, offsets and I_occ out
        "emit": no * (256 + 4 + 4 + 8 + 64) + 48 * T,                  # per occupied block: decoded tile, I_occ, id,
                                                                       # offset, cases in; vertices out
    }


def bytes_bj(stats, rate):
    """Bytes the method must move per extraction by the headline formula:
    compressed blocks read + decoded blocks written + vertices written."""
    return stats["n_new"] * (8 * rate + 256) + 48 * stats["num_triangles"]


def bytes_full(stats, rate, nb):
    """The headline bytes plus the range test's reads (8 B per block), the
    active decoded blocks read once and the masks and id lists."""
    return (bytes_bj(stats, rate) + 8 * nb + 256 * stats["n_active"] + nb / 8 + 12 * stats["n_active"])


# ---------------------------------------------------------------- CPU oracle baseline

def cpu_sample_volume(window, origin):
    """The oracle's input for the CPU baseline: the window of the benchmark
    field (the seeded input generator, on the GPU when there is one: it is
    bit-identical to the NumPy generator and much faster), encoded by the
    oracle's own encoder."""
    import oracle
    from synth import fields
    try:
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError
        import synth.gpu as sg
        sg.build()
        f = sg.gradient_noise(*window, SEED, origin=origin).cpu().numpy()
    except (ImportError, RuntimeError):
        f = fields.gradient_noise(*window, SEED, origin=origin)
    return oracle.encode_volume(f, RATE)


def cpu_oracle_sample(window, origin, isos, volume=None, check=None):
    """The oracle timed on the sample; `check(iso, result)` (untimed) sees
    each surface."""
    import oracle
    bits, bmin, bmax = volume if volume is not None else cpu_sample_volume(window, origin)
    tris, t = 0, 0.0
    for iso in isos:
        t0 = time.perf_counter()
        r = oracle.extract(bits, window, RATE, bmin, bmax, iso)
        t += time.perf_counter() - t0
        tris += r["num_triangles"]
        if check is not None:
            check(iso, r)
    return tris, t


def parity_checker(bc, window, volume):
    """The library on the same encoded sample, compared surface by surface
    with the oracle's: triangle counts, order and block ids exactly, and the
    largest distance between the library's float32 positions and the
    oracle's float64 interpolation of the same decoded samples."""
    bits, bmin, bmax = volume
    vol = bc.Volume(bits, window, RATE, bmin, bmax)
    out = {"triangles_equal": True, "blocks_equal": True, "max_abs_position_error_vs_fp64": 0.0, "triangles": 0}

    def check(iso, ref):
        m = vol.extract(iso)
        try:
            same = m.num_triangles == ref["num_triangles"]
            out["triangles_equal"] &= bool(same)
            out["triangles"] += int(m.num_triangles)
            if same and m.num_triangles:
                v = m.vertices.cpu().numpy().reshape(-1, 3, 4)
                err = float(np.abs(v[:, :, :3].astype(np.float64) - ref["local_pos"]).max())
                out["max_abs_position_error_vs_fp64"] = max(out["max_abs_position_error_vs_fp64"], err)
                out["blocks_equal"] &= bool(np.array_equal(v[:, :, 3].view(np.uint32),
                                                           np.repeat(ref["tri_block"][:, None], 3, axis=1)))
        finally:
            m.release()

    return vol, out, check


def _oracle_slab(args):
    """The oracle, as it stands, on one slab of block layers; returns
    (triangles, seconds)."""
    bits, bmin, bmax, dims, isos = args
    import oracle
    tris, t = 0, 0.0
    for iso in isos:
        t0 = time.perf_counter()
        tris += oracle.extract(bits, dims, RATE, bmin, bmax, iso)["num_triangles"]
        t += time.perf_counter() - t0
    return tris, t


def cpu_oracle_parallel(window, isos, volume):
    """The same sample on all cores: the encoded window split into slabs of
    whole block layers, one spawned process each (the parent holds a CUDA
    context), the oracle unchanged.  A slab also gets the first sample plane
    of the next slab's blocks, so its cells are exactly its own layers' and
    the triangles add up to the single-process count.  Returns (triangles,
    wall seconds of the extraction, processes)."""
    import concurrent.futures
    import multiprocessing as mp
    import oracle
    bits, bmin, bmax = volume
    nbx, nby, nbz = oracle.block_dims(window)
    layer = nbx * nby
    cores = max(1, min(os.cpu_count() or 1, nbz))
    per = -(-nbz // cores)
    jobs = []
    for bz0 in range(0, nbz, per):
        bz1 = min(bz0 + per, nbz) - 1
        last = min(bz1 + 1, nbz - 1)
        zs = min(4 * (bz1 - bz0 + 1) + 1, window[2] - 4 * bz0)
        rows = slice(bz0 * layer, (last + 1) * layer)
        jobs.append((bits[rows], bmin[rows], bmax[rows], (window[0], window[1], zs), isos))
    with concurrent.futures.ProcessPoolExecutor(len(jobs), mp_context=mp.get_context("spawn")) as ex:
        warm = [(j[0][:layer], j[1][:layer], j[2][:layer], (window[0], window[1], 4), isos[:1]) for j in jobs]
        list(ex.map(_oracle_slab, warm))                 # start every worker first
        t0 = time.perf_counter()
        out = list(ex.map(_oracle_slab, jobs))
        wall = time.perf_counter() - t0
    return sum(o[0] for o in out), wall, len(jobs)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from synth import fields
    f = fields.gradient_noise(*REF_WINDOW, SEED, origin=CPU_ORIGIN)
    bits, bmin, bmax = oracle.encode_volume(f, RATE)
    vox = int(np.prod(REF_WINDOW))

    def step():
        n = 0
        for iso in ISOS:
            n += oracle.extract(bits, REF_WINDOW, RATE, bmin, bmax, iso)["num_triangles"]
        return n

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    tris = 0
    for _ in range(args.steps):
        tris += step()
    dt = time.perf_counter() - t0
    value = tris / dt
    sample = (f"{REF_WINDOW[0]}x{REF_WINDOW[1]}x{REF_WINDOW[2]} window at {CPU_ORIGIN} of the 512^3 field, "
              f"5 isovalues per step, single-threaded plain C oracle (decode all blocks, range test, block MC)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "triangles/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "voxels_per_s": 5 * vox * args.steps / dt,
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "triangles/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "triangles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batch of 64 volumes

def measure_batch64(bc, sg, torch, stream, flush, steps):
    """64 volumes of uneven size (each axis log-uniform in [32, 256]), each
    with its own isovalue: one batch (one launch per stage for all volumes,
    replayed as a CUDA graph) against 64 iso_extract_into calls (the plain
    per-request path), from cold caches and from warm ones."""
    from synth import recipes
    recs = recipes.batch64_recipes()
    vols = []
    for r in recs:
        f = sg.generate(r)
        bits, bmin, bmax = bc.encode_field(f, r.rate)
        torch.cuda.synchronize()
        del f
        vols.append(bc.Volume(bits, r.dims, r.rate, bmin, bmax))
    isos = np.array([r.isovalues[0] for r in recs], np.float32)
    voxels = float(sum(np.prod(r.dims) for r in recs))
    b = bc.Batch(vols)
    _, offs, _ = b.extract(isos)
    total = int(offs[-1])
    out = torch.empty((total + 1024, 3, 4), dtype=torch.float32, device="cuda")
    parts = [out[int(offs[i]):int(offs[i + 1])] for i in range(len(vols))]

    def timed(fn, cold):
        ms = []
        for _ in range(max(3, steps) + 2):
            if cold:
                for v in vols:
                    v.cache_reset()
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms[2:]))

    def batch_call():
        b.extract_into(isos, out)

    def plain_calls():
        for i, v in enumerate(vols):
            v.extract_into(float(isos[i]), parts[i])

    res = {"volumes": len(vols), "voxels": voxels, "triangles": total}
    for cold in (True, False):
        key = "cold" if cold else "warm"
        tb, tp = timed(batch_call, cold), timed(plain_calls, cold)
        res[key] = {"batch_ms": tb, "plain_ms": tp, "speedup": tp / tb,
                    "batch_triangles_per_s": total / (tb / 1000.0), "plain_triangles_per_s": total / (tp / 1000.0)}
    tune = b.tune(isos, out, trials=2)
    tb = timed(batch_call, True)
    res["tuned"] = {"shape": tune["shape"], "cold_batch_ms": tb, "tuner_default_ms": tune["default_ms"],
                    "tuner_tuned_ms": tune["tuned_ms"], "cold_speedup_vs_plain": res["cold"]["plain_ms"] / tb}
    res["what"] = ("batch: iso_batch_extract (one launch per stage over all 64 volumes, CUDA graph); plain: 64 "
                   "iso_extract_into calls in sequence; device time (CUDA events) per whole batch, median")
    b.release()
    for v in vols:
        v.release()
    return res


# ---------------------------------------------------------------- our arm

RENDER_SIZE = (1920, 1080)
RENDER_ISO = 0.0


def measure_render(bc, vol, torch, stream, tmax, vmax, frames=10):
    """The rendering step (Section 4.6.2): the isovalue-0 surface drawn at
    1920x1080 from an orbit camera, as the float4 soup, the compact soup and
    the indexed mesh.  Each frame is one iso_render call (fragment clear,
    rasterisation, shading), timed with CUDA events back to back."""
    from synth import cameras
    w, h = RENDER_SIZE
    m = cameras.orbit(DIMS, 30.0, 25.0, distance_factor=1.1, aspect=w / h)
    light = (0.3, -0.5, 0.8)
    frag = torch.empty((h, w), dtype=torch.int64, device="cuda")
    rgba = torch.empty((h, w), dtype=torch.int32, device="cuda")
    soup = torch.empty((tmax + 1024, 3, 4), dtype=torch.float32, device="cuda")
    packed = torch.empty((tmax + 1024, 3, 2), dtype=torch.int32, device="cuda")
    v4 = torch.empty((vmax + 1024, 4), dtype=torch.float32, device="cuda")
    idx = torch.empty((tmax + 1024, 3), dtype=torch.int32, device="cuda")
    T = vol.extract_into(RENDER_ISO, soup)["num_triangles"]
    vol.extract_packed_into(RENDER_ISO, packed)
    V = vol.extract_indexed_into(RENDER_ISO, v4, idx)["num_vertices"]
    cases = {"float4_soup": (soup, None, 48.0 * T), "compact_soup": (packed, None, 24.0 * T),
             "indexed_float4": (v4, idx, 16.0 * V + 12.0 * T)}
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    out = {"workload": f"noise512 isovalue {RENDER_ISO}: {T} triangles, {w}x{h}, orbit camera (azimuth 30, "
                       f"elevation 25 degrees)", "triangles": T}
    for name, (verts, ind, vbytes) in cases.items():
        st = None
        for _ in range(3):
            _, _, st = bc.render(verts, T, DIMS, m, light, w, h, indices=ind, fragments=frag, rgba=rgba, stats=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(frames):
            bc.render(verts, T, DIMS, m, light, w, h, indices=ind, fragments=frag, rgba=rgba)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / frames
        # vertices read once, fragments cleared and read back by shading, image written
        nbytes = vbytes + w * h * (8 + 8 + 4)
        out[name] = {"ms_per_frame": ms, "fps": 1000.0 / ms, "triangles_per_s": T / (ms / 1000.0),
                     "drawn": st["drawn"], "big": st["big"], "alg_bytes_per_frame": nbytes,
                     "GBps": nbytes / (ms / 1000.0) / 1e9, "frac_of_measured_hbm": nbytes / (ms / 1000.0) / 1e9 / peak}
    covered = int((frag != -1).sum())
    out["pixels_covered"] = covered
    # implicit ray casting of the same surface over the block macrocell grid
    # (the cache already holds the isovalue's blocks: the call's front
    # decodes nothing new)
    cam = cameras.pinhole_orbit(DIMS, 30.0, 25.0, distance_factor=1.1, fovy_deg=45.0, aspect=w / h)
    hits = torch.empty((h, w), dtype=torch.int64, device="cuda")
    for _ in range(2):
        _, _, cst = vol.raycast(RENDER_ISO, *cam, light, w, h, hits=hits, rgba=rgba)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(frames):
        vol.raycast(RENDER_ISO, *cam, light, w, h, hits=hits, rgba=rgba)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / frames
    out["raycast"] = {"ms_per_frame": ms, "fps": 1000.0 / ms, "rays_per_s": w * h / (ms / 1000.0),
                      "hits": cst["hits"], "n_active": cst["n_active"], "n_new": cst["n_new"],
                      "what": "iso_raycast per frame: range test, cache update (no new blocks), one thread per "
                              "pixel over blocks whose 2x2x2 range holds the isovalue, then cells"}
    del hits
    out["what"] = ("iso_render per frame: fragment clear, one thread per small triangle, one warp per triangle "
                   "over 32 pixel centres, 64-bit atomicMin on (depth, triangle), Lambert shading to RGBA8")
    del soup, packed, v4, idx, frag, rgba
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_03254_gb300 as bc
    import synth.gpu as sg

    nb = int(np.prod(bc.block_dims(DIMS)))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        field = sg.gradient_noise(*DIMS, SEED)
        bits, bmin, bmax = bc.encode_field(field, RATE)
        torch.cuda.synchronize()
        del field
        vol = bc.Volume(bits, DIMS, RATE, bmin, bmax)
        # size the output buffer from one pass over the isovalues
        tmax = 0
        per_iso = []
        for iso in ISOS:
            m = vol.extract(iso)
            tmax = max(tmax, m.num_triangles)
            per_iso.append(m.stats)
            m.release()
        out = torch.empty((tmax + 1024, 3, 4), dtype=torch.float32, device="cuda")
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        lat = []

        def step(record=None):
            vol.cache_reset()
            tris = 0
            stats = []
            for iso in ISOS:
                t0 = time.perf_counter()
                st = vol.extract_into(iso, out)
                if record is not None:
                    record.append(time.perf_counter() - t0)
                tris += st["num_triangles"]
                stats.append(st)
            return tris, stats

        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        total_tris = 0
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                ev[i][0].record(stream)
                tris, stats = step(lat)
                ev[i][1].record(stream)
                total_tris += tris
            torch.cuda.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in ev]
        total_s = sum(step_ms) / 1000.0
        if world > 1:
            total_s, total_tris = reduce_over_ranks(total_s, total_tris, "cuda")

        # per-kernel durations (same steps, events between the kernels)
        vol.set_profiling(True)
        stage_ms = {k: 0.0 for k in bc.Volume.STAGES}
        stage_b = {k: 0.0 for k in KERNELS}
        prof_steps = max(1, min(args.steps, 5))
        for _ in range(prof_steps):
            flush.zero_()
            vol.cache_reset()
            for iso in ISOS:
                st = vol.extract_into(iso, out)
                ms = vol.stage_times()
                for k in stage_ms:
                    stage_ms[k] += ms[k]
                for k, nbytes in stage_bytes(st, RATE, nb).items():
                    stage_b[k] += nbytes
        vol.set_profiling(False)

        # whole extractions from a cold cache (every active block decoded),
        # against the bytes the method must move
        cold_ms, cold_b, cold_t, cold_full = 0.0, 0.0, 0, 0.0
        for _ in range(prof_steps):
            for iso in ISOS:
                vol.cache_reset()
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                with torch.cuda.nvtx.range("cold_extraction"):     # selects these launches in profiles
                    st = vol.extract_into(iso, out)
                e1.record(stream)
                torch.cuda.synchronize()
                cold_ms += e0.elapsed_time(e1)
                cold_b += bytes_bj(st, RATE)
                cold_full += bytes_full(st, RATE, nb)
                cold_t += st["num_triangles"]
        n_cold = prof_steps * len(ISOS)

        # the same steps with the compact 8-byte vertices (NEXT-1)
        outp = torch.empty((tmax + 1024, 3, 2), dtype=torch.int32, device="cuda")
        vol.set_profiling(True)
        p_ms, p_emit, p_tris = 0.0, 0.0, 0
        for _ in range(prof_steps):
            flush.zero_()
            vol.cache_reset()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for iso in ISOS:
                st = vol.extract_packed_into(iso, outp)
                p_emit += vol.stage_times()["emit"]
                p_tris += st["num_triangles"]
            e1.record(stream)
            torch.cuda.synchronize()
            p_ms += e0.elapsed_time(e1)
        vol.set_profiling(False)
        packed = {"triangles_per_s": p_tris / (p_ms / 1000.0), "ms_per_step": p_ms / prof_steps,
                  "emit_ms_per_surface": p_emit / (prof_steps * len(ISOS)), "bytes_per_triangle": 24,
                  "what": "the same cold-cache 5-isovalue steps writing 8-byte vertices (10-bit block-local "
                          "codes + block id), with per-kernel events on"}
        del outp

        # the same steps writing the within-block indexed mesh (NEXT-3), both
        # vertex formats: sized by one pass, then timed like the packed ones
        empty_v = torch.empty((0, 4), dtype=torch.float32, device="cuda")
        empty_i = torch.empty((0, 3), dtype=torch.int32, device="cuda")
        vmax = max(vol.extract_indexed_into(iso, empty_v, empty_i, check=False)["num_vertices"] for iso in ISOS)
        idx_buf = torch.empty((tmax + 1024, 3), dtype=torch.int32, device="cuda")
        indexed = {}
        for fmt, width, dt, vbytes in (("float4", 4, torch.float32, 16), ("packed", 2, torch.int32, 8)):
            vbuf = torch.empty((vmax + 1024, width), dtype=dt, device="cuda")
            vol.set_profiling(True)
            i_ms, i_emit, i_count, i_tris, i_verts = 0.0, 0.0, 0.0, 0, 0
            for _ in range(prof_steps):
                flush.zero_()
                vol.cache_reset()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for iso in ISOS:
                    st = vol.extract_indexed_into(iso, vbuf, idx_buf)
                    ms = vol.stage_times()
                    i_emit += ms["emit"]
                    i_count += ms["count"]
                    i_tris += st["num_triangles"]
                    i_verts += st["num_vertices"]
                e1.record(stream)
                torch.cuda.synchronize()
                i_ms += e0.elapsed_time(e1)
            vol.set_profiling(False)
            n_s = prof_steps * len(ISOS)
            indexed[fmt] = {"triangles_per_s": i_tris / (i_ms / 1000.0), "ms_per_step": i_ms / prof_steps,
                            "emit_ms_per_surface": i_emit / n_s, "count_ms_per_surface": i_count / n_s,
                            "vertices_per_triangle": i_verts / i_tris,
                            "bytes_per_triangle": (i_verts * vbytes + 12 * i_tris) / i_tris}
            del vbuf
        del idx_buf
        indexed["what"] = ("the same cold-cache 5-isovalue steps writing the indexed mesh: one vertex per cut edge "
                           "of each block's window, uint32 index triples, per-kernel events on")

        render = measure_render(bc, vol, torch, stream, tmax, vmax)

        # the full-volume baselines of the paper's comparisons: decode every block
        # into a dense field; and the extraction with the range test off (every
        # block decoded into the cache and visited, from an empty cache)
        dense = torch.empty((DIMS[2], DIMS[1], DIMS[0]), dtype=torch.float32, device="cuda")
        d_ms = []
        for _ in range(4):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bc.decode_volume(bits, DIMS, RATE, out=dense)
            e1.record(stream)
            torch.cuda.synchronize()
            d_ms.append(e0.elapsed_time(e1))
        # the naive data-parallel marching cubes over that dense field (no
        # blocks, no cache): classify every cell, compact, count, scan, emit
        nv_out = torch.empty((tmax + 1024, 3, 4), dtype=torch.float32, device="cuda")
        bc.mc_dense(dense, ISOS[0], out=nv_out)
        n_ms, n_tris = 0.0, 0
        for iso in ISOS:
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, nst, _ = bc.mc_dense(dense, iso, out=nv_out)
            e1.record(stream)
            torch.cuda.synchronize()
            n_ms += e0.elapsed_time(e1)
            n_tris += nst["num_triangles"]
        del nv_out
        del dense
        d_med = float(np.median(d_ms[1:]))
        a_ms, a_tris = 0.0, 0
        for iso in ISOS:
            vol.cache_reset()
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = vol.extract_all_blocks_into(iso, out)
            e1.record(stream)
            torch.cuda.synchronize()
            a_ms += e0.elapsed_time(e1)
            a_tris += st["num_triangles"]
        baselines = {
            "dense_decode": {"ms": d_med, "decoded_GBps": float(np.prod(DIMS)) * 4 / (d_med / 1000.0) / 1e9,
                             "compressed_GBps": nb * RATE * 8 / (d_med / 1000.0) / 1e9,
                             "what": "iso_decode_volume: every block into a dense float32 field"},
            "naive_dense_mc": {"ms_per_surface": n_ms / len(ISOS), "triangles_per_s": n_tris / (n_ms / 1000.0),
                               "what": "iso_mc_dense over the decoded 512^3 field: every cell classified, the crossing "
                                       "cells compacted, counted, prefix-summed and emitted (two count readbacks per "
                                       "surface); the same triangles as the block path"},
            "all_blocks_extraction": {"ms_per_surface": a_ms / len(ISOS),
                                      "triangles_per_s": a_tris / (a_ms / 1000.0),
                                      "what": "range test off: all 2,097,152 blocks decoded and visited per "
                                              "surface (empty cache), same meshes"}}

        # end to end through the public API from pinned host memory
        e2e = None
        if not args.no_e2e:
            h_bits = bits.cpu().pin_memory()
            h_min = bmin.cpu().pin_memory()
            h_max = bmax.cpu().pin_memory()
            h2d = h_bits.numel() * 8 + h_min.numel() * 4 + h_max.numel() * 4
            e2e_steps = max(2, args.steps)

            load_s = []

            lanes = [torch.cuda.Stream(), torch.cuda.Stream()]

            def load(lane=None):
                t1 = time.perf_counter()
                # the bitstream's copy is queued on the volume's upload stream
                # (ISO_ASYNC_UPLOAD); the call returns once the ranges' copy,
                # the hulls and the rest of the load's work are queued on the
                # volume's stream (`lane`: its own, else the current one)
                kw = {} if lane is None else {"stream": ctypes.c_void_p(lane.cuda_stream)}
                v = bc.Volume(h_bits, DIMS, RATE, h_min, h_max, async_upload=True, **kw)
                load_s.append(time.perf_counter() - t1)
                return v

            def extract_all(v):
                n = 0
                for iso in ISOS:
                    m = v.extract(iso)
                    n += m.num_triangles
                    m.release()
                return n

            def serial(k):
                # load, five surfaces, release; one volume at a time
                n = 0
                for _ in range(k):
                    v = load()
                    n += extract_all(v)
                    v.release()
                return n

            def streamed(k):
                # double buffering: volume i + 1 is loaded (its bitstream
                # uploading on the copy engine) before volume i's surfaces are
                # extracted, so each upload overlaps the previous volume's work;
                # consecutive volumes run on two streams, so the next volume's
                # load (ranges' copy, hulls) does not queue ahead of this
                # volume's surfaces; every volume is still uploaded and read
                # back inside the run
                n = 0
                nxt = load(lanes[0])
                for i in range(k):
                    cur = nxt
                    if i + 1 < k:
                        nxt = load(lanes[(i + 1) % 2])
                    n += extract_all(cur)
                    cur.release()
                return n

            def timed(fn, k):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                n = fn(k)
                torch.cuda.synchronize()
                return n, time.perf_counter() - t0

            serial(1)
            streamed(2)
            load_s.clear()
            n_ser, dt_ser = timed(serial, e2e_steps)
            n_str, dt_str = timed(streamed, e2e_steps)
            e2e = {"value": n_str / dt_str, "unit": "triangles/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": 2 * CTL_BYTES * len(ISOS), "ms_per_step": 1000 * dt_str / e2e_steps,
                   "steps": e2e_steps, "load_ms": 1000 * float(np.median(load_s)),
                   "includes": "per step: iso_load_volume from pinned host buffers (ranges, allocation, block "
                               "hulls; the bitstream's upload queued on the copy engine), 5 x iso_extract "
                               "(exact-size device meshes, count readbacks), release; volume i + 1 is loaded "
                               "(on the other of two streams) before volume i's surfaces are extracted, so its "
                               "upload overlaps them (the first volume's upload is not overlapped and is inside "
                               "the timed run)",
                   "serial": {"value": n_ser / dt_ser, "ms_per_step": 1000 * dt_ser / e2e_steps,
                              "what": "the same steps one volume at a time: load, five surfaces, release"}}
        vol.release()
        batch = None if args.no_batch else measure_batch64(bc, sg, torch, stream, flush, args.steps)
        del out, flush
        torch.cuda.empty_cache()
        serve = None
        if not args.no_serve and rank == 0:
            bc.release_cached_memory()              # the earlier legs' memory back to the device
            torch.cuda.empty_cache()
            try:
                serve = serving_summary(measure_serving(bc, torch, SERVE_LEG_SCALE, SERVE_LEG_REQUESTS,
                                                        batches=(2, 8), sweeps=False))
            except Exception as e:                  # reported in the line; the other legs stand
                serve = {"error": f"{type(e).__name__}: {e}"}
            bc.release_cached_memory()
            torch.cuda.empty_cache()
        configs = None if (args.no_configs or rank != 0) else measure_configs(bc, torch)

    if rank != 0:
        dist.barrier() if world > 1 else None
        return
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "measured" if peaks else "fallback"
    dominant = max(KERNELS, key=lambda k: stage_ms[k])
    n_launch = prof_steps * len(ISOS)
    ach = stage_b[dominant] / n_launch / (stage_ms[dominant] / n_launch / 1000.0) / 1e9
    stages = {}
    for k in KERNELS:
        ms = stage_ms[k] / n_launch
        gbs = (stage_b[k] / n_launch) / (ms / 1000.0) / 1e9 if ms > 0 and stage_b[k] > 0 else None
        stages[k] = {"kernel": KERNEL_OF[k][0], "ms_per_surface": ms, "alg_bytes_per_surface": stage_b[k] / n_launch,
                     "GBps": gbs, "frac_of_measured_hbm": (gbs / peak) if gbs else None}
    stages["prep"] = {"ms_per_surface": stage_ms["prep"] / n_launch}
    cold_gbs = cold_b / (cold_ms / 1000.0) / 1e9
    cold = {"ms_per_surface": cold_ms / n_cold, "bytes_per_surface": cold_b / n_cold, "GBps": cold_gbs,
            "frac": cold_gbs / peak, "triangles_per_s": cold_t / (cold_ms / 1000.0),
            "bytes": "n_new*(8R + 256) + 48T: compressed blocks read, decoded blocks written, vertices written",
            "full_bytes_per_surface": cold_full / n_cold,
            "full_frac": cold_full / (cold_ms / 1000.0) / 1e9 / peak,
            "full_bytes": "the above + 8 per block (ranges) + 256 per active block (read once) + masks and ids",
            "what": "one whole extraction (all kernels, count readback) from an empty cache, device time"}
    lat_ms = sorted(1000 * x for x in lat)
    value = total_tris / total_s
    ms_per_step = 1000 * total_s / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "triangles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "voxels_per_s": len(ISOS) * float(np.prod(DIMS)) * args.steps * world / total_s,
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                       "what": "host time of one iso_extract_into call (cache update, decode, triangles, count readback)"},
        "config": {"workload": WORKLOAD, "dims": list(DIMS), "rate_bits": RATE, "isovalues": list(ISOS),
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write, untimed)",
                   "triangles_per_surface": [s["num_triangles"] for s in per_iso],
                   "active_blocks_per_surface": [s["n_active"] for s in per_iso],
                   "occupied_blocks_per_surface": [s["n_occupied"] for s in per_iso],
                   "active_fraction": [round(s["n_active"] / nb, 4) for s in per_iso],
                   "occupied_fraction": [round(s["n_occupied"] / nb, 4) for s in per_iso],
                   "cache_hit_rate_per_surface_in_a_step": [
                       round(1.0 - st["n_new"] / st["n_active"], 4) if st["n_active"] else None for st in stats],
                   "parallelism": f"{world} independent replica(s)"},
        "roofline": {"bound": "hbm", "what": "one whole extraction from an empty cache (every kernel, count "
                     "readback), device time, against n_new*(8R + 256) + 48T bytes per surface",
                     "achieved": cold_gbs, "peak": peak, "unit": "GB/s", "frac": cold_gbs / peak,
                     "peak_source": f"{peak_src} hbm_gbs (copy)",
                     "traffic": extraction_traffic(),
                     "alg_bytes_per_launch": cold_b / n_cold,
                     "dominant_kernel": {"kernel": KERNEL_OF[dominant][0], "achieved": ach, "frac": ach / peak,
                                         "alg_bytes_per_launch": stage_b[dominant] / n_launch,
                                         "traffic": profile_traffic(KERNEL_OF[dominant][1], KERNEL_OF[dominant][0])}},
        "roofline_cold_extraction": cold,
        "packed_vertices": packed,
        "indexed_mesh": indexed,
        "render": render,
        "full_volume_baselines": baselines,
        "batch64": batch,
        "stages": stages,
        "serving": serve,
        "configs": configs,
        "gpu_launches": args.steps * (KERNELS_PER_RESET + KERNELS_PER_SURFACE * len(ISOS)),
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    if world > 1:
        dist.barrier()
    if not args.no_cpu_baseline and world == 1:
        sample = cpu_sample_volume(CPU_WINDOW, CPU_ORIGIN)
        pvol, parity, check = parity_checker(bc, CPU_WINDOW, sample)
        tris, dt = cpu_oracle_sample(CPU_WINDOW, CPU_ORIGIN, ISOS, volume=sample, check=check)
        pvol.release()
        line["parity"] = dict(parity, unit="voxel", sample=f"the CPU baseline's {CPU_WINDOW[0]}x{CPU_WINDOW[1]}x"
                              f"{CPU_WINDOW[2]} window, 5 isovalues, through iso_extract",
                              tolerance=1e-5)
        line["cpu_baseline"] = {
            "value": tris / dt, "unit": "triangles/s", "cores": 1, "kind": "oracle",
            "sample": f"{CPU_WINDOW[0]}x{CPU_WINDOW[1]}x{CPU_WINDOW[2]} window at {CPU_ORIGIN} of the same field, "
                      f"5 isovalues, {dt:.1f} s single-threaded (decode every block, range test, block MC)",
            "voxels_per_s": len(ISOS) * float(np.prod(CPU_WINDOW)) / dt}
        ptris, pdt, procs = cpu_oracle_parallel(CPU_WINDOW, ISOS, sample)
        line["cpu_baseline"]["all_cores"] = {
            "value": ptris / pdt, "unit": "triangles/s", "cores": procs,
            "sample": f"the same encoded window in {procs} slabs of whole block layers, one spawned process each "
                      f"running the oracle unchanged, {pdt:.1f} s wall, {ptris} triangles "
                      f"({'equal to' if ptris == tris else 'differing from'} the single-process count)",
            "voxels_per_s": len(ISOS) * float(np.prod(CPU_WINDOW)) / pdt}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- serving

SERVE_BUDGET_BYTES = 64e9          # decoded-block cache budget of the serving volume (scaled with its area)
SERVE_LEG_SCALE = 0.25             # the default run's serving leg: x and y at a quarter (1/16 of the samples)
SERVE_LEG_REQUESTS = 300
SERVE_VERTEX_BUDGET = 48e9         # finished meshes held by the server at once (not scaled with the volume)


def measure_configs(bc, torch, reps=4):
    """The other single-volume configurations, each extracted whole through
    iso_extract_into (device time, CUDA events on the volume's stream):
    sphere64 (64^3 sphere distance field, 16 bits/value, isovalue 0: the
    correctness case) and channel2k (2048 x 2048 x 1024 channel-flow field,
    4 bits/value, isovalue at the 70th percentile of the decoded data).  For
    each: the surface from an empty cache (median of `reps`, the cache reset
    before each) and warm (the same isovalue again), triangles and voxels
    per second, and the cold extraction against n_new*(8R + 256) + 48T bytes
    and the measured copy peak."""
    from synth import recipes, volumes
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    res = {}
    for rec in (recipes.SPHERE64, recipes.CHANNEL2K):
        bits, bmin, bmax = volumes.encode_recipe(rec)
        iso = rec.isovalues[0] if rec.isovalues else volumes.percentile_isovalue(bits, rec.dims, rec.rate,
                                                                                 rec.percentile, seed=3)
        vol = bc.Volume(bits, rec.dims, rec.rate, bmin, bmax)
        del bits, bmin, bmax
        torch.cuda.empty_cache()
        st = vol.extract_into(iso, torch.empty((1, 3, 4), dtype=torch.float32, device="cuda"), check=False)
        T = st["num_triangles"]
        out = torch.empty((max(T, 1), 3, 4), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()

        def timed(cold):
            ms = []
            for _ in range(reps):
                if cold:
                    vol.cache_reset()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s2 = vol.extract_into(iso, out)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            return float(np.median(ms)), s2

        cold_ms, sc = timed(True)
        warm_ms, _ = timed(False)
        nvox = float(np.prod(rec.dims))
        nb = int(np.prod(bc.block_dims(rec.dims)))
        alg = sc["n_new"] * (8 * rec.rate + 256) + 48 * sc["num_triangles"]
        res[rec.name] = {
            "dims": list(rec.dims), "rate_bits": rec.rate, "isovalue": iso, "triangles": sc["num_triangles"],
            "active_fraction": round(sc["n_active"] / nb, 4), "cold_ms": cold_ms, "warm_ms": warm_ms,
            "cold_triangles_per_s": sc["num_triangles"] / (cold_ms / 1000.0),
            "warm_triangles_per_s": sc["num_triangles"] / (warm_ms / 1000.0),
            "cold_voxels_per_s": nvox / (cold_ms / 1000.0), "warm_voxels_per_s": nvox / (warm_ms / 1000.0),
            "cold_alg_bytes": alg, "cold_GBps": alg / (cold_ms / 1000.0) / 1e9,
            "cold_frac_of_measured_hbm": alg / (cold_ms / 1000.0) / 1e9 / peak}
        del out
        vol.release()
        torch.cuda.empty_cache()
    res["what"] = ("other single-volume configurations through iso_extract_into, device time: the surface from an "
                   "empty cache and warm, and the cold extraction against n_new*(8R + 256) + 48T bytes")
    return res


def measure_serving(bc, torch, scale, n, batches=(4,), sweeps=True):
    """The request loop on the serving volume (the channel-flow recipe, x and
    y scaled by `scale`): Poisson arrivals at 0.8 / the plain path's median
    service time, isovalues a reflecting random walk over the [p5, p95]
    decoded percentiles (step 0.02 of the range), served by the batched
    server (each max_batch in `batches`) and, on the same schedule, by the
    plain per-request path; a warm single request both ways; optionally
    sweeps up and down the same range."""
    import dataclasses
    from paper_2009_03254_gb300 import serving
    from synth import recipes, volumes
    rec = recipes.SERVE_DNS
    if scale != 1.0:
        nx, ny, nz = rec.dims
        sx = max(4, int(round(nx * scale / 4)) * 4)
        sy = max(4, int(round(ny * scale / 4)) * 4)
        rec = dataclasses.replace(rec, dims=(sx, sy, nz))
    scale_area = rec.dims[0] * rec.dims[1] / float(recipes.SERVE_DNS.dims[0] * recipes.SERVE_DNS.dims[1])
    t0 = time.time()
    bits, bmin, bmax = volumes.encode_recipe(rec)
    t_gen = time.time() - t0
    p5, p50, p95 = (volumes.percentile_isovalue(bits, rec.dims, rec.rate, q, seed=3) for q in (0.05, 0.5, 0.95))
    budget = int(SERVE_BUDGET_BYTES * scale_area)
    vertex_budget = int(SERVE_VERTEX_BUDGET)       # a memory cap: the same at every scale
    vol = bc.Volume(bits, rec.dims, rec.rate, bmin, bmax, cache_budget_bytes=budget, initial_cache_fraction=0.01)
    compressed = bits.numel() * 8
    del bits, bmin, bmax
    torch.cuda.empty_cache()
    # plain service time at the median isovalue (warm), for the arrival rate
    svc = []
    for _ in range(4):
        t1 = time.perf_counter()
        m = vol.extract(p50)
        svc.append(time.perf_counter() - t1)
        t_med = m.num_triangles
        m.release()
    median_svc = float(np.median(svc[1:]))
    rate = 0.8 / median_svc
    isos = serving.random_walk_isovalues(n, p5, p95, 5)
    arrivals = serving.poisson_arrivals(n, rate, 1)
    over_rate = 1.25 / median_svc                  # more than the plain path can serve
    over_arrivals = serving.poisson_arrivals(n, over_rate, 2)

    def drive(backend, arr, iso_list):
        torch.cuda.synchronize()
        tw = time.perf_counter()
        res = serving.RequestLoop(backend).run(arr, iso_list)
        wall = time.perf_counter() - tw
        tris = sum(r["triangles"] for r in res)
        out = serving.latency_summary(res)
        out.update({"triangles_per_s": tris / wall, "wall_s": wall, "triangles": tris,
                    "failed": sum(1 for r in res if r["status"] not in (serving.ISO_OK, serving.REJECTED))})
        return out

    # one request alone, warm cache: the plain call against a one-request tick
    single = {"plain_ms": [], "served_ms": []}
    probe = bc.Server(vol, max_batch=1, vertex_budget_bytes=vertex_budget)
    for _ in range(5):
        t1 = time.perf_counter()
        m = vol.extract(p50)
        single["plain_ms"].append(1e3 * (time.perf_counter() - t1))
        m.release()
        tk = probe.submit(float(p50))
        t1 = time.perf_counter()
        probe.step()
        single["served_ms"].append(1e3 * (time.perf_counter() - t1))
        st, m = probe.take(tk)
        if m is not None:
            m.release()
    probe.release()
    single = {"plain_ms": float(np.median(single["plain_ms"][1:])), "served_ms": float(np.median(single["served_ms"][1:]))}
    vol.cache_reset()
    plain = drive(serving.PlainBackend(vol), arrivals, isos)
    served = {}
    for mb in batches:
        vol.cache_reset()
        srv = bc.Server(vol, max_batch=mb, vertex_budget_bytes=vertex_budget)
        served[mb] = drive(srv, arrivals, isos)
        srv.release()
    # overload: arrivals at 1.25x the plain path's service rate
    vol.cache_reset()
    over = {"arrival_rate_per_s": over_rate, "plain": drive(serving.PlainBackend(vol), over_arrivals, isos)}
    mb = batches[-1]
    vol.cache_reset()
    srv = bc.Server(vol, max_batch=mb, vertex_budget_bytes=vertex_budget)
    over["served"] = drive(srv, over_arrivals, isos)
    over["max_batch"] = mb
    srv.release()
    sw = {}
    if sweeps:
        mb = batches[len(batches) // 2]
        srv = bc.Server(vol, max_batch=mb, vertex_budget_bytes=vertex_budget)
        for name, seq in (("sweep_up", np.linspace(p5, p95, 100)), ("sweep_down", np.linspace(p95, p5, 100))):
            seq = seq.astype(np.float32)
            burst = np.zeros(len(seq))                   # all queued at once: throughput of each path
            vol.cache_reset()
            sp = drive(serving.PlainBackend(vol), burst, seq)
            vol.cache_reset()
            ss = drive(srv, burst, seq)
            sw[name] = {"plain_triangles_per_s": sp["triangles_per_s"], "served_triangles_per_s": ss["triangles_per_s"],
                        "plain_wall_s": sp["wall_s"], "served_wall_s": ss["wall_s"]}
        srv.release()
    vol.release()
    torch.cuda.empty_cache()
    return {"workload": f"serve_dns: {rec.dims[0]}x{rec.dims[1]}x{rec.dims[2]} channel-flow field (seed {rec.seed}, "
                        f"{rec.octaves} octaves, coarsest period {rec.base_period}), {rec.rate} bits/value, cache "
                        f"budget {budget / 1e9:.1f} GB",
            "requests": n, "arrival_rate_per_s": rate, "plain_median_service_ms": 1e3 * median_svc,
            "isovalue_range": [p5, p95], "median_isovalue": p50, "triangles_at_median": t_med,
            "compressed_bytes": compressed, "generate_encode_s": t_gen, "vertex_budget_bytes": vertex_budget,
            "plain": plain, "served": served, "overload": over, "single_request_warm": single, "sweeps": sw}


def serving_summary(sv):
    """The served-vs-plain figures of measure_serving, compact."""
    best = min(sv["served"], key=lambda mb: sv["served"][mb].get("p99_ms", float("inf")))
    s, p = sv["served"][best], sv["plain"]
    return {"workload": sv["workload"], "requests": sv["requests"], "arrival_rate_per_s": round(sv["arrival_rate_per_s"], 1),
            "max_batch": best,
            "served": {"p50_ms": s.get("p50_ms"), "p99_ms": s.get("p99_ms"), "triangles_per_s": s["triangles_per_s"],
                       "failed": s["failed"]},
            "plain": {"p50_ms": p.get("p50_ms"), "p99_ms": p.get("p99_ms"), "triangles_per_s": p["triangles_per_s"],
                      "failed": p["failed"]},
            "by_max_batch": {str(mb): [round(v.get("p50_ms", 0), 2), round(v.get("p99_ms", 0), 2),
                                       round(v["triangles_per_s"] / 1e9, 3)] for mb, v in sv["served"].items()},
            "single_request_warm_ms": {"plain": round(sv["single_request_warm"]["plain_ms"], 3),
                                       "served": round(sv["single_request_warm"]["served_ms"], 3)},
            "overload": {"arrival_rate_per_s": round(sv["overload"]["arrival_rate_per_s"], 1),
                         "max_batch": sv["overload"]["max_batch"],
                         "served": [round(sv["overload"]["served"].get("p50_ms", 0), 2),
                                    round(sv["overload"]["served"].get("p99_ms", 0), 2),
                                    round(sv["overload"]["served"]["triangles_per_s"] / 1e9, 3)],
                         "plain": [round(sv["overload"]["plain"].get("p50_ms", 0), 2),
                                   round(sv["overload"]["plain"].get("p99_ms", 0), 2),
                                   round(sv["overload"]["plain"]["triangles_per_s"] / 1e9, 3)]},
            "what": "Poisson isovalue requests at 0.8x the plain path's service rate (overload: 1.25x), latency "
                    "arrival -> mesh written; [p50 ms, p99 ms, G triangles/s]; meshes identical to the plain "
                    "path's (tested)"}


def run_serve(args):
    """The serving workload alone (full size unless --serve-scale), one line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_03254_gb300 as bc
    import synth.gpu as sg
    sg.build()
    sv = measure_serving(bc, torch, args.serve_scale, args.requests, batches=(2, 4, 8))
    summ = serving_summary(sv)
    best = summ["max_batch"]
    line = {
        "metric": "p50/p99 isovalue-change latency under Poisson requests, served vs plain path",
        "value": summ["served"]["p50_ms"], "unit": "ms", "higher_is_better": False, "n_gpus": 1,
        "steps": args.requests, "warmup": 1, "dtype": "f32", "data": "synthetic", "scaling": "weak",
        "vs_baseline": None,
        "config": {"workload": sv["workload"], "requests": sv["requests"],
                   "arrival_rate_per_s": sv["arrival_rate_per_s"], "plain_median_service_ms": sv["plain_median_service_ms"],
                   "isovalue_range": sv["isovalue_range"], "median_isovalue": sv["median_isovalue"],
                   "triangles_at_median": sv["triangles_at_median"], "compressed_bytes": sv["compressed_bytes"],
                   "generate_encode_s": sv["generate_encode_s"],
                   "server": {"max_batch": best, "vertex_budget_bytes": sv["vertex_budget_bytes"]}},
        "served": sv["served"], "plain": sv["plain"], "overload": sv["overload"], "sweeps": sv["sweeps"],
        "single_request_warm": sv["single_request_warm"], "p99_ms": summ["served"]["p99_ms"],
    }
    print(json.dumps(line), flush=True)


def main():
    global DIMS, WORKLOAD
    args = parse()
    if args.dims != 512:
        DIMS = (args.dims,) * 3
        WORKLOAD = WORKLOAD.replace("noise512: 512^3", f"noise{args.dims}: {args.dims}^3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
