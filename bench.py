#!/usr/bin/env python
"""Benchmark of the DOT hot path on GB300: forward and forward+backward Mrays/s.

Workload (N = 1): the NeRF-synthetic-shaped scene (depth-9 octree, 2.9 M leaves, SH degree 3,
FP16 leaves, FP32 arithmetic) seen by 100 cameras of 800x800 on a radius-4 hemisphere (focal
1111).  One step renders all 100 views in one launch (64 M rays).  Extra keys: forward+backward
on 2^16-ray batches from those views, the refine pass (signal, selection, prune/sample), the
roofline of the forward kernel, the FP64 CPU oracle on a bounded sample, and end-to-end
throughput through host buffers.  Multi-GPU: every rank renders its own copy of the workload
(weak scaling; the only collectives are the barrier and the max of the timings).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s fwd & fwd+bwd at 800² SH-deg3; serve p50/p99 ms vs plain launch"
WORKLOAD = "nerf_synthetic_d9_sh3_f16_100x800x800"
BATCH = 1 << 16


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="dot", choices=["dot", "reference"])
    p.add_argument("--views", type=int, default=100)
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="target CPU time of the oracle baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--quick", action="store_true",
                   help="skip the training-loop and Tanks&Temples-shaped measurements")
    p.add_argument("--serve-seconds", type=float, default=20.0,
                   help="length of each serving trace (Poisson arrivals at 200 and 2000 req/s)")
    p.add_argument("--serve-repeats", type=int, default=3,
                   help="serving traces per rate and server (other seeds)")
    p.add_argument("--serve-requests", type=int, default=None,
                   help="shorthand for traces of this many requests at 200 req/s, one repeat")
    a = p.parse_args()
    if a.serve_requests is not None:
        a.serve_seconds, a.serve_repeats = a.serve_requests / 200.0, 1
    return a


# ----------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200", "-i",
                                       str(index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------------------------
def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as tdist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(rays_per_rank_step: int, steps: int, ws: int, total_ms: float) -> float:
    """Whole-job Mrays/s: every rank renders its own copy of the workload (weak scaling), so the
    job processes ws times the rays of one rank in the slowest rank's time."""
    return rays_per_rank_step * steps * ws / (total_ms / 1e3) / 1e6


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources that define the forward march kernel: a profile taken on other sources is stale
MARCH_SOURCES = ("internal.cuh", "march.cuh", "march_launch.cuh", "render_fwd.cu")


def csrc_hash() -> str:
    """Hash of the code (comments and whitespace removed) of the forward march's sources."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2307_15333_gb300", "csrc")
    for f in MARCH_SOURCES:
        with open(os.path.join(d, f)) as fh:
            code = re.sub(r"/\*.*?\*/", " ", fh.read(), flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(f.encode() + " ".join(code.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag: str):
    """DRAM bytes per launch from the committed ncu summary of this kernel and workload, if the
    kernel sources are unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    s = re.search(r"csrc_sha:\s*([0-9a-f]+)", txt)
    if not m or not s or s.group(1) != csrc_hash():
        return None
    return float(m.group(1))


class OracleSample:
    """The FP64 oracle as it stands, on the host cores, over a strided pixel sample of the views
    sized to a time budget (the oracle's tree and parameters are built once)."""

    def __init__(self, scene, cams):
        import oracle
        import seeded_inputs as si
        self.oracle, self.si = oracle, si
        self.scene, self.cams = scene, cams
        self.t = oracle.scene_tree(scene)
        sig, sh = si.leaf_params(self.t["leaf_key"], self.t["leaf_inside"], scene)
        self.s64 = si.storage_to_f64(sig, scene.storage)
        self.h64 = si.storage_to_f64(sh, scene.storage)
        self.lo, self.size = oracle.root_of(scene)

    def _render(self, o, d, threads):
        self.oracle.render(self.t, self.lo, self.size, self.s64, self.h64, self.scene.sh_degree,
                           o, d, threads=threads)

    def rays(self, budget_s: float, threads: int):
        """A strided sample of every view whose render takes about budget_s."""
        W, H = self.cams[0].width, self.cams[0].height
        stride = 4096
        while True:          # calibrate on growing samples until one takes a second
            pix = np.arange(0, W * H, stride)
            o, d = self.si.camera_rays(self.cams[0], pix)
            t0 = time.perf_counter()
            self._render(o, d, threads)
            dt = max(time.perf_counter() - t0, 1e-6)
            if dt > 1.0 or stride == 1:
                break
            stride = max(1, stride // 4)
        rate = len(pix) / dt
        want = max(1000, int(rate * budget_s))
        stride = max(1, (W * H * len(self.cams)) // want)
        os_, ds_ = [], []
        for v, cam in enumerate(self.cams):
            o, d = self.si.camera_rays(cam, np.arange(v % stride, W * H, stride))
            os_.append(o)
            ds_.append(d)
        which = "every pixel" if stride == 1 else f"every {stride}-th pixel"
        desc = f"{which} of the {len(self.cams)} {W}x{H} views"
        return np.concatenate(os_), np.concatenate(ds_), desc

    def time(self, o, d, threads):
        t0 = time.perf_counter()
        self._render(o, d, threads)
        return time.perf_counter() - t0


def pixel_errors(got, ref, fp32_exact: bool) -> dict:
    """Per-ray error of GPU pixels against the oracle's: absolute, and relative to
    max(|oracle|, 1e-2); rays beyond the stated tolerance (FP32 exact: 1e-5 relative, the
    grazing-ray exceptions; 16-bit: 2e-3 absolute)."""
    got = np.asarray(got, np.float64).reshape(ref.shape)
    a = np.abs(got - ref)
    r = a / np.maximum(np.abs(ref), 1e-2)
    a_ray, r_ray = a.max(axis=1), r.max(axis=1)
    beyond = r_ray > 1e-5 if fp32_exact else a_ray > 2e-3
    return {"rays": int(ref.shape[0]), "max_abs": float(a.max()),
            "p99_abs": float(np.percentile(a_ray, 99)), "max_rel": float(r.max()),
            "p99_rel": float(np.percentile(r_ray, 99)),
            "tolerance": "1e-5 relative per channel" if fp32_exact else "2e-3 absolute per channel",
            "rays_beyond": int(beyond.sum()), "frac_beyond": float(beyond.mean())}


def grad_errors(got, ref, absum, floor) -> dict:
    """Error of FP32 gradient sums against the oracle's as a fraction of the 16-bit tolerance
    (2e-3 of the entry's summed term magnitudes + floor; <= 1 is within it), and the leaves with
    an entry beyond it."""
    got = np.asarray(got, np.float64).reshape(ref.shape)
    d = np.abs(got - ref)
    live = absum > 0
    q = d[live] / (2e-3 * absum[live] + floor)
    bad = (d > 2e-3 * absum + floor).reshape(ref.shape[0], -1).any(axis=1)
    n_live = int(live.reshape(ref.shape[0], -1).any(axis=1).sum())
    return {"entries": int(live.sum()), "leaves": n_live, "floor": float(floor),
            "max_err_over_tolerance": float(q.max()),
            "p99_err_over_tolerance": float(np.percentile(q, 99)),
            "leaves_beyond": int(bad.sum()), "frac_leaves_beyond": float(bad.sum() / max(n_live, 1))}


def parity_report(threads: int, sampler=None) -> dict:
    """Error of the GPU path against the FP64 oracle on every configuration, measured in the CPU
    baseline leg (the oracle's own leg): the tiny FP32 scene on all 4096 pixels of its camera, the
    NeRF-synthetic-shaped FP16 scene and the Tanks&Temples-shaped BF16 scene on seeded pixel
    samples of their views, and the gradients of one 2^16-ray training batch of the FP16 scene
    through the fused pass (dL/dC taken from the GPU, the backward from the oracle; rays whose
    transmittance comes within 0.1% of eps_T are set aside, the discrete early-termination
    decision)."""
    import torch

    import oracle
    import seeded_inputs as si
    import paper_2307_15333_gb300 as dot
    out = {}
    opts = dot.render_opts(background=(1.0, 1.0, 1.0), eps_T=1e-4)

    def gpu_render(tree, o, d):
        rgb = torch.empty(o.shape[0], 3, device="cuda")
        dot.dot_render_forward(tree, dot.rays_buffer(torch.from_numpy(o).cuda(),
                                                     torch.from_numpy(d).cuda()), opts, rgb)
        torch.cuda.synchronize()
        return rgb.cpu().numpy()

    def full_params(t, sc, leaves=None):
        if leaves is None:
            sig, sh = si.leaf_params(t["leaf_key"], t["leaf_inside"], sc)
            return si.storage_to_f64(sig, sc.storage), si.storage_to_f64(sh, sc.storage)
        L = t["leaf_key"].size
        s64 = np.zeros(L)
        h64 = np.zeros((L, 3, sc.n_coeffs))
        sig, sh = si.leaf_params(t["leaf_key"][leaves], t["leaf_inside"][leaves], sc)
        s64[leaves] = si.storage_to_f64(sig, sc.storage)
        h64[leaves] = si.storage_to_f64(sh, sc.storage)
        return s64, h64

    # tiny FP32 scene, every pixel (exact mode)
    sc, cams = si.config_tiny()
    tree = dot.octree_from_scene(sc)
    t = oracle.scene_tree(sc)
    lo, size = oracle.root_of(sc)
    s64, h64 = full_params(t, sc)
    o, d = si.camera_rays(cams[0])
    ref, _, _ = oracle.render(t, lo, size, s64, h64, sc.sh_degree, o, d, eps_T=1e-4, threads=threads)
    out["tiny_f32_64x64"] = pixel_errors(gpu_render(tree, o, d), ref, True)
    tree.free()

    # NeRF-synthetic-shaped FP16 scene: 200 seeded pixels of each of the 100 views (the oracle
    # tree and parameters of the baseline's sampler when given)
    sc, cams = si.config_nerf_synthetic(100)
    tree = dot.octree_from_scene(sc)
    if sampler is not None:
        t, lo, size, s64, h64 = sampler.t, sampler.lo, sampler.size, sampler.s64, sampler.h64
    else:
        t = oracle.scene_tree(sc)
        lo, size = oracle.root_of(sc)
        s64, h64 = full_params(t, sc)
    rng = np.random.default_rng(31)
    oo, dd = zip(*[si.camera_rays(c, rng.choice(c.width * c.height, 200, replace=False)) for c in cams])
    o, d = np.concatenate(oo), np.concatenate(dd)
    ref, _, _ = oracle.render(t, lo, size, s64, h64, sc.sh_degree, o, d, eps_T=1e-4, threads=threads)
    out["nerf_synthetic_f16_800"] = pixel_errors(gpu_render(tree, o, d), ref, False)

    # gradients of one 2^16-ray batch through the fused pass
    o, d = si.ray_batch(cams, BATCH, seed=8123)
    _, _, _, margin = oracle.render(t, lo, size, s64, h64, sc.sh_degree, o, d, eps_T=1e-4,
                                    margin=True, threads=threads)
    keep = margin > 1e-3
    o, d = np.ascontiguousarray(o[keep]), np.ascontiguousarray(d[keep])
    R = o.shape[0]
    ref, _, _ = oracle.render(t, lo, size, s64, h64, sc.sh_degree, o, d, eps_T=1e-4, threads=threads)
    tgt = np.where(ref > 0.5, ref - 0.45, ref + 0.45).astype(np.float32)
    L, K = tree.n_leaves, sc.n_coeffs
    rgb, g = torch.empty(R, 3, device="cuda"), torch.empty(R, 3, device="cuda")
    gs, gsh = torch.zeros(L, device="cuda"), torch.zeros(L, 3, K, device="cuda")
    dot.dot.dot_render_forward_backward_mse(
        tree, dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()), opts,
        torch.from_numpy(tgt).cuda(), rgb, g, gs, gsh)
    torch.cuda.synchronize()
    g64 = g.cpu().numpy().astype(np.float64)
    rs, rsh, asg, ash = oracle.backward(t, lo, size, s64, h64, sc.sh_degree, o, d, g64, eps_T=1e-4)
    floor = 1e-5 * np.abs(g64).max()
    out["nerf_synthetic_f16_grad_b16"] = {
        "rays": R, "rays_set_aside_near_eps_T": int((~keep).sum()),
        "pixels": pixel_errors(rgb.cpu().numpy(), ref, False),
        "dsigma": grad_errors(gs.cpu().numpy(), rs, asg, floor),
        "dsh": grad_errors(gsh.cpu().numpy(), rsh, ash, floor)}
    tree.free()
    del s64, h64, t

    # Tanks&Temples-shaped BF16 scene: 64 seeded pixels of each of the 150 views (the oracle gets
    # the parameters of the leaves these rays cross)
    sc, cams = si.config_tanks_temples()
    tree = dot.octree_from_scene(sc)
    t = oracle.scene_tree(sc)
    lo, size = oracle.root_of(sc)
    rng = np.random.default_rng(32)
    oo, dd = zip(*[si.camera_rays(c, rng.choice(c.width * c.height, 64, replace=False)) for c in cams])
    o, d = np.concatenate(oo), np.concatenate(dd)
    crossed = np.unique(np.concatenate([oracle.segments(t, lo, size, o[i], d[i])[0]
                                        for i in range(o.shape[0])]))
    s64, h64 = full_params(t, sc, crossed)
    ref, _, _ = oracle.render(t, lo, size, s64, h64, sc.sh_degree, o, d, eps_T=1e-4, threads=threads)
    out["tanks_temples_bf16_1080p"] = pixel_errors(gpu_render(tree, o, d), ref, False)
    tree.free()
    return out


def oracle_baseline(scene, cams, budget_s: float, threads: int, sampler=None):
    """The oracle timed once on a sample of about budget_s seconds."""
    sm = sampler or OracleSample(scene, cams)
    o, d, desc = sm.rays(budget_s, threads)
    dt = sm.time(o, d, threads)
    return {"value": o.shape[0] / dt / 1e6, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
            "sample": f"{desc} ({o.shape[0]} rays, FP64 forward render, {dt:.1f} s)"}


def measure_l2_read(local: int):
    """L2 read bandwidth for the two-level roofline: the library's L2-only streaming kernel over
    device buffers of several sizes (the resident ones are served by L2), CUDA events around a
    call of many passes, SM clocks sampled meanwhile.  Also one buffer far larger than L2 as a
    check against the measured HBM figure."""
    import torch

    from paper_2307_15333_gb300 import dot as d
    stream = torch.cuda.current_stream()
    sizes_mb = (8, 16, 32, 48, 64, 96)
    out = {"kernel": "dot_probe_l2_read (ld.global.cg 16-byte loads, whole waves)", "by_size": {}}
    clocks = Clocks(local)
    for mb in sizes_mb + (4096,):
        buf = torch.ones(mb << 20, dtype=torch.uint8, device="cuda")
        passes = max(2, (2048 if mb < 4096 else 8) * 16 // mb)
        d.dot_probe_l2_read(buf, 2)
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            d.dot_probe_l2_read(buf, passes)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out["by_size"][f"{mb}MB"] = (mb << 20) * passes / (best / 1e3) / 1e9
        del buf
    out["clocks"] = clocks.stop()
    resident = [out["by_size"][f"{mb}MB"] for mb in sizes_mb]
    out["l2_read_gbs"] = max(resident)
    out["hbm_read_gbs_same_kernel"] = out["by_size"]["4096MB"]
    return out


def two_level(compulsory_bytes, sample_bytes, t_meas_s, hbm_gbs, l2_gbs):
    """Two-level roofline: t_roof = max(compulsory / HBM bandwidth, sample / L2 bandwidth)."""
    t_hbm = compulsory_bytes / (hbm_gbs * 1e9)
    t_l2 = sample_bytes / (l2_gbs * 1e9)
    t_roof = max(t_hbm, t_l2)
    return {"compulsory_bytes": compulsory_bytes, "sample_bytes": sample_bytes,
            "t_hbm_ms": t_hbm * 1e3, "t_l2_ms": t_l2 * 1e3, "t_roof_ms": t_roof * 1e3,
            "t_meas_ms": t_meas_s * 1e3, "frac": t_roof / t_meas_s,
            "bound": "l2" if t_l2 >= t_hbm else "hbm"}


def measure_serving(args, refined_tree):
    """Continuous batching (slot tables replayed as CUDA graphs, two in flight; one slot launch
    per storage / SH-degree group of the trees, on forked streams) against one launch per
    request, on the same seeded Poisson traces over the four resident trees: the tiny FP32 SH-1
    scene, the tree the training run left after its refines, and two seed variants of the
    NeRF-synthetic-shaped scene (FP16, SH degree 3).  Each rate runs several traces (other
    seeds) through both servers."""
    import torch

    import seeded_inputs as si
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300 import serve
    scenes, refined, poses = si.config_serving()
    trees = [refined_tree if ref else dot.octree_from_scene(s) for s, ref in zip(scenes, refined)]
    opts = dot.render_opts(background=(1.0, 1.0, 1.0), eps_T=1e-4)
    free, _ = torch.cuda.mem_get_info()
    pool_floats = int(min(free // 8, 1 << 28))            # admission pool: an eighth of free HBM
    res = {"trees": [s.name + (" (after training refines)" if r else "") for s, r in zip(scenes, refined)],
           "leaves": [t.n_leaves for t in trees],
           "storage_sh_degree": [[int(t.storage), int(t.sh_degree)] for t in trees],
           "slot_groups": serve.slot_groups(trees),
           "resolutions": si.SERVE_RESOLUTIONS, "pool_MB": pool_floats * 4 / 1e6,
           "trace_seconds": args.serve_seconds, "repeats": args.serve_repeats,
           "latency": "arrival to completion observed by the host loop"}
    servers = {"batched": serve.BatchedServer(trees, opts, pool_floats),
               "plain": serve.PlainServer(trees, opts, pool_floats)}
    for srv in servers.values():                          # warm-up
        srv.run(serve.poisson_trace(50, 200.0, 4, si.SERVE_RESOLUTIONS, poses, seed=1))
    torch.cuda.synchronize()
    for rate in (200.0, 2000.0):
        n = int(rate * args.serve_seconds)
        runs = {"batched": [], "plain": []}
        for rep in range(args.serve_repeats):
            for mode in ("batched", "plain") if rep % 2 == 0 else ("plain", "batched"):
                trace = serve.poisson_trace(n, rate, 4, si.SERVE_RESOLUTIONS, poses, seed=2 + rep)
                torch.cuda.synchronize()
                servers[mode].run(trace)
                rays = sum(r.width * r.height for r in trace)
                span = max(r.done for r in trace) - trace[0].arrival
                runs[mode].append(dict(serve.percentiles(trace), mrays_s=rays / span / 1e6,
                                       requests=n, seed=2 + rep))
        ratio = [b["p99_ms"] / p["p99_ms"] for b, p in zip(runs["batched"], runs["plain"])]
        row = {m: {"runs": r,
                   "p50_ms": [x["p50_ms"] for x in r], "p99_ms": [x["p99_ms"] for x in r],
                   "mrays_s": [x["mrays_s"] for x in r]} for m, r in runs.items()}
        row["batched_over_plain_p99"] = {"each": ratio, "min": min(ratio), "max": max(ratio)}
        row["batched_p99_below_plain_every_run"] = all(x < 1.0 for x in ratio)
        res[f"rate_{int(rate)}_per_s"] = row
    del servers
    torch.cuda.synchronize()
    for t in trees:
        t.free()
    return res


def alg_bytes_of(stats, n_rays, storage_bytes, K):
    """Algorithmic bytes of one forward launch: the leaf payload of every occupied segment
    (density + SH row), the density of every other segment, one child word per segment, and the
    12-byte colour of every ray."""
    P = (1 + 3 * K) * storage_bytes
    seg, occ = stats["segments"], stats["occupied"]
    return occ * P + (seg - occ) * storage_bytes + seg * 4 + n_rays * 12


def grad_bytes_per_occupied(K):
    """FP32 gradient update of one occupied segment: dL/dsigma and the 3K SH gradients."""
    return 4 * (1 + 3 * K)


def alg_bytes_bwd(stats, n_rays, storage_bytes, K):
    """Algorithmic bytes of one backward launch (the march recomputed): the forward's leaf and
    node reads, the gradient update of every occupied segment, and dL/dC and C of every ray."""
    return (alg_bytes_of(stats, n_rays, storage_bytes, K) - n_rays * 12
            + stats["occupied"] * grad_bytes_per_occupied(K) + n_rays * 24)


def alg_bytes_fused(stats, n_rays, storage_bytes, K):
    """Algorithmic bytes of one fused training pass: the forward's leaf and node reads, the
    gradient update of every occupied segment, and per ray the target read and C and dL/dC
    written."""
    return (alg_bytes_of(stats, n_rays, storage_bytes, K) - n_rays * 12
            + stats["occupied"] * grad_bytes_per_occupied(K) + n_rays * 36)


def sum_stats(tree, rays_list, opts):
    """Segment counts summed over several ray sets (counting passes, not timed)."""
    from paper_2307_15333_gb300 import dot as d
    tot = {"segments": 0, "occupied": 0, "rays": 0}
    for r in rays_list:
        st = d.dot_render_stats(tree, r, opts)
        tot["segments"] += st["segments"]
        tot["occupied"] += st["occupied"]
        tot["rays"] += d.n_rays_of(r)
    return tot


def timed(fn, n, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(n):
        fn(i)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def measure_training(scene, cams, steps: int):
    """Algorithm 1 on the NeRF-synthetic-shaped scene: optimisation steps on 2^16-ray batches
    (one fused launch of the forward with the SUM_ALPHA signal, the MSE gradient and the backward
    with touched-leaf flags, then RMSProp of the touched leaves with their gradients zeroed and the
    decay of the others deferred) against targets rendered from a copy of the tree with other
    seeded parameters (same cells, other seed), then one refine (recursive pruning at the
    20th-percentile signal, sampling of the top 5%)."""
    import dataclasses

    import torch

    import seeded_inputs as si
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300.train import Trainer
    stream = torch.cuda.current_stream()
    tree = dot.octree_from_scene(scene)
    ref = dot.octree_from_scene(dataclasses.replace(scene, seed=scene.seed + 1))
    opts = dot.render_opts(background=(1.0, 1.0, 1.0), eps_T=1e-4)
    nb = 8
    batches, targets = [], []
    for i in range(nb):
        o, d = si.ray_batch(cams, BATCH, seed=9000 + i)
        r = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
        t = torch.empty(BATCH, 3, device="cuda")
        dot.dot_render_forward(ref, r, opts, t)
        batches.append(r)
        targets.append(t)
    ref.free()
    tr = Trainer(tree, opts, dot.dot.rmsprop_opts(), signal_mode=dot.dot.DOT_SIGNAL_SUM_ALPHA)
    for i in range(5):
        tr.step(batches[i % nb], targets[i % nb])
    torch.cuda.synchronize()
    tr.loss_sum.zero_()
    n = max(50, steps)
    ms = timed(lambda i: tr.step(batches[i % nb], targets[i % nb]), n, stream)
    loss = float(tr.loss_sum) / n
    L0 = tr.L
    q = float(torch.quantile(tr.signal[tr.signal > 0].float()[:1 << 24], 0.2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = tr.refine(q, 0.05, depth_cap=11, recursive=True, canonical=True)
    torch.cuda.synchronize()
    refine_ms = (time.perf_counter() - t0) * 1e3
    out = {"value": BATCH * n / (ms / 1e3) / 1e6, "unit": "Mrays/s", "iters_per_s": n / (ms / 1e3),
           "ms_per_iter": ms / n, "batch_rays": BATCH, "iters": n, "mean_batch_mse": loss,
           "leaves": L0, "step": "fwd+signal, mse grad, bwd (+touched flags), sparse rmsprop (touched leaves, "
                   "deferred decay)+zero grad",
           "refine": {"ms": refine_ms, "tau": q, "gamma": 0.05, "recursive": True,
                      "pruned_groups_per_pass": [p["n_pruned_groups"] for p in res["passes"]],
                      "leaves_after": res["n_leaves"]},
           # the training schedule of the workload: a refine every 1000 iterations
           "iters_per_s_with_refine_every_1000": 1000.0 / ((1000 * ms / n + refine_ms) / 1e3)}
    tree.free()
    return out


def measure_train_config3(iters: int = 3000, refine_every: int = 1000, keep_tree: bool = False):
    """Algorithm 1 on the differentiable-training configuration as specified: the tiny sphere
    scene (depth 4, FP32 leaves, SH degree 1) trained toward targets rendered from a seeded
    perturbed copy of its parameters (density x U(0.8, 1.2), SH + N(0, 0.1)), on 2^16-ray
    batches drawn from its 100 views of 800x800 (a pool of 100 batches, one epoch = one pass
    over them in a permuted order), with the fused training step, the MAX_WEIGHT signal and a
    refine every 1000 iterations (leaves at or below the 20% quantile of the signal
    prune-marked, top 5% sampled, depth cap D + 2), all through Trainer.fit.  Reports iterations/s, the time of each refine, the
    leaves after each, and the loss curve (mean batch MSE of every epoch).  Returns (result, the
    trained tree if keep_tree else None)."""
    import torch

    import seeded_inputs as si
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300.train import Trainer
    scene, cams = si.config_train()
    tree = dot.octree_from_scene(scene)
    ex = tree.export()
    sg, shg = si.perturbed_params(ex["sigma"], ex["sh"], seed=2002)
    goal = dot.dot.dot_tree_import(dict(ex, sigma=sg, sh=shg))
    opts = dot.render_opts(background=(1.0, 1.0, 1.0), eps_T=1e-4)
    pool = 100
    batches, keep = [], []
    for i in range(pool):
        o, d = si.ray_batch(cams, BATCH, seed=20000 + i)
        ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
        r = dot.rays_buffer(ot, dt)
        t = torch.empty(BATCH, 3, device="cuda")
        dot.dot_render_forward(goal, r, opts, t)
        batches.append((r, t))
        keep.append((ot, dt))
    torch.cuda.synchronize()
    goal.free()
    rng = np.random.default_rng(2003)

    def epoch(i):
        return [batches[j] for j in rng.permutation(pool)]
    tr = Trainer(tree, opts, dot.dot.rmsprop_opts(), signal_mode=dot.dot.DOT_SIGNAL_MAX_WEIGHT)
    leaves = [tree.n_leaves]
    pruned = []

    def on_refine(i, plan):
        leaves.append(plan["n_leaves"])
        pruned.append(sum(p["n_pruned_groups"] for p in plan["passes"]))
    F = dot.dot.DOT_SELECT_FRACTION
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = tr.fit(epoch, epochs=iters // pool, T=refine_every // pool, tau=0.2, gamma=0.05,
                    depth_cap=scene.max_depth + 2, recursive=False,
                    prune_mode=dot.dot.DOT_SELECT_QUANTILE, sample_mode=F, on_refine=on_refine)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    assert tree.status() == 0
    step_s = wall - sum(tr.refine_ms) / 1e3
    out = {"workload": "tiny_sphere_d4_sh1_f32_train_100x800x800", "batch_rays": BATCH,
           "iters": iters, "refine_every": refine_every, "refines": len(tr.refine_ms),
           "iters_per_s": iters / step_s, "iters_per_s_with_refines": iters / wall,
           "refine_ms": tr.refine_ms, "leaves_after_each_refine": leaves,
           "loss_per_epoch": losses, "epoch_iters": pool,
           "loss_first_last": [losses[0], losses[-1]],
           "targets": "render of a perturbed copy (density x U(0.8,1.2), SH + N(0,0.1), seed 2002)",
           "step": "fused fwd + MSE grad + bwd, MAX_WEIGHT signal, sparse RMSProp",
           "select": "prune at the 20% quantile of the signal, sample top 5% (rank), depth cap 6",
           "pruned_groups_per_refine": pruned}
    if not keep_tree:
        tree.free()
        tree = None
    return out, tree


def measure_compressed(scene, cams, steps: int):
    """The compressed model of Sec. 4.1 on the NeRF-synthetic-shaped scene: median-cut palette
    of 2^16 SH rows, then the forward render of all views from the 4-byte leaf records; PSNR of
    the compressed render against the uncompressed one."""
    import math

    import torch

    import paper_2307_15333_gb300 as dot
    stream = torch.cuda.current_stream()
    tree = dot.octree_from_scene(scene)
    W, H = cams[0].width, cams[0].height
    cam_t = dot.cameras_tensor(cams)
    order_t = torch.from_numpy(dot.dot.dot_camera_order(cam_t.cpu().numpy())).cuda()
    rays = dot.rays_cameras(cam_t, W, H, order_t)
    R = len(cams) * W * H
    opts = dot.render_opts(background=(1.0, 1.0, 1.0), eps_T=1e-4)
    ref = torch.empty(R, 3, device="cuda")
    dot.dot_render_forward(tree, rays, opts, ref)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dot.dot.dot_compress_sh(tree, 16)
    quant_s = time.perf_counter() - t0
    rgb = torch.empty(R, 3, device="cuda")
    st = dot.dot_render_stats(tree, rays, opts)
    K = scene.n_coeffs
    seg, occ = st["segments"], st["occupied"]
    ab = occ * 3 * K * 2 + seg * (4 + 4) + R * 12      # palette row + record + child word
    dot.dot_render_forward(tree, rays, opts, rgb)
    torch.cuda.synchronize()
    n = max(5, min(steps, 50))
    ms = timed(lambda i: dot.dot_render_forward(tree, rays, opts, rgb), n, stream)
    mse = float(((rgb - ref) ** 2).mean())
    hbm, kind = peaks()
    out = {"value": R * n / (ms / 1e3) / 1e6, "unit": "Mrays/s", "ms_per_step": ms / n,
           "palette_rows": 1 << 16, "quantise_s": quant_s,
           "psnr_vs_uncompressed_db": 10 * math.log10(1.0 / mse) if mse > 0 else None,
           "roofline_frac": ab / (ms / n / 1e3) / 1e9 / hbm, "peak_kind": kind,
           "alg_bytes_per_launch": ab,
           "per_unit": {"occupied_segment_B": 3 * K * 2 + 8, "empty_segment_B": 8,
                        "ray_output_B": 12}}
    tree.free()
    return out


def measure_tanks_temples(steps: int):
    """Forward (all 150 views of 1920x1080 in one launch, 311 M rays) and forward+backward
    (2^16-ray batches) on the Tanks&Temples-shaped scene (depth 10, BF16 leaves, SH degree 3)."""
    import torch

    import seeded_inputs as si
    import paper_2307_15333_gb300 as dot
    stream = torch.cuda.current_stream()
    scene, cams = si.config_tanks_temples()
    tree = dot.octree_from_scene(scene)
    W, H = cams[0].width, cams[0].height
    cam_t = dot.cameras_tensor(cams)
    order_t = torch.from_numpy(dot.dot.dot_camera_order(cam_t.cpu().numpy())).cuda()
    rays = dot.rays_cameras(cam_t, W, H, order_t)
    R = len(cams) * W * H
    opts = dot.render_opts(background=(1.0, 1.0, 1.0), eps_T=1e-4)
    rgb = torch.empty(R, 3, device="cuda")
    st = dot.dot_render_stats(tree, rays, opts)
    ab = alg_bytes_of(st, R, 2, scene.n_coeffs)
    dot.dot_render_forward(tree, rays, opts, rgb)
    torch.cuda.synchronize()
    n = max(3, min(steps, 10))
    ms = timed(lambda i: dot.dot_render_forward(tree, rays, opts, rgb), n, stream)
    hbm, kind = peaks()
    L, K = tree.n_leaves, scene.n_coeffs
    batches = []
    for i in range(8):
        o, d = si.ray_batch(cams, BATCH, seed=11000 + i)
        batches.append(dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()))
    g = torch.full((BATCH, 3), 1e-3, device="cuda")
    brgb = torch.empty(BATCH, 3, device="cuda")
    gs = torch.zeros(L, device="cuda")
    gsh = torch.zeros(L, 3, K, device="cuda")

    def pair(i):
        r = batches[i % 8]
        dot.dot_render_forward(tree, r, opts, brgb)
        dot.dot_render_backward(tree, r, opts, g, brgb, gs, gsh)
    for i in range(8):
        pair(i)
    torch.cuda.synchronize()
    pms = timed(pair, 100, stream)
    bst = sum_stats(tree, batches, opts)
    b_pair = (alg_bytes_of(bst, bst["rays"], 2, K) + alg_bytes_bwd(bst, bst["rays"], 2, K)) / 8
    # forward + backward over all 150 views in one batch (311 M rays per pair)
    gfull = torch.full((R, 3), 1e-6, device="cuda")
    dot.dot_render_forward(tree, rays, opts, rgb)
    dot.dot_render_backward(tree, rays, opts, gfull, rgb, gs, gsh)
    torch.cuda.synchronize()
    fpairs = 2
    fms = timed(lambda i: (dot.dot_render_forward(tree, rays, opts, rgb),
                           dot.dot_render_backward(tree, rays, opts, gfull, rgb, gs, gsh)),
                fpairs, stream)
    del gfull
    f_pair = ab + alg_bytes_bwd(st, R, 2, K)
    # distinct occupied leaves the 311 M rays touch (a max-weight signal pass, not timed): the
    # compulsory bytes of the forward and of a forward + backward pair over all views
    touched = torch.zeros(L, dtype=torch.float32, device="cuda")
    dot.dot_accumulate_signal(tree, rays, opts, dot.dot.DOT_SIGNAL_MAX_WEIGHT, touched)
    u_leaf = int(torch.count_nonzero(touched))
    del touched
    n_empty = int((tree.sigma <= 0).sum())
    P = 2 * (1 + 3 * K)
    comp_fwd = u_leaf * P + tree.n_nodes * 32 + n_empty * 2 + R * 12
    comp_pair = 2 * comp_fwd + u_leaf * 2 * grad_bytes_per_occupied(K) + R * 12
    out = {"workload": "tanks_temples_d10_sh3_bf16_150x1920x1080", "leaves": L,
           "nodes": tree.n_nodes, "rays_per_step": R,
           "fwd": {"value": R * n / (ms / 1e3) / 1e6, "unit": "Mrays/s", "ms_per_step": ms / n,
                   "roofline_frac": ab / (ms / n / 1e3) / 1e9 / hbm, "peak_kind": kind,
                   "alg_bytes_per_launch": ab, "segments_per_ray": st["segments"] / R,
                   "occupied_per_ray": st["occupied"] / R},
           "fwd_bwd": {"value": BATCH * 100 / (pms / 1e3) / 1e6, "unit": "Mrays/s",
                       "batch_rays": BATCH, "ms_per_pair": pms / 100, "alg_bytes_per_pair": b_pair,
                       "roofline_frac": b_pair / (pms / 100 / 1e3) / 1e9 / hbm},
           "fwd_bwd_full_batch": {"value": R * fpairs / (fms / 1e3) / 1e6, "unit": "Mrays/s",
                                  "batch_rays": R, "ms_per_pair": fms / fpairs,
                                  "alg_bytes_per_pair": f_pair,
                                  "roofline_frac": f_pair / (fms / fpairs / 1e3) / 1e9 / hbm},
           "compulsory": {"occupied_leaves_touched": u_leaf, "fwd_bytes": comp_fwd,
                          "pair_bytes": comp_pair}}
    tree.free()
    return out


# ----------------------------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ----------------------------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import seeded_inputs as si
    scene, cams = si.config_nerf_synthetic(args.views)
    threads = os.cpu_count() or 1
    # every step renders the same bounded sample; the whole run stays within about a minute or two
    per_step = min(2.0, max(0.25, args.cpu_seconds / max(1, args.steps)))
    sm = OracleSample(scene, cams)
    o, d, desc = sm.rays(per_step, threads)
    vals = []
    for i in range(args.warmup + args.steps):
        dt = sm.time(o, d, threads)
        if i >= args.warmup:
            vals.append({"value": o.shape[0] / dt / 1e6, "ms": dt * 1e3,
                         "sample": f"{desc} ({o.shape[0]} rays, FP64 forward render, {dt:.2f} s)"})
    v = statistics.median([b["value"] for b in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mrays/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median([b["ms"] for b in vals]),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": vals[-1]["sample"]},
            "cpu_baseline": {"value": v, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------------------------
# the GB300 arm
# ----------------------------------------------------------------------------------------------
def run_dot(args):
    import torch
    import torch.distributed as tdist

    import seeded_inputs as si
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300.render import render_views

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            tdist.barrier()

    def max_over_ranks(x: float) -> float:
        return globals()["max_over_ranks"](x, ws)

    scene, cams = si.config_nerf_synthetic(args.views)
    W, H = cams[0].width, cams[0].height
    tree = dot.octree_from_scene(scene)
    L = tree.n_leaves
    N_nodes = tree.n_nodes                                # the headline tree (refined later)
    cam_t = dot.cameras_tensor(cams)
    # views rendered in a nearest-neighbour chain so that consecutive views reuse L2
    order_t = torch.from_numpy(dot.dot.dot_camera_order(cam_t.cpu().numpy())).cuda()
    rays = dot.rays_cameras(cam_t, W, H, order_t)
    R = len(cams) * W * H
    opts = dot.render_opts(background=(1.0, 1.0, 1.0), eps_T=1e-4)
    rgb = torch.empty(R, 3, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # algorithmic bytes of one launch (counting pass, not timed)
    st = dot.dot_render_stats(tree, rays, opts)
    bs = 2                                                # FP16 storage
    K = scene.n_coeffs
    P = (1 + 3 * K) * bs                                  # leaf payload of an occupied segment
    seg, occ = st["segments"], st["occupied"]
    alg_bytes = alg_bytes_of(st, R, bs, K)

    # ---- forward: W warm-up steps, K timed steps, one launch each ----
    for _ in range(args.warmup):
        dot.dot_render_forward(tree, rays, opts, rgb)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_wall = time.perf_counter()
    for a, b in ev:
        a.record(stream)
        dot.dot_render_forward(tree, rays, opts, rgb)
        b.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = ev[0][0].elapsed_time(ev[-1][1])
    total_ms = max_over_ranks(total_ms)
    value = weak_scaling_value(R, args.steps, ws, total_ms)
    mean_launch_s = statistics.mean(launch_ms) / 1e3
    assert tree.status() == 0
    # distinct occupied leaves one launch touches (a max-weight signal pass, not timed)
    touched = torch.zeros(L, dtype=torch.float32, device="cuda")
    dot.dot_accumulate_signal(tree, rays, opts, dot.dot.DOT_SIGNAL_MAX_WEIGHT, touched)
    u_leaf = int(torch.count_nonzero(touched))
    del touched
    n_empty = int((tree.sigma <= 0).sum())

    # ---- forward + backward on 2^16-ray batches (fixed synthetic dL/dC) ----
    nb = 8
    batches = []
    for i in range(nb):
        o, d = si.ray_batch(cams, BATCH, seed=7000 + i)
        batches.append(dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()))
    g = torch.from_numpy(np.random.default_rng(1).normal(0, 1e-3, (BATCH, 3)).astype(np.float32)).cuda()
    brgb = torch.empty(BATCH, 3, device="cuda")
    gs = torch.zeros(L, device="cuda")
    gsh = torch.zeros(L, 3, K, device="cuda")
    pairs = max(200, 2 * args.steps)
    for i in range(3 * nb):
        r = batches[i % nb]
        dot.dot_render_forward(tree, r, opts, brgb)
        dot.dot_render_backward(tree, r, opts, g, brgb, gs, gsh)
    torch.cuda.synchronize()
    barrier()
    clocks2 = Clocks(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(pairs):
        r = batches[i % nb]
        dot.dot_render_forward(tree, r, opts, brgb)
        dot.dot_render_backward(tree, r, opts, g, brgb, gs, gsh)
    e1.record(stream)
    torch.cuda.synchronize()
    clk2 = clocks2.stop()
    fb_ms = max_over_ranks(e0.elapsed_time(e1))
    bst = sum_stats(tree, batches, opts)                  # the nb batches (counting pass)
    b_pair = (alg_bytes_of(bst, bst["rays"], bs, K) + alg_bytes_bwd(bst, bst["rays"], bs, K)) / nb
    b_fused = alg_bytes_fused(bst, bst["rays"], bs, K) / nb
    # distinct occupied leaves one batch touches (max-weight signal passes, not timed)
    u_occ_b = []
    for r in batches:
        tb = torch.zeros(L, dtype=torch.float32, device="cuda")
        dot.dot_accumulate_signal(tree, r, opts, dot.dot.DOT_SIGNAL_MAX_WEIGHT, tb)
        u_occ_b.append(int(torch.count_nonzero(tb)))
        del tb
    u_occ_b16 = statistics.mean(u_occ_b)
    fwd_bwd = {"value": BATCH * pairs * ws / (fb_ms / 1e3) / 1e6, "unit": "Mrays/s",
               "batch_rays": BATCH, "pairs": pairs, "ms_per_pair": fb_ms / pairs,
               "grad": "fixed synthetic dL/dC; FP32 gradients accumulate across pairs",
               "alg_bytes_per_pair": b_pair,
               "roofline_frac": b_pair / (fb_ms / pairs / 1e3) / 1e9 / peaks()[0],
               "clocks": clk2}

    # ---- the same batches through the fused training pass (forward, MSE gradient and backward
    # in one launch; the backward scatters from each ray's recorded segments) ----
    tgt = torch.full((BATCH, 3), 0.5, dtype=torch.float32, device="cuda")
    gfused = torch.empty(BATCH, 3, device="cuda")
    for i in range(3 * nb):
        dot.dot.dot_render_forward_backward_mse(tree, batches[i % nb], opts, tgt, brgb, gfused, gs, gsh)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(pairs):
        dot.dot.dot_render_forward_backward_mse(tree, batches[i % nb], opts, tgt, brgb, gfused, gs, gsh)
    e1.record(stream)
    torch.cuda.synchronize()
    fu_ms = max_over_ranks(e0.elapsed_time(e1))
    fwd_bwd["fused_mse"] = {"value": BATCH * pairs * ws / (fu_ms / 1e3) / 1e6, "unit": "Mrays/s",
                            "batch_rays": BATCH, "passes": pairs, "ms_per_pass": fu_ms / pairs,
                            "pass": "forward + MSE gradient + backward in one launch",
                            "alg_bytes_per_pass": b_fused,
                            "roofline_frac": b_fused / (fu_ms / pairs / 1e3) / 1e9 / peaks()[0]}
    del tgt, gfused

    # ---- forward + backward over all views in one batch (64 M rays per pair) ----
    gfull = torch.full((R, 3), 1e-6, dtype=torch.float32, device="cuda")
    for _ in range(2):
        dot.dot_render_forward(tree, rays, opts, rgb)
        dot.dot_render_backward(tree, rays, opts, gfull, rgb, gs, gsh)
    torch.cuda.synchronize()
    full_pairs = 5
    e0.record(stream)
    for _ in range(full_pairs):
        dot.dot_render_forward(tree, rays, opts, rgb)
        dot.dot_render_backward(tree, rays, opts, gfull, rgb, gs, gsh)
    e1.record(stream)
    torch.cuda.synchronize()
    ff_ms = max_over_ranks(e0.elapsed_time(e1))
    f_pair = alg_bytes + alg_bytes_bwd(st, R, bs, K)
    fwd_bwd["full_batch"] = {"value": R * full_pairs * ws / (ff_ms / 1e3) / 1e6,
                             "unit": "Mrays/s", "batch_rays": R, "pairs": full_pairs,
                             "ms_per_pair": ff_ms / full_pairs, "alg_bytes_per_pair": f_pair,
                             "roofline_frac": f_pair / (ff_ms / full_pairs / 1e3) / 1e9 / peaks()[0]}
    del gfull

    # ---- end to end through host buffers (pinned cameras in, pinned images out) ----
    cams_host = cam_t.cpu().pin_memory()
    out_host = torch.empty(len(cams), H, W, 3, dtype=torch.float32, pin_memory=True)
    ws_views = torch.empty(dot.dot.dot_render_views_host_workspace(len(cams), W, H),
                           dtype=torch.uint8, device="cuda")
    for _ in range(2):
        render_views(tree, cams_host, W, H, opts, out_host, workspace=ws_views)
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        render_views(tree, cams_host, W, H, opts, out_host, workspace=ws_views)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": R * e2e_steps * ws / e2e_s / 1e6, "unit": "Mrays/s",
           "h2d_bytes_per_step": int(cams_host.numel() * 4),
           "d2h_bytes_per_step": int(out_host.numel() * 4),
           "call": "dot_render_views_host (host cameras in, pinned host images out, written in "
                   "place by the render launch)"}
    del ws_views

    # ---- refine pass (signal, selection, prune / sample), once, on the resident tree ----
    sig = torch.zeros(L, device="cuda")
    pm = torch.empty(L, dtype=torch.uint8, device="cuda")
    sm = torch.empty(L, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in batches:
        dot.dot_accumulate_signal(tree, r, opts, dot.dot.DOT_SIGNAL_MAX_WEIGHT, sig)
    dot.dot_select_masks(tree, sig, dot.select_opts(dot.dot.DOT_SELECT_FRACTION, 0.2,
                                                    dot.dot.DOT_SELECT_FRACTION, 0.05), pm, sm)
    counts = dot.dot_refine_plan(tree, pm, sm, 11)
    lm = torch.empty(counts["n_leaves"], dtype=torch.int32, device="cuda")
    dot.dot_refine_prune(tree, pm, sm, 11, lm)
    torch.cuda.synchronize()
    refine_ms = (time.perf_counter() - t0) * 1e3
    refine = {"ms": refine_ms, "leaves_before": L, "leaves_after": counts["n_leaves"],
              "signal": f"MAX_WEIGHT over {nb} x 2^16 rays", "select": "bottom 20% / top 5%"}
    # the refined tree keeps its cells in appended order; renumbering restores Morton order
    rgb2 = torch.empty(R, 3, dtype=torch.float32, device="cuda")
    dot.dot_render_forward(tree, rays, opts, rgb2)
    torch.cuda.synchronize()
    ms_app = timed(lambda i: dot.dot_render_forward(tree, rays, opts, rgb2), 5, stream) / 5
    perm = torch.empty(counts["n_leaves"], dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    dot.dot.dot_tree_canonicalize(tree, perm)
    torch.cuda.synchronize()
    canon_ms = (time.perf_counter() - t0) * 1e3
    dot.dot_render_forward(tree, rays, opts, rgb2)
    torch.cuda.synchronize()
    ms_can = timed(lambda i: dot.dot_render_forward(tree, rays, opts, rgb2), 5, stream) / 5
    refine["forward_after_refine_ms"] = {"appended_order": ms_app, "canonical_order": ms_can,
                                         "canonicalize_ms": canon_ms}
    del rgb2, perm

    train_res = measure_training(scene, cams, args.steps) if rank == 0 and not args.quick else None
    train3_res, serve_res = None, None
    if rank == 0:
        # the training configuration's run (a shorter one with --quick) leaves the refined tree
        # that the serving measurement keeps resident
        train3_res, trained = (measure_train_config3(keep_tree=True) if not args.quick else
                               measure_train_config3(iters=300, refine_every=100, keep_tree=True))
        serve_res = measure_serving(args, trained)
    tt_res = measure_tanks_temples(args.steps) if rank == 0 and not args.quick else None
    comp_res = measure_compressed(scene, cams, args.steps) if rank == 0 and not args.quick else None

    hbm, peak_kind = peaks()
    achieved = alg_bytes / mean_launch_s / 1e9
    traffic = profiled_traffic("render_fwd_nerf_synthetic_800")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "march_kernel<__half,16,kFwd,false>",
                "alg_bytes_per_launch": alg_bytes,
                "per_unit": {"occupied_segment_B": P + 4, "empty_segment_B": bs + 4,
                             "ray_output_B": 12},
                "segments_per_ray": seg / R, "occupied_per_ray": occ / R,
                "occupied_leaves_touched": u_leaf}
    # compulsory bytes: what one launch must move at least once from HBM
    compulsory = u_leaf * P + N_nodes * 32 + n_empty * bs + R * 12
    roofline["compulsory"] = {
        "bytes": compulsory,
        "what": "distinct occupied leaves x payload + every node row + every empty density "
                "+ 12 B per ray",
        "t_at_peak_ms": compulsory / (hbm * 1e9) * 1e3, "t_meas_ms": mean_launch_s * 1e3}

    # the two-level roofline with a measured L2 read bandwidth
    if rank == 0:
        l2 = measure_l2_read(local)
        comp_fused = u_occ_b16 * (P + 2 * grad_bytes_per_occupied(K)) + BATCH * 36
        roofline["two_level"] = {
            "l2": l2,
            "forward": two_level(compulsory, alg_bytes, mean_launch_s, hbm, l2["l2_read_gbs"]),
            "fused_pass_b16": two_level(comp_fused, b_fused, fu_ms / pairs / 1e3, hbm,
                                        l2["l2_read_gbs"]),
            "fused_compulsory": "distinct occupied leaves of the batch x (payload + FP32 gradient "
                                "read and write) + 36 B per ray"}
        # forward + backward over all 64 M rays: each pass reads what a forward must, and the
        # backward also reads and writes the touched leaves' FP32 gradients and reads dL/dC
        comp_pair = 2 * compulsory + u_leaf * 2 * grad_bytes_per_occupied(K) + R * 12
        fb = fwd_bwd["full_batch"]
        roofline["two_level"]["fwd_bwd_full_batch"] = two_level(
            comp_pair, fb["alg_bytes_per_pair"], fb["ms_per_pair"] / 1e3, hbm, l2["l2_read_gbs"])
        roofline["two_level"]["pair_compulsory"] = (
            "2 x the forward's compulsory bytes + the touched leaves' FP32 gradients read and "
            "written + 12 B of dL/dC per ray")
        if tt_res is not None:
            c = tt_res["compulsory"]
            tt_res["fwd"]["two_level"] = two_level(
                c["fwd_bytes"], tt_res["fwd"]["alg_bytes_per_launch"],
                tt_res["fwd"]["ms_per_step"] / 1e3, hbm, l2["l2_read_gbs"])
            tb = tt_res["fwd_bwd_full_batch"]
            tb["two_level"] = two_level(c["pair_bytes"], tb["alg_bytes_per_pair"],
                                        tb["ms_per_pair"] / 1e3, hbm, l2["l2_read_gbs"])

    cpu, parity = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sampler = OracleSample(scene, cams)
        cpu = oracle_baseline(scene, cams, args.cpu_seconds, os.cpu_count() or 1, sampler)
        cpu["single_thread"] = oracle_baseline(scene, cams, 2.0, 1, sampler)
        parity = parity_report(os.cpu_count() or 1, sampler if len(cams) == 100 else None)
        del sampler

    line = {"metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "leaves": L, "nodes": N_nodes,
                       "views": len(cams), "width": W, "height": H, "rays_per_step": R,
                       "sh_degree": scene.sh_degree, "leaf_storage": "f16",
                       "l2": "inputs larger than L2, no flush: leaves %.0f MB + nodes %.0f MB + "
                             "ropes %.0f MB vs 129 MB L2" % (L * P / 1e6, N_nodes * 32 / 1e6,
                                                            L * 24 / 1e6),
                       "eps_T": 1e-4, "parallelism": f"replicas{ws}"},
            "clocks": clk, "e2e": e2e, "gpu_launches": args.steps, "roofline": roofline,
            "cpu_baseline": cpu, "parity": parity, "fwd_bwd": fwd_bwd, "refine": refine, "train": train_res,
            "train_config3": train3_res,
            "tanks_temples": tt_res, "compressed": comp_res, "serve": serve_res,
            "wall_s_timed": t_wall}
    if rank == 0:
        print(json.dumps(line))
    tree.free()
    if ws > 1:
        tdist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_dot(args)


if __name__ == "__main__":
    main()
