#!/usr/bin/env python
"""Benchmark: element-pair assemblies per second of the nonlocal FEM assembly on GB300.

Workload (default): the 720,000-triangle structured mesh of [-0.01, 1.01]^2 (600 x 600
cells split by their "/" diagonal), constant kernel 4/(pi delta^4) with delta = 0.01,
nocaps ball, 7-point outer and inner rules, FP32-bulk arithmetic. One step = one
nlfem_assemble on the resident mesh with its cached pair list and pattern (values
only: quadrature of every ordered pair, segmented reduction into CSR, load vector).
The pair list, contributions and index (tens of GB) are far larger than L2, so every
step streams from HBM. Also reported: the same step in plain FP64, the cold assembly
(pair search + pattern + values), the step end to end through the C ABI with host
buffers (steady on a resident mesh, and cold from the host mesh), the roofline of the
quadrature kernel and the FP64 CPU oracle on a sample.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]
Under torchrun (N > 1) every rank assembles its own replica of the workload (no
collective on the data path); value = pairs of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "720k": dict(mesh="cfg720k", kernel="constant", delta=0.01, ball="nocaps", quad_outer=7, quad_inner=7,
                 desc="structured 600x600 cells on [-0.01,1.01]^2 (720,000 triangles), constant kernel, "
                      "delta=0.01, nocaps, 7-point outer/inner rules"),
    "720k_small": dict(mesh="s200", kernel="constant", delta=0.03, ball="nocaps", quad_outer=7, quad_inner=7,
                       desc="structured 200x200 cells on [-0.01,1.01]^2 (80,000 triangles), constant kernel, "
                            "delta=0.03 (the delta/h of the 720k workload), nocaps, 7-point rules"),
    "cfg5": dict(mesh="cfg5", kernel="constant", delta=0.01, ball="nocaps", quad_outer=7, quad_inner=7,
                 desc="structured h=0.002 on [-0.01,1.01]^2 (520,200 triangles), constant kernel, delta=0.01, "
                      "nocaps, 7-point rules"),
    "cfg5_small": dict(mesh="s204", kernel="constant", delta=0.025, ball="nocaps", quad_outer=7, quad_inner=7,
                       desc="structured 204x204 cells on [-0.01,1.01]^2 (83,232 triangles, h=0.005), constant "
                            "kernel, delta=0.025=5h (the ties of configuration 5), nocaps, 7-point rules"),
    "cfg2": dict(mesh="cfg2", kernel="fractional", s=0.5, delta=0.1, ball="approxcaps", quad_outer=16,
                 quad_inner=16,
                 desc="jittered Delaunay h=0.01 on [-0.1,1.1]^2 (~29k triangles), fractional s=0.5, delta=0.1, "
                      "approxcaps, 16-point rules, singular rule (5^4 Gauss) on touching pairs"),
    "cfg3": dict(mesh="cfg3", kernel="peridynamic", delta=0.02, ball="nocaps", quad_outer=7, quad_inner=7,
                 desc="structured h=0.005 on [-0.02,1.02]^2 (86,528 triangles), bond-based peridynamics, "
                      "delta=0.02, 2 dofs per node, 7-point rules"),
    "cfg1": dict(mesh="cfg1", kernel="constant", delta=0.1, ball="nocaps", quad_outer=7, quad_inner=7,
                 desc="structured h=0.05 on [-0.1,1.1]^2 (1152 triangles), constant kernel, delta=0.1"),
    "inf_e5": dict(mesh="paper_e5", kernel="constant", delta=0.2, ball="infinity", quad_outer=7, quad_inner=7,
                   desc="Sec. 3.3 infinity-ball problem at its largest horizon: structured spacing 0.00625 on "
                        "[-0.2,0.7]^2 (41,472 triangles), constant kernel c=3/(4 delta^4), delta=0.2, "
                        "infinity norm ball cut exactly, 7-point rules"),
    "inf_jit": dict(mesh="paper_e5_jit", kernel="constant", delta=0.2, ball="infinity", quad_outer=7, quad_inner=7,
                    desc="the inf_e5 problem on a jittered Delaunay mesh (spacing 0.00625 on [-0.2,0.7]^2, "
                         "3% jitter, about 41,500 triangles): infinity ball without grid-aligned sides"),
    "inf_small": dict(mesh="paper_e5_small", kernel="constant", delta=0.1, ball="infinity", quad_outer=7,
                      quad_inner=7,
                      desc="Sec. 3.3 infinity-ball problem at delta=0.1: structured spacing 0.00625 on [-0.1,0.6]^2 "
                           "(25,088 triangles), constant kernel c=3/(4 delta^4), infinity norm ball, 7-point rules"),
}

# algorithmic work per unit (FMA = 2 flops, a MUFU op = 1): the fixed weights of the
# measurement plan, counted on the device by nlfem_system_census
FLOPS_PER_EVAL = {"constant": 14, "fractional": 14 + 3, "peridynamic": 14 + 7 + 2 * 8}  # per (x_p, y_q)
FLOPS_PER_OUTER = 90            # kk / kl finalisation of an outer point with a nonempty polygon
FLOPS_VERTEX_TESTS = 15         # three vertex-in-ball tests per (x_p, E_l) of a cut pair
FLOPS_EDGES = 3 * 23            # three edge quadratics (with sqrt) per cut (x_p, E_l)
FLOPS_CAPS = 3 * 14             # up to three cap centres per cut (x_p, E_l), approxcaps only
FLOPS_SUBTRI_POINT = 8 + 6      # point mapping and barycentric basis per point of a sub-triangle
FLOPS_DUFFY_POINT = 40          # FP64 flops per point of the singular rule (plus one pow / rsqrt)
CONTRIB_ENTRIES = {1: 21, 2: 84}


def make_mesh(name):
    from synth import meshes
    if name == "s200":
        return meshes.structured(-0.01, 1.01, 200, name="structured200")
    if name == "s204":
        return meshes.structured(-0.01, 1.01, 204, name="structured204")
    if name == "paper_e5":
        return meshes.paper_square(0.2, 0.00625)
    if name == "paper_e5_jit":
        return meshes.jittered_delaunay(-0.2, 0.7, 144, 0.03, seed=2207039216)
    if name == "paper_e5_small":
        return meshes.paper_square(0.1, 0.00625)
    return {"cfg720k": meshes.cfg720k_mesh, "cfg5": meshes.cfg5_mesh, "cfg2": meshes.cfg2_mesh,
            "cfg3": meshes.cfg3_mesh, "cfg1": meshes.cfg1_mesh}[name]()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, exe="nvidia-smi", first_wait_s=3.0):
        self.index = index
        self.exe = exe
        self.first_wait_s = first_wait_s
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen([self.exe, f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return self
        # the sampler takes a moment to start: let its first sample arrive before the timed
        # region begins, so that the samples cover that region (bounded wait)
        t0 = time.perf_counter()
        while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < self.first_wait_s:
            time.sleep(0.01)
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
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(ngpus):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    """The largest x over the ranks (the slowest replica's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, ws, ms_max):
    """Whole-job throughput of ws independent replicas: all ranks' units over the slowest time."""
    return units_per_rank * ws / (ms_max * 1e-3)


def time_steps(fn, steps, warmup, ws, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    outs = [fn() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return max_over_ranks(ms, ws), outs


def oracle_sample(m, wl, seconds_target=15.0, threads=0):
    """Time the FP64 oracle on a bounded sample of outer elements; returns (pairs/s, desc, cores)."""
    import oracle
    kw = {k: wl[k] for k in ("kernel", "delta", "ball", "quad_outer", "quad_inner") if k in wl}
    if "s" in wl:
        kw["s"] = wl["s"]
    stride = max(1, m.K // 1500)
    sub = np.arange(0, m.K, stride, dtype=np.int32)
    t = time.perf_counter()
    S = oracle.assemble(m, elem_subset=sub, threads=threads, **kw)
    dt = time.perf_counter() - t
    rate = S.counts["pairs"] / dt
    if dt < seconds_target / 4 and stride > 1:   # grow the sample to ~seconds_target of CPU work
        stride = max(1, int(stride * dt / seconds_target))
        sub = np.arange(0, m.K, stride, dtype=np.int32)
        t = time.perf_counter()
        S = oracle.assemble(m, elem_subset=sub, threads=threads, **kw)
        dt = time.perf_counter() - t
        rate = S.counts["pairs"] / dt
    cores = threads if threads > 0 else (os.cpu_count() or 1)
    desc = (f"outer elements k = 0 mod {stride} ({len(sub)} of {m.K}), {S.counts['pairs']} ordered pairs, "
            f"{dt:.1f} s")
    return rate, desc, cores, dt


def traffic_from_profiles(kernel_name, workload):
    """dram bytes per launch recorded in profiles/ for this kernel and workload (None if absent)."""
    p = os.path.join(ROOT, "profiles", f"{kernel_name}_{workload}.json")
    try:
        d = json.load(open(p))
        return d.get("dram_bytes_per_launch")
    except Exception:
        return None


def peaks_tflops(pk):
    """FP32 and FP64 vector peaks from the unit counts and the maximum SM clock, and the HBM peak."""
    sm_max = pk.get("sm_max_mhz", 2070.0)
    fp32 = 152 * 128 * 2 * sm_max * 1e6 / 1e12      # TFLOP/s: 128 FP32 lanes per SM, FMA = 2
    fp64 = 152 * 2 * 2 * sm_max * 1e6 / 1e12        # 2 FP64 FMA lanes per SM and clock
    return fp32, fp64, pk.get("hbm_gbs", 6800.0)


def kernel_rooflines(wl, census, info0, timed, npairs, ndof, pk, sing32):
    """Achieved algorithmic FLOP/s (or bytes/s) of every kernel of the FP32-bulk step against
    the peak of the pipe its arithmetic runs on (the singular rule: FP64 or FP32)."""
    fp32_peak, fp64_peak, hbm_peak = peaks_tflops(pk)
    fpe = FLOPS_PER_EVAL[wl["kernel"]]
    nqi = wl["quad_inner"]

    def mean(key):
        return statistics.mean(i[key] for i in timed)

    ms_whole, ms_cut, ms_close, ms_sums = mean("ms_whole"), mean("ms_cut"), mean("ms_close"), mean("ms_sums")
    red_ms = mean("ms_reduce")
    flops_whole = census["evals_whole"] * fpe + (census["evals_whole"] // nqi) * FLOPS_PER_OUTER
    flops_cut = (census["evals_cut"] * fpe + census["nonempty_points_cut"] * FLOPS_PER_OUTER
                 + census["outer_points_cut"] * FLOPS_VERTEX_TESTS
                 + census["cut_points_cut"] * (0 if wl["ball"] == "infinity" else
                                               FLOPS_EDGES + (FLOPS_CAPS if wl["ball"] == "approxcaps" else 0))
                 + census["subtri_evals_cut"] * FLOPS_SUBTRI_POINT)
    flops_duffy = census["duffy_points"] * FLOPS_DUFFY_POINT
    nc = 1 if ndof == 1 else 3
    sums_bytes = npairs * (24 * nc + 4)                          # ll records (gathered) and transposed pair ids
    conv_bytes = (info0["n_upper"] * 8 * nc + info0["nnz"] // (ndof * ndof) * 4  # fixed-point entries, columns
                  + info0["nnz"] // 2 * 8 + info0["nnz"] * 8)     # transposed positions, values written

    def rate(x, ms, scale):
        return x / (ms * 1e-3) / scale if ms > 0 else 0.0

    kernels = {
        "k_trunc_whole": {"bound": "alu", "ms": ms_whole, "units": info0["pairs_whole"],
                          "achieved": rate(flops_whole, ms_whole, 1e12), "peak": fp32_peak, "unit": "TFLOP/s",
                          "pipe": "fp32"},
        "k_trunc_cut": {"bound": "alu", "ms": ms_cut, "units": census["outer_points_cut"] // wl["quad_outer"],
                        "achieved": rate(flops_cut, ms_cut, 1e12), "peak": fp32_peak, "unit": "TFLOP/s",
                        "pipe": "fp32"},
        "k_ll_sums": {"bound": "hbm", "ms": ms_sums, "units": npairs,
                      "achieved": rate(sums_bytes, ms_sums, 1e9), "peak": hbm_peak, "unit": "GB/s"},
        "k_acc_to_csr": {"bound": "hbm", "ms": red_ms, "units": info0["n_upper"],
                         "achieved": rate(conv_bytes, red_ms, 1e9), "peak": hbm_peak, "unit": "GB/s"},
    }
    if census["singular_pairs"]:
        kernels["k_duffy"] = {"bound": "alu", "ms": ms_close, "units": census["singular_pairs"],
                              "achieved": rate(flops_duffy, ms_close, 1e12),
                              "peak": fp32_peak if sing32 else fp64_peak, "unit": "TFLOP/s",
                              "pipe": "fp32" if sing32 else "fp64"}
    for k in kernels.values():
        k["frac"] = k["achieved"] / k["peak"]
    if wl["ball"] == "infinity":
        kernels["k_trunc_cut"]["note"] = ("FP32 quadrature work only: the square's Sutherland-Hodgman cut runs in "
                                          "FP32 with exact decisions or, near ties, in FP64 (FP64-pipe bound on "
                                          "grids aligned with the square)")
    return kernels


def fp64_roofline(kernels, canon64_ms, pk):
    """The FP64 path's canonical kernel (every standard-rule pair, whole and cut) does the
    algorithmic work of the FP32-bulk whole- and cut-pair kernels (the plan's weights), on the
    FP64 pipe."""
    _, fp64_peak, _ = peaks_tflops(pk)
    flops = sum(kernels[k]["achieved"] * kernels[k]["ms"] * 1e9 for k in ("k_trunc_whole", "k_trunc_cut"))
    achieved = flops / (canon64_ms * 1e-3) / 1e12 if canon64_ms > 0 else 0.0
    return {"bound": "alu", "kernel": "k_trunc<double>", "ms": canon64_ms, "achieved": achieved,
            "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak, "pipe": "fp64"}


def rel_frobenius(sa, sb):
    """||val_a - val_b|| / ||val_b|| of two systems on the same pattern (on the device)."""
    import torch
    _, ca, va = sa.csr_views()
    _, cb, vb = sb.csr_views()
    assert torch.equal(ca, cb), "patterns differ"
    return float(torch.linalg.vector_norm(va - vb) / torch.linalg.vector_norm(vb))


def measure_config(name, steps, warmup, local, pk, with_cpu=True, variants=()):
    """One benchmark configuration besides the headline: the FP32-bulk cached step timed with
    CUDA events (clocks sampled during it), plain FP64 on the same GPU, the error of the bulk
    result against the FP64 path, the per-kernel roofline and an oracle sample; variants:
    the same step with another arithmetic of the singular rule or of the cut geometry."""
    import torch
    from paper_2207_03921_gb300 import Mesh, assemble
    wl = WORKLOADS[name]
    m = make_mesh(wl["mesh"])
    ndof = 2 if wl["kernel"] == "peridynamic" else 1
    kw = {k: wl[k] for k in ("kernel", "delta", "ball", "quad_outer", "quad_inner") if k in wl}
    if "s" in wl:
        kw["s"] = wl["s"]
    stream = torch.cuda.current_stream()
    f = torch.as_tensor(np.random.default_rng(0).standard_normal(m.M * ndof)).cuda()
    mesh = Mesh.from_synth(m, ndof)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = assemble(mesh, precision="fp32_bulk", f_nodal=f, **kw)
    torch.cuda.synchronize()
    cold_ms = (time.perf_counter() - t0) * 1e3
    info0 = S.info()
    census = S.census()
    npairs = info0["npairs"]
    del S
    out = {"desc": wl["desc"], "pairs": npairs, "nnz": info0["nnz"], "cold_ms": cold_ms,
           "singular_precision": "fp64" if census["singular_pairs"] else None, "geometry_precision": "fp32"}

    def timed_bulk(extra, nsteps):
        infos = []

        def step():
            infos.append(assemble(mesh, precision="fp32_bulk", f_nodal=f, **kw, **extra).info())

        with ClockSampler(local) as clk:
            ms, _ = time_steps(step, nsteps, warmup, 1, stream)
        return ms / nsteps, infos[warmup:], clk.summary()

    ms_step, timed, clocks = timed_bulk({}, steps)
    out.update({"ms_per_step": ms_step, "value": npairs / (ms_step * 1e-3), "unit": "pairs/s", "clocks": clocks,
                "breakdown_ms": {k: statistics.mean(i["ms_" + k] for i in timed)
                                 for k in ("whole", "cut", "close", "sums", "reduce")}})
    kernels = kernel_rooflines(wl, census, info0, timed, npairs, ndof, pk, sing32=False)
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    out["roofline"] = dict(kernels[dom], kernel=dom, kernels=kernels)
    # plain FP64 on the same GPU, and the error of the bulk result against it (the FP64 path
    # equals the oracle to 1e-12 entrywise in the parity tests)
    S64 = assemble(mesh, precision="fp64", f_nodal=f, **kw)   # warm-up (slot index built on first use)
    del S64
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    S64 = assemble(mesh, precision="fp64", f_nodal=f, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    out["fp64_plain"] = {"ms_per_step": ms64, "value": npairs / (ms64 * 1e-3),
                         "speedup_fp32_bulk_over_fp64": ms64 / ms_step}
    Sb = assemble(mesh, precision="fp32_bulk", f_nodal=f, **kw)
    out["error_vs_fp64"] = rel_frobenius(Sb, S64)
    del Sb
    out["variants"] = {}
    for vname, extra in variants:
        ms_v, _, clk_v = timed_bulk(extra, max(3, steps // 2))
        Sv = assemble(mesh, precision="fp32_bulk", f_nodal=f, **kw, **extra)
        out["variants"][vname] = {"settings": extra, "ms_per_step": ms_v, "value": npairs / (ms_v * 1e-3),
                                  "error_vs_fp64": rel_frobenius(Sv, S64), "clocks": clk_v}
        del Sv
    del S64, mesh
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if with_cpu:
        rate, desc, cores, dt = oracle_sample(m, wl, seconds_target=4.0)
        out["cpu_baseline"] = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": desc}
    return out


def run_serving(budget_gb=40, slots=8):
    """The serving stream of 512 assemble+solve requests (Poisson, 200/s): p50/p99 latency."""
    from paper_2207_03921_gb300.serving import Server, make_request
    from synth import meshes
    t = time.perf_counter()
    specs = meshes.serving_requests()
    reqs = [make_request(sp, meshes.request_mesh(sp)) for sp in specs]
    gen_s = time.perf_counter() - t
    srv = Server(budget_bytes=int(budget_gb) << 30, slots=slots)
    st = srv.run(reqs, realtime=True)
    srv.close()
    out = st.summary()
    errs = [r.error for r in st.results if r.error]
    out.update({"stream": "512 requests, Poisson 200/s, jittered Delaunay meshes of 500-50k triangles "
                          "(log-uniform), delta in {0.05, 0.1, 0.2}, constant (nocaps) or fractional "
                          "s in {0.25, 0.75} (approxcaps, singular rule on touching pairs), FP32 bulk, "
                          "CG to 1e-10 with FP64 refinement",
                "budget_gb": budget_gb, "slots": slots, "mesh_generation_s": gen_s,
                "max_rel_residual": max((r.rel_residual for r in st.results if r.error is None), default=None),
                "errors": errs[:3]})
    return out


def run_reference(args):
    """The oracle (the reference arm of this project): FP64 CPU assembly on a bounded sample."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    m = make_mesh(wl["mesh"])
    vals = []
    desc = cores = None
    for _ in range(args.warmup):
        oracle_sample(m, wl, seconds_target=3.0)
    for _ in range(args.steps):
        rate, desc, cores, dt = oracle_sample(m, wl, seconds_target=6.0)
        vals.append(rate)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": "element-pair assemblies/s", "value": v, "unit": "pairs/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"]},
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="720k", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--mode", default="bench", choices=["bench", "profile", "serving"],
                    help="profile: one cold and one cached FP32-bulk assembly, nothing else (for ncu); "
                         "serving: the request stream alone")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving stream")
    ap.add_argument("--configs", default="cfg1,cfg2,cfg3,cfg5",
                    help="further configurations measured beside the headline workload (comma list, or none)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2207_03921_gb300 import Mesh, assemble, autotune, binding

    ws, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    if args.mode == "serving":
        line = {"metric": "serving latency (arrival to u on the host)", "unit": "ms", "higher_is_better": False,
                "n_gpus": ws, "data": "synthetic"}
        line.update(run_serving())
        line["value"] = line["p99_ms"]
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    stream = torch.cuda.current_stream()
    wl = WORKLOADS[args.workload]
    m = make_mesh(wl["mesh"])
    ndof = 2 if wl["kernel"] == "peridynamic" else 1
    kw = {k: wl[k] for k in ("kernel", "delta", "ball", "quad_outer", "quad_inner") if k in wl}
    if "s" in wl:
        kw["s"] = wl["s"]
    rng = np.random.default_rng(0)
    f = torch.as_tensor(rng.standard_normal(m.M * ndof)).cuda()
    mesh = Mesh.from_synth(m, ndof)

    if args.mode == "profile":
        for prec in ("fp32_bulk", "fp32_bulk"):
            assemble(mesh, precision=prec, f_nodal=f, **kw)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "profile", "workload": args.workload}), flush=True)
        return

    # cold assembly: pair search + pattern + values
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = assemble(mesh, precision="fp32_bulk", f_nodal=f, **kw)
    torch.cuda.synchronize()
    cold_ms = (time.perf_counter() - t0) * 1e3
    info0 = S.info()
    census = S.census()
    npairs = info0["npairs"]
    del S

    # launch shape of the bulk kernels picked by the autotuner (results do not depend on it)
    tuned = autotune(mesh, **kw)

    # steady FP32-bulk steps
    infos = []

    def step():
        s = assemble(mesh, precision="fp32_bulk", f_nodal=f, **kw)
        infos.append(s.info())
        return None

    with ClockSampler(local) as clk:
        ms, _ = time_steps(step, args.steps, args.warmup, ws, stream)
    timed = infos[args.warmup:]
    ms_step = ms / args.steps
    value = replica_value(npairs, ws, ms_step)
    quad_ms = statistics.mean(i["ms_quadrature"] for i in timed)
    red_ms = statistics.mean(i["ms_reduce"] for i in timed)

    # plain FP64 on the same GPU
    infos.clear()
    ms64_step = quad64_ms = None
    if args.fp64_steps > 0:
        ms64, _ = time_steps(lambda: infos.append(assemble(mesh, precision="fp64", f_nodal=f, **kw).info()),
                             args.fp64_steps, 1, ws, stream)
        ms64_step = ms64 / args.fp64_steps
        quad64_ms = statistics.mean(i["ms_quadrature"] for i in infos[1:])
        canon64_ms = statistics.mean(i["ms_cut"] for i in infos[1:])

    # end to end through the C ABI with host buffers: pinned verts/elems/labels/f -> mesh, assemble,
    # CSR values + load vector back to pinned host memory
    hv = torch.as_tensor(m.verts).pin_memory()
    he = torch.as_tensor(m.elems).pin_memory()
    hl = torch.as_tensor(m.elem_label).pin_memory()
    hf = f.cpu().pin_memory()
    p = binding.make_params(precision="fp32_bulk", **kw)
    e2e_steps = max(1, min(3, args.steps))
    out_val = out_F = None
    h2d = hv.numel() * 8 + he.numel() * 4 + hl.numel() + hf.numel() * 8
    d2h = 0

    def e2e_step():
        nonlocal out_val, out_F, d2h
        mh = binding.nlfem_mesh_create(hv, he, hl, ndof, stream)
        sh = binding.nlfem_assemble(mh, p, hf, stream)
        rp, col, val, n, nnz = binding.nlfem_system_csr(sh)
        if out_val is None:
            out_val = torch.empty(nnz, dtype=torch.float64).pin_memory()
            out_F = torch.empty(n, dtype=torch.float64).pin_memory()
        # device -> pinned host copies of the result through torch views
        from paper_2207_03921_gb300.api import _DevView
        vv = torch.as_tensor(_DevView(val, nnz, "<f8", None), device="cuda")
        fv = torch.as_tensor(_DevView(binding.nlfem_system_rhs(sh), n, "<f8", None), device="cuda")
        out_val.copy_(vv, non_blocking=True)
        out_F.copy_(fv, non_blocking=True)
        torch.cuda.synchronize()
        d2h = nnz * 8 + n * 8
        binding.nlfem_system_destroy(sh)
        binding.nlfem_mesh_destroy(mh)
        return None

    e2e_ms, _ = time_steps(e2e_step, e2e_steps, 1, ws, stream)
    e2e_cold_value = replica_value(npairs, ws, e2e_ms / e2e_steps)
    h2d_cold, d2h_cold = h2d, d2h

    # the steady step end to end: a mesh handle uploaded once from the pinned host arrays (its
    # first assembly, untimed, builds the pair list and pattern), then per step the load data
    # from pinned host memory -> nlfem_assemble -> CSR values and F to pinned host memory
    mh_res = binding.nlfem_mesh_create(hv, he, hl, ndof, stream)

    def e2e_cached_step():
        nonlocal out_val, out_F, d2h
        sh = binding.nlfem_assemble(mh_res, p, hf, stream)
        rp, col, val, n, nnz = binding.nlfem_system_csr(sh)
        from paper_2207_03921_gb300.api import _DevView
        vv = torch.as_tensor(_DevView(val, nnz, "<f8", None), device="cuda")
        fv = torch.as_tensor(_DevView(binding.nlfem_system_rhs(sh), n, "<f8", None), device="cuda")
        out_val.copy_(vv, non_blocking=True)
        out_F.copy_(fv, non_blocking=True)
        torch.cuda.synchronize()
        d2h = nnz * 8 + n * 8
        binding.nlfem_system_destroy(sh)
        return None

    e2e_ms, _ = time_steps(e2e_cached_step, max(3, min(10, args.steps)), 2, ws, stream)
    e2e_value = replica_value(npairs, ws, e2e_ms / max(3, min(10, args.steps)))
    binding.nlfem_mesh_destroy(mh_res)
    h2d = hf.numel() * 8

    # roofline of the dominant kernel: the longest of the bulk quadrature kernels (FP32 ALU),
    # the close-list kernel (the singular rule, FP64 ALU), the per-element sums and the
    # conversion of the fixed-point entries into CSR (HBM)
    pk = peaks()
    clk_sum = clk.summary()
    kernels = kernel_rooflines(wl, census, info0, timed, npairs, ndof, pk, sing32=False)
    ms_whole, ms_cut, ms_close, ms_sums = (statistics.mean(i[k] for i in timed)
                                           for k in ("ms_whole", "ms_cut", "ms_close", "ms_sums"))
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    d = kernels[dom]
    peak_src = {"alu": "derived: 152 SMs x (128 FP32 | 2 FP64) lanes x 2 x max SM clock",
                "hbm": "MEASURED_PEAKS hbm_gbs" if "hbm_gbs" in pk else "fallback 6.8 TB/s"}
    roof = {"bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
            "frac": d["frac"], "traffic": traffic_from_profiles(dom, args.workload), "kernel": dom,
            "ms_per_launch": d["ms"], "peak_source": peak_src[d["bound"]], "kernels": kernels}

    line = {
        "metric": "element-pair assemblies/s", "value": value, "unit": "pairs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("f32 (truncation quadrature, cut geometry with decisions equal to f64) + i64 fixed-point sums "
                  "+ f64 (singular rule, near ties, CSR values)"),
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "precision": "fp32_bulk",
                   "step": "nlfem_assemble with cached pair list and pattern",
                   "l2": "working set larger than L2 (pair lists, kl ranks and per-pair ll records stream from HBM)",
                   "pairs": npairs, "nnz": info0["nnz"], "parallelism": "replicas" if ws > 1 else "single GPU",
                   "autotune_shape": {"whole_pairs_blocks_per_sm": tuned[0], "cut_pairs_blocks_per_sm": tuned[1],
                                      "cut_pairs_outer_points_per_chunk": tuned[2]}},
        "roofline": roof,
        "fp64_plain": ({"value": npairs * ws / (ms64_step * 1e-3), "ms_per_step": ms64_step,
                        "quadrature_ms": quad64_ms, "speedup_fp32_bulk_over_fp64": ms64_step / ms_step,
                        "roofline": fp64_roofline(kernels, canon64_ms, pk)}
                       if ms64_step else None),
        "breakdown_ms": {"quadrature": quad_ms, "whole_pairs": ms_whole, "cut_pairs": ms_cut,
                         "close_list": ms_close, "ll_sums": ms_sums, "to_csr": red_ms, "cold_total": cold_ms,
                         "pairs_search": info0["ms_pairs"], "pattern_and_index": info0["ms_pattern"]},
        "cold": {"value": npairs / (cold_ms * 1e-3), "ms": cold_ms},
        "census": census,
        "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "pinned host load data -> nlfem_assemble on a resident mesh handle (pair list and "
                        "pattern cached) -> CSR values and F to pinned host memory",
                "cold": {"value": e2e_cold_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d_cold,
                         "d2h_bytes_per_step": d2h_cold,
                         "path": "pinned host mesh -> nlfem_mesh_create -> nlfem_assemble (pair search, "
                                 "pattern, values) -> CSR values and F to pinned host memory"}},
        # per timed step: whole-pair and cut-pair kernels, the ll sums, the scale check, fixed
        # point to CSR, load vector (6; the pilot pass and the scale pick ran once, at the first
        # assembly on the pattern); with a close list also its kernel and its records' pass, and
        # under the singular rule the copy of the mirrored orders' blocks
        "gpu_launches": args.steps * (6 + (3 if census["singular_pairs"] else
                                           2 if census["evals_canonical"] else 0)),
        "clocks": clk_sum,
    }
    # the other benchmark configurations, each with its own clocks, FP64 comparison, error
    # against the FP64 path, roofline and oracle sample; the precision variants of the FP32-bulk
    # path (singular rule in FP32, cut geometry in FP64) beside the default split
    geo64 = ("geometry_fp64", {"geometry_precision": "fp64"})
    sing32 = ("singular_fp32", {"singular_precision": "fp32"})
    if ws == 1 and args.configs != "none":
        del mesh
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        mesh = None
        line["configs"] = {}
        vsteps = max(3, min(10, args.steps))
        for cname in [c for c in args.configs.split(",") if c and c != args.workload]:
            var = {"cfg2": (sing32, geo64), "cfg3": (geo64,)}.get(cname, ())
            try:
                line["configs"][cname] = measure_config(cname, vsteps, args.warmup, local, pk,
                                                        with_cpu=not args.no_cpu, variants=var)
            except Exception as e:  # reported; the headline numbers stand
                line["configs"][cname] = {"error": f"{type(e).__name__}: {e}"}
        # the headline workload's error against FP64 and its cut geometry in FP64
        try:
            v = measure_config(args.workload, vsteps, args.warmup, local, pk, with_cpu=False, variants=(geo64,))
            line["precision"] = {"error_vs_fp64": v["error_vs_fp64"], "variants": v["variants"],
                                 "singular_precision": v["singular_precision"],
                                 "geometry_precision": v["geometry_precision"]}
        except Exception as e:
            line["precision"] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_serving:
        del mesh
        torch.cuda.synchronize()
        try:
            line["serving"] = run_serving()
        except Exception as e:  # reported, the assembly numbers stand
            line["serving"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and ws == 1 and not args.no_cpu:
        rate, desc, cores, dt = oracle_sample(m, wl)
        line["cpu_baseline"] = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": desc}
        # the same oracle on one core, a smaller sample
        rate1, desc1, _, _ = oracle_sample(m, wl, seconds_target=8.0, threads=1)
        line["cpu_baseline"]["single_core"] = {"value": rate1, "sample": desc1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
