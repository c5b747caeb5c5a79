#!/usr/bin/env python
"""Benchmark: radiosity RHS/s of the compressed F.X Jacobi solve.

Workload (the terrain configuration the metric is quoted on): a 200 x 200
seeded fBm DEM (Hurst 0.8, RMS slope 15 deg, 10 m spacing) with an embedded
1 km spherical-cap crater -> 79,202 triangles; quadtree with 64-facet
leaves; F compressed at tol 1e-3 in FP32; E = direct solar flux for sun
positions at 10 deg elevation (azimuth sweep); albedo 0.12; Jacobi to
rtol 1e-6.  One step = one vf_solve of R right-hand sides (default R = 1,
the single-RHS configuration): permute in, the device-side Jacobi loop
(phase-1/phase-2 multiply with the fused update), permute out.

Reported beside the headline: the same solve with the uncompressed dense
FP32 F (25 GB) on the same GPU, the roofline of the multiply kernel pair
(algorithmic bytes / CUDA-event time vs the measured HBM copy bandwidth),
an end-to-end number through vf_solve_host (host buffers, copies in the
timed region), SM clocks sampled during the timed region, and the CPU
oracle timed on a bounded sample of rows.

--impl reference times the CPU oracle (plain FP64 dense F, numpy) on the
host cores instead, on a bounded row sample, as the reference arm.
"""
from __future__ import annotations

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

METRIC = "radiosity RHS/s of compressed F·X solve vs dense & plain FP32, at rel err 1e-3"
WORKLOAD = "fbm200_crater_79202tri_quadtree64_tol1e-3"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--rhs", type=int, default=1)
    p.add_argument("--dem-size", type=int, default=200, help="DEM side (200 -> 79,202 facets); smaller for profiling")
    p.add_argument("--tol", type=float, default=1e-3)
    p.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp8"])
    p.add_argument("--no-dense", action="store_true", help="skip the dense-F comparison")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--cpu-rows", type=int, default=128, help="rows of F in the CPU oracle sample")
    p.add_argument("--no-batched", action="store_true", help="skip the batched (tensor-core) section")
    p.add_argument("--batch-rhs", type=int, default=1440, help="RHS (sun positions) of the batched section")
    p.add_argument("--multimesh", type=int, default=32, help="meshes of the multi-mesh section (0: skip)")
    p.add_argument("--multimesh-max-side", type=int, default=200,
                   help="largest DEM side of the multi-mesh section (51 -> 5,000 facets, 200 -> 79,202)")
    p.add_argument("--multimesh-rhs", type=int, default=256, help="RHS per mesh in the multi-mesh section")
    p.add_argument("--no-tol-sweep", action="store_true", help="skip the terrain at tol 1e-2 and 1e-4")
    p.add_argument("--profile-batched", action="store_true",
                   help="only run --steps refined solves of --batch-rhs suns, BF16 (or --precision fp8) "
                        "sweeps on the tensor cores (for a profiler's launch list)")
    p.add_argument("--profile-apply", action="store_true",
                   help="only run --warmup + --steps tensor-core multiplies of --batch-rhs seeded columns in "
                        "--precision (bf16 or fp8; outside any CUDA graph, for a profiler)")
    p.add_argument("--no-config4", action="store_true", help="skip the 522,242-facet precision section")
    p.add_argument("--config4-only", action="store_true",
                   help="run only the 522,242-facet precision section (with its oracle check)")
    p.add_argument("--config4-side", type=int, default=512, help="DEM side of the precision section (512 -> 522,242)")
    p.add_argument("--config4-rows", type=int, default=4096, help="oracle-sampled rows of the precision section")
    p.add_argument("--steady-s", type=float, default=2.0,
                   help="seconds of back-to-back steps after the timed K (a steady-state cross-check)")
    return p.parse_args()


def synth_dirs(R: int):
    import synth
    return synth.sun_directions(R, 10.0)


def max_over_ranks(x: float, world: int, device: str) -> float:
    """The largest of every rank's x (a time): the job is as slow as its slowest replica."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_all_ranks: int, seconds: float) -> float:
    """Units processed by all replicas per second of the slowest one (weak scaling)."""
    return units_all_ranks / seconds


def lunar_day_dirs(R: int):
    """R sun directions over one lunar day: an azimuth sweep at 1.5 deg elevation."""
    import synth
    return synth.sun_directions(R, 1.5)


def workload_inputs(R: int, side: int = 200):
    import synth
    v, f = synth.fbm_dem_mesh(n=side, spacing=10.0, hurst=0.8, seed=1, rms_slope_deg=15.0, crater_diameter=1000.0)
    dirs = synth.sun_directions(R, 10.0)
    return v, f, dirs


# ------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle
class CpuOracle:
    """The oracle's dense FP64 multiply (the work of one Jacobi sweep) on a
    bounded, seeded sample of rows of F, extrapolated to the full solve:
    t_solve = sweeps * (N / rows) * t_rows.  Building the sampled rows
    (visibility by the oracle's BVH, then Eq. FF-def) is setup, untimed."""

    def __init__(self, v, f, dirs, rows: int, R: int):
        import numpy as np

        import oracle
        self.om = oracle.mesh(v, f)
        rng = np.random.default_rng(7)
        self.rows = rows
        self.S = np.sort(rng.choice(self.om.n, size=rows, replace=False))
        self.Fs = oracle.F_rows(self.om, self.S)
        self.E = oracle.insolation(self.om, dirs[:R], 1365.0)
        self.R = R

    def batched_check(self, v, f, host):
        """The batched solve's error against the oracle on this sample's rows:
        per column ||B_S - T(B)_S|| / ||T(B)_S|| with T(B)_S = E_S + rho F_S B,
        one exact oracle Jacobi step from the GPU's B (within a factor
        1 +- rho/(1 - rho) of the error against the oracle's exact B*); E_S
        is the oracle's own insolation for the batch's suns."""
        from oracle import sampled
        t0 = time.time()
        with sampled.SampledOracle(v, f, self.S) as so:
            Eo = so.insolation_rows(host["dirs"], 1365.0)
            workers = so.workers
        Bg = host["B"]
        TB = Eo + host["rho"] * (self.Fs @ Bg)
        nr = np.linalg.norm(TB, axis=0)
        live = nr > 0
        err = np.linalg.norm(Bg[self.S] - TB, axis=0)[live] / nr[live]
        return {"rows": int(self.rows), "seed": 7, "columns": int(live.sum()), "workers": workers,
                "solve_rel_err_vs_oracle": float(err.max()), "median": float(np.median(err)),
                "oracle_s": round(time.time() - t0, 1),
                "reference": "oracle FP64 F rows and insolation on the sampled rows; E_S + rho F_S B"}

    def measure(self, sweeps: int, seconds: float):
        reps = 0
        t0 = time.perf_counter()
        while True:
            _ = self.Fs @ self.E
            reps += 1
            if time.perf_counter() - t0 >= seconds:
                break
        t_rows = (time.perf_counter() - t0) / reps
        t_solve = sweeps * (self.om.n / self.rows) * t_rows
        try:
            import threadpoolctl
            cores = max(int(i.get("num_threads", 1)) for i in threadpoolctl.threadpool_info())
        except Exception:
            cores = os.cpu_count()
        return {"value": self.R / t_solve, "unit": "RHS/s", "cores": cores, "kind": "oracle",
                "sample": f"dense FP64 F, {self.rows} of {self.om.n} rows (seeded), y = F_S E timed over "
                          f"{reps} repeats ({reps * t_rows:.1f} s), extrapolated x{self.om.n / self.rows:.0f} "
                          f"rows x {sweeps} sweeps"}


# ------------------------------------------------------------- precision workload
C4_RHO = 0.12


def config4_inputs(side: int = 512):
    """512 x 512 seeded fBm DEM (Hurst 0.8, 5 m spacing, RMS slope 15 deg,
    seed 2, no crater): 522,242 triangles; 256 suns over one lunar day."""
    import synth
    v, f = synth.fbm_dem_mesh(n=side, spacing=5.0, hurst=0.8, seed=2, rms_slope_deg=15.0, crater_diameter=None)
    return v, f, synth.sun_directions(256, 1.5)


def c4_workload(n: int) -> str:
    return f"fbm{int(round((n / 2) ** 0.5)) + 1}_5m_{n}tri_quadtree64_tol1e-3"


def events_ms(fn, reps: int, st) -> float:
    """Mean time of fn() over reps back-to-back calls, CUDA events on st."""
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        fn()
    b.record(st)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_config4(a, dev, peak, st):
    """The precision workload on the GPU: assembly, the FP32 single-RHS
    multiply, the 256-RHS BF16 tensor-core solve with split-BF16 refinement
    (and the FP8 solve), the tensor multiply's roofline.  Returns the
    result object and what the oracle check needs (host copies)."""
    import torch

    from paper_2209_07632_gb300 import vf
    v, f, dirs = config4_inputs(a.config4_side)
    t0 = time.time()
    prob = vf.build_problem(v, f, kind="quad", leaf_size=64, tol=1e-3, device=dev,
                            precisions=("fp32", "bf16", "fp8"))
    t_asm = time.time() - t0
    n = prob.mesh.n
    h = prob.hmat
    R = dirs.shape[0]
    E = torch.empty((R, n), device="cuda", dtype=torch.float32)
    vf.vf_mesh_insolation(prob.mesh, dirs, 1365.0, E)
    perm = torch.tensor(vf.vf_tree_perm(prob.tree).astype(np.int64), device="cuda")
    # FP32 single-RHS multiply (the plain compressed apply): tree order, CUDA events
    X1 = E[:1, perm].contiguous()
    Y1 = torch.empty_like(X1)
    for _ in range(3):
        vf.vf_apply_tree(h, X1, Y1)
    torch.cuda.synchronize()
    ms1 = events_ms(lambda: vf.vf_apply_tree(h, X1, Y1), 20, st)
    b32 = vf.vf_hmat_bytes(h, "fp32") + n * 8
    single_rhs = 1000.0 / ms1
    # the batched BF16 solve: tensor-core sweeps, split-BF16 residual refinement
    B = torch.empty_like(E)
    kw = dict(rho=C4_RHO, rtol=1e-4, precision="bf16", refine=True)
    t1 = time.time()
    sb = vf.vf_solve(h, E, B, **kw)
    torch.cuda.synchronize()
    t_first = time.time() - t1
    sb = vf.vf_solve(h, E, B, **kw)
    torch.cuda.synchronize()
    bms = events_ms(lambda: vf.vf_solve(h, E, B, **kw), 5, st)
    # the tensor multiply alone (128 and 256 RHS, BF16)
    Xb = E[:, perm].contiguous()
    Yb = torch.empty_like(Xb)
    tm = {}
    for r in (128, 256):
        for _ in range(2):
            vf.vf_apply_tree(h, Xb[:r], Yb[:r], precision="bf16")
        torch.cuda.synchronize()
        ms = events_ms(lambda: vf.vf_apply_tree(h, Xb[:r], Yb[:r], precision="bf16"), 10, st)
        alg = vf.vf_hmat_bytes(h, "bf16") + n * r * 6
        tm[str(r)] = {"ms": round(ms, 4), "alg_bytes": alg, "hbm_frac": round(alg / (ms / 1e3) / 1e9 / peak, 4)}
    tpages = vf.vf_hmat_tensor_bytes(h, 1)
    # the FP8 tensor multiply (kind::f8f6f4; FP8 panels: 1 byte read per RHS entry, FP32 result)
    tm8 = {}
    for r in (128, 256):
        for _ in range(2):
            vf.vf_apply_tree(h, Xb[:r], Yb[:r], precision="fp8")
        torch.cuda.synchronize()
        ms = events_ms(lambda: vf.vf_apply_tree(h, Xb[:r], Yb[:r], precision="fp8"), 10, st)
        alg = vf.vf_hmat_bytes(h, "fp8") + n * r * 5
        tm8[str(r)] = {"ms": round(ms, 4), "alg_bytes": alg, "hbm_frac": round(alg / (ms / 1e3) / 1e9 / peak, 4)}
    tpages8 = vf.vf_hmat_tensor_bytes(h, 3)
    # FP8 sweeps on the tensor cores with the same refinement
    B8 = torch.empty_like(E)
    kw8 = dict(rho=C4_RHO, rtol=1e-4, precision="fp8", refine=True)
    s8 = vf.vf_solve(h, E, B8, **kw8)
    torch.cuda.synchronize()
    ms8 = events_ms(lambda: vf.vf_solve(h, E, B8, **kw8), 2, st)
    # the three multiplies of all 256 suns (for the apply check), each after
    # the handle's cached pages and workspaces are released (the 256-column
    # FP32 multiply alone holds ~20 GB of T scratch at this size)
    Y32, Ybf, Yf8 = torch.empty_like(E), torch.empty_like(E), torch.empty_like(E)
    for prec, Y in (("fp32", Y32), ("bf16", Ybf), ("fp8", Yf8)):
        torch.cuda.synchronize()
        vf.vf_hmat_trim(h)
        torch.cuda.empty_cache()
        vf.vf_apply(h, E, Y, precision=prec)
    torch.cuda.synchronize()
    vf.vf_hmat_trim(h)
    res = {"workload": c4_workload(n), "facets": n, "rhs": R, "tol": 1e-3, "rho": C4_RHO,
           "suns": "lunar-day azimuth sweep at 1.5 deg elevation",
           "assembly_s": round(t_asm, 1),
           "assembly": {k: prob.stats[k] for k in ("nblocks", "bytes", "probes", "max_rank", "t_visibility",
                                                   "t_probe", "t_total")},
           "bytes": {p: vf.vf_hmat_bytes(h, p) for p in ("fp32", "bf16", "fp8")},
           "value": round(R / (bms / 1e3), 1), "unit": "RHS/s", "ms_per_solve": round(bms, 3),
           "precision": "bf16 factors and RHS on tcgen05 tensor cores, FP32 accumulation; "
                        "split-BF16 residual refinement with FP64 update, rtol 1e-4",
           "sweeps": sb["sweeps"], "refinements": sb["refinements"], "converged": sb["converged"],
           "first_solve_s": round(t_first, 2),
           "fp32_single_rhs_multiply": {"ms": round(ms1, 4), "rhs_per_s": round(single_rhs, 1),
                                        "hbm_frac": round(b32 / (ms1 / 1e3) / 1e9 / peak, 4)},
           "x_fp32_single_rhs_apply": round((R / (bms / 1e3)) / single_rhs, 2),
           "tensor_multiply": tm, "hbm_frac": tm["128"]["hbm_frac"], "tensor_page_bytes": tpages,
           "fp8_solve": {"value": round(R / (ms8 / 1e3), 1), "unit": "RHS/s", "ms_per_solve": round(ms8, 3),
                         "sweeps": s8["sweeps"], "refinements": s8["refinements"], "converged": s8["converged"],
                         "precision": "fp8 e4m3 factors and RHS on tcgen05 tensor cores (kind::f8f6f4), "
                                      "power-of-two scales per RHS column, row and SVD rank column, FP32 "
                                      "accumulation; split-BF16 residual refinement with FP64 update, rtol 1e-4",
                         "tensor_multiply": tm8, "hbm_frac": tm8["128"]["hbm_frac"],
                         "tensor_page_bytes": tpages8}}
    host = {"v": v, "f": f, "dirs": dirs, "n": n,
            "E": E.double().cpu().numpy().T, "B": B.double().cpu().numpy().T,
            "B8": B8.double().cpu().numpy().T, "Y32": Y32.double().cpu().numpy().T,
            "Ybf": Ybf.double().cpu().numpy().T, "Yf8": Yf8.double().cpu().numpy().T}
    del prob, h, E, B, B8, Xb, Yb, X1, Y1, Y32, Ybf, Yf8, perm
    return res, host


def config4_oracle_check(host, nrows: int):
    """The oracle on nrows rows sampled without replacement (seed 7): its F
    rows (Eq. FF-def, its own visibility) and insolation; errors per
    column over the sampled rows (max over columns).  The solve's reference
    is one exact oracle Jacobi step from the GPU's B, T(B)_S = E_S + rho F_S B:
    since T contracts by rho ||F|| <= rho, |B* - T(B)| <= rho/(1-rho) |B* - B|,
    so this sampled error is within a factor 1 +- 0.14 of the error against
    the oracle's exact solution B*."""
    from oracle import sampled
    n = host["n"]
    rows = np.sort(np.random.default_rng(7).choice(n, nrows, replace=False))
    t0 = time.time()
    with sampled.SampledOracle(host["v"], host["f"], rows) as so:
        ip, ix, dv = so.F_rows_sparse()
        Eo = so.insolation_rows(host["dirs"], 1365.0)
        workers = so.workers
    t_or = time.time() - t0

    def colerr(got, ref):
        nr = np.linalg.norm(ref, axis=0)
        live = nr > 0
        return float((np.linalg.norm(got - ref, axis=0)[live] / nr[live]).max()), int(live.sum())

    E = host["E"]
    FE = sampled.csr_matmul(ip, ix, dv, E)
    out = {"rows": nrows, "seed": 7, "workers": workers, "oracle_s": round(t_or, 1)}
    out["insolation_max_abs_err_rel_to_max"] = float(np.abs(E[rows] - Eo).max() / max(Eo.max(), 1e-300))
    out["apply_fp32_rel_err"], live = colerr(host["Y32"][rows], FE)
    out["apply_bf16_rel_err"], _ = colerr(host["Ybf"][rows], FE)
    out["apply_fp8_rel_err"], _ = colerr(host["Yf8"][rows], FE)
    out["columns"] = live
    for key, name in (("B", "solve_bf16_refined_rel_err"), ("B8", "solve_fp8_refined_rel_err")):
        Bg = host[key]
        TB = Eo + C4_RHO * sampled.csr_matmul(ip, ix, dv, Bg)
        out[name], _ = colerr(Bg[rows], TB)
    out["reference"] = ("oracle FP64 F rows (own BVH visibility, Eq. FF-def) and insolation on the sampled rows; "
                        "solve reference E_S + rho F_S B (one exact oracle Jacobi step from the GPU's B)")
    return out


# ------------------------------------------------------------- main
def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if a.impl == "reference":
        if rank != 0:
            return
        v, f, dirs = workload_inputs(max(a.rhs, 1), a.dem_size)
        # the oracle's Jacobi takes the sweeps the GPU solve takes on this workload (4 at rtol 1e-6)
        sweeps = 4
        co = CpuOracle(v, f, dirs, a.cpu_rows, a.rhs)
        # each step: a timed sample of the oracle's rows, sized so the whole run stays near two minutes
        per = min(1.0, max(0.05, 120.0 / (a.warmup + a.steps)))
        samples = [co.measure(sweeps, seconds=per) for _ in range(a.warmup + a.steps)]
        val = sorted(s["value"] for s in samples[a.warmup:])[len(samples[a.warmup:]) // 2]
        cb = dict(samples[-1])
        cb["value"] = val
        line = {"metric": METRIC, "value": val, "unit": "RHS/s", "n_gpus": a.gpus, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": 1000.0 * a.rhs / val, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD if a.dem_size == 200 else f"fbm{a.dem_size}_crater",
                           "facets": int(co.om.n), "rhs_per_gpu": a.rhs, "tol": a.tol},
                "impl": "reference", "cpu_baseline": cb,
                "e2e": {"value": val, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_07632_gb300 import vf

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    st = torch.cuda.current_stream()

    if a.config4_only:
        c4, host = run_config4(a, dev, peak, st)
        if not a.no_cpu:
            c4["oracle_check"] = config4_oracle_check(host, a.config4_rows)
        print(json.dumps({"config4": c4}))
        return

    if a.profile_apply:
        prec = a.precision if a.precision != "fp32" else "bf16"
        v, f, _ = workload_inputs(1, a.dem_size)
        prob = vf.build_problem(v, f, kind="quad", leaf_size=64, tol=a.tol, device=dev,
                                precisions=("fp32", "bf16", "fp8"))
        gen = torch.Generator(device="cpu").manual_seed(5)
        X = torch.rand((a.batch_rhs, prob.mesh.n), generator=gen).cuda()
        Y = torch.empty_like(X)
        for _ in range(a.warmup + a.steps):
            vf.vf_apply_tree(prob.hmat, X, Y, precision=prec)
        torch.cuda.synchronize()
        print(json.dumps({"profile_apply": True, "precision": prec, "facets": prob.mesh.n, "rhs": a.batch_rhs,
                          "multiplies": a.warmup + a.steps}))
        return

    if a.profile_batched:
        prec = a.precision if a.precision != "fp32" else "bf16"  # the sweeps' precision (tensor cores)
        v, f, _ = workload_inputs(1, a.dem_size)
        prob = vf.build_problem(v, f, kind="quad", leaf_size=64, tol=a.tol, device=dev,
                                precisions=("fp32", "bf16", "fp8"))
        Eb = torch.empty((a.batch_rhs, prob.mesh.n), device="cuda", dtype=torch.float32)
        vf.vf_mesh_insolation(prob.mesh, lunar_day_dirs(a.batch_rhs), 1365.0, Eb)
        Bb = torch.empty_like(Eb)
        for _ in range(a.warmup + a.steps):
            vf.vf_solve(prob.hmat, Eb, Bb, rho=0.12, rtol=1e-4, precision=prec, refine=True)
        torch.cuda.synchronize()
        print(json.dumps({"profile_batched": True, "facets": prob.mesh.n, "rhs": a.batch_rhs, "solves": a.steps}))
        return

    R = a.rhs
    v, f, dirs = workload_inputs(R, a.dem_size)
    t0 = time.time()
    prob = vf.build_problem(v, f, kind="quad", leaf_size=64, tol=a.tol, device=dev,
                            precisions=("fp32", "bf16", "fp8"))
    t_setup = time.time() - t0
    n = prob.mesh.n
    E = torch.empty((R, n), device="cuda", dtype=torch.float32)
    vf.vf_mesh_insolation(prob.mesh, dirs, 1365.0, E)
    B = torch.empty_like(E)
    rho = 0.12
    rtol = 1e-6

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    solve_kw = dict(rho=rho, rtol=rtol, precision=a.precision, refine=a.precision != "fp32")
    for _ in range(max(a.warmup, 3)):
        stats = vf.vf_solve(prob.hmat, E, B, **solve_kw)
    sweeps = stats["sweeps"]
    barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    kernels = 0
    ev0.record(st)
    for _ in range(a.steps):
        stats = vf.vf_solve(prob.hmat, E, B, **solve_kw)
        kernels += stats["kernels"]
    ev1.record(st)
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / a.steps, world, "cuda")
    # steady state: back-to-back steps for at least --steady-s seconds (not
    # part of the K timed steps; a cross-check of ms_per_step with the clocks
    # sampled over a longer window)
    steady = None
    if a.steady_s > 0:
        nst = max(1, int(a.steady_s * 1000.0 / max(ms, 1e-3)))
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(st)
        for _ in range(nst):
            vf.vf_solve(prob.hmat, E, B, **solve_kw)
        s1.record(st)
        barrier()
        sms = max_over_ranks(s0.elapsed_time(s1) / nst, world, "cuda")
        steady = {"steps": nst, "seconds": round(sms * nst / 1000.0, 2), "ms_per_step": round(sms, 4),
                  "value": round(whole_job_rate(world * R, sms / 1000.0), 3)}
    clk = clocks.stop()
    value = whole_job_rate(world * R, ms / 1000.0)

    # ---- roofline of the multiply (phase 1 + phase 2), tree order, on `st`
    Xt = E.clone()
    Yt = torch.empty_like(Xt)
    for _ in range(5):
        vf.vf_apply_tree(prob.hmat, Xt, Yt, precision=a.precision)
    torch.cuda.synchronize()
    reps = 50
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(st)
    for _ in range(reps):
        vf.vf_apply_tree(prob.hmat, Xt, Yt, precision=a.precision)
    k1.record(st)
    torch.cuda.synchronize()
    mult_ms = k0.elapsed_time(k1) / reps
    alg_bytes = vf.vf_hmat_bytes(prob.hmat, a.precision) + n * R * 8
    achieved = alg_bytes / (mult_ms / 1000.0) / 1e9
    traffic = None
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", "multiply_traffic.json")))
        if prof.get("workload") == WORKLOAD and prof.get("rhs") == R and prof.get("precision") == a.precision:
            traffic = prof.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": "multiply = k_phase1 + k_p1_reduce + k_phase2", "alg_bytes_per_launch": alg_bytes,
                "ms_per_launch": round(mult_ms, 4),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if peaks else "fallback 6.8 TB/s"}

    # ---- end to end through vf_solve_host (pinned host buffers, copies timed)
    Eh = E.cpu().pin_memory().numpy()
    Bh = torch.empty((R, n), dtype=torch.float32).pin_memory().numpy()
    for _ in range(2):
        vf.vf_solve_host(prob.hmat, Eh, Bh, **solve_kw)
    barrier()
    e0 = time.perf_counter()
    for _ in range(a.steps):
        vf.vf_solve_host(prob.hmat, Eh, Bh, **solve_kw)
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - e0) / a.steps, world, "cuda")
    e2e = {"value": whole_job_rate(world * R, e2e_s), "unit": "RHS/s", "h2d_bytes_per_step": n * R * 4,
           "d2h_bytes_per_step": n * R * 4}

    # ---- batched: 1,440 sun positions over one lunar day (azimuth sweep at
    # 1.5 deg elevation) on the same mesh, BF16 sweeps on the tensor cores
    # (tcgen05, FP32 accumulation) with split-BF16 residual refinement; the
    # autotuner picks the path and the RHS block, and RHS blocks of 64, 256
    # and 1440 are timed as well
    batched = None
    batched_host = None
    if not a.no_batched and rank == 0:
        Rb = a.batch_rhs
        Eb = torch.empty((Rb, n), device="cuda", dtype=torch.float32)
        vf.vf_mesh_insolation(prob.mesh, lunar_day_dirs(Rb), 1365.0, Eb)
        Bb = torch.empty_like(Eb)
        Bref = torch.empty_like(Eb)
        vf.vf_solve(prob.hmat, Eb, Bref, rho=rho, rtol=rtol)  # FP32 CUDA-core solve: the accuracy reference
        bkw = dict(rho=rho, rtol=1e-4, precision="bf16", refine=True)
        t_tune = time.time()
        tune = vf.vf_autotune(prob.hmat, "bf16", Rb)
        t_tune = time.time() - t_tune

        def time_solves(steps):
            for _ in range(2):
                sb = vf.vf_solve(prob.hmat, Eb, Bb, **bkw)
            torch.cuda.synchronize()
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(st)
            for _ in range(steps):
                sb = vf.vf_solve(prob.hmat, Eb, Bb, **bkw)
            b1.record(st)
            torch.cuda.synchronize()
            return b0.elapsed_time(b1) / steps, sb

        blocks = {}
        for w in (64, 256, Rb):
            if w > Rb:
                continue
            vf.vf_tune_set(prob.hmat, "bf16", Rb, rb=8, tensor=1, rhs_block=0 if w == Rb else w)
            wms, _ = time_solves(3)
            blocks[str(w)] = round(Rb / (wms / 1000.0), 1)
        vf.vf_tune_set(prob.hmat, "bf16", Rb, rb=tune["rb"], tensor=tune["tensor"], rhs_block=tune["rhs_block"])
        bms, sb = time_solves(max(3, min(a.steps, 20)))
        live = Bref.norm(dim=1) > 0
        brel = float(((Bb - Bref).norm(dim=1)[live] / Bref.norm(dim=1)[live]).max().item())
        # the tensor-core multiply alone (panels of 128, BF16), tree order
        Xb = Eb[:128].clone()
        Yb = torch.empty_like(Xb)
        for _ in range(3):
            vf.vf_apply_tree(prob.hmat, Xb, Yb, precision="bf16")
        torch.cuda.synchronize()
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        m0.record(st)
        for _ in range(20):
            vf.vf_apply_tree(prob.hmat, Xb, Yb, precision="bf16")
        m1.record(st)
        torch.cuda.synchronize()
        tms = m0.elapsed_time(m1) / 20
        bf16_bytes = vf.vf_hmat_bytes(prob.hmat, "bf16") + n * 128 * (2 + 4)
        tpages = vf.vf_hmat_tensor_bytes(prob.hmat, 1)
        single_apply = 1.0 / (mult_ms / 1000.0)  # FP32 single-RHS multiply, RHS/s
        batched = {"value": round(Rb / (bms / 1000.0), 1), "unit": "RHS/s", "rhs": Rb, "ms_per_solve": round(bms, 3),
                   "suns": "lunar-day azimuth sweep at 1.5 deg elevation",
                   "precision": "bf16 factors and RHS on tcgen05 tensor cores, FP32 accumulation; "
                                "split-BF16 residual refinement with FP64 update",
                   "autotuned": dict(tune, seconds=round(t_tune, 2)), "rhs_per_s_by_rhs_block": blocks,
                   "rtol": 1e-4, "sweeps": sb["sweeps"], "refinements": sb["refinements"],
                   "max_rel_diff_vs_fp32_solve": brel,
                   "x_fp32_single_rhs_apply": round(Rb / (bms / 1000.0) / single_apply, 2),
                   "x_fp32_single_rhs_solve": round(Rb / (bms / 1000.0) / (value / world), 2),
                   "tensor_multiply": {"ms": round(tms, 4), "rhs": 128,
                                       "alg_bytes": bf16_bytes,
                                       "hbm_frac": round(bf16_bytes / (tms / 1000.0) / 1e9 / peak, 4),
                                       "page_bytes": tpages,
                                       "page_frac": round((tpages["total"] + n * 128 * 6) / (tms / 1000.0) / 1e9 / peak,
                                                          4)}}
        # the same solve with FP8 sweeps on the tensor cores (kind::f8f6f4)
        # and the same split-BF16 refinement; the FP8 multiply of 128 RHS
        B8 = torch.empty_like(Eb)
        kw8 = dict(rho=rho, rtol=1e-4, precision="fp8", refine=True)
        for _ in range(2):
            s8 = vf.vf_solve(prob.hmat, Eb, B8, **kw8)
        torch.cuda.synchronize()
        ms8 = events_ms(lambda: vf.vf_solve(prob.hmat, Eb, B8, **kw8), 3, st)
        rel8 = float(((B8 - Bref).norm(dim=1)[live] / Bref.norm(dim=1)[live]).max().item())
        for _ in range(3):
            vf.vf_apply_tree(prob.hmat, Xb, Yb, precision="fp8")
        torch.cuda.synchronize()
        tms8 = events_ms(lambda: vf.vf_apply_tree(prob.hmat, Xb, Yb, precision="fp8"), 20, st)
        fp8_bytes = vf.vf_hmat_bytes(prob.hmat, "fp8") + n * 128 * (1 + 4)
        tpages8 = vf.vf_hmat_tensor_bytes(prob.hmat, 3)
        batched["fp8"] = {"value": round(Rb / (ms8 / 1000.0), 1), "unit": "RHS/s", "ms_per_solve": round(ms8, 3),
                          "precision": "fp8 e4m3 factors and RHS on tcgen05 tensor cores (kind::f8f6f4), "
                                       "power-of-two scales per RHS column, row and SVD rank column; "
                                       "split-BF16 residual refinement with FP64 update",
                          "rtol": 1e-4, "sweeps": s8["sweeps"], "refinements": s8["refinements"],
                          "converged": s8["converged"], "max_rel_diff_vs_fp32_solve": rel8,
                          "tensor_multiply": {"ms": round(tms8, 4), "rhs": 128, "alg_bytes": fp8_bytes,
                                              "hbm_frac": round(fp8_bytes / (tms8 / 1000.0) / 1e9 / peak, 4),
                                              "page_bytes": tpages8}}
        batched_host = {"B": Bb.double().cpu().numpy().T, "B8": B8.double().cpu().numpy().T,
                        "dirs": lunar_day_dirs(Rb), "rho": rho}
        del Eb, Bb, Bref, Xb, Yb, B8
        # the autotuner's candidate workspaces and the tensor pages of this
        # section are released before the many-mesh section needs the memory
        vf.vf_hmat_trim(prob.hmat)
        torch.cuda.empty_cache()

    # ---- many meshes in one launch per phase: K seeded fBm terrains (every
    # other one with a crater) of growing size, each with its own suns, one
    # vf_solve_batched on their block-diagonal stack against a loop of
    # per-mesh vf_solve calls
    multimesh = None
    if a.multimesh > 0 and rank == 0:
        import synth
        K = a.multimesh
        # the batching workload's meshes: sides 51 .. max side, seeds 100 + k,
        # a crater of half the domain width on even seeds
        specs = synth.batch_mesh_specs(count=K)
        for sp_ in specs:
            sp_["n"] = int(round(51 + (a.multimesh_max_side - 51) * (sp_["n"] - 51) / 149.0))
        mm0 = time.time()
        ps = []
        for sp_ in specs:
            mv, mf = synth.fbm_dem_mesh(n=sp_["n"], spacing=sp_["spacing"], hurst=sp_["hurst"], seed=sp_["seed"],
                                        rms_slope_deg=15.0, crater_diameter=sp_["crater_diameter"])
            ps.append(vf.build_problem(mv, mf, kind="quad", leaf_size=64, tol=a.tol, device=dev,
                                       precisions=("fp32", "bf16")))
        t_mm_setup = time.time() - mm0
        Rm = a.multimesh_rhs
        Es = []
        for k, p_ in enumerate(ps):
            Ek = torch.empty((Rm, p_.mesh.n), device="cuda", dtype=torch.float32)
            vf.vf_mesh_insolation(p_.mesh, synth.sun_directions(Rm, 5.0 + k % 10, 7.0 * k), 1365.0, Ek)
            Es.append(Ek)
        Bs = [torch.empty_like(e_) for e_ in Es]
        Bl = [torch.empty_like(e_) for e_ in Es]
        mkw = dict(rho=rho, rtol=1e-4, precision="bf16", refine=True)
        hs = [p_.hmat for p_ in ps]
        steps_mm = 5
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        # the loop of per-mesh solves first; then its workspaces and tensor
        # pages are released so the stack's fit beside the meshes' matrices
        for _ in range(2):
            for p_, e_, b_ in zip(ps, Es, Bl):
                vf.vf_solve(p_.hmat, e_, b_, **mkw)
        torch.cuda.synchronize()
        q0.record(st)
        for _ in range(steps_mm):
            for p_, e_, b_ in zip(ps, Es, Bl):
                vf.vf_solve(p_.hmat, e_, b_, **mkw)
        q1.record(st)
        torch.cuda.synchronize()
        loop_ms = q0.elapsed_time(q1) / steps_mm
        for h_ in hs:
            vf.vf_hmat_trim(h_)
        for _ in range(2):
            vf.vf_solve_batched(hs, Es, Bs, **mkw)
        torch.cuda.synchronize()
        q0.record(st)
        for _ in range(steps_mm):
            sm = vf.vf_solve_batched(hs, Es, Bs, **mkw)
        q1.record(st)
        torch.cuda.synchronize()
        bat_ms = q0.elapsed_time(q1) / steps_mm
        diff = 0.0
        for b_, l_ in zip(Bs, Bl):
            live = l_.norm(dim=1) > 0
            diff = max(diff, float(((b_ - l_).norm(dim=1)[live] / l_.norm(dim=1)[live]).max().item()))
        facets = [p_.mesh.n for p_ in ps]
        multimesh = {"value": round(K * Rm / (bat_ms / 1000.0), 1), "unit": "RHS/s", "meshes": K,
                     "facets_min_max_total": [min(facets), max(facets), sum(facets)], "rhs_per_mesh": Rm,
                     "ms_per_batched_solve": round(bat_ms, 3), "ms_per_loop_of_solves": round(loop_ms, 3),
                     "x_vs_loop": round(loop_ms / bat_ms, 2), "max_rel_diff_vs_loop": diff,
                     "sweeps": sm[0]["sweeps"], "refinements": sm[0]["refinements"],
                     "converged": all(x["converged"] for x in sm), "setup_s": round(t_mm_setup, 1),
                     "precision": "bf16 tensor-core sweeps + split-BF16 refinement, rtol 1e-4"}
        del ps, Es, Bs, Bl, hs
        import gc
        gc.collect()
        torch.cuda.empty_cache()

    # ---- the uncompressed dense FP32 F on the same GPU
    dense = None
    if not a.no_dense and rank == 0:
        hd, _ = vf.vf_assemble(prob.mesh, prob.tree, storage="dense", precisions=("fp32",))
        Bd = torch.empty_like(E)
        for _ in range(2):
            vf.vf_solve(hd, E, Bd, rho=rho, rtol=rtol)
        torch.cuda.synchronize()
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        dsteps = max(3, a.steps // 4)
        d0.record(st)
        for _ in range(dsteps):
            sd = vf.vf_solve(hd, E, Bd, rho=rho, rtol=rtol)
        d1.record(st)
        torch.cuda.synchronize()
        dms = d0.elapsed_time(d1) / dsteps
        rel = float(((B - Bd).norm() / Bd.norm()).item())
        dense = {"value": R / (dms / 1000.0), "unit": "RHS/s", "ms_per_step": round(dms, 3),
                 "bytes": vf.vf_hmat_bytes(hd, "fp32"), "sweeps": sd["sweeps"],
                 "compressed_vs_dense_rel_err": rel, "speedup_compressed": round(value / world / (R / (dms / 1e3)), 2)}
        del hd
    # ---- the terrain at tol 1e-2 and 1e-4 (the headline is tol 1e-3): the
    # same single-RHS FP32 solve, its multiply's roofline and its error
    # against the uncompressed dense FP32 F's solve
    tol_sweep = None
    if not a.no_tol_sweep and rank == 0 and a.tol == 1e-3:
        tol_sweep = {"1e-3": {"value": round(value / world, 3), "ms_per_step": round(ms, 4),
                              "bytes_fp32": vf.vf_hmat_bytes(prob.hmat, "fp32"), "roofline_frac": roofline["frac"],
                              "rel_err_vs_dense_fp32": dense["compressed_vs_dense_rel_err"] if dense else None}}
        for tt in (1e-2, 1e-4):
            t_a = time.time()
            pt = vf.build_problem(v, f, kind="quad", leaf_size=64, tol=tt, device=dev, precisions=("fp32",))
            t_a = time.time() - t_a
            Bt_ = torch.empty_like(E)
            for _ in range(3):
                vf.vf_solve(pt.hmat, E, Bt_, rho=rho, rtol=rtol)
            tms_ = events_ms(lambda: vf.vf_solve(pt.hmat, E, Bt_, rho=rho, rtol=rtol), max(20, a.steps), st)
            Xt_ = E.clone()
            Yt_ = torch.empty_like(Xt_)
            for _ in range(3):
                vf.vf_apply_tree(pt.hmat, Xt_, Yt_)
            mms_ = events_ms(lambda: vf.vf_apply_tree(pt.hmat, Xt_, Yt_), 50, st)
            ab_ = vf.vf_hmat_bytes(pt.hmat, "fp32") + n * R * 8
            tol_sweep[f"{tt:.0e}"] = {
                "value": round(R / (tms_ / 1e3), 3), "ms_per_step": round(tms_, 4), "assembly_s": round(t_a, 1),
                "bytes_fp32": vf.vf_hmat_bytes(pt.hmat, "fp32"),
                "roofline_frac": round(ab_ / (mms_ / 1e3) / 1e9 / peak, 4),
                "rel_err_vs_dense_fp32": float(((Bt_ - Bd).norm() / Bd.norm()).item()) if dense else None}
            del pt, Bt_, Xt_, Yt_

    # ---- the 522,242-facet precision workload (after the terrain's buffers are freed)
    setup_info = {"workload": WORKLOAD if a.dem_size == 200 else f"fbm{a.dem_size}_crater_{n}tri", "facets": n,
                  "l2": "inputs larger than L2 (compressed F %.0f MB)" % (vf.vf_hmat_bytes(prob.hmat, a.precision) / 1e6),
                  "assembly": {k: prob.stats[k] for k in ("nblocks", "bytes", "probes", "max_rank", "t_visibility",
                                                          "t_probe", "t_total")}}
    config4 = None
    c4_host = None
    if not a.no_config4 and rank == 0 and world == 1:
        import gc
        del prob, E, B, Xt, Yt
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        config4, c4_host = run_config4(a, dev, peak, st)
        gc.collect()
        torch.cuda.empty_cache()

    # ---- the CPU baseline leg: the oracle timed on a bounded sample of the
    # terrain's rows; the same sampled oracle rows state the batched solve's
    # error, and the precision workload's oracle rows its errors
    cpu = None
    if not a.no_cpu and rank == 0 and world == 1:
        co = CpuOracle(v, f, dirs, a.cpu_rows, R)
        cpu = co.measure(sweeps, seconds=10.0)
        if batched_host is not None:
            batched["oracle_check"] = co.batched_check(v, f, batched_host)
            batched["fp8"]["oracle_check"] = co.batched_check(v, f, dict(batched_host, B=batched_host["B8"]))
        if c4_host is not None:
            config4["oracle_check"] = config4_oracle_check(c4_host, a.config4_rows)
            chk = config4["oracle_check"]
            config4["err_vs_oracle"] = chk["solve_bf16_refined_rel_err"]
            config4["meets_1e-3"] = bool(chk["solve_bf16_refined_rel_err"] <= 1e-3)

    line = {"metric": METRIC, "value": round(value, 3), "unit": "RHS/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "fp8e4m3"}[a.precision],
            "data": "synthetic",
            "config": {"workload": setup_info["workload"], "facets": n, "rhs_per_gpu": R, "tol": a.tol, "rho": rho,
                       "rtol": rtol, "sweeps": sweeps, "l2": setup_info["l2"],
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "setup_s": round(t_setup, 2)},
            "roofline": roofline, "e2e": e2e, "gpu_launches": kernels, "clocks": clk, "steady": steady,
            "batched": batched, "multimesh": multimesh, "dense_fp32": dense, "tol_sweep": tol_sweep,
            "config4": config4,
            "cpu_baseline": cpu, "assembly": setup_info["assembly"]}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
