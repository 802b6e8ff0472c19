"""Benchmark of the hot path: per-frequency boundary-regularised BIE solves followed by the field
evaluation and Fourier synthesis of the space-time scattered field.

Workload (one step): two sound-hard unit spheres, 720 quadratic elements / 1442 nodes each
(N = 2884), surface gap 0.1, incident Gaussian plane-wave pulse along the axis; 512 wavenumbers
k_m = m/32 (ka in (0, 16]) solved in mixed precision (FP32 assembly with float-float phases,
tcgen05 TF32 LU, float-float iterative refinement, FP64 re-solve of flagged wavenumbers), field on
a 128 x 128 grid of the plane z = 0 over [-5, 5]^2, synthesis of 1024 time samples.

Metric: frequency solves per second of the whole path (each solve carries its share of the field
evaluation and synthesis), with space-time points per second and the per-phase times alongside.
Accuracy gate (after the timed steps): every one of the 512 surface solutions is compared with a
solution of the FP64-accurate system (each wavenumber re-assembled with float-float bulk pairs and
FP64 near pairs, refined with FP64 residuals to a backward error of 1e-13), one wavenumber with the
CPU oracle's direct solve, and a few with the plain FP64 GPU path; a solve whose relative L2 error
exceeds 1e-6 is not counted in `value`.  Rooflines divide by rates measured in the same run
(bie_measure_peaks: FP32 FMA for the field kernel, tcgen05 TF32 for the LU).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BEM freq solves/s & space-time pts/s at rel err <=1e-6 vs FP64; roofline frac"
UNIT = "freq_solves/s"
TOL = 1e-6  # relative L2 error of a counted solve against the FP64-accurate system


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_workload():
    from workloads import config_two_spheres_mixed
    return config_two_spheres_mixed()


def bench_config(w, args, world: int) -> dict:
    """The workload description, identical in both arms."""
    return {"workload": "two_spheres_N2884_Nk512_M16384_Nt1024", "N": int(w.mesh.N), "E": int(w.mesh.E),
            "Nk": len(w.k), "ka_max": float(w.k[-1]), "M": int(w.xobs.shape[0]), "Nt": w.Nt,
            "pulses": int(w.pulses.shape[0]), "parallelism": f"{world} independent replica(s), one per GPU",
            "l2": f"working set ({args.batch} x 133 MB systems per batch) larger than L2; no flush needed",
            "mixed_batch": args.batch}


class RankGroup:
    """One process per GPU, launched by torchrun (RANK, WORLD_SIZE, LOCAL_RANK, MASTER_* from the
    environment).  The frequency sweep shards into independent replicas, so there is no
    data-path collective: the group only brackets the timed region with barriers, takes the
    maximum of the ranks' times, and lets rank 0 report."""

    def __init__(self, backend: str = "nccl", device=None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": device} if backend == "nccl" and device is not None else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    @property
    def is_root(self) -> bool:
        return self.rank == 0

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, x: float, device=None) -> float:
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=device if self.backend == "nccl" else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def job_throughput(units_per_rank_step: int, world: int, steps: int, t_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank_step * world * steps / (t_ms / 1e3)


# ----------------------------------------------------------------------------- GPU arm ----
def run_ours(args):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    grp = RankGroup("nccl", dev)
    rank, world = grp.rank, grp.world

    import __graft_entry__

    __graft_entry__.build()
    from paper_1706_07919_gb300 import Solver
    from paper_1706_07919_gb300 import binding as B

    w = build_workload()
    Nk, M, Nt, P = len(w.k), w.xobs.shape[0], w.Nt, w.pulses.shape[0]
    peaks = B.bie_measure_peaks(local)  # pipe rates of this GPU (roofline denominators)
    stream = torch.cuda.Stream(dev)
    sol = Solver(local, stream)
    sol.set_geometry(w.mesh.nodes, w.mesh.elems, w.mesh.normals, w.mesh.bc)
    sol.set_incident_plane_wave(w.direction)
    sol.set_option("mixed.tcgen05", args.tc)
    sol.set_option("mixed.lu_block", args.lu_block)
    sol.set_option("mixed.lu_panel", args.lu_panel)
    sol.set_option("mixed.lu_tile", args.lu_tile)
    sol.set_option("mixed.asm_kb", args.asm_kb)
    sol.set_option("field.variant", args.field_variant)
    sol.set_option("mixed.batch", args.batch)
    midx = np.arange(1, Nk + 1, dtype=np.int64)

    with torch.cuda.stream(stream):
        xo = torch.tensor(w.xobs, dtype=torch.float64, device=dev)
        pulses = torch.tensor(w.pulses, dtype=torch.float64, device=dev)
        surf = torch.empty((Nk, 2, w.mesh.N), dtype=torch.complex128, device=dev)
        T = torch.empty((Nk, M), dtype=torch.complex128, device=dev)
        S = torch.empty((P, Nt // 2 + 1), dtype=torch.complex128, device=dev)
        out = torch.empty((P, M, Nt), dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    reports = {}

    def step(record=False):
        if record:
            ev[0].record(stream)
        reports["rep"] = sol.solve_frequencies(w.k, B.BIE_MODE_MIXED, out=surf)[1]
        if record:
            ev[1].record(stream)
        sol.eval_field(xo, w.k, surf, B.BIE_MODE_MIXED, out=T)
        if record:
            ev[2].record(stream)
        sol.pulse_spectrum(pulses, out=S)
        sol.synthesize(T, midx, S, Nt, torch.float32, out=out)
        if record:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    phase = np.zeros(3)
    grp.barrier()
    torch.cuda.synchronize(dev)
    launches0 = B.bie_kernel_launches()
    with ClockSampler(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(record=True)
            torch.cuda.synchronize(dev)
            phase += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])]
        t1.record(stream)
        torch.cuda.synchronize(dev)
        grp.barrier()
    t_ms = grp.max_over_ranks(t0.elapsed_time(t1), dev)
    launches = B.bie_kernel_launches() - launches0
    rep = reports["rep"]

    # ---- accuracy gate (outside the timed region) ----
    # (1) every wavenumber against the solution of the FP64-accurate system: re-assembly with
    #     float-float bulk pairs and FP64 near pairs, refinement with FP64 residuals to 1e-13
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sol.set_option("mixed.fallback_err_est", 1e-30)
    g0.record(stream)
    ref, rep_ref = sol.solve_frequencies(w.k, B.BIE_MODE_MIXED)
    g1.record(stream)
    torch.cuda.synchronize(dev)
    sol.set_option("mixed.fallback_err_est", 3e-7)  # back to the default
    err_all = (torch.linalg.norm((surf - ref).reshape(Nk, -1), dim=1) /
               torch.linalg.norm(ref.reshape(Nk, -1), dim=1)).cpu().numpy()
    ref_berr = max(r.backward_err for r in rep_ref)
    del ref
    n_over = int((err_all > TOL).sum())
    # (2) the plain FP64 GPU path (FP64 assembly and LU) on sampled wavenumbers
    rng = np.random.Generator(np.random.PCG64(2001))
    sample = np.sort(rng.choice(Nk, size=args.check, replace=False))
    ks = w.k[sample]
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    s64, _ = sol.solve_frequencies(ks, B.BIE_MODE_FP64)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    fp64_solves_per_s = len(ks) / (f0.elapsed_time(f1) / 1e3)
    errs = [(torch.linalg.norm(surf[i] - s64[j]) / torch.linalg.norm(s64[j])).item() for j, i in enumerate(sample)]
    T64 = sol.eval_field(xo, ks, s64, B.BIE_MODE_FP64)
    ferrs = [(torch.linalg.norm(T[i] - T64[j]) / torch.linalg.norm(T64[j])).item() for j, i in enumerate(sample)]
    del s64, T64

    # ---- phases of one more (untimed) sweep, for the LU's own roofline ----
    sol.set_option("mixed.phase_timing", 1)
    sol.solve_frequencies(w.k, B.BIE_MODE_MIXED)
    phases = B.bie_get_phase_times(sol.ctx)
    sol.set_option("mixed.phase_timing", 0)
    roof_lu = roofline_lu(w, phases, peaks)

    # ---- end to end through the C ABI with host buffers (copies inside the timed region) ----
    e2e = run_e2e(args, w, sol, B, dev, stream)
    solve_rate = Nk * args.steps / (phase[0] / 1e3)

    # ---- roofline of the dominant kernel: the field phase of the timed steps ----
    roof = roofline_field(w, phase[1] / args.steps, M, Nk, args.field_variant, peaks)

    # ---- the CPU oracle on a bounded sample; its surface solution also checks the GPU's ----
    cpu = None
    if grp.is_root and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args, w)
        kk = cpu.pop("k_index")
        Por = cpu.pop("P")
        cpu_err = float(np.linalg.norm(surf[kk, 0].cpu().numpy() - Por) / np.linalg.norm(Por))
    else:
        cpu_err = None

    n_pass = Nk - n_over
    value = job_throughput(n_pass, world, args.steps, t_ms)
    pts = job_throughput(M * Nt * P, world, args.steps, t_ms)
    nfall = sum(1 for r in rep if r.flags & B.BIE_FLAG_FALLBACK_FP64)
    nre64 = sum(1 for r in rep if r.flags & B.BIE_FLAG_FP64_ASSEMBLY)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded meshes/points/pulse)",
        "config": bench_config(w, args, world),
        "space_time_pts_per_s": pts,
        "phase_ms_per_step": {"solve": phase[0] / args.steps, "field": phase[1] / args.steps,
                              "spectrum_synthesis": phase[2] / args.steps},
        "accuracy": {"tolerance": TOL, "solves_counted": n_pass, "solves_over_tolerance": n_over,
                     "max_rel_err_vs_fp64_system_all_k": float(err_all.max()),
                     "median_rel_err_vs_fp64_system": float(np.median(err_all)),
                     "fp64_system_reference": "all 512 wavenumbers re-assembled (float-float bulk, FP64 near "
                                              "pairs) and refined with FP64 residuals",
                     "fp64_system_max_backward_err": ref_berr,
                     "fp64_system_ms": g0.elapsed_time(g1),
                     "max_rel_err_vs_oracle": cpu_err,
                     "oracle_k": float(w.k[kk]) if cpu is not None else None,
                     "sampled_k": [float(x) for x in ks], "max_rel_err_surface_vs_fp64_path": max(errs),
                     "max_rel_err_field_vs_fp64_path": max(ferrs), "fp64_reassembled": nre64,
                     "fp64_full_solves": nfall, "max_refine_iters": max(r.iters for r in rep)},
        "fp64_path": {"solves_per_s": fp64_solves_per_s, "sample": f"{len(ks)} wavenumbers, same N",
                      "mixed_solve_phase_speedup": solve_rate / fp64_solves_per_s},
        "clocks": clk.summary(),
        "e2e": e2e,
        "roofline": roof,
        "roofline_lu": roof_lu,
        "peaks_measured": peaks,
        "gpu_launches": int(launches),
    }
    sol.close()
    if not args.no_learned:
        line["learned"] = run_learned(args, dev, stream)
    if not args.no_uneven:
        line["uneven"] = run_uneven(args, dev)
    if not args.no_large:
        line["large"] = run_large(args, dev, stream, peaks)
    if not args.no_paper:
        line["paper"] = run_paper(args, dev, stream)
    if grp.is_root:
        line["cpu_baseline"] = cpu
        print(json.dumps(line))
    grp.close()


def run_learned(args, dev, stream):
    """The learned-warm-start sweep (BIE_MODE_LEARNED) on the spheroid workload: hard prolate
    spheroid (1, 1, 2), N = 2562, 1024 wavenumbers over ka in (0, 20]; every 8th solved directly,
    the network trained on those, the rest by GMRES from its prediction.  Timed next to the
    mixed direct path on the same wavenumbers and to GMRES from a zero start; accuracy on sampled
    GMRES-solved wavenumbers against the FP64 GPU path."""
    import torch

    from workloads import config_spheroid_learned
    from paper_1706_07919_gb300 import Solver
    from paper_1706_07919_gb300 import binding as B

    w = config_spheroid_learned()
    Nk = len(w.k)
    sol = Solver(dev.index if dev.index is not None else 0, stream)
    sol.set_geometry(w.mesh.nodes, w.mesh.elems, w.mesh.normals, w.mesh.bc)
    sol.set_incident_plane_wave(w.direction)
    sol.set_option("mixed.batch", args.batch)
    sol.set_option("learned.epochs", args.epochs)
    with torch.cuda.stream(stream):
        surf = torch.empty((Nk, 2, w.mesh.N), dtype=torch.complex128, device=dev)
        surf_d = torch.empty_like(surf)

    def timed(mode, out):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        _, rep = sol.solve_frequencies(w.k, mode, out=out)
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t, rep

    sol.solve_frequencies(w.k[:64], B.BIE_MODE_LEARNED)  # warm-up (module load, graph paths)
    t_l, rep_l = timed(B.BIE_MODE_LEARNED, surf)
    info = sol.learned_info()
    t_d, _ = timed(B.BIE_MODE_MIXED, surf_d)
    starts = {}
    for code, name in ((0, "zero"), (2, "nearest_anchor"), (3, "anchor_interpolant")):
        sol.set_option("learned.x0", code)
        t_s, _ = timed(B.BIE_MODE_LEARNED, surf_d)
        inf = sol.learned_info()
        starts[name] = {"solves_per_s": Nk / t_s, "mean_arnoldi_steps": inf["mean_iters"],
                        "x0_rel_err": inf["x0_rel_err"], "krylov_fallback": inf["krylov_fallback"]}
    starts["network"] = {"solves_per_s": Nk / t_l, "mean_arnoldi_steps": info["mean_iters"],
                         "x0_rel_err": info["x0_rel_err"], "krylov_fallback": info["krylov_fallback"]}
    t_z = Nk / starts["zero"]["solves_per_s"]
    info_z = {"mean_iters": starts["zero"]["mean_arnoldi_steps"], "krylov_fallback": starts["zero"]["krylov_fallback"]}
    sol.set_option("learned.x0", 1)
    # accuracy: sampled wavenumbers that GMRES solved, against the FP64 path
    rng = np.random.Generator(np.random.PCG64(3002))
    gm = [i for i, r in enumerate(rep_l) if r.path == B.BIE_MODE_LEARNED]
    sample = np.sort(rng.choice(gm, size=min(args.check, len(gm)), replace=False)) if gm else np.array([], int)
    errs = []
    if len(sample):
        s64, _ = sol.solve_frequencies(w.k[sample], B.BIE_MODE_FP64)
        errs = [(torch.linalg.norm(surf[i] - s64[j]) / torch.linalg.norm(s64[j])).item()
                for j, i in enumerate(sample)]
    sol.close()
    return {"workload": "spheroid_1_1_2_N2562_Nk1024_ka20", "solves_per_s": Nk / t_l,
            "mixed_direct_solves_per_s": Nk / t_d, "zero_start_solves_per_s": Nk / t_z,
            "anchors": info["anchors"], "krylov": info["krylov"], "krylov_fallback": info["krylov_fallback"],
            "epochs": info["epochs"], "train_ms": info["train_ms"], "first_loss": info["first_loss"],
            "last_loss": info["last_loss"], "x0_rel_err": info["x0_rel_err"], "mean_arnoldi_steps": info["mean_iters"],
            "max_arnoldi_steps": info["max_iters"],
            "phase_ms": {name: info[name] for name in ("anchors_ms", "train_ms", "assembly_ms", "predict_ms",
                                                       "gmres_ms", "estimate_ms", "redo_ms")},
            "zero_start_mean_arnoldi_steps": info_z["mean_iters"],
            "zero_start_krylov_fallback": info_z["krylov_fallback"],
            "starts": starts,
            "sampled_k": [float(w.k[i]) for i in sample], "max_rel_err_surface_vs_fp64": max(errs) if errs else None,
            "timing": "wall clock around each synchronising call (host-side setup included)"}


def run_paper(args, dev, stream):
    """The paper's own experiments (Sec. 4) on the device: (1) the 1002-node soft sphere with the
    pulse of Eq. (pulse) (2N_c = 4, alpha = 0.1, w = 20.1a), 64 frequencies, the field at the two
    points of Table I and the 80 x 80 snapshot grid, synthesised from all frequencies and from the
    5, 10, 20 dominant ones (chosen on the device): Table I's RMS errors; (2) eight incident
    directions on the same sphere sharing each wavenumber's factor, against eight separate sweeps;
    (3) the peak total-field amplification of the two hard spheres 3a apart and of the tilted hard
    bowl.  Wall clock around synchronising calls."""
    import torch

    from workloads import config_paper_sphere, config_paper_two_spheres, config_paper_bowl
    from paper_1706_07919_gb300 import Solver
    from paper_1706_07919_gb300 import binding as B

    out = {}
    w = config_paper_sphere(bc=1)
    sol = Solver(dev.index if dev.index is not None else 0, stream)
    sol.set_geometry(w.mesh.nodes, w.mesh.elems, w.mesh.normals, w.mesh.bc)
    sol.set_incident_plane_wave(w.direction)
    xo = torch.tensor(w.xobs, dtype=torch.float64, device=dev)
    pulses = torch.tensor(w.pulses, dtype=torch.float64, device=dev)
    sol.solve_frequencies(w.k[:8], B.BIE_MODE_MIXED)  # warm-up
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    surf, _ = sol.solve_frequencies(w.k, B.BIE_MODE_MIXED)
    T = sol.eval_field(xo, w.k, surf, B.BIE_MODE_MIXED)
    S = sol.pulse_spectrum(pulses)
    m_all = np.arange(len(w.k))
    p_all = sol.synthesize(T, m_all, S, w.Nt)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t
    pall = p_all[0, :2].cpu().numpy()
    rms = {}
    for K in (5, 10, 20):
        sel = sol.top_frequencies(S, w.Nt, K)
        pK = sol.synthesize(T[torch.tensor(sel, device=dev)].contiguous(), sel, S, w.Nt)[0, :2].cpu().numpy()
        r = 100.0 * np.sqrt(((pK - pall) ** 2).mean(axis=-1)) / np.abs(pall).max(axis=-1)
        rms[str(K)] = [float(r[0]), float(r[1])]
    out["sphere_table1"] = {"workload": "soft sphere N1002, Eq. pulse 2Nc=4 alpha=0.1 w=20.1, 64 k, 6350 points x 128 steps",
                            "rms_percent_at_-1.1a_-4a": rms, "printed": {"5": [4.4, 4.9], "10": [1.6, 1.7], "20": [0.5, 0.6]},
                            "solves_per_s": len(w.k) / dt,
                            "space_time_pts_per_s": w.xobs.shape[0] * w.Nt / dt}
    # several incident directions sharing each factor
    rng = np.random.Generator(np.random.PCG64(6001))
    dirs = rng.standard_normal((8, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    sm, _ = sol.solve_frequencies_multi(w.k, dirs, B.BIE_MODE_MIXED)
    torch.cuda.synchronize(dev)
    t_multi = time.perf_counter() - t
    t = time.perf_counter()
    errs = []
    for d in range(len(dirs)):
        sol.set_incident_plane_wave(dirs[d])
        s1, _ = sol.solve_frequencies(w.k, B.BIE_MODE_MIXED)
        errs.append((torch.linalg.norm(s1 - sm[:, d]) / torch.linalg.norm(s1)).item())
    torch.cuda.synchronize(dev)
    t_sep = time.perf_counter() - t
    sol.close()
    out["directions"] = {"workload": "soft sphere N1002, 64 k x 8 seeded directions", "solves_per_s": 64 * 8 / t_multi,
                         "separate_sweeps_solves_per_s": 64 * 8 / t_sep, "speedup": t_sep / t_multi,
                         "max_rel_diff_vs_separate": max(errs)}
    # amplification of the total field
    for name, w2, paper in (("two_spheres_3a", config_paper_two_spheres(), 1.8), ("bowl", config_paper_bowl(), 4.5)):
        s2 = Solver(dev.index if dev.index is not None else 0, stream)
        s2.set_geometry(w2.mesh.nodes, w2.mesh.elems, w2.mesh.normals, w2.mesh.bc)
        s2.set_incident_plane_wave(w2.direction)
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        surf2, _ = s2.solve_frequencies(w2.k, B.BIE_MODE_MIXED)
        xo2 = torch.tensor(w2.xobs, dtype=torch.float64, device=dev)
        T2 = s2.eval_field(xo2, w2.k, surf2, B.BIE_MODE_MIXED)
        inc = torch.tensor(np.exp(1j * np.outer(w2.k, w2.xobs @ w2.direction)), device=dev)
        S2 = s2.pulse_spectrum(torch.tensor(w2.pulses, device=dev))
        m2 = np.arange(len(w2.k))
        ptot = s2.synthesize((T2 + inc).contiguous(), m2, S2, w2.Nt)
        pinc = s2.synthesize(inc.contiguous(), m2, S2, w2.Nt)
        ratio = (ptot.abs().max() / pinc.abs().max()).item()
        torch.cuda.synchronize(dev)
        out[name] = {"N": int(w2.mesh.N), "points": int(w2.xobs.shape[0]), "peak_total_over_incident": ratio,
                     "paper": paper, "seconds": time.perf_counter() - t}
        s2.close()
    return out


def run_large(args, dev, stream, peaks=None):
    """The lattice workload (4 x 4 x 2 sound-soft spheres, N = 20 544) on a bounded sample: the
    zero-frequency term k = 0 (soft bodies scatter at k = 0, and the Gaussian pulse has a non-zero
    mean) plus `--large-nk` consecutive wavenumbers from the middle of the sweep -- by default 17,
    so that the sample is one batch of 18 systems, the batch the full 2048-wavenumber sweep is cut
    into on this GPU's memory -- solved in mixed precision, their field on the full 256 x 256 plane
    and the synthesis of the eight pulses at 4096 samples.  CUDA events on the library's stream
    around each phase."""
    import torch

    from workloads import config_lattice_large
    from paper_1706_07919_gb300 import Solver
    from paper_1706_07919_gb300 import binding as B

    w = config_lattice_large()
    nk = args.large_nk
    i0 = len(w.k) // 2 - nk // 2
    idx = np.arange(i0, i0 + nk, dtype=np.int64)
    ks = np.concatenate([[0.0], w.k[idx]])
    midx = np.concatenate([[0], idx + 1])  # frequency index m of each wavenumber (k_m = m dk), m = 0 first
    M, Nt, P = w.xobs.shape[0], w.Nt, w.pulses.shape[0]
    sol = Solver(dev.index if dev.index is not None else 0, stream)
    sol.set_geometry(w.mesh.nodes, w.mesh.elems, w.mesh.normals, w.mesh.bc)
    sol.set_incident_plane_wave(w.direction)
    with torch.cuda.stream(stream):
        xo = torch.tensor(w.xobs, dtype=torch.float64, device=dev)
        pulses = torch.tensor(w.pulses, dtype=torch.float64, device=dev)
        out = torch.empty((P, M, Nt), dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    sol.set_option("mixed.phase_timing", 1)  # one batch: no graph replay to lose
    l0 = B.bie_kernel_launches()
    ev[0].record(stream)
    surf, rep = sol.solve_frequencies(ks, B.BIE_MODE_MIXED)
    ev[1].record(stream)
    solve_launches = B.bie_kernel_launches() - l0
    ph = B.bie_get_phase_times(sol.ctx)
    T = sol.eval_field(xo, ks, surf, B.BIE_MODE_MIXED)
    ev[2].record(stream)
    S = sol.pulse_spectrum(pulses)
    sol.synthesize(T, midx, S, Nt, torch.float32, out=out)
    ev[3].record(stream)
    torch.cuda.synchronize(dev)
    t_solve, t_field, t_syn = (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]))
    sol.close()
    return {"workload": "lattice_4x4x2_soft_N20544", "N": int(w.mesh.N), "wavenumbers": len(ks),
            "k": [float(x) for x in ks], "solves_per_s": len(ks) / (t_solve / 1e3),
            "field_evals_per_s": M * w.mesh.E * 16 * len(ks) / (t_field / 1e3), "points": M, "pulses": P, "Nt": Nt,
            "phase_ms": {"solve": t_solve, "field": t_field, "spectrum_synthesis": t_syn},
            "batches": ph["batches"], "systems_per_batch": ph["systems"] / max(1, ph["batches"]),
            "fp64_reassembled": sum(1 for r in rep if r.flags & B.BIE_FLAG_FP64_ASSEMBLY),
            "max_backward_err": max(r.backward_err for r in rep),
            "solve_phase_ms": {k_: ph[k_] for k_ in ("assembly_ms", "factor_ms", "refine_ms", "reassembly_ms")},
            "lu_tflops": ph["systems"] * (8.0 / 3.0) * float(w.mesh.N) ** 3 / (ph["factor_ms"] * 1e-3) / 1e12,
            "roofline_lu": None if not peaks else {
                "bound": "tensor", "unit": "TFLOP/s", "peak": peaks["tf32_tflops"],
                "achieved": ph["systems"] * (8.0 / 3.0) * float(w.mesh.N) ** 3 / (ph["factor_ms"] * 1e-3) / 1e12,
                "frac": ph["systems"] * (8.0 / 3.0) * float(w.mesh.N) ** 3 / (ph["factor_ms"] * 1e-3) / 1e12
                        / peaks["tf32_tflops"],
                "note": "(8/3) N^3 per system over the factorisation phase (CUDA events), blocked LU with "
                        "cooperative panels, against the tcgen05 TF32 rate measured in the same run"},
            "solve_kernel_launches": int(solve_launches)}


def run_uneven(args, dev):
    """The uneven batch (64 seeded configurations of 1-8 spheres and ellipsoids, N 162 .. 7976)
    through the scheduler: a bounded sample of `--uneven-nk` wavenumbers over (0, 8] per
    configuration (the full workload has 256), run with 4 workers (one context and stream each,
    largest job first) and with 1 worker; wall clock around each synchronising run."""
    import torch

    from workloads import uneven_configuration
    from paper_1706_07919_gb300 import binding as B

    nk = args.uneven_nk
    k = (8.0 / nk) * np.arange(1, nk + 1, dtype=np.float64)
    meshes = [uneven_configuration(i)[0] for i in range(64)]
    outs = [torch.empty((nk, 2, m.N), dtype=torch.complex128, device=dev) for m in meshes]
    res = {}
    for workers in (args.uneven_workers, 1):
        sched = B.bie_sched_create(dev.index if dev.index is not None else 0, workers, None)
        jobs = [B.bie_sched_add(sched, m.nodes, m.elems, m.normals, m.bc, [0.0, 0.0, 1.0], k, B.BIE_MODE_MIXED, o)
                for m, o in zip(meshes, outs)]
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        st = B.bie_sched_run(sched)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t
        B.bie_sched_destroy(sched)
        res[workers] = (dt, st, jobs)
    dt4, st4, jobs4 = res[args.uneven_workers]
    flagged = sum(1 for j in jobs4 for r in j.reports() if r.flags & B.BIE_FLAG_FP64_ASSEMBLY)
    worst = max(r.backward_err for j in jobs4 for r in j.reports())
    Ns = [m.N for m in meshes]
    return {"workload": "uneven_64_configs_N162_to_7976", "wavenumbers_per_config": nk,
            "solves": 64 * nk, "solves_per_s": 64 * nk / dt4, "solves_per_s_one_worker": 64 * nk / res[1][0],
            "workers": args.uneven_workers, "wall_s": dt4, "busy_s": st4["busy_ms"] / 1e3, "sum_N": int(sum(Ns)),
            "max_N": int(max(Ns)), "fp64_reassembled": flagged, "max_backward_err": worst,
            "timing": "wall clock around bie_sched_run (mesh set-up of every job included)"}


def run_e2e(args, w, sol, B, dev, stream):
    """Same step through the public API with host buffers: host->device copies of the step's inputs
    (wavenumber list travels as a host argument; observation points and pulse samples from pinned
    host memory) and device->host copies of the surface solutions and the space-time field."""
    import torch

    Nk, M, Nt, P = len(w.k), w.xobs.shape[0], w.Nt, w.pulses.shape[0]
    hx = torch.tensor(w.xobs, dtype=torch.float64).pin_memory()
    hp = torch.tensor(w.pulses, dtype=torch.float64).pin_memory()
    hsurf = torch.empty((Nk, 2, w.mesh.N), dtype=torch.complex128).pin_memory()
    hout = torch.empty((P, M, Nt), dtype=torch.float32).pin_memory()
    midx = np.arange(1, Nk + 1, dtype=np.int64)
    steps = max(1, min(args.steps, 2))

    def one():
        with torch.cuda.stream(stream):
            xo = hx.to(dev, non_blocking=True)
            pl = hp.to(dev, non_blocking=True)
        surf, _ = sol.solve_frequencies(w.k, B.BIE_MODE_MIXED)
        T = sol.eval_field(xo, w.k, surf, B.BIE_MODE_MIXED)
        S = sol.pulse_spectrum(pl)
        o = sol.synthesize(T, midx, S, Nt, torch.float32)
        with torch.cuda.stream(stream):
            hsurf.copy_(surf, non_blocking=True)
            hout.copy_(o, non_blocking=True)
        stream.synchronize()

    one()
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    for _ in range(steps):
        one()
    dt = time.perf_counter() - t
    return {"value": Nk * steps / dt, "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": int(hx.numel() * 8 + hp.numel() * 8 + Nk * 8),
            "d2h_bytes_per_step": int(hsurf.numel() * 16 + hout.numel() * 4)}


def roofline_field(w, field_ms, M, Nk, variant, peaks):
    """The dominant kernel of the step is the field evaluation (Eq. BRIEFdmn), FP32-ALU-bound:
    algorithmic flops per (point, quadrature point, k) x evaluations / the field phase's device time
    in the timed steps (CUDA events on the library's stream; the phase also holds the foot-point
    projection and the interpolation to quadrature points, about 1 % of it), against the FP32 FMA
    rate measured in the same run (bie_measure_peaks)."""
    EQ = w.mesh.E * 16
    evals = M * EQ * Nk
    flops_per_eval = FIELD_FLOPS_PER_EVAL
    achieved = flops_per_eval * evals / (field_ms * 1e-3) / 1e12
    peak = peaks["ffma_tflops"]
    launches = (Nk + FIELD_BATCH - 1) // FIELD_BATCH
    name = {1: "k_field32c<16,64,4,64>", 2: "k_field32c<16,128,3,32>"}.get(variant, "k_field32b")
    return {"kernel": name + " (Eq. BRIEFdmn, float-float phases)", "bound": "alu",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": FIELD_LAUNCH_DRAM_BYTES.get(variant), "traffic_unit": "bytes per launch",
            "evals_per_s": evals / (field_ms * 1e-3), "flops_per_eval": flops_per_eval,
            "launches_per_step": launches, "ms_per_launch": field_ms / launches,
            "peak_source": f"measured in this run: FP32 FMA micro-benchmark on {peaks['sm_count']} SMs "
                           "(bie_measure_peaks)"}


def roofline_lu(w, phases, peaks):
    """The blocked LU of the mixed path (panels, row swaps, U-block solves and tcgen05 trailing
    updates): useful flops (8/3) N^3 per wavenumber (complex LU) over the factorisation phase's
    device time in one untimed sweep of the 512 wavenumbers with phase timing on (CUDA events
    around the factorisation of each batch), against the tcgen05 TF32 rate measured in the same
    run (bie_measure_peaks)."""
    N = w.mesh.N
    flops = phases["systems"] * (8.0 / 3.0) * float(N) ** 3
    t = phases["factor_ms"] * 1e-3
    achieved = flops / t / 1e12 if t > 0 else None
    peak = peaks["tf32_tflops"]
    return {"kernel": "blocked complex LU (k_leaf, k_swap_trsm, k_trsm64, tc2::k_update_tc2)", "bound": "tensor",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved and peak else None, "flops_per_system": (8.0 / 3.0) * float(N) ** 3,
            "systems": phases["systems"], "factor_ms": phases["factor_ms"],
            "phase_ms": {k: phases[k] for k in ("assembly_ms", "factor_ms", "refine_ms", "reassembly_ms")},
            "peak_source": "measured in this run: tcgen05.mma kind::tf32 M128 N256 micro-benchmark "
                           "(bie_measure_peaks)"}


# wavenumbers per field launch of the library (bie_eval_field)
FIELD_BATCH = 512

# DRAM bytes (read + write) of one launch of the field kernel in this configuration (512
# wavenumbers x 16 384 points) per kernel variant, from an ncu capture of a launch of exactly
# that shape (`bench.py --case field512`): 221.8 MB read (tables and surface values) and 105.9 MB
# written (the 134 MB field, part of it still in L2 when the launch ends).  Variants without an
# entry have no capture of the current kernel.
FIELD_LAUNCH_DRAM_BYTES = {2: 221_766_912 + 105_931_520}

# algorithmic flops of one field evaluation (one observation point, one quadrature point, one k),
# counted on the FP64 formula: 2 distances (3 sub, 3 mul, 2 add, sqrt, div = 10 each), the
# foot-point projection nu0.r and nu.nu0 (5 each), 3 complex exponentials (sin, cos, 1 mul = 3
# each), G and dG for both sources (2 + 8 each), g, f, dg, df (5), Pt and dPt (16), the integrand
# (2 complex mul + 3 complex sub = 14) and the accumulation (4)
FIELD_FLOPS_PER_EVAL = 10 * 2 + 5 * 2 + 3 * 3 + 10 * 2 + 5 + 16 + 14 + 4


def cpu_baseline(args, w):
    """The CPU FP64 oracle on a bounded sample of the same workload, all host cores."""
    import oracle

    oracle.build()
    cores = oracle.num_threads()
    rng = np.random.Generator(np.random.PCG64(2002))
    kidx = rng.choice(len(w.k), size=1, replace=False)
    pts = w.xobs[rng.choice(w.xobs.shape[0], size=args.cpu_points, replace=False)]
    t = time.perf_counter()
    for i in kidx:
        P, Pn = oracle.solve_frequency(w.mesh, w.k[i], w.direction)
    t_solve = (time.perf_counter() - t) / len(kidx)
    t = time.perf_counter()
    oracle.field(w.mesh, w.k[kidx[0]], P, Pn, pts)
    t_pts = time.perf_counter() - t
    t_field = t_pts * (w.xobs.shape[0] / len(pts))
    per_k = t_solve + t_field
    return {"value": 1.0 / per_k, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(kidx)} wavenumber solve(s) (assembly+LU+solve, N={w.mesh.N}) and the field at "
                      f"{len(pts)} of {w.xobs.shape[0]} points; value = 1 / (solve time + field time scaled "
                      "to all points); synthesis not counted",
            "seconds_per_frequency": per_k, "sample_wall_s": t_solve * len(kidx) + t_pts,
            "k_index": int(kidx[0]), "P": P}


# ------------------------------------------------------------------------- reference arm ----
def run_reference(args):
    """The oracle as the reference arm, timed on the host cores: each step is one bounded sample
    (one frequency solve at N = 2884 plus the field at --cpu-points of the 16 384 points, the same
    sample as the GPU arm's cpu_baseline leg); `ms_per_step` is the measured wall time per sample,
    `value` extrapolates each sample to whole frequency solves (field at every point)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = build_workload()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    vals = []
    for _ in range(args.warmup):      # warm-up samples (page-in, thread pool start), untimed
        cpu_baseline(args, w)
    t = time.perf_counter()
    cb = None
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(args, w)
        vals.append(cb["value"])
    dt = time.perf_counter() - t
    value = float(np.mean(vals))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded meshes/points/pulse)", "impl": "reference",
            "config": bench_config(w, args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "extrapolation": "ms_per_step is the measured wall time of one sample; value = 1 / (seconds per "
                             "frequency solve with the field at all points), from each sample's timings",
            "wall_s": dt}
    print(json.dumps(line))


def run_case(args):
    """Small cases for profiler captures (no timing, no output line): `lu` factors and refines four
    two-sphere systems (k = 3.15 .. 3.25); `field` evaluates the field of eight wavenumbers at 2048
    of the 16 384 plane points from a constant surface solution; `batch` runs one batch of the
    benchmark (128 wavenumbers, k = 8.03 .. 12.0: solves and the field at all points); `learned`
    runs the learned sweep on 128 spheroid wavenumbers (k = 5.02 .. 7.5, 20 training epochs);
    `field512` evaluates the field of all 512 wavenumbers at all 16 384 points from a constant
    surface solution (the shape of the benchmark's field launch, without its solves);
    `step` runs one benchmark step once (cold: the geometry tables are built inside it); `lattice`
    solves one batch of the lattice (k = 0 and 8 wavenumbers, N = 20 544) with phase timing;
    `lu_n8004` solves two wavenumbers on two spheres of 4002 nodes (N = 8004, deferred block 512,
    cooperative panels; a few GB on the device)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1706_07919_gb300 import Solver
    from paper_1706_07919_gb300 import binding as B

    w = build_workload()
    sol = Solver(0)
    sol.set_geometry(w.mesh.nodes, w.mesh.elems, w.mesh.normals, w.mesh.bc)
    sol.set_option("mixed.tcgen05", args.tc)
    sol.set_option("mixed.lu_block", args.lu_block)
    sol.set_option("mixed.lu_panel", args.lu_panel)
    sol.set_option("mixed.lu_tile", args.lu_tile)
    sol.set_option("mixed.asm_kb", args.asm_kb)
    sol.set_option("field.variant", args.field_variant)
    if args.case == "phases":  # one untimed sweep, then one with phase timing (device times per phase)
        sol.set_incident_plane_wave(w.direction)
        sol.set_option("mixed.batch", args.batch)
        sol.solve_frequencies(w.k, B.BIE_MODE_MIXED)
        sol.set_option("mixed.phase_timing", 1)
        sol.solve_frequencies(w.k, B.BIE_MODE_MIXED)
        ph = B.bie_get_phase_times(sol.ctx)
        flops = ph["systems"] * (8.0 / 3.0) * float(w.mesh.N) ** 3
        ph["lu_tflops"] = flops / (ph["factor_ms"] * 1e-3) / 1e12
        print("case phases:", json.dumps(ph))
    elif args.case == "step":
        sol.set_incident_plane_wave(w.direction)
        sol.set_option("mixed.batch", args.batch)
        xo = torch.tensor(w.xobs, dtype=torch.float64, device="cuda")
        pulses = torch.tensor(w.pulses, dtype=torch.float64, device="cuda")
        surf, _ = sol.solve_frequencies(w.k, B.BIE_MODE_MIXED)
        T = sol.eval_field(xo, w.k, surf, B.BIE_MODE_MIXED)
        S = sol.pulse_spectrum(pulses)
        sol.synthesize(T, np.arange(1, len(w.k) + 1, dtype=np.int64), S, w.Nt, torch.float32)
        print("case step: one benchmark step")
    elif args.case == "learned":
        from workloads import config_spheroid_learned
        ws = config_spheroid_learned()
        s2 = Solver(0)
        s2.set_geometry(ws.mesh.nodes, ws.mesh.elems, ws.mesh.normals, ws.mesh.bc)
        s2.set_option("learned.epochs", 20)
        surf, rep = s2.solve_frequencies(ws.k[256:384], B.BIE_MODE_LEARNED)
        print("case learned:", s2.learned_info())
        s2.close()
    elif args.case == "batch":
        ks = w.k[256:384]
        surf, rep = sol.solve_frequencies(ks, B.BIE_MODE_MIXED)
        xo = torch.tensor(w.xobs, device="cuda")
        T = sol.eval_field(xo, ks, surf, B.BIE_MODE_MIXED)
        print("case batch: flagged", sum(1 for r in rep if r.flags & B.BIE_FLAG_FP64_ASSEMBLY), tuple(T.shape))
    elif args.case == "lu":
        sol.set_option("mixed.fallback_err_est", 1.0)
        surf, rep = sol.solve_frequencies(w.k[100:104], B.BIE_MODE_MIXED)
        print("case lu: refinement corrections", [r.iters for r in rep])
    elif args.case == "lu16":  # one batch of 16 systems (a few GB on the device)
        sol.set_option("mixed.fallback_err_est", 1.0)
        sol.set_option("mixed.batch", 16)
        surf, rep = sol.solve_frequencies(w.k[100:116], B.BIE_MODE_MIXED)
        print("case lu16: refinement corrections", [r.iters for r in rep])
    elif args.case == "lattice":  # one lattice batch: k = 0 and 8 wavenumbers, N = 20 544, phase timing
        from workloads import config_lattice_large
        wl = config_lattice_large()
        ks = np.concatenate([[0.0], wl.k[np.linspace(0, len(wl.k) - 1, 8).round().astype(np.int64)]])
        s2 = Solver(0)
        s2.set_geometry(wl.mesh.nodes, wl.mesh.elems, wl.mesh.normals, wl.mesh.bc)
        s2.set_incident_plane_wave(wl.direction)
        s2.set_option("mixed.phase_timing", 1)
        surf, rep = s2.solve_frequencies(ks, B.BIE_MODE_MIXED)
        ph = B.bie_get_phase_times(s2.ctx)
        ph["lu_tflops"] = ph["systems"] * (8.0 / 3.0) * float(wl.mesh.N) ** 3 / (ph["factor_ms"] * 1e-3) / 1e12
        print("case lattice:", json.dumps(ph), "max backward error", max(r.backward_err for r in rep))
        s2.close()
    elif args.case == "lu_n8004":  # two spheres of 4002 nodes, 2 wavenumbers, deferred block 512 (a few GB)
        from workloads import ico_sphere, merge_meshes, scale_translate
        s0 = ico_sphere(10)
        m = merge_meshes([scale_translate(s0, 1.0, (0, 0, -1.05)), scale_translate(s0, 1.0, (0, 0, 1.05))])
        s2 = Solver(0)
        s2.set_geometry(m.nodes, m.elems, m.normals, m.bc)
        s2.set_option("mixed.batch", 2)
        s2.set_option("mixed.lu_block", 512)
        s2.set_option("mixed.reassembly_group", 1)
        s2.set_option("mixed.fallback_err_est", 1.0)
        s2.set_option("mixed.phase_timing", 1)
        surf, rep = s2.solve_frequencies(np.array([3.3, 7.7]), B.BIE_MODE_MIXED)
        ph = B.bie_get_phase_times(s2.ctx)
        print("case lu_n8004: factor_ms", ph["factor_ms"], "refinement corrections", [r.iters for r in rep])
        s2.close()
    elif args.case == "field512":
        ks = w.k
        surf = torch.full((len(ks), 2, w.mesh.N), 0.3 + 0.1j, dtype=torch.complex128, device="cuda")
        xo = torch.tensor(w.xobs, device="cuda")
        ms = []
        for _ in range(3):
            t0 = time.perf_counter()
            T = sol.eval_field(xo, ks, surf, B.BIE_MODE_MIXED)  # synchronises
            ms.append(1e3 * (time.perf_counter() - t0))
        print("case field512:", tuple(T.shape), "variant", args.field_variant, "ms", [round(x, 1) for x in ms])
    elif args.case == "field_sample":  # all 512 wavenumbers at every 8th point (profiler captures)
        surf = torch.full((len(w.k), 2, w.mesh.N), 0.3 + 0.1j, dtype=torch.complex128, device="cuda")
        xo = torch.tensor(w.xobs[::8], device="cuda")
        T = sol.eval_field(xo, w.k, surf, B.BIE_MODE_MIXED)
        print("case field_sample:", tuple(T.shape))
    elif args.case == "reassembly4":  # four wavenumbers forced through the FP64 re-assembly (profiler captures)
        sol.set_incident_plane_wave(w.direction)
        sol.set_option("mixed.batch", 4)
        sol.set_option("mixed.reassembly_group", 4)
        sol.set_option("mixed.fallback_err_est", 1e-30)
        surf, rep = sol.solve_frequencies(w.k[[100, 200, 300, 400]], B.BIE_MODE_MIXED)
        print("case reassembly4: flags", [r.flags for r in rep], "backward errors", [r.backward_err for r in rep])
    else:
        ks = w.k[496:504]
        surf = torch.full((len(ks), 2, w.mesh.N), 0.3 + 0.1j, dtype=torch.complex128, device="cuda")
        xo = torch.tensor(w.xobs[::8], device="cuda")
        T = sol.eval_field(xo, ks, surf, B.BIE_MODE_MIXED)
        print("case field:", tuple(T.shape))
    torch.cuda.synchronize()
    sol.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lu-block", type=int, default=256, help="columns of the deferred LU update (128, 256, 512)")
    ap.add_argument("--lu-panel", type=int, default=64, help="panel width of the deferred LU update (64, 32)")
    ap.add_argument("--lu-tile", type=int, default=256, help="real columns of the LU update tile (256, 128)")
    ap.add_argument("--field-variant", type=int, default=2,
                    help="mixed field kernel: 2 (128 points per CTA, 32-point tiles), 1 (64 points), 0 (k_field32b)")
    ap.add_argument("--asm-kb", type=int, default=2,
                    help="FP32 bulk assembly: wavenumbers per thread (2, 1) or 0 for the general kernel")
    ap.add_argument("--tc", type=int, default=3,
                    help="LU trailing update: 3 TMA-fed tcgen05 deferred over 256 columns, 2 after every 64-column "
                         "panel, 1 register-staged tcgen05, 0 SIMT")
    ap.add_argument("--check", type=int, default=4)
    ap.add_argument("--cpu-points", dest="cpu_points", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", dest="no_learned", action="store_true",
                    help="skip the learned-warm-start sweep on the spheroid workload")
    ap.add_argument("--epochs", type=int, default=60, help="training epochs of the learned warm start")
    ap.add_argument("--no-large", dest="no_large", action="store_true",
                    help="skip the lattice (N = 20544) sample")
    ap.add_argument("--large-nk", dest="large_nk", type=int, default=17,
                    help="wavenumbers of the lattice sample")
    ap.add_argument("--no-paper", dest="no_paper", action="store_true",
                    help="skip the paper's own experiments (Table I, directions, amplification)")
    ap.add_argument("--no-uneven", dest="no_uneven", action="store_true",
                    help="skip the uneven multi-configuration batch through the scheduler")
    ap.add_argument("--uneven-nk", dest="uneven_nk", type=int, default=8,
                    help="wavenumbers per configuration of the uneven batch sample")
    ap.add_argument("--uneven-workers", dest="uneven_workers", type=int, default=4)
    ap.add_argument("--case", choices=["lu", "lu16", "lu_n8004", "lattice", "lattice_full", "field", "field512",
                                       "field_sample", "reassembly4", "batch", "learned", "step", "peaks", "phases",
                                       "uneven_full"],
                    default=None,
                    help="run one small case for a profiler capture instead of the benchmark")
    args = ap.parse_args()
    if args.case == "uneven_full":  # the whole uneven workload: 64 configurations x 256 wavenumbers
        import torch
        import __graft_entry__
        __graft_entry__.build()
        from paper_1706_07919_gb300 import binding as B
        from workloads import config_uneven_batch
        ws = config_uneven_batch()
        dev = torch.device("cuda", 0)
        outs = [torch.empty((len(w.k), 2, w.mesh.N), dtype=torch.complex128, device=dev) for w in ws]
        res = {}
        for workers in (args.uneven_workers, 1):
            sched = B.bie_sched_create(0, workers, None)
            jobs = [B.bie_sched_add(sched, w.mesh.nodes, w.mesh.elems, w.mesh.normals, w.mesh.bc, w.direction, w.k,
                                    B.BIE_MODE_MIXED, o) for w, o in zip(ws, outs)]
            torch.cuda.synchronize(dev)
            util = subprocess.Popen(["nvidia-smi", "-i", "0", "--query-gpu=utilization.gpu", "--format=csv,noheader,nounits",
                                     "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            t = time.perf_counter()
            st = B.bie_sched_run(sched)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t
            util.terminate()
            u = [float(x) for x in util.communicate(timeout=5)[0].split() if x.strip().replace('.', '', 1).isdigit()]
            B.bie_sched_destroy(sched)
            ns = sum(len(w.k) for w in ws)
            reps = [r for j in jobs for r in j.reports()]
            full = [r for r in reps if r.flags & B.BIE_FLAG_FALLBACK_FP64]
            worst = max(r.backward_err for r in reps if not r.flags & B.BIE_FLAG_FALLBACK_FP64)
            res[workers] = {"solves": ns, "wall_s": dt, "solves_per_s": ns / dt, "busy_s": st["busy_ms"] / 1e3,
                            "gpu_util_median_pct": float(np.median(u)) if u else None,
                            "fp64_reassembled": sum(1 for r in reps if r.flags & B.BIE_FLAG_FP64_ASSEMBLY),
                            "fp32_refactored": sum(1 for r in reps if r.flags & B.BIE_FLAG_FP32_REFACTOR),
                            "fp64_full_solves": len(full), "max_backward_err_refined": worst}
        print(json.dumps({"case": "uneven_full", "workload": "uneven_64_configs_N162_to_7976_Nk256",
                          "workers": res[args.uneven_workers], "one_worker": res[1],
                          "speedup": res[1]["wall_s"] / res[args.uneven_workers]["wall_s"]}))
        return
    if args.case == "lattice_full":  # the whole lattice workload: k = 0 and 2048 wavenumbers, 8 pulses
        import torch
        import __graft_entry__
        __graft_entry__.build()
        from paper_1706_07919_gb300 import Solver
        from paper_1706_07919_gb300 import binding as B
        from workloads import config_lattice_large
        wl = config_lattice_large()
        ks = np.concatenate([[0.0], wl.k])
        midx = np.arange(len(ks), dtype=np.int64)
        dev = torch.device("cuda", 0)
        sol = Solver(0)
        sol.set_geometry(wl.mesh.nodes, wl.mesh.elems, wl.mesh.normals, wl.mesh.bc)
        sol.set_incident_plane_wave(wl.direction)
        xo = torch.tensor(wl.xobs, dtype=torch.float64, device=dev)
        pulses = torch.tensor(wl.pulses, dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        surf, rep = sol.solve_frequencies(ks, B.BIE_MODE_MIXED)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        T = sol.eval_field(xo, ks, surf, B.BIE_MODE_MIXED)
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        S = sol.pulse_spectrum(pulses)
        out = sol.synthesize(T, midx, S, wl.Nt, torch.float32)
        torch.cuda.synchronize(dev)
        t3 = time.perf_counter()
        M, P, Nt = wl.xobs.shape[0], wl.pulses.shape[0], wl.Nt
        ok = [r for r in rep if not r.flags & B.BIE_FLAG_NOT_CONVERGED]
        print(json.dumps({"case": "lattice_full", "workload": "lattice_4x4x2_soft_N20544_Nk2048_M65536_Nt4096_P8",
                          "N": int(wl.mesh.N), "wavenumbers": len(ks), "points": M, "pulses": P, "Nt": Nt,
                          "solve_s": t1 - t0, "field_s": t2 - t1, "spectrum_synthesis_s": t3 - t2,
                          "solves_per_s": len(ks) / (t1 - t0),
                          "space_time_pts_per_s": M * Nt * P / ((t2 - t1) + (t3 - t2)),
                          "field_evals_per_s": M * wl.mesh.E * 16 * len(ks) / (t2 - t1),
                          "fp64_reassembled": sum(1 for r in rep if r.flags & B.BIE_FLAG_FP64_ASSEMBLY),
                          "fp32_refactored": sum(1 for r in rep if r.flags & B.BIE_FLAG_FP32_REFACTOR),
                          "fp64_full_solves": sum(1 for r in rep if r.flags & B.BIE_FLAG_FALLBACK_FP64),
                          "not_converged": len(rep) - len(ok),
                          "max_backward_err": max(r.backward_err for r in rep),
                          "output_finite": bool(torch.isfinite(out).all().item()),
                          "timing": "wall clock around each synchronising phase"}))
        sol.close()
        return
    if args.case == "peaks":  # the pipe micro-benchmarks alone, as one JSON line
        import torch
        import __graft_entry__
        __graft_entry__.build()
        from paper_1706_07919_gb300 import binding as B
        pk = B.bie_measure_peaks(0)
        pk["gpu"] = torch.cuda.get_device_name(0)
        print(json.dumps(pk))
        return
    if args.case:
        run_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
