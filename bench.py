#!/usr/bin/env python
"""Throughput of the GB300 IOBM transport solve (channel-solves per second).

Workload (one step): the 6-atom wire of Gaussian wells plus s/p Kleinman-
Bylander projectors on a 48x48x160 grid (h = 0.35 bohr) between r_s = 3.28
jellium electrodes, 32 energies uniform in [E_F - 2 eV, E_F + 0.5 eV], every
open incident channel of every energy solved to ||b - A psi|| / ||b|| <= 1e-8
(FP64 residual) by the mixed-precision solver (complex FP32 COCG iterations,
FP64 residual replacement and projection), then T and G.  One step = channel
set-up + the batched solve + projection, inputs resident on the device.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "channel-solves/sec at 1e-6 G0 (mixed vs FP64 GPU); stencil HBM GB/s vs peak"
UNIT = "channel-solves/s"
# Roofline kernels: per COCG iteration kernel, the algorithmic HBM bytes per
# RHS-point (complex FP32 vectors, 8 B per element) and per grid point of a launch,
# and the measured DRAM bytes per RHS-point (ncu dram__bytes_read.sum +
# dram__bytes_write.sum of one launch of the first COCG iteration with all 56 RHS of
# the 8-energy wire48 case active), None until captured for the kernel as it stands.
ROOFLINE_KERNELS = {
    # p = z + beta p_old, q = (r - V z) + beta q_old: read z r p_old q_old, write p q
    "operator": {"kernel": "k_pq_update<float> (implicit operator form: direction and "
                           "operator update + p^T q partials)",
                 "bytes_rhs_point": 48.0, "bytes_point": 4.0,
                 "dram_rhs_point": (670682368 + 288807168) / (56 * 368640)},
    # x += alpha p, r -= alpha q, forward plane FFTs: read x p r q, write x r spectrum
    "update_fft": {"kernel": "k_update_fft_ct<float,48> (x, r update + forward plane FFTs)",
                   "bytes_rhs_point": 56.0, "bytes_point": 0.0,
                   "dram_rhs_point": (660668672 + 435869696) / (56 * 368640)},
    # z-sweeps in place: read the spectrum, write the forward sweep, read it back, write z
    "zsweep": {"kernel": "k_zsolve<float,4> (free-propagator z-sweeps per lateral mode)",
               "bytes_rhs_point": 32.0, "bytes_point": 0.0,
               "dram_rhs_point": (229594368 + 196402432) / (56 * 368640)},
    # inverse plane FFTs + dots: read spectrum and r, write z
    "ifft": {"kernel": "k_ifft_dots_ct<float,48> (inverse plane FFTs + r^T z, |r|^2 partials)",
             "bytes_rhs_point": 24.0, "bytes_point": 0.0,
             "dram_rhs_point": (330364672 + 119505152) / (56 * 368640)},
}
ROOFLINE_STAGE = "update_fft"   # the kernel with the largest share of the bench step
# The explicit-form stencil (fused p = z + beta p_old, FD operator + V, p^T q): 32 B per
# RHS-point (read z and p_old, write p and q) + 4 B per point (V) per launch; DRAM bytes
# per RHS-point from an ncu capture, None until captured for the kernel as it stands.
# Kernel per stencil variant (iobm_set_tiling) on the 48-point rows of the bench wire.
STENCIL_KERNELS = {
    0: "k_stencil_blk<48,4,4,4> (explicit form: fused p update + FD operator + p^T q; "
       "4 rows per thread, bulk-copy staged)",
    1: "k_stencil_rows<float,4> (register-pipelined rows)",
    3: "k_stencil_rows_tma<48,4> (one row per thread, bulk-copy staged)",
    4: "k_stencil_ring<48,4> (explicit form: fused p update + FD operator + p^T q; "
       "operand planes in a shared-memory ring, one thread per point, bulk-copy staged)",
}
STENCIL_BYTES_RHS_POINT = 32.0
# ncu captures of one full-load launch on 56 RHS (bench.py --workload stencil
# --stencil-rhs 56 --stencil-variant V): DRAM bytes read + written per RHS-point
STENCIL_DRAM_BYTES_PER_RHS_POINT = {0: (402582528 + 289049344) / (56 * 368640)}
WORKLOAD = ("wire48: 6-atom wire, Gaussian wells (0.5 Ha, width 1.5 bohr, spacing 6.8 bohr) "
            "+ s/p KB projectors (radius 3 bohr), 48x48x160 grid, h=0.35 bohr, 9-point FD, "
            "r_s=3.28 jellium, 32 energies in [E_F-2eV, E_F+0.5eV], all open channels, "
            "mixed precision, Fourier preconditioner")


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="iobm_clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() in ("active", "1"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (subprocess: thread count fixed before numpy loads)

ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import iobm_synth as S
from oracle import transport
jn = S.wire12_copy()
E = float(jn.energies[0])
n = 0
t0 = time.perf_counter()
reps = 0
while True:
    sol = transport.solve(jn, E)
    n += sol.n_open
    reps += 1
    if time.perf_counter() - t0 > {budget} or reps >= {max_reps}:
        break
dt = time.perf_counter() - t0
print(json.dumps({{"solves": n, "seconds": dt, "reps": reps, "G": sol.G, "n_open": sol.n_open}}))
"""


def run_oracle(budget_s: float, max_reps: int = 1000):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, budget=budget_s, max_reps=max_reps)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=600)
    if out.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


ORACLE_SAMPLE = ("FP64 oracle (scipy sparse LU of the assembled operator with dense Eq. 8 "
                 "self-energy blocks) on the 12x12x40 copy of the same wire (h=1.4 bohr, same "
                 "atoms and projector shapes) at E_F, all open channels; the oracle cannot "
                 "factor the 48x48x160 operator (dense 9216^2 end blocks)")


def cpu_baseline_entry(budget_s=12.0):
    r = run_oracle(budget_s)
    return {"value": r["solves"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": ORACLE_SAMPLE + f"; {r['reps']} repetitions, {r['seconds']:.1f} s",
            "cpu_model": cpu_model(), "threads": 1, "host_cores": os.cpu_count(),
            "paper_context": PAPER_CPU_CONTEXT}


# ---------------------------------------------------------------------------

def reduce_over_ranks(dist, device, elapsed, units):
    """Whole-job (elapsed, units) of a replicated run, one process per GPU: the slowest
    rank's elapsed time and the units every rank processed (dist None: one process)."""
    if dist is None:
        return float(elapsed), float(units)
    import torch
    t = torch.tensor([float(elapsed), float(units)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
    dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    steps = []
    for i in range(args.warmup + args.steps):
        r = run_oracle(budget_s=1.0, max_reps=1)
        if i >= args.warmup:
            steps.append(r)
    solves = sum(r["solves"] for r in steps)
    secs = sum(r["seconds"] for r in steps)
    value = solves / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference_sample": ORACLE_SAMPLE},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": ORACLE_SAMPLE + "; one repetition per step",
                             "cpu_model": cpu_model(), "threads": 1,
                             "host_cores": os.cpu_count(), "paper_context": PAPER_CPU_CONTEXT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


GOLDEN_WIRE48 = os.path.join(ROOT, "tests", "golden", "wire48_gmres.json")


def oracle_accuracy(jn, E, mixed, fp64):
    """Conductance error of both solvers against the stored oracle values of the
    wire48 energies (FP64 preconditioned GMRES to 1e-12 on the matrix-free Eq. 7
    operator, written by tests/golden/make_wire48_gmres.py, which calls only the oracle)."""
    import numpy as np
    if jn.name != "wire48" or jn.seed != 1000 or len(E) != 32 or not os.path.exists(GOLDEN_WIRE48):
        return {}
    with open(GOLDEN_WIRE48) as f:
        gd = json.load(f)
    idx = [e["index"] for e in gd["energies"]]
    Gref = np.array([e["G"] for e in gd["energies"]])
    if not np.allclose(E[idx], [e["E"] for e in gd["energies"]], rtol=0, atol=1e-15):
        return {}
    return {"oracle_energies": idx,
            "oracle": "FP64 preconditioned GMRES, relative residual <= 1e-12 (stored values)",
            "max_abs_dG_mixed_vs_oracle_G0": float(np.max(np.abs(mixed.G[idx] - Gref))),
            "max_abs_dG_fp64_vs_oracle_G0": float(np.max(np.abs(fp64.G[idx] - Gref)))}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip():
                return v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model", "CPU part") and v.strip():
                    return v.strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


PAPER_CPU_CONTEXT = ("paper (Sec. III, Table I): serial runs on a 3.25 GHz Intel Xeon workstation; "
                     "no absolute times are printed (Figs. 2-3), only CG iteration counts per "
                     "incident wave: about 14,000 unpreconditioned and 6,000-12,000 with the "
                     "Eq. 10 preconditioner on 36x36-lateral Na wires")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def native_arm(args, rank, world, local_rank):
    import numpy as np
    import torch

    import iobm_synth as S
    from paper_1009_5300_gb300 import IOBMSolver, build_library

    build_library()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    jn = S.wire48(junction_id=rank, n_energies=args.energies)
    E = jn.energies
    opt_kw = {}
    if args.delta is not None:
        opt_kw["refine_delta"] = args.delta
    if args.chunk is not None:
        opt_kw["chunk"] = args.chunk
    solver = IOBMSolver.from_junction(jn, precision="mixed", device=dev, **opt_kw)
    nrhs_int = solver._count_rhs(np.ascontiguousarray(E), None)
    ws_bytes = solver.workspace_size(nrhs_int)

    # warm-up
    for _ in range(args.warmup):
        res = solver.solve(E)
        print(f"[bench] warm-up solve: {res.device_ms:.1f} ms device, {res.nrhs} channels, "
              f"iterations mean {res.iterations.mean():.1f} max {res.iterations.max()}, "
              f"replacements mean {res.replacements.mean():.1f}, converged {res.converged}",
              file=sys.stderr, flush=True)
    barrier()

    sampler = ClockSampler(local_rank)
    solver.profile(ROOFLINE_STAGE)
    sampler.start()
    stream = torch.cuda.current_stream(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(solver.solve(E))
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    kern_ms, kern_launches = solver.kernel_stats()
    solver.profile(False)

    solves = sum(r.nrhs for r in results)
    converged = all(r.converged for r in results)
    iters_total = sum(r.iterations_total for r in results)
    launches = sum(r.launches for r in results)
    max_res = max(float(r.residual.max()) for r in results)
    ms_max, solves_all = reduce_over_ranks(dist, dev, ms, solves)
    value = solves_all / (ms_max / 1000.0)

    # roofline of the dominant kernel: algorithmic bytes of its launches (per
    # RHS-point for every active RHS-iteration, plus the per-point tables once a
    # launch) over its CUDA-event time inside the timed region
    npts = jn.npts
    rk = ROOFLINE_KERNELS[ROOFLINE_STAGE]
    alg_bytes = rk["bytes_rhs_point"] * npts * iters_total + rk["bytes_point"] * npts * kern_launches
    peak, peak_kind = load_peaks()
    roof = None
    if kern_launches > 0 and kern_ms > 0:
        achieved = alg_bytes / (kern_ms / 1000.0) / 1e9
        rhs_points = npts * iters_total / kern_launches
        dram = rk["dram_rhs_point"]
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": dram * rhs_points if dram is not None else None,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                   "launch on the 8-energy case (56 RHS), scaled by RHS-points"
                                   if dram is not None else "not captured for this kernel"),
                "kernel": rk["kernel"],
                "launches": kern_launches,
                "avg_launch_ms": kern_ms / kern_launches,
                "alg_bytes_per_launch": alg_bytes / kern_launches,
                "peak_source": f"{peak_kind} hbm_gbs"}

    extra = {}
    if rank == 0 and not args.no_fp64:
        # the explicit FD stencil kernel (fused p update + operator + p^T q) on the same
        # workload: one solve with the explicit operator form, its launches timed
        sx = IOBMSolver.from_junction(jn, precision="mixed", device=dev, op_form="explicit")
        sx.solve(E[:8])                   # warm
        sx.profile("operator")
        rx = sx.solve(E[:8])
        st_ms, st_launches = sx.kernel_stats()
        sx.profile(False)
        sx.close()
        if st_launches > 0 and st_ms > 0:
            st_bytes = (STENCIL_BYTES_RHS_POINT * npts * rx.iterations_total
                        + 4.0 * npts * st_launches)
            st_ach = st_bytes / (st_ms / 1000.0) / 1e9
            # the same kernel at full load: every internal RHS of the bench step active
            # (workspace 6.7 GB, larger than L2), tiling picked by the autotuner
            sx2 = IOBMSolver.from_junction(jn, precision="mixed", device=dev, op_form="explicit")
            zc, var = sx2.autotune(nrhs_int)
            fl_ms = sx2.time_operator(nrhs_int, reps=20)
            sx2.close()
            fl_ach = (STENCIL_BYTES_RHS_POINT * npts * nrhs_int + 4.0 * npts) / (fl_ms / 1e3) / 1e9
            dram = STENCIL_DRAM_BYTES_PER_RHS_POINT.get(var)
            extra["stencil_roofline"] = {
                "kernel": STENCIL_KERNELS.get(var, f"stencil variant {var}"),
                "bound": "hbm", "achieved": fl_ach, "peak": peak, "unit": "GB/s",
                "frac": fl_ach / peak, "avg_launch_ms": fl_ms,
                "alg_bytes_per_launch": STENCIL_BYTES_RHS_POINT * npts * nrhs_int + 4.0 * npts,
                "traffic": dram * npts * nrhs_int if dram else None,
                "sample": f"full load: {nrhs_int} RHS of the bench wire all active, 20 timed "
                          f"launches (iobm_time_operator), autotuned tiling z-chunk {zc}, "
                          f"variant {var}",
                "in_solve": {"achieved": st_ach, "frac": st_ach / peak,
                             "launches": st_launches, "avg_launch_ms": st_ms / st_launches,
                             "sample": "one explicit-form solve of the first 8 energies (its "
                                       "late launches run few RHS)",
                             "iterations_mean": float(rx.iterations.mean())}}
        # plain FP64 GPU solver on the same work: every energy of the step in one batch,
        # same tolerance, timed the same way as the mixed step
        s64 = IOBMSolver.from_junction(jn, precision="fp64", device=dev)
        r64 = s64.solve(E)                # warm
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n64 = 2
        e0.record(stream)
        for _ in range(n64):
            r64 = s64.solve(E)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1) / n64
        s64.close()
        rm = results[-1]
        extra["fp64_solver"] = {"value": r64.nrhs / (ms64 / 1000.0), "unit": UNIT,
                                "ms_per_step": ms64,
                                "sample": f"the same step: all {len(E)} energies in one batch "
                                          f"({r64.nrhs} channel-solves), {n64} timed solves",
                                "converged": bool(r64.converged),
                                "iterations_mean": float(r64.iterations.mean())}
        extra["mixed_vs_fp64_speedup"] = value / extra["fp64_solver"]["value"]
        acc = {"max_abs_dG_mixed_vs_fp64_G0": float(np.max(np.abs(rm.G - r64.G))),
               "max_residual": max_res, "all_converged": converged, "tol": 1e-8}
        acc.update(oracle_accuracy(jn, E, rm, r64))
        extra["accuracy"] = acc

    if rank == 0 and not args.no_samples:
        extra["workload_samples"] = {"uneven_batch": batch_sample(dev, stream),
                                     "wire128": wire128_sample(dev, stream)}

    # end to end through the public API with host buffers: create (H2D of V and
    # the projector tables from pinned memory), solve, read T, R, G back
    e2e = None
    if not args.no_e2e:
        Vp = torch.from_numpy(jn.V).pin_memory()
        csr = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in jn.projector_csr()]
        Ep = torch.from_numpy(np.ascontiguousarray(E)).pin_memory()
        h2d = Vp.numel() * 8 + sum(a.numel() * a.element_size() for a in csr) + Ep.numel() * 8
        d2h = 0
        barrier()
        t0 = time.perf_counter()
        e2e_steps = max(1, args.steps)
        for _ in range(e2e_steps):
            s = IOBMSolver(jn.nx, jn.ny, jn.nz, jn.hx, jn.hy, jn.hz, jn.nf, Vp.numpy(), jn.rs,
                           projectors=[a.numpy() for a in csr], precision="mixed", device=dev)
            s._ws = solver._ws  # reuse the torch-allocated workspace
            r = s.solve(Ep.numpy())
            d2h = (r.T.size + r.R.size + r.G.size) * 8 + r.nrhs * 32
            s._ws = None
            s.close()
        barrier()
        dt, e2e_solves = reduce_over_ranks(dist, dev, time.perf_counter() - t0, r.nrhs * e2e_steps)
        e2e = {"value": e2e_solves / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_entry()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "c64+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "channel_solves_per_step": results[0].nrhs,
                           "internal_rhs": nrhs_int, "grid_points": npts,
                           "workspace_bytes": ws_bytes,
                           "l2": "inputs larger than L2 (workspace %.1f GB > 129 MB)"
                                 % (ws_bytes / 1e9),
                           "parallelism": f"replicas x{world} (one junction per GPU)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "iterations_mean": iters_total / max(1, sum(len(r.status) for r in results)),
                "converged": converged}
        line.update(extra)
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _timed(stream, fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1)


def batch_sample(dev, stream, n_junctions=16, n_energies=4):
    """A stated sample of the uneven many-junction workload: the first n_junctions of
    its seeded generator at n_energies energies each (the first, middle-ish and last of
    [E_F - 1 eV, E_F + 0.5 eV]), one iobm_solve_batch graph launch, autotuned tiling."""
    import numpy as np
    import iobm_synth as S
    from paper_1009_5300_gb300 import IOBMSolver, solve_batch
    jns = [S.batch_junction(j, n_energies=n_energies) for j in range(n_junctions)]
    sols = [IOBMSolver.from_junction(jn, precision="mixed", device=dev) for jn in jns]
    solve_batch(sols[:1], [jns[0].energies[:1]], autotune=True)          # warm
    res, ms = _timed(stream, lambda: solve_batch(sols, [jn.energies for jn in jns], autotune=True))
    n = sum(r.nrhs for r in res)
    out = {"value": n / (ms / 1000.0), "unit": UNIT, "ms": ms, "channel_solves": n,
           "converged": bool(all(r.converged for r in res)),
           "iterations_mean": float(np.mean(np.concatenate([r.iterations for r in res]))),
           "sample": f"junctions 0-{n_junctions - 1} of the 256-junction uneven workload "
                     f"(lateral {sorted(set(j.nx for j in jns))}, N_z {min(j.nz for j in jns)}-"
                     f"{max(j.nz for j in jns)}), {n_energies} energies each in "
                     f"[E_F-1eV, E_F+0.5eV], one graph launch (timed region includes the "
                     f"autotuner and host channel set-up)"}
    for sol in sols:
        sol.close()
    return out


def wire128_sample(dev, stream, n_channels=32):
    """A stated sample of the 128x128x256 large cross-section workload: the first
    n_channels open channels at E_F in one batch."""
    import iobm_synth as S
    from paper_1009_5300_gb300 import IOBMSolver
    jn = S.wire128()
    E = jn.e_fermi
    sol = IOBMSolver.from_junction(jn, precision="mixed", device=dev)
    sol.solve([E], channels=[0])                                            # warm
    res, ms = _timed(stream, lambda: sol.solve([E], channels=list(range(n_channels))))
    out = {"value": res.nrhs / (ms / 1000.0), "unit": UNIT, "ms": ms, "channel_solves": res.nrhs,
           "n_open": int(res.n_open[0]), "converged": bool(res.converged),
           "iterations_mean": float(res.iterations.mean()),
           "iteration_phase_ms": res.device_ms,
           "sample": f"the first {n_channels} of the {int(res.n_open[0])} open channels at E_F of "
                     "the 128x128x256 wire (h=0.3, 7 deep wells, s/p/d KB), one batch"}
    sol.close()
    return out


BATCH_WORKLOAD = ("uneven batch: {n} junctions (lateral N from the 2,3,5-smooth set in [24, 64], "
                  "N_z in [96, 256], h=0.35 bohr, 2-8 Gaussian wells, r_s in [2, 4]), {e} energies "
                  "each in [E_F-1eV, E_F+0.5eV], all open channels, mixed precision, Fourier "
                  "preconditioner, autotuned stencil tiling, one graph launch per group")


def batch_arm(args, rank, world, local_rank):
    """Many junctions of uneven size: groups sized to the free device memory, each
    group solved by one iobm_solve_batch (one graph launch, a device-side WHILE loop
    per junction).  Junctions are dealt round-robin to the ranks."""
    import numpy as np
    import torch

    import iobm_synth as S
    from paper_1009_5300_gb300 import IOBMSolver, build_library, solve_batch

    build_library()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ids = list(range(rank, args.junctions, world))
    jns = [S.batch_junction(j, n_energies=args.batch_energies) for j in ids]

    # warm-up: the first junction at two energies, untimed
    w = IOBMSolver.from_junction(jns[0], precision="mixed", device=dev)
    solve_batch([w], [jns[0].energies[:2]], autotune=True)
    w.close()
    torch.cuda.synchronize(dev)

    # RHS counts and workspace sizes decide the groups (host-side, untimed)
    sols = [IOBMSolver.from_junction(jn, precision="mixed", device=dev) for jn in jns]
    need = []
    for sol, jn in zip(sols, jns):
        nrhs = sol._count_rhs(np.ascontiguousarray(jn.energies), None)
        need.append(sol.workspace_size(max(nrhs, 1)))
    free, _ = torch.cuda.mem_get_info(dev)
    budget = 0.7 * free
    groups, cur, cur_b = [], [], 0
    for i, b in enumerate(need):
        if cur and cur_b + b > budget:
            groups.append(cur)
            cur, cur_b = [], 0
        cur.append(i)
        cur_b += b
    if cur:
        groups.append(cur)

    sampler = ClockSampler(local_rank)
    sampler.start()
    stream = torch.cuda.current_stream(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    solves, converged, iters = 0, True, 0
    ev0.record(stream)
    for g in groups:
        res = solve_batch([sols[i] for i in g], [jns[i].energies for i in g], autotune=True)
        for r in res:
            solves += r.nrhs
            converged &= bool(r.converged)
            iters += r.iterations_total
        for i in g:
            sols[i].release_workspace()   # free this group's workspace before the next one
        torch.cuda.empty_cache()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms, solves_all = reduce_over_ranks(dist, dev, ev0.elapsed_time(ev1), solves)
    if rank == 0:
        line = {"metric": METRIC, "value": solves_all / (ms / 1000.0), "unit": UNIT,
                "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "c64+f64", "data": "synthetic",
                "config": {"workload": BATCH_WORKLOAD.format(n=args.junctions, e=args.batch_energies),
                           "junctions": args.junctions, "channel_solves": int(solves_all),
                           "groups_rank0": len(groups), "l2": "inputs larger than L2",
                           "parallelism": f"junctions dealt to {world} replica(s)"},
                "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clocks,
                "iterations_mean": iters / max(1, solves), "converged": converged}
        print(json.dumps(line), flush=True)
    for sol in sols:
        sol.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


WIRE128_WORKLOAD = ("wire128: 7-atom wire at 4.3 bohr spacing, Gaussian wells (2.0 Ha, width 1.5 bohr) "
                    "+ s/p/d KB projectors, 128x128x256 grid, h=0.3 bohr, 9-point FD, r_s=2.0 jellium "
                    "(109 open channels at E_F), {e} energies, every open channel in batches of {b} "
                    "channels, mixed precision, Fourier preconditioner (two-pass plane FFTs)")


def wire128_arm(args, rank, world, local_rank):
    """The large cross-section workload: every open channel of each energy, solved in
    batches of --batch channels (one solve per batch), energies dealt to the ranks."""
    import numpy as np
    import torch

    import iobm_synth as S
    from paper_1009_5300_gb300 import IOBMSolver, build_library

    build_library()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    jn = S.wire128()
    Es = jn.energies[: args.wire128_energies][rank::world]
    sol = IOBMSolver.from_junction(jn, precision="mixed", device=dev)
    sol.solve(Es[:1], channels=list(range(min(args.batch, 4))))   # warm-up
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local_rank)
    sampler.start()
    stream = torch.cuda.current_stream(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    solves, iters, converged = 0, 0, True
    ev0.record(stream)
    for E in Es:
        n_open = sol.open_channels(float(E))[0].shape[0]
        for c0 in range(0, n_open, args.batch):
            res = sol.solve([E], channels=list(range(c0, min(c0 + args.batch, n_open))))
            solves += res.nrhs
            iters += res.iterations_total
            converged &= bool(res.converged)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    if rank == 0:
        line = {"metric": METRIC, "value": solves * world / (ms / 1000.0), "unit": UNIT,
                "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "c64+f64", "data": "synthetic",
                "config": {"workload": WIRE128_WORKLOAD.format(e=len(Es), b=args.batch),
                           "channel_solves": solves, "grid_points": jn.npts,
                           "l2": "inputs larger than L2",
                           "parallelism": f"energies dealt to {world} replica(s)"},
                "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clocks,
                "iterations_mean": iters / max(1, solves), "converged": converged}
        print(json.dumps(line), flush=True)
    sol.close()
    return 0


# Sec. III solvers on the synthetic sodium-wire series (iobm_synth.na_wire), every open
# channel at E_F, FP64 iterations as in the paper: (b) the self-energy as the dense
# N_f N_xy matrix and (c) through the lateral FFT, both unpreconditioned; (d) with the
# Eq. 10 preconditioner at alpha = 3.0, 2.4, 1.8; and the default free-propagator
# preconditioner.  Explicit operator form for (b)-(d) (the dense matrix is what (b)
# multiplies every iteration).
ABLATION_SOLVERS = [
    ("b_dense_sigma", dict(use_precond="none", op_form="explicit", sigma_form="dense")),
    ("c_fft_sigma", dict(use_precond="none", op_form="explicit", sigma_form="fft")),
    ("d_eq10_alpha3.0", dict(use_precond="eq10", alpha=3.0, op_form="explicit")),
    ("d_eq10_alpha2.4", dict(use_precond="eq10", alpha=2.4, op_form="explicit")),
    ("d_eq10_alpha1.8", dict(use_precond="eq10", alpha=1.8, op_form="explicit")),
    ("free_propagator", dict()),
]


def ablation_solve(jn, kw, dev, precision):
    """Solves of every open channel at E_F, CUDA events on the solver's stream: the
    first (cold: tables, graphs and for (b) the dense matrices built inside), and a
    second (warm) one when the first took under 20 s; returns the warm time if taken."""
    import torch
    from paper_1009_5300_gb300 import IOBMSolver

    sol = IOBMSolver.from_junction(jn, precision=precision, device=dev, max_iter_mixed=100000,
                                   max_iter=100000, **kw)
    E = float(jn.energies[0])
    stream = torch.cuda.current_stream(dev)

    def timed():
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        res = sol.solve([E])
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        return res, ev0.elapsed_time(ev1)

    res, ms = timed()
    kind = "cold"
    if ms < 20000.0:
        res, ms = timed()
        kind = "warm"
    out = {"ms": ms, "timed": kind, "iterations_mean": float(res.iterations.mean()),
           "G": float(res.G[0]), "n_open": int(res.nrhs), "converged": bool(res.converged)}
    sol.close()
    return out


def ablation_arm(args, rank, world, local_rank):
    """Solver ablation of Sec. III (Figs. 2-3, Table I) on the synthetic sodium-wire
    series: per N_atom the time and iterations of each solver, same conductance."""
    import torch
    import iobm_synth as S
    from paper_1009_5300_gb300 import build_library

    build_library()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    rows = []
    for natom in args.ablation_atoms:
        jn = S.na_wire(natom)
        row = {"natom": natom, "grid": [jn.nx, jn.ny, jn.nz]}
        for name, kw in ABLATION_SOLVERS:
            row[name] = ablation_solve(jn, kw, dev, args.ablation_precision)
        Gs = [row[name]["G"] for name, _ in ABLATION_SOLVERS]
        row["max_dG_G0"] = max(Gs) - min(Gs)
        rows.append(row)
        if rank == 0:
            print(json.dumps(row), flush=True)
    if rank == 0:
        print(json.dumps({"workload": "ablation", "precision": args.ablation_precision,
                          "solvers": [n for n, _ in ABLATION_SOLVERS], "rows": rows}), flush=True)
    return 0


def stencil_arm(args, rank, world, local_rank):
    """The explicit-form FD stencil kernel alone at full load: --stencil-rhs RHS of the
    48x48x160 wire, every RHS active, --steps timed launches after --warmup (iobm_time_operator),
    tiling --stencil-variant / --stencil-zchunk (variant -1: the autotuner's choice)."""
    import torch
    import iobm_synth as S
    from paper_1009_5300_gb300 import IOBMSolver, build_library

    build_library()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    jn = S.wire48()
    sol = IOBMSolver.from_junction(jn, precision="mixed", device=dev, op_form="explicit")
    nrhs = args.stencil_rhs
    if args.stencil_variant < 0:
        zc, var = sol.autotune(nrhs)
    else:
        zc, var = args.stencil_zchunk, args.stencil_variant
        sol.set_tiling(zc, var)
    sol.time_operator(nrhs, reps=max(1, args.warmup))
    ms = sol.time_operator(nrhs, reps=max(1, args.steps))
    sol.close()
    npts = jn.npts
    alg = STENCIL_BYTES_RHS_POINT * npts * nrhs + 4.0 * npts
    peak, kind = load_peaks()
    if rank == 0:
        print(json.dumps({"workload": "stencil", "kernel": STENCIL_KERNELS.get(var, str(var)),
                          "zchunk": zc, "variant": var, "nrhs": nrhs,
                          "avg_launch_ms": ms, "achieved_gbs": alg / (ms / 1e3) / 1e9,
                          "frac": alg / (ms / 1e3) / 1e9 / peak, "peak_source": kind}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--energies", type=int, default=32)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-samples", action="store_true",
                    help="skip the stated samples of the uneven-batch and 128x128x256 workloads")
    ap.add_argument("--delta", type=float, default=None,
                    help="FP64 residual replacement factor of the mixed solver (library default)")
    ap.add_argument("--chunk", type=int, default=None,
                    help="COCG iterations per captured graph (library default)")
    ap.add_argument("--stencil-rhs", type=int, default=228,
                    help="RHS of the stencil-only measurement (--workload stencil)")
    ap.add_argument("--stencil-variant", type=int, default=-1,
                    help="stencil variant of --workload stencil (-1: autotuned)")
    ap.add_argument("--stencil-zchunk", type=int, default=32,
                    help="z-planes per CTA of --workload stencil with an explicit variant")
    ap.add_argument("--workload", choices=["wire48", "batch", "wire128", "stencil", "ablation"],
                    default="wire48",
                    help="wire48: the 48x48x160 wire (default line); batch: the uneven "
                         "many-junction workload solved in grouped graph launches; wire128: "
                         "the 128x128x256 large cross-section wire; stencil: the explicit-form "
                         "FD stencil kernel alone at full load; ablation: the Sec. III solvers "
                         "on the synthetic sodium-wire series")
    ap.add_argument("--ablation-atoms", type=int, nargs="+", default=[3, 4, 5, 6, 7, 8])
    ap.add_argument("--ablation-precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--wire128-energies", type=int, default=8)
    ap.add_argument("--batch", type=int, default=32, help="channels per solve (wire128)")
    ap.add_argument("--junctions", type=int, default=256)
    ap.add_argument("--batch-energies", type=int, default=16)
    args = ap.parse_args()
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload == "batch":
        return batch_arm(args, rank, world, local_rank)
    if args.workload == "wire128":
        return wire128_arm(args, rank, world, local_rank)
    if args.workload == "stencil":
        return stencil_arm(args, rank, world, local_rank)
    if args.workload == "ablation":
        return ablation_arm(args, rank, world, local_rank)
    return native_arm(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
