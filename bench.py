"""Benchmark: batched solves of (E - H_ef) psi = Phi over many energies on one GB300.

Workload (default): the 2-state, 2-mode conical-intersection model with 80 x 80 oscillator
functions (N = 12,800 unknowns), 256 incident energies on (0, 3] eV, v_i = 0, both partial
waves (512 systems), true relative residual 1e-8, complex-FP32 Krylov iterations inside FP64
iterative refinement.  One step = one vbk_solve call over the whole batch (level-shift
tables, preconditioner factorisation, Krylov iterations, refinement).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (sparse LU per
energy, complex128) on a bounded sample of the same workload instead.
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

METRIC = "energy points solved/s at rel. residual 1e-8, mixed vs FP64; matvec HBM GB/s"
UNIT = "energy points/s"


def load_json(name):
    p = os.path.join(ROOT, name)
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return None


def workload():
    import workloads as w

    spec = w.WORKLOADS["ci2d_batched"]
    return spec["model"](), spec["eps"], spec["vi"]


REFERENCE_ENERGIES_PER_STEP = 128  # half of the grid, evenly spaced, per reference step

WORKLOAD_NAME = ("ci2d_batched: 2 states x 80 x 80 oscillator functions (N=12800), 256 incident energies "
                 "on (0,3] eV, v_i=(0,0), 2 partial waves = 512 systems, tol 1e-8")


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self):
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        idx = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", idx, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx = float(s[1])
                for k, nm in enumerate(names):
                    if s[4 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------- roofline model
def kernel_bytes_per_unit(name, N, nmu, c, p_band):
    """Algorithmic bytes one kernel moves per system-iteration: the vectors and tables the method
    must read and write once (c bytes per complex entry, N unknowns, n_mu waves per energy)."""
    if name == "matvec":
        return (2 * c + c / nmu) * N          # read x, write y, diagonal shared by the n_mu waves
    if name == "cocg_update":
        return 6 * c * N                      # x, r read+write; p, q read
    if name == "cocg_update_jacobi":
        return (7 * c + c / nmu) * N
    if name == "cocg_p":
        return 3 * c * N                      # z read, p read+write
    if name == "block_apply":
        return (2 * c + (p_band + 1) * c / nmu) * N  # r in, z out, L D L^T factor shared by the waves
    if name == "point_precond":
        return (2 * c + c / nmu) * N
    if name == "cocg_resident":
        # one COCG iteration (matvec x in / y out, updates of x, r, p, q, z: (2 + 7) c N) plus the
        # diagonal and reciprocal tables shared by the n_mu waves; p and q stay in shared memory
        # and x, r in L2 across iterations, so DRAM traffic is far below this algorithmic figure
        return (9 * c + 2 * c / nmu) * N
    return None


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the kernel
    source changed since the counters were taken."""
    import hashlib

    rec = (load_json(os.path.join("profiles", "ncu_traffic.json")) or {}).get(kernel)
    if not rec:
        return None
    path = os.path.join(ROOT, rec["source_file"])
    if not os.path.exists(path) or hashlib.sha1(open(path, "rb").read()).hexdigest() != rec["source_sha1"]:
        return None
    scale = {"B": 1, "kB": 1e3, "MB": 1e6}[rec.get("traffic_unit", "B")]
    return rec["traffic_bytes_per_launch"] * scale


def roofline(model_N, nmu, stats, timings, opts, peaks):
    c = 8 if opts.precision == 1 else 16
    units = sum(s["iterations"] for s in stats)
    # dominant kernel by total time
    name, (launches, ms) = max(timings.items(), key=lambda kv: kv[1][1])
    p_band = 4 if opts.precond_span == 0x5 else 0
    bname = name
    if name == "cocg_update" and opts.precond_span == 0:
        bname = "cocg_update_jacobi"
    bpu = kernel_bytes_per_unit(bname, model_N, nmu, c, p_band)
    peak = (peaks or {}).get("hbm_gbs")
    peak_note = "measured" if peak else "fallback"
    peak = peak or 6800.0
    if bpu is None or launches == 0:
        return {"kernel": name, "bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                "traffic": None, "peak_source": peak_note}
    total_bytes = bpu * units
    achieved = total_bytes / (ms * 1e-3) / 1e9
    traffic = measured_traffic(name)
    return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "peak_source": peak_note,
            "bytes_per_launch": round(total_bytes / launches), "launches": launches,
            "avg_launch_us": round(ms * 1e3 / launches, 2), "share_of_step": None}


# ------------------------------------------------------------------------------ replicas
def job_rate(t_step_ms, units_per_rank, world, dist=None, device="cpu"):
    """Step time and whole-job throughput of `world` replicas.  Every rank solves its own copy
    of the workload (the systems are independent: no data-path collective); the step time is
    the maximum over ranks, and value = world * units / time."""
    if dist is not None and world > 1:
        import torch

        tt = torch.tensor([float(t_step_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step_ms = float(tt.item())
    return t_step_ms, world * units_per_rank / (t_step_ms * 1e-3)


# ------------------------------------------------------------------------------ oracle
_ORACLE_DESC = None


def _oracle_init():
    """Worker set-up: one BLAS/OpenMP thread per process (the energies are the parallel axis) and
    the workload's model description built once."""
    global _ORACLE_DESC
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    _ORACLE_DESC = workload()[0]


def _oracle_energy(args):
    """One incident energy of the workload: A(E) by the oracle, sparse LU, both partial waves."""
    from oracle import vibronic as o

    eps_i, vi = args
    desc = _ORACLE_DESC
    E = o.total_energy(desc, float(eps_i), vi)
    o.solve_many(desc, E, [o.phi(desc, E, vi, mu) for mu in range(o.n_partial_waves(desc))])
    return 0


class OraclePool:
    """The CPU oracle over all host cores: one process per core (spawned, never forked: the parent
    may already hold a CUDA context), one energy per task."""

    def __init__(self, cores=None):
        import concurrent.futures as cf
        import multiprocessing as mp

        self.cores = cores or os.cpu_count() or 1
        self.ex = cf.ProcessPoolExecutor(max_workers=self.cores, mp_context=mp.get_context("spawn"),
                                         initializer=_oracle_init)
        list(self.ex.map(_oracle_energy, [(1.0, [0, 0])] * self.cores))  # start-up outside the timing

    def rate(self, eps, vi, n_sample):
        """Oracle energies/s on a bounded, evenly spaced sample of the energy grid (all of it when
        n_sample >= its size)."""
        idx = np.linspace(0, eps.size - 1, min(n_sample, eps.size)).round().astype(int)
        t0 = time.perf_counter()
        list(self.ex.map(_oracle_energy, [(float(eps[k]), list(vi[0])) for k in idx]))
        dt = time.perf_counter() - t0
        return idx.size / dt, dt, idx.size

    def close(self):
        self.ex.shutdown()


def run_reference(args, rank):
    if rank != 0:
        return
    _, eps, vi = workload()
    pool = OraclePool()
    per_step = REFERENCE_ENERGIES_PER_STEP
    for _ in range(args.warmup):
        pool.rate(eps, vi, per_step)
    times = []
    for _ in range(args.steps):
        _, dt, per_step = pool.rate(eps, vi, per_step)
        times.append(dt)
    pool.close()
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "complex128", "data": "synthetic (seeded model)",
        "config": {"workload": WORKLOAD_NAME, "solver": "sparse LU (SuperLU) per energy, 2 right-hand sides"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "blas_threads": 1, "kind": "oracle",
                         "sample": f"{per_step} evenly spaced energies of the 256-point grid per step, "
                                   f"one energy per process over {pool.cores} processes"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------- ours
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--method", default="cocg", choices=["cocg", "gmres"])
    ap.add_argument("--precond", type=int, default=0, help="span mask (0 = Jacobi, 0x5 = M^g, -1 = none)")
    ap.add_argument("--restart", type=int, default=64)
    ap.add_argument("--inner-tol", type=float, default=1e-5)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 comparisons and the CPU baseline")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2307_13483_gb300 as vbk
    from oracle import vibronic as o

    desc, eps, vi = workload()
    model = vbk.Model(desc)
    N, nmu = model.N, model.n_mu
    opts = vbk.vbk_default_opts(method=args.method, precision="mixed", precond_span=args.precond, tol=1e-8,
                                restart=args.restart, inner_tol=args.inner_tol, max_refine=100)
    psi = torch.empty((eps.size, len(vi), nmu, N), dtype=torch.complex128, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        psi, stats = vbk.vbk_solve(model, eps, vi, opts, psi=psi)
    # timed steps: device time of each solve (CUDA events on the launch stream); the L2 is
    # flushed between steps outside the events
    sampler = ClockSampler()
    sampler.start()
    barrier()
    stream = torch.cuda.current_stream()
    step_ms = []
    launches = 0
    all_stats = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        psi, stats = vbk.vbk_solve(model, eps, vi, opts, psi=psi)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        launches += vbk.vbk_last_launch_count(model)
        all_stats.extend(stats)
    barrier()
    clocks = sampler.stop()
    n_energies = eps.size * len(vi)
    t_step, value = job_rate(sum(step_ms) / len(step_ms), n_energies, world, dist, "cuda")
    converged = all(s["status"] == "converged" for s in all_stats)
    worst = max(s["rel_residual"] for s in all_stats)
    iters = [s["iterations"] for s in stats]
    # per-kernel CUDA-event timings: the same solves once more with an event pair around every
    # launch (direct launches instead of graphs), for the roofline of the dominant kernel
    timing_opts = vbk.vbk_default_opts(method=args.method, precision="mixed", precond_span=args.precond, tol=1e-8,
                                       restart=args.restart, inner_tol=args.inner_tol, max_refine=100, timing=1)
    timings = {}
    prof_stats = []
    prof_ms = 0.0
    n_prof = max(1, min(2, args.steps))
    for k in range(n_prof):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        psi, stats_p = vbk.vbk_solve(model, eps, vi, timing_opts, psi=psi)
        b.record(stream)
        b.synchronize()
        prof_ms += a.elapsed_time(b)
        for nm, (nl, ms) in vbk.vbk_kernel_timings(model).items():
            t = timings.setdefault(nm, [0, 0.0])
            t[0] += nl
            t[1] += ms
        prof_stats.extend(stats_p)
    peaks = load_json("MEASURED_PEAKS.json")
    roof = roofline(N, nmu, prof_stats, {k: tuple(v) for k, v in timings.items()}, opts, peaks)
    if roof.get("kernel") in timings and prof_ms > 0:
        roof["share_of_step"] = round(timings[roof["kernel"]][1] / prof_ms, 4)
    roof["timed_in"] = f"{n_prof} profiled step(s) after the timed steps, one event pair per launch"
    # matvec HBM GB/s (part of the metric): the batched operator kernel alone, through vbk_matvec
    # with per-kernel CUDA-event timing, on a working set of 2.6 x L2: the 256 energies of the
    # workload x 6 vectors each (1536 systems; x and y 157 MB each in FP32, the diagonal tables
    # 26 MB).  Every kernel variant valid for the model is timed (best of 3 launches); the fastest
    # is reported with its algorithmic bytes (x in, y out, the diagonal once per energy).
    matvec_gbs = {}
    if rank == 0:
        peak = (peaks or {}).get("hbm_gbs") or 6800.0
        nvec = 6
        E_tot = np.array([o.total_energy(desc, float(e), vi[0]) for e in eps])
        gen = torch.Generator(device="cuda").manual_seed(2307)
        xm = torch.complex(torch.randn((eps.size, nvec, N), device="cuda", dtype=torch.float64, generator=gen),
                           torch.randn((eps.size, nvec, N), device="cuda", dtype=torch.float64, generator=gen))
        vbk.vbk_set_op_timing(model, True)
        for prec, c, name in ((vbk.VBK_MIXED, 8, "fp32"), (vbk.VBK_FP64, 16, "fp64")):
            per_var = {}
            for v in range(16):
                best = None
                for _ in range(3):
                    try:
                        vbk.vbk_matvec(model, E_tot, xm, precision=prec, variant=v)
                    except vbk.VbkError:
                        break  # variant not available for this model and precision
                    nl, ms = vbk.vbk_kernel_timings(model).get("matvec", (0, 0.0))
                    if nl == 1 and ms > 0:
                        best = ms if best is None else min(best, ms)
                if best is not None:
                    per_var[v] = best
            bpu = (2 * c + c / nvec) * N
            nsys_m = eps.size * nvec
            if not per_var:
                matvec_gbs[name] = {"error": "no matvec variant ran"}
                continue
            vb = min(per_var, key=per_var.get)
            achieved = bpu * nsys_m / (per_var[vb] * 1e-3) / 1e9
            matvec_gbs[name] = {"achieved": round(achieved, 1), "frac": round(achieved / peak, 4),
                                "kernel_us": round(per_var[vb] * 1e3, 2), "variant": vb,
                                "variants_us": {str(k): round(t * 1e3, 1) for k, t in sorted(per_var.items())},
                                "batch": f"{nsys_m} systems (256 energies x {nvec} vectors) in one launch, "
                                         f"{bpu * nsys_m / 1e6:.0f} MB of algorithmic traffic"}
        vbk.vbk_set_op_timing(model, False)
        del xm
        matvec_gbs["bytes_per_unit"] = "(2c + c/6) N per system: x in, y out, the diagonal once per energy (6 vectors each)"
        matvec_gbs["peak_source"] = "measured" if (peaks or {}).get("hbm_gbs") else "fallback"

    extras = {}
    if not args.no_extras and rank == 0:
        # end to end through the public API: host energies in, cross sections back to the host
        vf = o.open_levels(desc, o.total_energy(desc, float(eps[-1]), vi[0]))
        vf_h = np.asarray(vf, dtype=np.int32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            psi, _ = vbk.vbk_solve(model, eps, vi, opts, psi=psi)
            sig = vbk.vbk_cross_sections(model, eps, vi, psi, vf_h)
            sig_h = sig.cpu()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        extras["e2e"] = {"value": n_energies / e2e_s, "unit": UNIT,
                         "h2d_bytes_per_step": int(eps.nbytes + np.asarray(vi, np.int32).nbytes + vf_h.nbytes),
                         "d2h_bytes_per_step": int(sig_h.numel() * 8)}
        # FP64 batched (same workload, every Krylov iteration in FP64)
        o64 = vbk.vbk_default_opts(method=args.method, precision="fp64", precond_span=args.precond, tol=1e-8,
                                   restart=args.restart, max_refine=100)
        psi, st64 = vbk.vbk_solve(model, eps, vi, o64, psi=psi, check=False)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        psi, st64 = vbk.vbk_solve(model, eps, vi, o64, psi=psi, check=False)
        b.record()
        b.synchronize()
        extras["fp64_batched"] = {"value": n_energies / (a.elapsed_time(b) * 1e-3), "unit": UNIT,
                                  "converged": all(s["status"] == "converged" for s in st64)}
        # plain FP64 single-energy solves (GMRES + Jacobi, one energy per call), 16 energies
        o1 = vbk.vbk_default_opts(method="gmres", precision="fp64", precond_span=0, tol=1e-8, restart=64,
                                  max_refine=200)
        sel = np.linspace(0, eps.size - 1, 16).round().astype(int)
        psi1 = torch.empty((1, 1, nmu, N), dtype=torch.complex128, device="cuda")
        vbk.vbk_solve(model, eps[sel[:1]], vi, o1, psi=psi1, check=False)
        torch.cuda.synchronize()
        a.record()
        for kk in sel:
            vbk.vbk_solve(model, eps[kk:kk + 1], vi, o1, psi=psi1, check=False)
        b.record()
        b.synchronize()
        extras["fp64_single_energy"] = {"value": sel.size / (a.elapsed_time(b) * 1e-3), "unit": UNIT,
                                        "method": "GMRES(64) + Jacobi, FP64, one energy per call"}
        # the generalized model of Sec. II.C (Table II parameters, q-dependent continuum coupling,
        # non-local level shift of Eq. FE): 40 x 40 basis, 64 incident energies on (0, 5] eV,
        # FP64 COCG with the M^g blocks (spanning d and u), tol 1e-8
        import workloads as w

        gdesc = w.gen_ecd_model(40, 40)
        gmodel = vbk.Model(gdesc)
        geps = w.eps_grid(5.0, 64)
        og = vbk.vbk_default_opts(method="cocg", precision="fp64", precond_span=0x5, tol=1e-8, max_iter=20000,
                                  max_refine=100)
        vbk.vbk_solve(gmodel, geps, vi, og, check=False)
        torch.cuda.synchronize()
        a.record()
        _, stg = vbk.vbk_solve(gmodel, geps, vi, og, check=False)
        b.record()
        b.synchronize()
        extras["generalized_model"] = {
            "value": geps.size / (a.elapsed_time(b) * 1e-3), "unit": UNIT,
            "workload": "Table II model (Sec. II.C), 2 x 40 x 40 (N=3200), 64 energies on (0,5] eV x 2 waves, "
                        "FP64 COCG + M^g, tol 1e-8",
            "converged": all(s["status"] == "converged" for s in stg),
            "iterations_max": int(np.max(stg.iterations))}
        gmodel.close()
        # CPU oracle over all host cores on the whole energy grid of the workload
        pool = OraclePool()
        rate, dt, n_done = pool.rate(eps, vi, eps.size)
        pool.close()
        extras["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": pool.cores, "blas_threads": 1, "kind": "oracle",
                                  "sample": f"{n_done} of 256 energies, sparse LU per energy (both waves), one energy per "
                                            f"process over {pool.cores} processes, {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 Krylov + double-float (2 x f32) refinement residual and solution; f64 output", "data": "synthetic (seeded model, no dataset)",
            "config": {"workload": WORKLOAD_NAME, "method": args.method, "precond_span": args.precond,
                       "inner_tol": args.inner_tol, "restart": args.restart,
                       "l2": "256 MB buffer written between timed steps (outside the step events)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "matvec_hbm_gbs": matvec_gbs,
            "gpu_launches": launches,
            "clocks": clocks,
            "converged": converged, "worst_rel_residual": worst,
            "iterations": {"min": min(iters), "median": float(np.median(iters)), "max": max(iters)},
            "kernel_ms": {k: round(v[1] / n_prof, 3) for k, v in sorted(timings.items(), key=lambda kv: -kv[1][1])},
            "profiled_ms_per_step": round(prof_ms / n_prof, 3),
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
