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


def rank_energies(eps_max, n_per_rank, rank, world):
    """The incident energies rank `rank` of `world` solves: every world-th point, from `rank`, of
    the grid eps_k = eps_max k / (n_per_rank world), k = 1..n_per_rank world.  Each rank gets
    n_per_rank distinct energies spread over the whole range (the same mix of easy and hard
    systems), the ranks together the full grid; at world = 1 it is the workload's own grid."""
    k = np.arange(1, n_per_rank * world + 1, dtype=np.float64)
    return (eps_max * k / (n_per_rank * world))[rank::world].copy()


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
    if name in ("cocg_resident", "solve_resident", "solve_cluster"):
        # one COCG iteration (matvec x in / y out, updates of x, r, p, q, z: (2 + 7) c N) plus the
        # diagonal and reciprocal tables shared by the n_mu waves; p and q stay in shared memory
        # and x, r in L2 across iterations, so DRAM traffic is far below this algorithmic figure.
        # The fused kernels also form the refinement residuals, which this figure leaves out.
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
_ORACLE_DESC = {}


def _oracle_init():
    """Worker set-up: one BLAS/OpenMP thread per process (the energies are the parallel axis)."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _oracle_model(name):
    """The workload's model description, built once per worker process."""
    import workloads as w

    if name not in _ORACLE_DESC:
        _ORACLE_DESC[name] = w.WORKLOADS[name]["model"]()
    return _ORACLE_DESC[name]


def _oracle_energy(args):
    """One (incident energy, initial level) of a workload: A(E) by the oracle, sparse LU, every
    partial wave."""
    from oracle import vibronic as o

    eps_i, vi, name = args if len(args) == 3 else (*args, "ci2d_batched")
    desc = _oracle_model(name)
    E = o.total_energy(desc, float(eps_i), vi)
    o.solve_many(desc, E, [o.phi(desc, E, vi, mu) for mu in range(o.n_partial_waves(desc))])
    return 0


def _oracle_gradient(args):
    """Adjoint-workload loss gradient contribution of one incident energy (the oracle's dense-LU
    adjoint)."""
    from oracle import vibronic as o

    eps_i, vi, vf, target, thetas = args
    desc = _oracle_model("ci2d_adjoint")
    return o.loss_gradient_adjoint(desc, [eps_i], vi, vf, target[None, :], thetas)


def _oracle_init_probe(_):
    from oracle import vibronic  # noqa: F401  (imports numpy / scipy in the worker)

    return 0


class OraclePool:
    """The CPU oracle over all host cores: one process per core (spawned, never forked: the parent
    may already hold a CUDA context), one energy per task."""

    def __init__(self, cores=None):
        import concurrent.futures as cf
        import multiprocessing as mp

        self.cores = cores or os.cpu_count() or 1
        # one BLAS thread per worker, in the environment the spawned workers start with (before
        # their numpy import); the parent's own setting is restored
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})
        try:
            self.ex = cf.ProcessPoolExecutor(max_workers=self.cores, mp_context=mp.get_context("spawn"),
                                             initializer=_oracle_init)
            list(self.ex.map(_oracle_init_probe, range(self.cores)))  # start-up outside the timing
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def rate(self, eps, vi, n_sample, name="ci2d_batched"):
        """Oracle (energy, initial level) points/s on a bounded, evenly spaced sample of the energy
        grid (all of it when n_sample >= its size), for every initial level in vi."""
        idx = np.linspace(0, eps.size - 1, min(n_sample, eps.size)).round().astype(int)
        tasks = [(float(eps[k]), list(v), name) for k in idx for v in vi]
        t0 = time.perf_counter()
        list(self.ex.map(_oracle_energy, tasks))
        dt = time.perf_counter() - t0
        return len(tasks) / dt, dt, len(tasks)

    def map(self, fn, tasks):
        return list(self.ex.map(fn, tasks))

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


# --------------------------------------------------------------- the other configurations
def _timed(fn, reps=1):
    """Device time of fn() (CUDA events on the current stream), best of reps, after one warm-up."""
    import torch

    out = fn()
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        out = fn()
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    return best, out


def _top_kernels(vbk, model, k=5):
    t = vbk.vbk_kernel_timings(model)
    tot = sum(v[1] for v in t.values()) or 1.0
    return {nm: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / tot, 3)}
            for nm, v in sorted(t.items(), key=lambda kv: -kv[1][1])[:k]}


SPAN_STATES_BEND = 0x1 | 0x4 | 0x8  # d, bend x, bend y of the CO2-like model


def level_energy(desc, v):
    """Harmonic level energy E_v = sum_m omega_m (v_m + 1/2) of the neutral (the model's input)."""
    return float(sum(m["omega"] * (k + 0.5) for m, k in zip(desc["modes"], v)))


def open_final_levels(desc, E):
    """Multi-indices v_f with E_vf < E (open final channels), last mode fastest."""
    grids = np.meshgrid(*[np.arange(m["n"]) for m in desc["modes"]], indexing="ij")
    en = sum(m["omega"] * (g + 0.5) for m, g in zip(desc["modes"], grids))
    return [list(map(int, idx)) for idx in np.argwhere(en < E)]


def stencil_points(desc):
    """Largest number of off-diagonal stencil points of a discrete state: per term q^k the offsets
    -k, -k+2, .. k of each mode (their product over modes), the zero offset of a diagonal block
    folded into the diagonal, off-diagonal terms acting in both blocks."""
    import itertools

    count = [0] * desc["n_states"]
    for t in desc["terms"]:
        sets = [range(-k, k + 1, 2) for k in t.get("pow", [0] * len(desc["modes"]))]
        n = sum(1 for off in itertools.product(*sets) if t["d"] != t["dp"] or any(off))
        count[t["d"]] += n
        if t["d"] != t["dp"]:
            count[t["dp"]] += n
    return max(count)


def fp64_peak_tflops():
    """FP64 arithmetic roof of this GPU, measured in this run: cuBLAS DGEMM (torch.mm in float64,
    2048^3), CUDA events around 20 products after 3 untimed ones."""
    import torch

    n, reps = 2048, 20
    gen = torch.Generator(device="cuda").manual_seed(7)
    a = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=gen)
    b = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=gen)
    for _ in range(3):
        torch.mm(a, b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        torch.mm(a, b)
    e1.record()
    torch.cuda.synchronize()
    return 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12


def config_extras(vbk, pool, peaks):
    """Configurations 1, 3, 4 and 5 of the workload list, each timed on the GPU (CUDA events) with
    its dominant kernels (a run with per-kernel timing) and the oracle timed beside it."""
    import torch
    import scipy.linalg as sla
    import workloads as w
    from oracle import vibronic as o

    out = {}
    peak = (peaks or {}).get("hbm_gbs") or 6800.0
    # ---- 1: one energy, 40 x 40 (N = 3200), FP64 GMRES(64) + Jacobi to 1e-10
    spec = w.WORKLOADS["ci2d_single"]
    desc, eps, vi = spec["model"](), spec["eps"], spec["vi"]
    m = vbk.Model(desc)
    o1 = vbk.vbk_default_opts(method="gmres", precision="fp64", precond_span=0, tol=1e-10, restart=64, max_refine=400)
    ms, (_, st) = _timed(lambda: vbk.vbk_solve(m, eps, vi, o1), reps=5)
    vbk.vbk_solve(m, eps, vi, vbk.vbk_default_opts(method="gmres", precision="fp64", precond_span=0, tol=1e-10,
                                                   restart=64, max_refine=400, timing=1))
    E = o.total_energy(desc, float(eps[0]), vi[0])
    A = o.a_matrix(desc, E).toarray()
    rhs = np.stack([o.phi(desc, E, vi[0], mu) for mu in range(o.n_partial_waves(desc))], axis=1)
    t0 = time.perf_counter()
    sla.lu_solve(sla.lu_factor(A), rhs)
    t_lu = time.perf_counter() - t0
    out["config1_single_energy"] = {
        "value": 1.0 / (ms * 1e-3), "unit": UNIT, "ms_per_solve": round(ms, 3),
        "workload": "2 states x 40 x 40 (N=3200), eps_i = 1 eV, v_i = 0, both waves; FP64 GMRES(64) + Jacobi, tol 1e-10",
        "converged": all(x["status"] == "converged" for x in st), "iterations": [int(x) for x in st.iterations],
        "kernel_ms": _top_kernels(vbk, m),
        "bound": "latency: one system whose vectors (51 KB) stay in L2; every Arnoldi step is a chain of dependent "
                 "launches",
        "cpu_baseline": {"value": 1.0 / t_lu, "unit": UNIT, "kind": "oracle", "cores": os.cpu_count(),
                         "blas_threads": "library default", "sample": f"dense LU of A (3200 x 3200), {t_lu:.2f} s"}}
    m.close()
    # ---- 4: uneven batch, 80 x 80, 128 eps_i on (0, 4] x the 4 lowest levels x 2 waves = 1024
    # systems, mixed COCG to 1e-8, then cross sections and the 1 meV EELS spectrum
    spec = w.WORKLOADS["ci2d_uneven"]
    desc, eps = spec["model"](), spec["eps"]
    vi = w.lowest_levels(desc, 4)
    m = vbk.Model(desc)
    o4 = vbk.vbk_default_opts(method="cocg", precision="mixed", precond_span=0, tol=1e-8)
    vf = w.lowest_levels(desc, 24)
    de = np.arange(0.0, 4.0, 0.001)
    psi4 = torch.empty((eps.size, len(vi), m.n_mu, m.N), dtype=torch.complex128, device="cuda")

    def step4():
        p, st_ = vbk.vbk_solve(m, eps, vi, o4, psi=psi4)
        sg = vbk.vbk_cross_sections(m, eps, vi, p, vf)
        return vbk.vbk_eels(m, vi, vf, sg, de), st_

    ms, (_, st) = _timed(step4, reps=3)
    vbk.vbk_solve(m, eps, vi, vbk.vbk_default_opts(method="cocg", precision="mixed", precond_span=0, tol=1e-8, timing=1),
                  psi=psi4)
    rate, dt, nd = pool.rate(eps, vi, 16, "ci2d_uneven")
    out["config4_uneven_batch"] = {
        "value": eps.size * len(vi) / (ms * 1e-3), "unit": UNIT, "ms_per_step": round(ms, 3),
        "workload": "2 x 80 x 80 (N=12800), 128 eps_i on (0,4] eV x 4 lowest levels x 2 waves = 1024 systems, mixed "
                    "COCG tol 1e-8, then cross sections to 24 final levels and the EELS spectrum on a 1 meV grid",
        "converged": all(x["status"] == "converged" for x in st),
        "iterations": {"min": int(st.iterations.min()), "max": int(st.iterations.max())},
        "kernel_ms": _top_kernels(vbk, m),
        "cpu_baseline": {"value": rate, "unit": UNIT, "kind": "oracle", "cores": pool.cores, "blas_threads": 1,
                         "sample": f"{nd} (eps_i, v_i) points (16 energies x 4 levels), sparse LU, {dt:.1f} s"}}
    m.close()
    del psi4
    # ---- 5: adjoint gradient, 40 x 40 with the extra couplings, 256 eps_i, 10 final levels, 19 parameters
    spec = w.WORKLOADS["ci2d_adjoint"]
    desc, eps, vi = spec["model"](), spec["eps"], spec["vi"]
    vf = w.lowest_levels(desc, 10)
    nt = len(desc["terms"])
    thetas = list(range(nt)) + list(range(nt, nt + 2 * len(desc["channels"])))
    target = np.random.default_rng(2307134831).uniform(0.0, 1.0, (eps.size, len(vf)))
    tgt = torch.tensor(target[:, None, :], device="cuda")
    m = vbk.Model(desc)
    o5 = vbk.vbk_default_opts(method="cocg", precision="mixed", tol=1e-10, max_refine=100)

    def step5():
        p, _ = vbk.vbk_solve(m, eps, vi, o5)
        sg = vbk.vbk_cross_sections(m, eps, vi, p, vf)
        g, st_ = vbk.vbk_solve_adjoint(m, eps, vi, p, vf, 2.0 * (sg - tgt), thetas, o5)
        return g, st_

    ms, (g5, st) = _timed(step5, reps=3)
    sample = np.linspace(0, eps.size - 1, 16).round().astype(int)
    t0 = time.perf_counter()
    pool.map(_oracle_gradient, [(float(eps[k]), vi[0], vf, target[k], thetas) for k in sample])
    dt = time.perf_counter() - t0
    out["config5_adjoint"] = {
        "value": eps.size / (ms * 1e-3), "unit": UNIT, "ms_per_gradient": round(ms, 3),
        "workload": "2 x 40 x 40 with cubic / bilinear couplings (N=3200), 256 eps_i on (0,3] eV, 10 final levels, "
                    "L = sum (sigma - target)^2, gradient in 19 parameters: forward solves, cross sections, adjoint "
                    "solves and contractions (mixed COCG, tol 1e-10)",
        "adjoint_converged": all(x["status"] in ("converged", "zero_rhs") for x in st), "n_theta": len(thetas),
        "cpu_baseline": {"value": sample.size / dt, "unit": UNIT, "kind": "oracle", "cores": pool.cores,
                         "blas_threads": 1,
                         "sample": f"{sample.size} energies, dense-LU adjoint gradient per energy, {dt:.1f} s"}}
    m.close()
    # ---- 3: CO2-like, 3 states x 30 x 20 x 20 x 12 (N = 432,000), eps_i = 3 eV, three waves,
    # states x bend blocks: FP64 COCG, and mixed GMRES(256) (FP32 Arnoldi inside FP64 refinement)
    spec = w.WORKLOADS["co2_like"]
    desc, eps, vi = spec["model"](), spec["eps"], spec["vi"]
    m = vbk.Model(desc)
    res3 = {}
    for key, kw in (("fp64_cocg", dict(method="cocg", precision="fp64")),
                    ("mixed_gmres256", dict(method="gmres", precision="mixed", restart=256))):
        oc = vbk.vbk_default_opts(precond_span=SPAN_STATES_BEND, tol=1e-8, max_iter=20000, max_refine=100, **kw)
        ms, (_, st) = _timed(lambda: vbk.vbk_solve(m, eps, vi, oc, check=False), reps=1)
        res3[key] = {"seconds": round(ms * 1e-3, 3), "converged": all(x["status"] == "converged" for x in st),
                     "iterations": [int(x) for x in st.iterations],
                     "rel_residual_max": float(st.rel_residual.max())}
    ot = vbk.vbk_default_opts(method="cocg", precision="fp64", precond_span=SPAN_STATES_BEND, tol=1e-8, max_iter=20000,
                              max_refine=100, timing=1)
    _, stt = vbk.vbk_solve(m, eps, vi, ot, check=False)
    kt = vbk.vbk_kernel_timings(m)
    iters = int(stt.iterations.max())
    la = kt.get("block_apply_wide")
    roof3 = None
    if la and la[0] > 0:
        # level-blocked L D L^T apply: r in, z out per system, the factor levels once per energy
        # (shared by the 3 waves): 5 S x S blocks per level, K = L / S levels per block
        nb, L_blk, p_half = 30 * 12, 3 * 20 * 20, 120
        S_lv = 4 * ((p_half + 7) // 8)
        K = (L_blk + S_lv - 1) // S_lv
        factor_bytes = nb * K * 5 * S_lv * S_lv * 16
        per_launch = 3 * 2 * 16 * m.N + factor_bytes
        ach = per_launch * la[0] / (la[1] * 1e-3) / 1e9
        # FP64 arithmetic of one apply: per system and block 5 K - 6 products of an S x S complex
        # level block with a vector (K levels: D_k^-1, L_{k,k-1}, L_{k,k-2} forward, their
        # transposes backward), 8 flops per complex multiply-add
        flops = 3 * nb * (5 * K - 6) * S_lv * S_lv * 8
        tf = flops * la[0] / (la[1] * 1e-3) / 1e12
        fp64_peak = (peaks or {}).get("fp64_tflops_measured")
        roof3 = {"kernel": "block_apply_wide", "bound": "fp64", "achieved": round(tf, 3), "peak": fp64_peak,
                 "unit": "TFLOP/s", "frac": round(tf / fp64_peak, 4) if fp64_peak else None,
                 "flops_per_launch": int(flops), "peak_source": "cuBLAS DGEMM timed in this run",
                 "hbm": {"achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                         "bytes_per_launch": int(per_launch)},
                 "launches": la[0], "avg_launch_us": round(la[1] * 1e3 / la[0], 1)}
    # the oracle on a reduced basis (sparse LU at 12 x 8 x 8 x 6, N = 13,824)
    rdesc = w.co2_like_model(basis=(12, 8, 8, 6))
    E = o.total_energy(rdesc, 3.0, [0, 0, 0, 0])
    t0 = time.perf_counter()
    o.solve_many(rdesc, E, [o.phi(rdesc, E, [0, 0, 0, 0], mu) for mu in range(3)])
    t_red = time.perf_counter() - t0
    best = min(res3.values(), key=lambda r: r["seconds"])
    out["config3_co2_like"] = {
        "value": 1.0 / best["seconds"], "unit": UNIT,
        "workload": "CO2-like: 3 states x 30 x 20 x 20 x 12 (N=432,000), eps_i = 3 eV, v_i = 0, 3 waves, blocks over "
                    "states x 2D bend (1200 unknowns, half bandwidth 120), tol 1e-8",
        "solves": res3, "per_iteration_ms": round(sum(v[1] for v in kt.values()) / max(1, iters), 3),
        "kernel_ms": _top_kernels(vbk, m, 8), "roofline": roof3,
        "cpu_baseline": {"value": 1.0 / t_red, "unit": UNIT, "kind": "oracle", "cores": 1,
                         "sample": f"reduced basis 12 x 8 x 8 x 6 (N=13,824), sparse LU, 3 waves, {t_red:.1f} s "
                                   "(the full 4D LU does not fit the host)"}}
    m.close()
    return out


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
    ap.add_argument("--resident", type=int, default=1,
                    help="1: fused one-CTA solve, 2: one-CTA inner solves between host checks, 3: clusters, 0: grid-wide")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 comparisons and the CPU baseline")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workload configurations")
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

    desc, eps, vi = workload()
    if world > 1:  # distinct energies per rank (weak scaling: 256 per rank), no data-path collective
        eps = rank_energies(3.0, eps.size, rank, world)
    model = vbk.Model(desc)
    N, nmu = model.N, model.n_mu
    opts = vbk.vbk_default_opts(method=args.method, precision="mixed", precond_span=args.precond, tol=1e-8,
                                restart=args.restart, inner_tol=args.inner_tol, max_refine=100, resident=args.resident)
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
                                       restart=args.restart, inner_tol=args.inner_tol, max_refine=100, timing=1,
                                       resident=args.resident)
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
        E_tot = np.array([float(e) + level_energy(desc, vi[0]) for e in eps])
        gen = torch.Generator(device="cuda").manual_seed(2307)
        xm = torch.complex(torch.randn((eps.size, nvec, N), device="cuda", dtype=torch.float64, generator=gen),
                           torch.randn((eps.size, nvec, N), device="cuda", dtype=torch.float64, generator=gen))
        vbk.vbk_set_op_timing(model, True)
        for prec, c, name in ((vbk.VBK_MIXED, 8, "fp32"), (vbk.VBK_FP64, 16, "fp64")):
            per_var = {}
            for v in range(vbk.VBK_MATVEC_NVARIANTS):
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
        # the FP64 operator against the FP64 arithmetic roof (GB300 runs FP64 far below FP32):
        # per element and system 6 flops for the diagonal product and 4 per stencil point
        fp64_peak = fp64_peak_tflops()
        peaks = dict(peaks or {}, fp64_tflops_measured=fp64_peak)
        if "kernel_us" in matvec_gbs.get("fp64", {}):
            npts = stencil_points(desc)
            flops = (6 + 4 * npts) * N * eps.size * nvec
            tf = flops / (matvec_gbs["fp64"]["kernel_us"] * 1e-6) / 1e12
            matvec_gbs["fp64"]["alu"] = {"bound": "fp64", "achieved": round(tf, 3), "peak": round(fp64_peak, 3),
                                         "unit": "TFLOP/s", "frac": round(tf / fp64_peak, 4),
                                         "flops_per_unit": f"6 + 4 x {npts} stencil points per element and system",
                                         "peak_source": "cuBLAS DGEMM timed in this run"}
        matvec_gbs["bytes_per_unit"] = "(2c + c/6) N per system: x in, y out, the diagonal once per energy (6 vectors each)"
        matvec_gbs["peak_source"] = "measured" if (peaks or {}).get("hbm_gbs") else "fallback"

    extras = {}
    if not args.no_extras and rank == 0:
        # end to end through the public API: host energies in, cross sections back to the host
        vf = open_final_levels(desc, float(eps[-1]) + level_energy(desc, vi[0]))
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
        if not args.no_configs:
            extras["configs"] = config_extras(vbk, pool, peaks)
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
                       "resident": args.resident,
                       "inner_tol": args.inner_tol, "restart": args.restart,
                       "l2": "256 MB buffer written between timed steps (outside the step events)",
                       "parallelism": f"energies split over {world} rank(s), 256 each" if world > 1 else "1 GPU"},
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
