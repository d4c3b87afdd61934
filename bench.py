"""Benchmark: H·X throughput of the tight-binding Hamiltonian on the 1M-atom SiGe alloy.

Workload: Si0.7Ge0.3 random alloy of 50^3 conventional cells (1,000,000 atoms), hard walls,
bond lengths strained by U[-2%, 2%] with Harrison d^-2 scaling, sp3d5s* (10 orbitals, 10M
rows), seeded synthetic parameters.  One step = one application of the folded-spectrum
operator (H - sigma)^2 to a vector, i.e. two H·X products — the unit the folded-spectrum
Lanczos recurrence repeats (the paper times "500 Lanczos iterations").

value = algorithmic bytes of the H·X products of all ranks / max-over-ranks time (GB/s).
Algorithmic bytes per H·X: every stored bond block once (100 entries per bond), x and y once,
one species byte and one potential word per atom.

--impl reference: the CPU oracle (scipy CSR product from oracle/) on a bounded sample of the
same workload, on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "H·X GB/s vs HBM peak; s to 16 eigenpairs at 1M atoms; SCF time vs plain"
UNIT = "GB/s"
N_CELLS = 50
SAMPLE_NZ = 4          # CPU sample: 50 x 50 x 4 cells of the same recipe
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate (reported beside the DGEMM rate measured in the run)


# DRAM bytes (read + write) per bond of one FP64 stored H·X launch, by launch shape (CTA width,
# block rows per register batch): ncu capture of every shape on the 30^3-cell case of the alloy
# recipe (profiles/hx_kernel_f64_shapes_sige_alloy.md), scaled to a launch by its bonds
HX_F64_TRAFFIC_PER_BOND = {(32, 1): 1203.0, (32, 2): 922.4, (64, 1): 1190.2, (64, 2): 917.9, (96, 1): 1160.4,
                           (96, 2): 924.9, (128, 1): 1151.1, (128, 2): 917.2}
HX_F64_TRAFFIC_SOURCE = ("profiles/hx_kernel_f64_shapes_sige_alloy.md: ncu dram__bytes of each launch shape "
                         "at 30^3 cells, per bond x this launch's bonds")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def max_over_ranks(value, dist, device):
    """The slowest rank's time (the job's time) — every rank gets the same value."""
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, bytes_per_step, steps, seconds):
    """Whole-job throughput of weakly scaled replicas: all ranks' bytes over the slowest time."""
    return world * bytes_per_step * steps / seconds / 1e9


def alg_bytes_per_hx(nbonds, natoms, nrows, elem, vec_elem, matrix_free):
    h = 0 if matrix_free else nbonds * 100 * elem
    extra = natoms * (1 + 8) + (nbonds * 8 if matrix_free else 0)
    return h + 2 * nrows * vec_elem + extra


def flops_per_hx(nbonds, natoms, norb=10):
    return 2.0 * (2 * norb * norb * nbonds + norb * natoms)


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, max, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(tempfile.gettempdir(), f"omen_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload_config(cells, natoms, nbonds, rows, matrix_free, world):
    """The workload description both arms print (the reference arm times a bounded sample of it)."""
    return {"workload": f"Si0.7Ge0.3 alloy {cells}^3 cells ({natoms:,} atoms), hard wall, 2% bond "
                        "strain, sp3d5s*; step = folded operator (H-sigma)^2 x (two H·X)",
            "atoms": natoms, "bonds": nbonds, "rows": rows,
            "storage": "matrix-free" if matrix_free else "stored bond blocks",
            "l2": "no flush: H blocks exceed L2", "parallelism": f"replicas x{world}"}


def cpu_sample(seed=2):
    """Bounded CPU sample of the same recipe: 50 x 50 x SAMPLE_NZ cells, oracle CSR."""
    from oracle import hamiltonian
    spec = synth.lattice_spec(N_CELLS, N_CELLS, SAMPLE_NZ, (0, 0, 0), seed=seed, alloy_fraction=0.3, strain_amp=0.02)
    p = synth.draw_tb_params(seed, synth.SP3D5S, 2)
    H = hamiltonian.assemble(spec, p).tocsr()
    H.sort_indices()
    from oracle import lattice
    nb = len(lattice.find_bonds(spec.nx, spec.ny, spec.nz, spec.periodic).a)
    return spec, H, nb


def sample_config(spec, nb, H):
    return {"workload": f"Si0.7Ge0.3 alloy slab {spec.nx}x{spec.ny}x{spec.nz} cells ({spec.natoms:,} atoms) of the "
                        f"{N_CELLS}^3-cell recipe, hard wall, 2% bond strain, sp3d5s*; step = folded operator "
                        "(H-sigma)^2 x (two H·X)",
            "atoms": spec.natoms, "bonds": nb, "rows": H.shape[0], "nnz": int(H.nnz), "storage": "oracle CSR (FP64)",
            "parallelism": "host cores"}


def time_cpu_oracle(H, nbonds, natoms, min_seconds=10.0, min_steps=3, threads=0, sigma=0.3):
    """The oracle's folded-operator step (H - sigma)^2 x on the host cores: the plain OpenMP CSR
    loop of oracle/csr_matvec.c over `threads` threads (0 = all), steps repeated until
    min_seconds have passed.  Returns (GB/s algorithmic, seconds, steps, threads)."""
    from oracle import spmv
    nthr = threads or spmv.max_threads()
    x = synth.random_vectors(1, H.shape[0])[0]
    t = np.empty_like(x)
    y = np.empty_like(x)
    spmv.matvec(H, x, nthr, out=t)
    steps, t0 = 0, time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < min_seconds:
        spmv.matvec(H, x, nthr, out=t)
        t -= sigma * x
        spmv.matvec(H, t, nthr, out=y)
        y -= sigma * t
        steps += 1
    dt = time.perf_counter() - t0
    alg = 2 * alg_bytes_per_hx(nbonds, natoms, H.shape[0], 8, 8, False) * steps
    return alg / dt / 1e9, dt, steps, nthr


def time_cpu_scipy(H, nbonds, natoms, steps=5, sigma=0.3):
    """The same step with scipy's single-threaded CSR product (the oracle's own H @ x)."""
    x = synth.random_vectors(1, H.shape[0])[0]
    t0 = time.perf_counter()
    for _ in range(steps):
        t = H @ x - sigma * x
        H @ t - sigma * t
    dt = time.perf_counter() - t0
    return 2 * alg_bytes_per_hx(nbonds, natoms, H.shape[0], 8, 8, False) * steps / dt / 1e9


def run_reference(args, rank, world):
    if rank != 0:
        return
    t0 = time.perf_counter()
    spec, H, nb = cpu_sample()
    build_s = time.perf_counter() - t0
    time_cpu_oracle(H, nb, spec.natoms, min_seconds=0.0, min_steps=max(1, args.warmup))
    v, dt, steps, nthr = time_cpu_oracle(H, nb, spec.natoms, min_seconds=0.0, min_steps=args.steps)
    sample = (f"oracle CSR product (oracle/csr_matvec.c, OpenMP over {nthr} threads) of (H-sigma)^2 x on the "
              f"50x50x{SAMPLE_NZ}-cell slab named in config ({H.shape[0]} rows, {H.nnz} nnz), {steps} steps in "
              f"{dt:.2f} s; CSR assembly {build_s:.1f} s not timed")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            # the slab actually timed (the GPU arm's workload is the full 50^3-cell block of the
            # same recipe; GB/s counts the same algorithmic bytes per row and bond)
            "config": sample_config(spec, nb, H),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nthr, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_variants(ctx, omen, lat, p, natoms, nbonds, reps=50):
    """One H·X per variant (same workload): ms and algorithmic GB/s."""
    import torch
    out = {}
    for name, prec, mf, so in (("f64", omen.OMEN_F64, False, False), ("f64_df", omen.OMEN_F64_DF, False, False),
                               ("f32", omen.OMEN_F32, False, False), ("f32_matrix_free", omen.OMEN_F32, True, False),
                               ("c64_spin_orbit", omen.OMEN_F32, False, True)):
        ham = omen.omen_assemble_H(ctx, lat, p, precision=prec, matrix_free=mf, spin_orbit=so)
        el = 4 if prec == omen.OMEN_F32 else 8
        vel = el * (2 if so else 1)
        x = torch.zeros(ham.nrows * vel // 4, dtype=torch.float32, device="cuda")
        y = torch.empty_like(x)

        def timed():
            for _ in range(3):
                omen.omen_hx(ctx, ham, x, y)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                omen.omen_hx(ctx, ham, x, y)
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        ms = timed()
        alg = alg_bytes_per_hx(nbonds, natoms, ham.nrows, el, vel, mf)
        out[name] = {"ms": ms, "alg_GB": alg / 1e9, "GB_per_s": alg / ms / 1e6}
        if prec != omen.OMEN_F64_DF:
            tile = omen.omen_tune_hx(ctx, ham, prec, nvec=1, reps=5)
            mst = timed()
            out[name].update({"tuned_shape": [tile["threads"], tile["rows_per_batch"]], "tuned_ms": mst,
                              "tuned_GB_per_s": alg / mst / 1e6})
        del ham, x, y
    return out


def measure_lanczos(ctx, omen, ham, iters=500, basis=64):
    """The paper's benchmark unit (Section II-B): wall time of 500 Lanczos iterations, with the
    default full Gram–Schmidt update at every step, with the semi-orthogonal policy (overlaps
    measured every step) and with partial reorthogonalisation (overlaps estimated)."""
    import torch
    out = {}
    for name, pol in (("full_update", omen.OMEN_REORTH_FULL), ("semi_orthogonal", omen.OMEN_REORTH_SEMI),
                      ("partial_reorthogonalization", omen.OMEN_REORTH_PARTIAL)):
        omen.omen_set_reorthogonalization(ctx, pol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, info, st = omen.omen_eigs(ctx, ham, 16, omen.OMEN_LOWEST, tol=1e-30, block=1, basis=basis,
                                      max_iter=iters, raise_on_noconv=False)
        torch.cuda.synchronize()
        out[name] = {"iterations": info["iterations"], "seconds": time.perf_counter() - t0, "basis": basis,
                     "hx_count": info["hx_count"], "lowest": float(ev[0])}
    omen.omen_set_reorthogonalization(ctx, omen.OMEN_REORTH_FULL)
    return out


def measure_eigs_1m(ctx, omen, lat, p, nev=16, only=None):
    """Seconds to nev converged eigenpairs at 1M atoms (lowest end of the spectrum, where the
    thick-restart Lanczos converges): FP64; FP64-accurate double-float Krylov vectors on the FP32
    pipe; and spin-orbit complex64 + FP64 refinement."""
    import torch
    out = {}
    variants = [("f64", False, omen.OMEN_F64, 1e-9), ("f64_double_float", False, omen.OMEN_F64_DF, 1e-9),
                ("so_f32_refine64", True, omen.OMEN_F32_REFINE64, 1e-8)]
    if only == "so-all":
        # the spin-orbit precision comparison: raw complex64, complex64 + FP64 refinement, and
        # the complex128 solve as the reference for both
        variants = [("so_f64", True, omen.OMEN_F64, 1e-9), ("so_f32_raw", True, omen.OMEN_F32, 1e-5),
                    ("so_f32_refine64", True, omen.OMEN_F32_REFINE64, 1e-8)]
    evs = {}
    for name, so, prec, tol in variants:
        if only and only != "so-all" and name != only:
            continue
        ham = omen.omen_assemble_H(ctx, lat, p, spin_orbit=so, precision=prec)
        if name.endswith("partial_reorth"):
            omen.omen_set_reorthogonalization(ctx, omen.OMEN_REORTH_PARTIAL)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, info, st = omen.omen_eigs(ctx, ham, nev, omen.OMEN_LOWEST, tol=tol, block=1 if not so else 2,
                                      basis=96, max_iter=6000, raise_on_noconv=False)
        torch.cuda.synchronize()
        omen.omen_set_reorthogonalization(ctx, omen.OMEN_REORTH_FULL)
        out[name] = {"seconds": time.perf_counter() - t0, "converged": info["converged"], "tol_eV": tol,
                     "iterations": info["iterations"], "hx_count": info["hx_count"],
                     "max_error_bound": info["max_error_bound"], "max_residual_raw": info["max_residual_raw"],
                     "max_residual": info["max_residual"], "lowest": float(ev[0])}
        evs[name] = np.array(ev)
        if "so_f64" in evs and name != "so_f64":
            out[name]["max_abs_diff_vs_f64_eV"] = float(np.abs(evs[name] - evs["so_f64"]).max())
            out[name]["time_vs_f64"] = out[name]["seconds"] / out["so_f64"]["seconds"]
        del ham
    return out


def m2_sigma(ctx, omen, ham, seed=2):
    """The folded-spectrum shift of the alloy recipe: centre of the spectrum plus a seeded
    offset of up to 5% of its width, rounded to 1 meV (extremes from short Lanczos solves)."""
    lo, _, _ = omen.omen_eigs(ctx, ham, 1, omen.OMEN_LOWEST, tol=1e-4, block=1, basis=32, max_iter=2000,
                              raise_on_noconv=False)
    hi, _, _ = omen.omen_eigs(ctx, ham, 1, omen.OMEN_HIGHEST, tol=1e-4, block=1, basis=32, max_iter=2000,
                              raise_on_noconv=False)
    lo, hi = float(lo[0]), float(hi[0])
    return round(0.5 * (lo + hi) + synth.sigma_offset_fraction(seed) * (hi - lo), 3), lo, hi


def measure_m2_ladder(ctx, omen, sizes=(4, 5, 6, 8, 10), big=50, big_iters=2000, nev=16):
    """16 eigenpairs nearest a mid-spectrum shift by folded-spectrum Lanczos on the alloy recipe
    at growing sizes: iterations and time to the 1e-9 eV bound.  The folded gap of the 16th/17th
    pair shrinks as the square of the level spacing (~ width / rows), so the iteration count of a
    Krylov method grows about linearly with the rows; the largest size is run for a fixed budget
    and its residual recorded."""
    import torch
    out = []
    for n in list(sizes) + [big]:
        spec, p = synth.config_sige_alloy(n, seed=2)
        lat = omen.omen_build_lattice(ctx, spec)
        ham = omen.omen_assemble_H(ctx, lat, p)
        sigma, lo, hi = m2_sigma(ctx, omen, ham)
        cap = big_iters if n == big else 400000
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, info, st = omen.omen_eigs(ctx, ham, nev, omen.OMEN_NEAREST, sigma=sigma, tol=1e-9, block=1, basis=64,
                                      max_iter=cap, raise_on_noconv=False)
        torch.cuda.synchronize()
        ev = np.sort(np.asarray(ev))
        out.append({"cells": n, "rows": ham.nrows, "sigma": sigma, "spectrum": [lo, hi], "converged": info["converged"],
                    "iterations": info["iterations"], "hx_count": info["hx_count"], "restarts": info["restarts"],
                    "seconds": time.perf_counter() - t0, "max_residual": info["max_residual"],
                    "max_error_bound": info["max_error_bound"],
                    "mean_spacing_eV": float((ev[-1] - ev[0]) / (nev - 1))})
        print(json.dumps(out[-1]), flush=True)
        del ham, lat
    return out


def measure_charge_poisson(ctx, omen, lat, ham, spec, nstates=16, ng=256):
    """Rows a9-a12 at the 1M-atom scale: electrons per atom from nstates FP64 eigenvectors
    (omen_density_accum), cloud-in-cell deposit of the atom charges on an ng x ng x ng grid over the
    structure, the FP64 CG Poisson solve on that grid, and the trilinear gather back to the atoms.
    Algorithmic bytes: the eigenvectors once (density); per CG iteration 8 words per unknown
    (stencil input once, product written, x, r, p read and written)."""
    import torch
    from oracle import poisson  # grid description only (no computation)
    L = spec.nx * spec.a_nm
    grid = poisson.Grid(ng, ng, ng + 1, L, L, L)
    n = ham.nrows
    psi = torch.rand(nstates * n, dtype=torch.float64, device="cuda") - 0.5
    occ = np.linspace(1.0, 0.0, nstates)
    n_atom = torch.zeros(spec.natoms, dtype=torch.float64, device="cuda")
    out = {"grid": [grid.nx, grid.ny, grid.nz], "unknowns": grid.nx * grid.ny * (grid.nz - 1)}

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    t = timed(lambda: omen.omen_density_accum(ctx, ham, psi, nstates, occ, 1.0, n_atom))
    out["density_accum"] = {"states": nstates, "ms": t * 1e3, "GB_per_s": nstates * n * 8 / t / 1e9}
    q = (n_atom * -1.602176634e-19).contiguous()
    rho = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    t = timed(lambda: omen.omen_deposit(ctx, lat, grid, q, rho))
    out["deposit"] = {"ms": t * 1e3}
    phi = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    rho_s = rho + 1e6 * torch.rand(grid.shape, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = omen.omen_poisson(ctx, grid, rho_s, phi, rtol=1e-8, max_iter=50000)
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    nu = out["unknowns"]
    out["poisson_cg"] = {"iterations": info["iterations"], "seconds": tp, "ms_per_iteration": tp / info["iterations"] * 1e3,
                         "GB_per_s": 8 * 8 * nu * info["iterations"] / tp / 1e9, "rel_residual": info["rel_residual"]}
    # FP32 iterations, FP64 residual replacement: 7 FP32 words per unknown per iteration (stencil
    # input once; correction d, residual r and direction p read and written)
    phi32 = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = omen.omen_poisson(ctx, grid, rho_s, phi32, rtol=1e-8, max_iter=50000, precision=omen.OMEN_F32_REFINE64)
    torch.cuda.synchronize()
    tm = time.perf_counter() - t0
    out["poisson_cg_mixed"] = {"iterations": info["iterations"], "seconds": tm,
                               "ms_per_iteration": tm / info["iterations"] * 1e3,
                               "GB_per_s": 7 * 4 * nu * info["iterations"] / tm / 1e9,
                               "rel_residual": info["rel_residual"], "speedup_vs_fp64": tp / tm,
                               "max_abs_diff_vs_fp64_V": float((phi32 - phi).abs().max()),
                               "max_abs_phi_V": float(phi.abs().max())}
    del phi32
    phi_atom = torch.empty(spec.natoms, dtype=torch.float64, device="cuda")
    t = timed(lambda: omen.omen_gather(ctx, lat, grid, phi, phi_atom))
    out["gather"] = {"ms": t * 1e3}
    del psi
    return out


def measure_small_si(ctx, omen, n=8, nev=8):
    """Bulk Si 8^3 cells, periodic, sp3s* (20,480 rows, FP64): seconds to the 8 lowest
    eigenpairs at 1e-9 eV — single-vector Lanczos with and without graph replay of the steps,
    and block Lanczos (b = 8).  At this size every kernel is a few microseconds long, so the
    launch path, not HBM, sets the pace."""
    import torch
    spec, p = synth.config_si_periodic(n, seed=1)
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, p)
    out = {"rows": ham.nrows}
    for name, block, graphs in (("single_graphs", 1, True), ("single_direct", 1, False), ("block8", 8, True)):
        omen.omen_set_graph_capture(ctx, graphs)
        best = None
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev, info, st = omen.omen_eigs(ctx, ham, nev, omen.OMEN_LOWEST, tol=1e-9, block=block, basis=64,
                                          max_iter=4000, raise_on_noconv=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        out[name] = {"seconds": best, "iterations": info["iterations"], "converged": info["converged"],
                     "max_error_bound": info["max_error_bound"],
                     "ms_per_iteration": 1e3 * best / max(1, info["iterations"])}
    omen.omen_set_graph_capture(ctx, True)
    return out


def measure_cube_500(ctx, omen, n=80, iters=500):
    """The paper's 3-D benchmark unit (Section II-B, Fig. 3): 500 Lanczos iterations on a Si
    cube of 80^3 conventional cells (4,096,000 atoms, sp3d5s*, hard wall), FP64 and FP32."""
    import torch
    spec = synth.lattice_spec(n, n, n, (0, 0, 0), seed=11)
    p = synth.draw_tb_params(11, 10, 1)
    lat = omen.omen_build_lattice(ctx, spec)
    out = {"atoms": spec.natoms}
    for name, prec in (("f64", omen.OMEN_F64), ("f32", omen.OMEN_F32)):
        ham = omen.omen_assemble_H(ctx, lat, p, precision=prec)
        out[name] = measure_lanczos(ctx, omen, ham, iters=iters)
        out["rows"] = ham.nrows
        del ham
        torch.cuda.empty_cache()
    return out


def measure_hx_kbatch(ctx, omen, nxy=4, nz=80, nk=32, seed=7, reps=20):
    """The k-batched product alone: all nk wave vectors of the 4x4x80-cell delta layer per launch
    (complex64), default launch shape; also the profiling target of that kernel."""
    import torch
    spec = synth.lattice_spec(nxy, nxy, nz, (2, 2, 0), seed=seed)
    lam = synth.draw_kbatch_instances(seed)[0][2]
    U = synth.donor_sheet_potential(spec, seed, lam)
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, synth.gapped_si_params(), precision=omen.OMEN_F32, k=(0.0, 0.0, 0.0),
                               U_atom_dev=torch.from_numpy(U).cuda())
    ks = np.zeros((nk, 3))
    ks[:, 0] = np.linspace(0.0, 1.0, nk) * np.pi / (nxy * spec.a_nm)
    x = torch.ones(nk * ham.nrows, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        omen.omen_hx_kbatch(ctx, ham, ks, x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        omen.omen_hx_kbatch(ctx, ham, ks, x, y)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbonds = lat.counts()[1]
    # blocks (FP32) once per launch, complex64 vectors read and written once per k
    alg = nbonds * 100 * 4 + nk * ham.nrows * 8 * 2 + spec.natoms * 9
    return {"rows": ham.nrows, "k": nk, "ms": ms, "alg_GB": alg / 1e9, "GB_per_s": alg / ms / 1e6}


def measure_effmass(ctx, omen, n=256, reps=50, n_eig=64, nev=16):
    """The effective-mass product (7-point stencil) on an n^3 grid of Si conduction-band
    masses (periodic x, y; hard walls in z), FP64 / FP32 / complex (Bloch) vectors, one and four
    per launch; then the 16 lowest levels of an n_eig^3 box with a seeded random potential."""
    import torch
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    out = {"grid": [n, n, n], "points": n ** 3}
    for name, prec, bloch, nvec in (("f64", omen.OMEN_F64, False, 1), ("f32", omen.OMEN_F32, False, 1),
                                    ("c128_bloch", omen.OMEN_F64, True, 1), ("f64_4_vectors", omen.OMEN_F64, False, 4)):
        spec = synth.effmass_spec(n, n, n, seed=3, periodic=(2, 2, 0) if bloch else (1, 1, 0),
                                  kvec=(0.4, -0.3, 0.0) if bloch else None)
        ham = omen.omen_assemble_effmass(ctx, spec, precision=prec, U_dev=torch.from_numpy(spec.U).cuda())
        el = (4 if prec == omen.OMEN_F32 else 8) * (2 if bloch else 1)
        x = torch.ones(nvec * ham.nrows * el // 4, dtype=torch.float32, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            omen.omen_hx(ctx, ham, x, y, nvec=nvec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            omen.omen_hx(ctx, ham, x, y, nvec=nvec)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        # x read once and y written once per vector, the potential once per launch
        alg = nvec * 2 * el * ham.nrows + (4 if prec == omen.OMEN_F32 else 8) * ham.nrows
        out[name] = {"ms": ms, "alg_GB": alg / 1e9, "GB_per_s": alg / ms / 1e6,
                     "frac_of_measured_hbm": alg / ms / 1e6 / hbm}
        del ham, x, y
    spec = synth.effmass_spec(n_eig, n_eig, n_eig, seed=5, u_amp=0.05)
    ham = omen.omen_assemble_effmass(ctx, spec, U_dev=torch.from_numpy(spec.U).cuda())
    t0 = time.perf_counter()
    ev, info, _ = omen.omen_eigs(ctx, ham, nev, tol=1e-9, block=1, basis=64, max_iter=20000)
    out[f"eigs_{nev}_lowest_{n_eig}cubed_box"] = {
        "seconds": time.perf_counter() - t0, "converged": info["converged"], "iterations": info["iterations"],
        "hx_count": info["hx_count"], "max_error_bound": info["max_error_bound"], "lowest": float(ev[0])}
    return out


def measure_kbatch(ctx, omen, nxy=4, nz=80, nk=32, nev=8, seed=7):
    """Bands/s of the lockstep k-batched solve against one solve per k (same solver, nk = 1)."""
    import torch
    spec = synth.lattice_spec(nxy, nxy, nz, (2, 2, 0), seed=seed)
    p = synth.gapped_si_params()
    lam = synth.draw_kbatch_instances(seed)[0][2]
    U = synth.donor_sheet_potential(spec, seed, lam)
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, p, precision=omen.OMEN_F32, k=(0.0, 0.0, 0.0),
                               U_atom_dev=torch.from_numpy(U).cuda())
    ks = np.zeros((nk, 3))
    ks[:, 0] = np.linspace(0.0, 1.0, nk) * np.pi / (nxy * spec.a_nm)
    out = {"workload": f"delta-doped Si {nxy}x{nxy}x{nz} cells ({spec.natoms} atoms), donor sheet lambda_TF "
                       f"{lam:.2f} nm, sp3d5s* complex64, {nk} k along Gamma-X, {nev} bands per k"}
    out["tile_batched"] = omen.omen_tune_hx_kbatch(ctx, ham, nk, reps=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev, info, st = omen.omen_eigs_kbatch(ctx, ham, ks, nev, tol=1e-6, max_iter=20000, basis=64, raise_on_noconv=False)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    out["tile_per_k"] = omen.omen_tune_hx_kbatch(ctx, ham, 1, reps=5)
    t0 = time.perf_counter()
    for q in range(nk):
        ev1, _, _ = omen.omen_eigs_kbatch(ctx, ham, ks[q:q + 1], nev, tol=1e-6, max_iter=20000, basis=64,
                                          raise_on_noconv=False)
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    out["lowest"] = {"bands_per_s_batched": nk * nev / tb, "bands_per_s_per_k": nk * nev / tp,
                     "speedup": tp / tb, "converged": info["converged"], "max_residual": info["max_residual"]}
    # folded spectrum near the conduction-band edge, fixed step budget (does not converge here)
    steps = 200
    sigma = synth.GAPPED_SI_EC - 0.2
    omen.omen_tune_hx_kbatch(ctx, ham, nk, reps=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    omen.omen_eigs_kbatch(ctx, ham, ks, nev, which=omen.OMEN_NEAREST, sigma=sigma, tol=1e-12, max_iter=steps,
                          basis=64, raise_on_noconv=False)
    torch.cuda.synchronize()
    fb = time.perf_counter() - t0
    nper = 4
    omen.omen_tune_hx_kbatch(ctx, ham, 1, reps=5)
    t0 = time.perf_counter()
    for q in range(nper):
        omen.omen_eigs_kbatch(ctx, ham, ks[q:q + 1], nev, which=omen.OMEN_NEAREST, sigma=sigma, tol=1e-12,
                              max_iter=steps, basis=64, raise_on_noconv=False)
    torch.cuda.synchronize()
    fp = (time.perf_counter() - t0) / nper * nk
    out["folded_fixed_steps"] = {"steps": steps, "k_steps_per_s_batched": nk * steps / fb,
                                 "k_steps_per_s_per_k": nk * steps / fp, "speedup": fp / fb,
                                 "per_k_time": f"extrapolated from {nper} of {nk} wave vectors"}
    return out


def c5_kpoints(L):
    """The 4 x 4 Monkhorst-Pack mesh of the lateral zone, halved by time reversal (H(-k) is the
    complex conjugate of H(k)): 8 wave vectors (1/nm), weight 1/8 each."""
    ks = [(i / 8 * 2 * np.pi / L, j / 8 * 2 * np.pi / L, 0.0) for i in (1, 3) for j in (1, 3, -1, -3)]
    return np.array(ks), np.full(len(ks), 1.0 / len(ks))


def launch_hx_shapes(ctx, omen, cells):
    """Profiling aid: one FP64 stored H·X launch per compiled launch shape (CTA width 32, 64, 96,
    128 x block rows per batch 1, 2), in that order, on the alloy recipe at cells^3, so that one
    ncu capture of the 8 launches gives each shape's DRAM traffic per bond."""
    import torch
    spec, p = synth.config_sige_alloy(cells, seed=2)
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, p)
    x = torch.rand(ham.nrows, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    shapes = [(t, rb) for t in (32, 64, 96, 128) for rb in (1, 2)]
    for t, rb in shapes:
        omen.omen_hx_set_tile(ctx, ham, omen.OMEN_F64, t, rb)
        omen.omen_hx(ctx, ham, x, y)
    torch.cuda.synchronize()
    return {"cells": cells, "bonds": lat.counts()[1], "shapes_in_launch_order": shapes}


def measure_fp64_rate(ctx=None, omen=None, n=8192, reps=5):
    """GB300's FP64 rate as the library-side reference uses it: torch.matmul on float64 (cuBLAS
    DGEMM, 2 n^3 flops), best of reps after a warm-up, CUDA events; the FP64-bound product's
    roofline is reported against it."""
    import torch
    a = torch.rand((n, n), dtype=torch.float64, device="cuda")
    b = torch.rand((n, n), dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b, c
    out = {"n": n, "seconds": best, "tflops": 2.0 * n ** 3 / best / 1e12, "how": "torch.matmul float64 (cuBLAS DGEMM)"}
    if ctx is not None:
        out["fma_probe_tflops"] = omen.omen_probe_fp64_rate(ctx)
    return out


def measure_vff(ctx, omen, cells=N_CELLS, gtol=1e-8):
    """Valence-force-field relaxation of the alloy recipe (Keating, seeded constants, Si and Ge
    lattice constants, the box at the Si constant, hard walls): conjugate-gradient iterations,
    time, energy and largest force left."""
    import torch
    spec, _ = synth.config_sige_alloy(cells, seed=2)
    vp = synth.draw_vff_params(2)
    lat = omen.omen_build_lattice(ctx, spec)
    u = torch.zeros((3, spec.natoms), dtype=torch.float64, device="cuda")
    st = torch.empty(16 * spec.ncells, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info, status = omen.omen_relax_vff(ctx, lat, vp, u, gtol=gtol, max_iter=50000, strain_dev=st, raise_on_noconv=False)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s_np = st.cpu().numpy()
    return {"atoms": spec.natoms, "gtol_eV_per_nm": gtol, "seconds": dt, "iterations": info["iterations"],
            "converged": info["converged"], "energy_start_eV": info["energy_start"], "energy_eV": info["energy"],
            "max_force_eV_per_nm": info["max_force"], "ms_per_iteration": 1e3 * dt / max(1, info["iterations"]),
            "bond_strain_range": [float(s_np[s_np != 0].min()), float(s_np[s_np != 0].max())]}


def measure_c5_solve_cost(ctx, omen, nev=32, seed=5):
    """One zero-field eigen-solve of the 4x4x80-cell delta layer (10,240 atoms, 102,400 complex
    rows) at one wave vector of the 4x4 mesh: the 32 states nearest sigma = E_c - 0.4 E_g by
    folded-spectrum Lanczos (single vector and block 4), to the 1e-6 eV bound of the first SCF
    iteration.  One SCF iteration of the configured workload needs this for 8 wave vectors."""
    import torch
    spec, p, _ = synth.delta_layer(4, 80, seed=seed)
    L = 4 * spec.a_nm
    ks, _ = c5_kpoints(L)
    eg = synth.GAPPED_SI_EC - synth.GAPPED_SI_EV
    sigma = synth.GAPPED_SI_EC - 0.4 * eg
    lat = omen.omen_build_lattice(ctx, spec)
    ham = omen.omen_assemble_H(ctx, lat, p, k=tuple(ks[0]))
    out = {"workload": "delta-doped Si 4x4x80 cells (10,240 atoms, 102,400 complex rows), k = (1/8, 1/8) of the "
                       f"4x4 mesh, {nev} states nearest sigma, zero field", "runs": []}
    for block, basis in ((1, 96), (4, 96), (4, 256), (1, 384)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, info, st = omen.omen_eigs(ctx, ham, nev, omen.OMEN_NEAREST, sigma=sigma, tol=1e-6, block=block, basis=basis,
                                      max_iter=400000, raise_on_noconv=False)
        torch.cuda.synchronize()
        out["runs"].append({"block": block, "basis": basis, "seconds": time.perf_counter() - t0,
                            "steps": info["iterations"], "converged": info["converged"],
                            "bound": info["max_error_bound"], "levels_eV": [float(min(ev)), float(max(ev))]})
        print(json.dumps(out["runs"][-1]), flush=True)
    best = min(r["seconds"] for r in out["runs"] if r["converged"])
    out["per_scf_iteration_seconds_8k"] = 8 * best
    return out


def measure_scf(ctx, omen, nzc=16, n_train=12, n_test=2, train_steps=400, nev=8, block=1):
    """SCF iterations and wall time from the zero-field start and from the learned start.

    The network is trained here on self-consistent potentials that omen_scf itself produces
    for seeded doping profiles (training time reported separately); held-out profiles are
    then solved from both starts to the same 1e-6 V tolerance."""
    import torch
    from oracle import poisson  # grid description only (no computation)
    spec, p, _ = synth.delta_layer(1, nzc, seed=1)
    a = spec.a_nm
    grid = poisson.Grid(3, 3, round(nzc * a / 0.2), a, a, nzc * a)
    lat = omen.omen_build_lattice(ctx, spec)
    eg = synth.GAPPED_SI_EC - synth.GAPPED_SI_EV
    common = dict(kT=8.617333262e-5 * 4, kpts=[(0.0, 0.0, 0.0)], kweights=[1.0], nev=nev,
                  sigma=synth.GAPPED_SI_EC - 0.4 * eg, e_cut=0.5 * (synth.GAPPED_SI_EC + synth.GAPPED_SI_EV),
                  eig_tol=1e-10, eig_block=block, eig_basis=max(48, 3 * nev) if block == 1 else max(64, 4 * nev),
                  eig_max_iter=40000, mix=0.3, mix_history=6, tol_V=1e-6, max_iter=200)

    def solve(seed, phi):
        ns, w = synth.draw_doping(seed)
        rho = torch.from_numpy(synth.donor_rho_on_grid(ns, w, grid.nx, grid.ny, grid.nz, grid.Lz_nm)).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info, st = omen.omen_scf(ctx, lat, p, grid, phi, rho, n_electrons=ns * (a * 1e-7) ** 2, **common)
        torch.cuda.synchronize()
        return rho, info, time.perf_counter() - t0

    net = omen.omen_mlp_create(ctx, synth.mlp_init(7))
    X = torch.empty((n_train, 256), dtype=torch.float32, device="cuda")
    T = torch.empty((n_train, 256), dtype=torch.float32, device="cuda")
    t_data = time.perf_counter()
    ok, failed = 0, []
    for i in range(n_train):
        phi = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        try:
            rho, info, ts = solve(1000 + i, phi)
        except omen.OmenError as e:       # a profile whose loop did not finish is left out
            failed.append({"seed": 1000 + i, "error": str(e)[:120]})
            continue
        # progress on stderr (stdout carries the one result line)
        print(json.dumps({"scf_train": i, "iterations": info["iterations"], "seconds": ts}), file=sys.stderr, flush=True)
        omen.omen_mlp_features(ctx, net, grid, rho, X[ok])
        omen.omen_mlp_targets(ctx, net, grid, phi, T[ok])
        ok += 1
    t_data = time.perf_counter() - t_data
    t_train = time.perf_counter()
    for _ in range(train_steps):
        loss = omen.omen_mlp_train_step(ctx, net, X[:ok], T[:ok], ok, lr=1e-3, want_loss=False)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    zi, zt, li, lt = [], [], [], []
    for j in range(n_test):
        phi0 = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
        try:
            _, info0, s0 = solve(5000 + j, phi0)
        except omen.OmenError as e:
            failed.append({"seed": 5000 + j, "error": str(e)[:120]})
            continue
        ns, w = synth.draw_doping(5000 + j)
        rho = torch.from_numpy(synth.donor_rho_on_grid(ns, w, grid.nx, grid.ny, grid.nz, grid.Lz_nm)).cuda()
        phi1 = torch.empty(grid.shape, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        omen.omen_mlp_warm_start(ctx, net, grid, rho, phi1)
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t0
        try:
            _, info1, s1 = solve(5000 + j, phi1)
        except omen.OmenError as e:
            failed.append({"seed": 5000 + j, "start": "learned", "error": str(e)[:120]})
            continue
        zi.append(info0["iterations"]); zt.append(s0)
        li.append(info1["iterations"]); lt.append(s1 + t_inf)
        print(json.dumps({"scf_test": j, "zero_field": [info0["iterations"], s0], "learned": [info1["iterations"], s1 + t_inf]}),
              file=sys.stderr, flush=True)
    return {"workload": f"delta-doped Si 1x1x{nzc} cells ({spec.natoms} atoms, {spec.natoms * 10} rows), Gamma, "
                        f"grid {grid.nx}x{grid.ny}x{grid.nz}, {nev} states nearest sigma, Anderson mixing, tol 1e-6 V",
            "zero_field": {"iterations": zi, "seconds": zt, "mean_iterations": float(np.mean(zi))},
            "learned": {"iterations": li, "seconds": lt, "mean_iterations": float(np.mean(li)),
                        "includes": "network inference"},
            "time_ratio_zero_over_learned": float(np.sum(zt) / max(np.sum(lt), 1e-9)),
            "training": {"profiles": ok, "dataset_seconds": t_data, "adam_steps": train_steps,
                         "train_seconds": t_train},
            "left_out": failed}


def measure_kbatch_full(ctx, omen, nk=128, nev=8, seed=4, per_k_sample=4):
    """The k-batching workload: instances of drawn lateral sizes x 80 cells, each with its donor
    sheet, nk wave vectors along Gamma-X, nev lowest bands per k.  Three ways: every (instance, k)
    in one lockstep solve (one H·X launch per step over the whole work list); one lockstep solve
    per instance; one solve per k (time extrapolated from per_k_sample wave vectors per instance)."""
    import torch
    insts = []
    for idx, (nxy, nz, lam) in enumerate(synth.draw_kbatch_instances(seed)):
        spec = synth.lattice_spec(nxy, nxy, nz, (2, 2, 0), seed=seed + idx)
        U = synth.donor_sheet_potential(spec, seed + idx, lam)
        lat = omen.omen_build_lattice(ctx, spec)
        ham = omen.omen_assemble_H(ctx, lat, synth.gapped_si_params(), precision=omen.OMEN_F32, k=(0.0, 0.0, 0.0),
                                   U_atom_dev=torch.from_numpy(U).cuda())
        ks = np.zeros((nk, 3))
        ks[:, 0] = np.linspace(0.0, 1.0, nk) * np.pi / (nxy * spec.a_nm)
        insts.append(dict(nxy=nxy, spec=spec, lam=lam, lat=lat, ham=ham, ks=ks))
    bands = nk * nev * len(insts)
    # all instances in one lockstep solve
    tile_m = omen.omen_tune_hx_kbatch(ctx, insts[0]["ham"], nk, reps=5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    evm, infom, _ = omen.omen_eigs_kbatch_multi(ctx, [(d["ham"], d["ks"]) for d in insts], nev, tol=1e-6,
                                                max_iter=20000, basis=48, raise_on_noconv=False)
    torch.cuda.synchronize()
    tm = time.perf_counter() - t0
    out = []
    tot_b, tot_p = 0.0, 0.0
    for d, ev_multi in zip(insts, evm):
        ham, ks = d["ham"], d["ks"]
        tile_b = omen.omen_tune_hx_kbatch(ctx, ham, nk, reps=5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, info, st = omen.omen_eigs_kbatch(ctx, ham, ks, nev, tol=1e-6, max_iter=20000, basis=48, raise_on_noconv=False)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        tile_p = omen.omen_tune_hx_kbatch(ctx, ham, 1, reps=5)
        t0 = time.perf_counter()
        for q in np.linspace(0, nk - 1, per_k_sample).astype(int):
            omen.omen_eigs_kbatch(ctx, ham, ks[q:q + 1], nev, tol=1e-6, max_iter=20000, basis=48, raise_on_noconv=False)
        torch.cuda.synchronize()
        tp = (time.perf_counter() - t0) / per_k_sample * nk
        out.append({"lateral": d["nxy"], "atoms": d["spec"].natoms, "lambda_TF_nm": d["lam"], "batched_s": tb,
                    "per_k_s": tp, "converged": info["converged"], "max_residual": info["max_residual"],
                    "max_diff_multi_vs_batched_eV": float(np.abs(ev_multi - ev).max()),
                    "tile_batched": [tile_b["threads"], tile_b["rows_per_batch"]],
                    "tile_per_k": [tile_p["threads"], tile_p["rows_per_batch"]]})
        tot_b += tb
        tot_p += tp
    return {"instances": out, "bands": bands,
            "all_instances_one_solve": {"seconds": tm, "bands_per_s": bands / tm, "iterations": infom["iterations"],
                                        "converged": infom["converged"], "max_residual": infom["max_residual"],
                                        "tile": [tile_m["threads"], tile_m["rows_per_batch"]]},
            "bands_per_s_batched": bands / tot_b, "bands_per_s_per_k": bands / tot_p,
            "speedup_per_instance_batch": tot_p / tot_b, "speedup_one_solve": tot_p / tm,
            "per_k_time": f"extrapolated from {per_k_sample} wave vectors per instance"}


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_1003_4570_gb300 import omen
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    ctx = omen.omen_create(local_rank, stream.cuda_stream)
    prec = {"f64": omen.OMEN_F64, "f32": omen.OMEN_F32, "df": omen.OMEN_F64_DF}[args.precision]
    spec, p = synth.config_sige_alloy(args.cells, seed=2)
    lat = omen.omen_build_lattice(ctx, spec)
    natoms, nbonds = lat.counts()
    ham = omen.omen_assemble_H(ctx, lat, p, precision=prec, matrix_free=args.matrix_free)
    el = 4 if prec == omen.OMEN_F32 else 8
    if prec == omen.OMEN_F64_DF:   # double-float vectors: (hi, lo) FP32 pairs
        x64 = torch.rand(ham.nrows, dtype=torch.float64, device="cuda") * 2 - 1
        x = torch.empty((ham.nrows, 2), dtype=torch.float32, device="cuda")
        ctx.check(omen.lib().omen_convert_vectors(ctx.handle, x64.data_ptr(), omen.OMEN_F64, x.data_ptr(),
                                                  omen.OMEN_F64_DF, ham.nrows))
        del x64
    else:
        dt = torch.float64 if prec == omen.OMEN_F64 else torch.float32
        x = (torch.rand(ham.nrows, dtype=torch.float64, device="cuda") * 2 - 1).to(dt)
    t = torch.empty_like(x)
    y = torch.empty_like(x)
    sigma = 0.3
    # launch shape of the product: timed on this Hamiltonian by the library's tuner (identical
    # results for every shape); the double-float kernel has one shape
    if prec == omen.OMEN_F64_DF:
        tile = None
    elif args.tile:
        thr, rb = (int(v) for v in args.tile.split(","))
        omen.omen_hx_set_tile(ctx, ham, prec, thr, rb)
        tile = {"threads": thr or 128, "rows_per_batch": rb, "candidates": 0, "source": "--tile"}
    else:
        tile = omen.omen_tune_hx(ctx, ham, prec, nvec=1, reps=5)

    def step():
        omen.omen_hx(ctx, ham, x, t, 1, sigma)
        omen.omen_hx(ctx, ham, t, y, 1, sigma)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    if dist:
        ms = max_over_ranks(ms, dist, "cuda")
    alg = alg_bytes_per_hx(nbonds, natoms, ham.nrows, el, el, args.matrix_free)
    value = job_throughput(world, 2 * alg, args.steps, ms / 1e3)
    launch_ms = ms / (2 * args.steps)

    # end to end through the host-buffer entry point (pinned host x, y; copies timed)
    xh = (x if prec != omen.OMEN_F64_DF else x[:, 0].double()).cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    import ctypes
    L = omen.lib()
    for _ in range(2):
        ctx.check(L.omen_hx_host(ctx.handle, ham.handle, ctypes.c_void_p(xh.data_ptr()), ctypes.c_void_p(yh.data_ptr()), 1, sigma))
    e2e_steps = max(5, min(50, args.steps // 10))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.check(L.omen_hx_host(ctx.handle, ham.handle, ctypes.c_void_p(xh.data_ptr()), ctypes.c_void_p(yh.data_ptr()), 1, sigma))
    e2e_s = time.perf_counter() - t0
    if dist:
        e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e_val = job_throughput(world, alg, e2e_steps, e2e_s)

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    achieved_gbs = alg / (launch_ms / 1e3) / 1e9
    if prec == omen.OMEN_F64:
        fl = flops_per_hx(nbonds, natoms)
        achieved_tf = fl / (launch_ms / 1e3) / 1e12
        # DRAM bytes per launch of this kernel for the chosen shape: per-bond traffic from the
        # committed ncu capture of every shape, times this launch's bonds (not measured in this run)
        shape = (tile["threads"], tile["rows_per_batch"] or 1) if tile else None
        per_bond = HX_F64_TRAFFIC_PER_BOND.get(shape) if not args.matrix_free else None
        traffic = per_bond * nbonds if per_bond else None
        # the FP64 FMA rate measured now on this device (the library's probe), nominal beside it
        peak_tf = omen.omen_probe_fp64_rate(ctx)
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved_tf / peak_tf, "traffic": traffic,
                "frac_of_nominal_fp64": achieved_tf / FP64_PEAK_TFLOPS,
                "traffic_source": HX_F64_TRAFFIC_SOURCE if traffic else None,
                "kernel": "hx_kernel<double,10,real,stored>", "hbm_achieved_gbs": achieved_gbs,
                "hbm_frac_of_measured": achieved_gbs / hbm,
                "peak_source": "measured in this run: FP64 FMA rate (omen_probe_fp64_rate)"}
    else:
        kname = "hx_df_kernel<10>" if prec == omen.OMEN_F64_DF else "hx_kernel<float,10,real,stored>"
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                "frac": achieved_gbs / hbm, "traffic": None,
                "kernel": kname, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32", "df": "f32x2 (double-float)"}[args.precision],
              "data": "synthetic",
              "config": dict(workload_config(args.cells, natoms, nbonds, ham.nrows, args.matrix_free, world),
                             launch_shape=tile),
              "roofline": roof, "gpu_launches": 2 * args.steps,
              "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": ham.nrows * el,
                      "d2h_bytes_per_step": ham.nrows * el},
              "clocks": clk.summary()}
    if not args.no_extras and world == 1:
        # side measurements on one GPU only (a multi-GPU run measures the replicated product)
        result["hx_variants"] = measure_variants(ctx, omen, lat, p, natoms, nbonds)
        result["lanczos_500_iterations"] = measure_lanczos(ctx, omen, ham)
        ham_df = omen.omen_assemble_H(ctx, lat, p, precision=omen.OMEN_F64_DF)
        result["lanczos_500_iterations_double_float"] = measure_lanczos(ctx, omen, ham_df)
        del ham_df
        if args.cells == N_CELLS and prec == omen.OMEN_F64 and not args.matrix_free:
            result["charge_poisson_1M_atoms"] = measure_charge_poisson(ctx, omen, lat, ham, spec)
            del ham
            result["eigs_16_lowest_1M_atoms"] = measure_eigs_1m(ctx, omen, lat, p)
        result["eigs_8_lowest_si_8cubed"] = measure_small_si(ctx, omen)
        if args.cells == N_CELLS:
            result["lanczos_500_iterations_80cubed_si"] = measure_cube_500(ctx, omen)
        result["hx_kbatch"] = measure_hx_kbatch(ctx, omen)
        result["kbatch"] = measure_kbatch(ctx, omen)
        if args.cells == N_CELLS:
            # the full batching workload: 8 structures x 128 wave vectors (about two minutes)
            result["kbatch_full"] = measure_kbatch_full(ctx, omen)
        result["scf_learned_vs_zero"] = measure_scf(ctx, omen)
        result["effective_mass"] = measure_effmass(ctx, omen)
        if args.cells == N_CELLS:
            result["vff_relax_1M_atoms"] = measure_vff(ctx, omen)
    if rank == 0 and world == 1 and not args.no_cpu:
        t0 = time.perf_counter()
        cspec, H, cnb = cpu_sample()
        v, dtc, nsteps, nthr = time_cpu_oracle(H, cnb, cspec.natoms, min_seconds=10.0)
        v1 = time_cpu_scipy(H, cnb, cspec.natoms, steps=3)
        result["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": nthr, "kind": "oracle",
                                  "sample": f"oracle CSR product (oracle/csr_matvec.c, OpenMP, {nthr} threads) of "
                                            f"(H-sigma)^2 x, {nsteps} steps in {dtc:.1f} s on a 50x50x{SAMPLE_NZ}-cell "
                                            f"slab ({cspec.natoms} atoms, {H.shape[0]} rows) of the same recipe",
                                  "single_core_scipy_GB_per_s": v1}
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f64", choices=["f64", "f32", "df"],
                    help="f64 native FP64; f32; df double-float (FP64-accurate on the FP32 pipe)")
    ap.add_argument("--matrix-free", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the Lanczos and k-batch side measurements")
    ap.add_argument("--cells", type=int, default=N_CELLS, help="cells per edge (50 = the 1M-atom workload; "
                    "smaller only for profiling captures)")
    ap.add_argument("--scf-full", action="store_true",
                    help="one-off: warm-start network trained on 200 SCF solutions, 20 held-out profiles (minutes)")
    ap.add_argument("--scf-study", default="", metavar="NZ,NTRAIN,NTEST,NEV",
                    help="one-off: warm-start study on a 1x1xNZ-cell slab (NTRAIN training, NTEST held-out profiles, "
                         "NEV states per solve)")
    ap.add_argument("--kbatch-full", action="store_true",
                    help="one-off: the 8-instance x 128-k batching workload, batched vs per-k (minutes)")
    ap.add_argument("--only", default="", choices=["", "kbatch", "hx-kbatch", "scf", "small-si", "cube", "so-eigs",
                                                   "so-all", "effmass", "m2-ladder", "c5-solve", "hx-shapes", "vff", "eigs-1m",
                                                   "fp64-rate", "charge-poisson"],
                    help="profiling aid: run one side measurement alone and print its JSON")
    ap.add_argument("--poisson-grid", type=int, default=256, metavar="NG",
                    help="points per side of the Poisson grid of --only charge-poisson (profiling aid)")
    ap.add_argument("--tile", default="", metavar="THREADS,RB",
                    help="fix the H·X launch shape instead of tuning it (e.g. 64,2; profiling aid)")
    ap.add_argument("--lanczos-only", type=int, default=0, metavar="ITERS",
                    help="profiling aid: run only ITERS Lanczos iterations (FP64, basis 64) and print their time")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.scf_full:
        import torch
        from paper_1003_4570_gb300 import omen
        ctx = omen.omen_create(0, torch.cuda.current_stream().cuda_stream)
        print(json.dumps({"scf_full": measure_scf(ctx, omen, n_train=200, n_test=20, train_steps=2000)}))
        return
    if args.scf_study:
        import torch
        from paper_1003_4570_gb300 import omen
        ctx = omen.omen_create(0, torch.cuda.current_stream().cuda_stream)
        nz, ntr, nte, nev = (int(v) for v in args.scf_study.split(","))
        print(json.dumps({"scf_study": measure_scf(ctx, omen, nzc=nz, n_train=ntr, n_test=nte,
                                                   train_steps=max(400, 10 * ntr), nev=nev, block=4)}))
        return
    if args.kbatch_full:
        import torch
        from paper_1003_4570_gb300 import omen
        ctx = omen.omen_create(0, torch.cuda.current_stream().cuda_stream)
        print(json.dumps({"kbatch_full": measure_kbatch_full(ctx, omen)}))
        return
    if args.only:
        import torch
        from paper_1003_4570_gb300 import omen
        ctx = omen.omen_create(0, torch.cuda.current_stream().cuda_stream)
        if args.only == "eigs-1m":
            spec, p = synth.config_sige_alloy(args.cells, seed=2)
            lat = omen.omen_build_lattice(ctx, spec)
            print(json.dumps({args.only: measure_eigs_1m(ctx, omen, lat, p)}))
            return
        if args.only in ("so-eigs", "so-all"):
            spec, p = synth.config_sige_alloy(args.cells, seed=2)
            lat = omen.omen_build_lattice(ctx, spec)
            which = "so_f32_refine64" if args.only == "so-eigs" else "so-all"
            print(json.dumps({args.only: measure_eigs_1m(ctx, omen, lat, p, only=which)}))
            return
        if args.only == "charge-poisson":
            spec, p = synth.config_sige_alloy(args.cells, seed=2)
            lat = omen.omen_build_lattice(ctx, spec)
            ham = omen.omen_assemble_H(ctx, lat, p)
            print(json.dumps({"charge_poisson": measure_charge_poisson(ctx, omen, lat, ham, spec, ng=args.poisson_grid)}))
            return
        if args.only == "hx-shapes":
            print(json.dumps({"hx_shapes": launch_hx_shapes(ctx, omen, args.cells)}))
            return
        fn = {"kbatch": measure_kbatch, "hx-kbatch": measure_hx_kbatch, "scf": measure_scf,
              "small-si": measure_small_si, "cube": measure_cube_500, "effmass": measure_effmass,
              "m2-ladder": measure_m2_ladder, "c5-solve": measure_c5_solve_cost, "vff": measure_vff,
              "fp64-rate": measure_fp64_rate}[args.only]
        print(json.dumps({args.only: fn(ctx, omen)}))
        return
    if args.lanczos_only:
        import torch
        from paper_1003_4570_gb300 import omen
        ctx = omen.omen_create(0, torch.cuda.current_stream().cuda_stream)
        spec, p = synth.config_sige_alloy(args.cells, seed=2)
        lat = omen.omen_build_lattice(ctx, spec)
        prec = {"f64": omen.OMEN_F64, "f32": omen.OMEN_F32, "df": omen.OMEN_F64_DF}[args.precision]
        ham = omen.omen_assemble_H(ctx, lat, p, precision=prec)
        print(json.dumps({"lanczos": measure_lanczos(ctx, omen, ham, iters=args.lanczos_only), "cells": args.cells,
                          "precision": args.precision}))
        return
    run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
