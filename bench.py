#!/usr/bin/env python3
"""Benchmark of the online stage (Algorithm 2) on the large coupled workload: 5 levels of 1536 x 768 cells,
three torsional plates in tandem and a clamped flag, each in its own Omega_0 box (nf = 1608), in the mixed
mode against the plain FP64 path; the 3-level 512 x 256 flag is measured beside it.

One step = one full time step of the hot path: advection/right-hand side on every level, multidomain
coupling, the DST predictor solves on all levels, the FSI iteration (P B0 P^T assembly + solve + body
update) and the corrector solve.  B0 (Algorithm 1) is built once before timing and reported separately.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--precision fp32|fp64]

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on the context stream, with
an L2 flush (a 512 MiB buffer write) between timed steps outside the events.  value = cell-steps/s
summed over ranks (cells = sum over levels of nx*ny).  The reference arm times the FP64 CPU oracle.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

METRIC = "FSI cell-steps/s, mixed vs FP64 on GPU at <=1e-5 force err; p50/p99 step ms"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64"],
                    help="mixed: double fields, float transforms, finest level in increment form (the headline); "
                         "fp32: all-float fields; fp64: the plain FP64 path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--offline", action="store_true",
                    help="measure the offline stage instead (B0 for 8192 unknowns on a 1024^2 grid by both "
                         "methods, then the FP64 Cholesky factor of B0 + tau I) and print one JSON line")
    ap.add_argument("--serving", type=int, default=0,
                    help="serving mode: stream this many Poisson-arriving plate runs through the continuous-batching "
                         "server and print one JSON line")
    ap.add_argument("--no-comparator", action="store_true",
                    help="skip the true-E comparator runs (Sec. 5.1 speed-up experiment)")
    ap.add_argument("--comparator-only", action="store_true",
                    help="run only the true-E comparator and print its JSON object")
    ap.add_argument("--comparator-case", default="",
                    help="comparator workload to run (default: both); e.g. plate_128")
    ap.add_argument("--comparator-runs", default="",
                    help="comma-separated comparator runs (default: all), e.g. fp64_true_e")
    ap.add_argument("--oracle-worker", default="", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-budget", type=float, default=10.0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-level", default="", help=argparse.SUPPRESS)
    ap.add_argument("--horizon-steps", type=int, default=-1,
                    help="steps of the mixed-vs-FP64 history check (default: the workload's own horizon)")
    ap.add_argument("--profile-case", default="tandem", choices=["tandem", "tandem_full", "flag"],
                    help="profiling mode workload: the reduced tandem case (nf = 1608), the full five-level "
                         "tandem workload (one-pass launch lists only), or the reduced flag case")
    ap.add_argument("--profile-dst", default="fft", choices=["fft", "gemm"],
                    help="profiling mode: sine transforms by FFT passes or by tensor-core sine-matrix GEMMs "
                         "(the GEMM passes need --precision fp32)")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="profiling mode: build the --profile-case workload, run this many "
                         "eager (non-graph) steps and exit without timing (for ncu captures)")
    return ap.parse_args()


def workload():
    """The largest single-GPU configuration: 5 levels of 1536 x 768, three plates and a flag (nf = 1608)."""
    from paper_2103_06415_gb300 import workloads as wl
    return wl.tandem_1536x768_5lvl()


def secondary_workload():
    """The 3-level 512 x 256 flag, measured beside the headline with its 2000-step precision check."""
    from paper_2103_06415_gb300 import workloads as wl
    return wl.flag_512x256_3lvl()


def cells_per_step(w):
    return w["n_levels"] * w["nx"] * w["ny"]


def aggregate_replicas(local_ms, local_cell_steps, world):
    """Replicas only: every rank runs its own copy of the workload with no data-path collective.  The job
    time is the slowest rank's (MAX over ranks); the value is all ranks' cell-steps over that time."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([local_ms, local_cell_steps], dtype=torch.float64)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(tmax[0]), float(t[1]) / (float(tmax[0]) * 1e-3)
    return local_ms, local_cell_steps / (local_ms * 1e-3)


def _oracle_worker(path, budget_s):
    """Subprocess leg of oracle_sample: time the pickled oracle run's next steps, print one JSON line."""
    import pickle
    with open(path, "rb") as f:
        sim = pickle.load(f)
    n, t0 = 0, time.perf_counter()
    while True:
        sim.step()
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 50:
            break
    print(json.dumps({"steps": n, "seconds": el}), flush=True)


def _level_pair_seconds(w, nx, ny):
    """Wall time of the oracle's two level solves of a step (A_w^-1 then Lap^-1 by dense DSTs) on one level of
    nx x ny cells with the workload's spacing, Re and dt."""
    import numpy as np
    from oracle import grid as og
    lev = og.Level(nx, ny, w["h"], w["x0"], w["y0"])
    rhs = np.random.default_rng(1).standard_normal((ny - 1, nx - 1))
    zero = np.zeros(lev.shape)
    t0 = time.perf_counter()
    wv = og.solve_aw(rhs, zero, lev, w["re"], w["dt"])
    og.solve_lap(wv, zero, lev)
    return time.perf_counter() - t0


def oracle_level_sample(w):
    """The FP64 oracle as it stands cannot take one step of the 1536 x 768 x 5 workload in a bounded time (its
    first FSI iteration alone needs ~6400 B0 columns of full dense-DST solves), so its rate is sampled: the
    oracle's pair of level solves on one level of the workload's grid, timed once with every host core available
    to numpy's BLAS, and extrapolated to a step as (levels + 1) such pairs (every predictor level and the
    corrector).  Advection, the FSI iteration and the B0 columns are left out, so the figure is an upper bound
    on the oracle's rate.  At one BLAS thread the same pair is timed on a half-size level (nx/2 x ny/2) and
    scaled by the dense-DST operation count Nx Ny (Nx + Ny)."""
    cores = os.cpu_count()
    pairs = w["n_levels"] + 1
    t = _level_pair_seconds(w, w["nx"], w["ny"])
    out = dict(value=cells_per_step(w) / (pairs * t), unit="cell-steps/s", cores=cores, kind="oracle",
               sample="one pair of level solves (A_w^-1, Lap^-1; naive dense DST, numpy FP64) on one %d x %d level "
                      "of %s in %.1f s with all %d cores, extrapolated to a step as %d pairs; advection, FSI and "
                      "B0 columns not counted (an upper bound on the oracle's rate)"
                      % (w["nx"], w["ny"], w["name"], t, cores, pairs),
               ms_per_step=1e3 * pairs * t)
    env = dict(os.environ)
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    hx, hy = w["nx"] // 2, w["ny"] // 2
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-level", "%d,%d" % (hx, hy)], env=env,
                       capture_output=True, text=True, timeout=900)
    try:
        th = float(r.stdout.strip().splitlines()[-1])

        def ops(nx, ny):
            return (nx - 1) * (ny - 1) * ((nx - 1) + (ny - 1))
        t1 = th * ops(w["nx"], w["ny"]) / ops(hx, hy)
        out["one_thread"] = dict(value=cells_per_step(w) / (pairs * t1), unit="cell-steps/s", cores=1,
                                 sample="the same pair on a %d x %d level at one BLAS thread (%.1f s), scaled by "
                                        "the dense-DST operation count to %d x %d (%.0f s), %d pairs per step"
                                        % (hx, hy, th, w["nx"], w["ny"], t1, pairs),
                                 ms_per_step=1e3 * pairs * t1)
    except (ValueError, IndexError):
        pass
    return out


def oracle_sample(w, budget_s, one_thread_budget_s=None):
    """Time the FP64 oracle as it stands on a bounded prefix of the workload: one untimed first step (it also
    builds the B0 columns it touches), then the following steps in subprocesses started from that state --
    with every host core available to numpy's BLAS and, if one_thread_budget_s is given, with one thread."""
    import pickle
    from runners import oracle_sim
    sim = oracle_sim(w)
    t0 = time.perf_counter()
    sim.step()
    t_first = time.perf_counter() - t0
    fd, path = tempfile.mkstemp(suffix=".pkl")
    with os.fdopen(fd, "wb") as f:
        pickle.dump(sim, f)
    cores = os.cpu_count()
    out = None
    try:
        for threads, budget in ((cores, budget_s), (1, one_thread_budget_s)):
            if budget is None:
                continue
            env = dict(os.environ)
            for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
                env[k] = str(threads)
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-worker", path,
                                "--oracle-budget", str(budget)], env=env, capture_output=True, text=True,
                               timeout=600)
            rec = json.loads(r.stdout.strip().splitlines()[-1])
            val = cells_per_step(w) * rec["steps"] / rec["seconds"]
            entry = dict(value=val, unit="cell-steps/s", cores=threads, kind="oracle",
                         sample="%d steps of %s after 1 untimed step (%.1f s with all %d cores, incl. its B0 "
                                "columns); numpy FP64, naive dense-DST transforms, BLAS threads = %d"
                                % (rec["steps"], w["name"], t_first, cores, threads),
                         ms_per_step=1e3 * rec["seconds"] / rec["steps"])
            if out is None:
                out = entry
            else:
                out["one_thread"] = {k: entry[k] for k in ("value", "unit", "cores", "sample", "ms_per_step")}
    finally:
        os.unlink(path)
    return out


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_offline():
    """Offline stage of the b0_1024 workload (8192 sub-domain unknowns on 1024 x 1024): B0 assembly by the lattice
    Green's function (FP64) and by one DST solve per column (FP32 and FP64), then the FP64 Cholesky factor of
    B0 + tau I.  Wall times include a synchronisation; the factor's flops are n^3/3."""
    import torch
    from paper_2103_06415_gb300 import build as _b
    from paper_2103_06415_gb300 import workloads as wl
    _b.build()
    import paper_2103_06415_gb300 as lib
    from runners import gpu_context
    w = wl.b0_1024()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    out = {"metric": "offline stage: B0 assembly (8192 unknowns, 1024^2 grid) and FP64 Cholesky of B0 + tau I",
           "workload": w["name"], "unknowns": 8192, "columns_per_s": {}, "seconds": {}}
    n2 = 8192
    for name, prec, method in (("green_fp64", 0, 0), ("columns_fp32", 1, 1), ("columns_fp64", 0, 1)):
        c = gpu_context(w, precision=prec, b0_method=method, precompute=False)
        torch.cuda.synchronize()
        c.precompute()                       # warm-up (allocations, kernel attributes)
        c.close()
        c = gpu_context(w, precision=prec, b0_method=method, precompute=False)
        c.precompute()
        sec = c.stats()["b0_seconds"]
        out["seconds"][name] = sec
        out["columns_per_s"][name] = n2 / sec
        if name == "green_fp64":
            out["green_fill_gbs"] = n2 * n2 * 8 / sec / 1e9
            tau, fsec = c.factor_operator(1e-10)
            tau, fsec = c.factor_operator(1e-10)
            flops = n2 ** 3 / 3.0
            fp64 = lib.fma_rate(lib.FSI_PREC_FP64)
            out["cholesky"] = {"seconds": fsec, "tflops": flops / fsec / 1e12, "tau": tau,
                               "fp64_fma_peak_tflops_measured": fp64 / 1e12,
                               "frac_of_measured_fp64": flops / fsec / fp64}
        c.close()
    # second run: sixteen uneven boxes (256 ... 4096 points) on the same grid, built together
    boxes = wl.b0_1024_uneven_boxes()
    args = (w["nx"], w["ny"], w["x0"], w["y0"], w["h"], w["re"], w["dt"], boxes)
    uneven = {"boxes": len(boxes), "points": [], "seconds": {}, "columns_per_s": {}}
    for name, prec, method in (("green_fp64", 0, 0), ("columns_fp32", 1, 1)):
        lib.B0Set(*args, method=method, precision=prec).close()     # warm-up
        s = lib.B0Set(*args, method=method, precision=prec)
        uneven["points"] = [s.box(k)["n_sd"] for k in range(len(boxes))]
        sec = s.stats()["seconds"]
        s.close()
        uneven["seconds"][name] = sec
        uneven["columns_per_s"][name] = 2 * sum(uneven["points"]) / sec
    uneven["unknowns_total"] = 2 * sum(uneven["points"])
    uneven["b0_bytes_total"] = sum(8 * (2 * p) ** 2 for p in uneven["points"])
    uneven["green_fill_gbs"] = uneven["b0_bytes_total"] / uneven["seconds"]["green_fp64"] / 1e9
    out["uneven_subdomains"] = uneven
    out["hbm_peak_gbs"] = peaks.get("hbm_gbs")
    print(json.dumps(out), flush=True)


def run_serving(n_req):
    """Serving sample: a Poisson stream (20 req/s, real time) of independent
    torsional-plate runs on {128, 256, 512, 1024}^2 grids with steps drawn from [200, 400] (the config's
    200-2000 range shortened so the sample ends in seconds), FP32 fluid / FP64 FSI, admitted under an HBM
    budget and advanced together.  Prints aggregate cell-steps/s and per-step latency percentiles."""
    import numpy as np
    from paper_2103_06415_gb300 import build as _b
    from paper_2103_06415_gb300 import workloads as wl
    _b.build()
    import paper_2103_06415_gb300 as lib
    from paper_2103_06415_gb300 import serving
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    reqs = wl.serving_requests(n_req, steps=(200, 400))
    if world > 1:  # disjoint shares of the one stream, no collective on the data path
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
        dist.barrier()
    mine = serving.partition_requests(reqs, world, rank)
    srv = lib.Server(200 << 30)
    t0 = time.perf_counter()
    k, res, max_active = 0, [], 0
    while True:
        now = time.perf_counter() - t0
        while k < len(mine) and reqs[mine[k]][0] <= now:
            _, w, b, n = reqs[mine[k]]
            srv.submit(w, b, n, precision=lib.FSI_PREC_FP32, tag=mine[k])
            k += 1
        n_active = srv.step()
        max_active = max(max_active, n_active)
        res += srv.poll()
        if k == len(mine) and n_active == 0 and srv.stats()["queued"] == 0:
            break
        if n_active == 0 and k < len(mine):
            time.sleep(max(0.0, reqs[mine[k]][0] - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    st = srv.stats()
    local = {"cell_steps": st["cell_steps"], "wall": wall, "finished": len(res),
             "errors": sum(r["status"] != 0 for r in res), "max_active": max_active, "ticks": st["ticks"],
             "p50": [r["p50_step_ms"] for r in res], "p99": [r["p99_step_ms"] for r in res],
             "wait": [r["wait_ms"] for r in res]}
    srv.close()
    parts = gather_serving(local, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return
    agg = aggregate_serving(parts)
    out = {"metric": "serving: aggregate FSI cell-steps/s and per-step latency (Poisson stream of plate runs)",
           "requests": n_req, "n_gpus": world, "finished": agg["finished"], "errors": agg["errors"],
           "wall_s": agg["wall"], "cell_steps": agg["cell_steps"], "value": agg["value"],
           "unit": "cell-steps/s", "max_active": agg["max_active"], "ticks": agg["ticks"],
           "p50_step_ms": float(np.median(agg["p50"])), "p99_step_ms": float(np.percentile(agg["p99"], 99)),
           "mean_wait_ms": float(np.mean(agg["wait"])), "dtype": "f32 fluid / f64 FSI",
           "partition": "requests by decreasing cell-steps to the least-loaded rank (no data-path collective)"}
    print(json.dumps(out), flush=True)


def gather_serving(local, world):
    """Every rank's serving record on every rank (torch.distributed object gather; the records only)."""
    if world == 1:
        return [local]
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, local)
    return parts


def aggregate_serving(parts):
    """Whole-job figures from the ranks' records: work summed, time the slowest rank's, latencies pooled."""
    wall = max(p["wall"] for p in parts)
    cs = sum(p["cell_steps"] for p in parts)
    return {"wall": wall, "cell_steps": cs, "value": cs / wall, "finished": sum(p["finished"] for p in parts),
            "errors": sum(p["errors"] for p in parts), "max_active": max(p["max_active"] for p in parts),
            "ticks": sum(p["ticks"] for p in parts), "p50": [x for p in parts for x in p["p50"]],
            "p99": [x for p in parts for x in p["p99"]], "wait": [x for p in parts for x in p["wait"]]}


def run_comparator(args, timed_steps):
    """The speed-up experiment of Sec. 5.1 (Table eldgerror): mean step time of the sub-domain method against
    the true E, E^T at the body points (matrix-free conjugate gradients, one finest-level (C^T A C)^-1 per
    Krylov iteration), on the torsional plates of the flag grid and of plate_128 (body points at ds = h, and
    at the paper's ds = 2h) and on the flapping plates of Sec. 5.1 (cases 1, 2), FP64 and FP32, with the
    relative L2 difference of the deflection angle and the lift between the two couplings over the timed
    steps."""
    import numpy as np
    import torch
    import paper_2103_06415_gb300 as lib
    from paper_2103_06415_gb300 import workloads as wl
    from runners import gpu_context

    k = max(3, min(args.steps, 20))
    out = {"steps": k, "warmup": 3, "note": "true E: Krylov tolerance = relative residual of the CG solve "
                                            "(library default 1e-10 FP64, 1e-5 FP32; 1e-5 is also PETSc's "
                                            "default GMRES tolerance). The *_rel_l2 differences cover only the "
                                            "timed steps right after the impulsive start, where the lift is "
                                            "still transient; the comparison over 0 < t/T < 3 of Sec. 5.1 is "
                                            "a separate three-period run"}
    cases = ([args.comparator_case] if args.comparator_case
             else ["flag_512x256_3lvl_torsional", "plate_128", "plate_128_ds2h", "e1_flapping_case1",
                   "e1_flapping_case2"])
    only = set(x for x in args.comparator_runs.split(",") if x)
    for name in cases:
        # the flapping plates of Sec. 5.1 (E1): sub-domain runs with the sparse B0' (eps = 0.007; the dense
        # operator of the 58 k-point Omega_0 would hold 107 GB)
        w = wl.e1_flapping(int(name[-1])) if name.startswith("e1_") else getattr(wl, name)()
        drop = 0.007 if name.startswith("e1_") else 0.0
        last = len(w["bodies"]) - 1
        res = {}
        runs = [("fp64_subdomain", lib.FSI_PREC_FP64, 0, 0.0), ("fp64_true_e", lib.FSI_PREC_FP64, 1, 0.0),
                ("fp64_true_e_ktol1e-5", lib.FSI_PREC_FP64, 1, 1e-5), ("fp32_subdomain", lib.FSI_PREC_FP32, 0, 0.0),
                ("fp32_true_e", lib.FSI_PREC_FP32, 1, 0.0)]
        hist = {}
        for tag, prec, coupling, ktol in runs:
            if only and tag not in only:
                continue
            st = torch.cuda.Stream()
            c = gpu_context(w, precision=prec, stream=st.cuda_stream, coupling=coupling, krylov_tol=ktol,
                            drop_tol=drop if coupling == 0 else 0.0)
            c.advance(3)
            c.sync()
            kry0 = c.stats()["krylov_iters_total"]
            t = timed_steps(c, st, k)
            sts = c.stats()
            h = c.history(last)[-k:].copy()
            h[:, 1] = sum(c.history(b)[-k:, 1] for b in range(last + 1))    # lift of all bodies
            hist[tag] = h
            r = {"ms_per_step": float(np.mean(t)), "p50_ms": float(np.median(t)),
                 "fsi_iters_per_step": float(np.mean(h[:, 5])), "launches_last_step": sts["launches_per_step"]}
            if coupling == 1:
                r["krylov_iters_per_step"] = (sts["krylov_iters_total"] - kry0) / k
                r["krylov_tol"] = ktol if ktol > 0 else (1e-10 if prec == lib.FSI_PREC_FP64 else 1e-5)
            res[tag] = r
            c.close()
        for num, den, key in (("fp64_true_e", "fp64_subdomain", "fp64_speedup"),
                              ("fp32_true_e", "fp32_subdomain", "fp32_speedup"),
                              ("fp64_true_e_ktol1e-5", "fp64_subdomain", "fp64_speedup_ktol1e-5")):
            if num in res and den in res:
                res[key] = res[num]["ms_per_step"] / res[den]["ms_per_step"]
        if "fp64_subdomain" in hist and "fp64_true_e" in hist:
            for col, key in ((3, "theta"), (1, "lift")):
                a, b = hist["fp64_subdomain"][:, col], hist["fp64_true_e"][:, col]
                res[key + "_rel_l2_subdomain_vs_true_e"] = float(np.linalg.norm(a - b) /
                                                                 max(np.linalg.norm(b), 1e-300))
        if drop > 0:
            res["subdomain_drop_tol"] = drop
        res["body_points"] = sum(bb["n_pts"] for bb in w["bodies"])
        out[name] = res
    return out


def mixed_vs_fp64_horizon(w, n, make, lib, prec):
    """The timed path's error over the workload's whole horizon: n steps of its run (precision prec) and of
    the FP64 run from the same start, relative L2 difference of each force / deflection history (Eq.
    errortheta without the factor 100), beside the FP64 path's own sensitivity -- the same difference between
    two FP64 runs whose initial deflection differs by 1 part in 1e13 -- and the all-float FP32 mode's error."""
    import copy
    import numpy as np
    hist = {}
    runs = [("fp64", lib.FSI_PREC_FP64, 0.0), ("mixed", prec, 0.0), ("fp64_perturbed", lib.FSI_PREC_FP64, 1e-13)]
    if prec != lib.FSI_PREC_FP32:
        runs.append(("fp32", lib.FSI_PREC_FP32, 0.0))
    for tag, prec_k, rel in runs:
        wk = copy.deepcopy(w)
        for b in wk["bodies"]:
            if "tip_angle" in b:
                b["tip_angle"] *= 1.0 + rel
            elif "theta" in b:
                b["theta"] *= 1.0 + rel
        c, _, _ = make(prec_k, wk_override=wk)
        t0 = time.perf_counter()
        c.advance(n)
        c.sync()
        el = time.perf_counter() - t0
        hist[tag] = (np.stack([c.history(b) for b in range(len(w["bodies"]))]), el, c.stats()["inverse_rebuilds"])
        c.close()
    names = ("fx", "fy", "moment", "deflection")

    def rel_l2(a, b):
        out = {}
        for k, nm in enumerate(names):
            den = np.linalg.norm(b[:, :, k])
            if den > 0:
                out[nm] = float(np.linalg.norm(a[:, :, k] - b[:, :, k]) / den)
        return out

    ref = hist["fp64"][0]
    mixed = rel_l2(hist["mixed"][0], ref)
    env = rel_l2(hist["fp64_perturbed"][0], ref)
    out = {"mixed_vs_fp64_rel_l2": mixed, "mixed_within_1e-5": bool(max(mixed.values()) <= 1e-5),
           "fp64_perturbation_envelope_rel_l2": env}
    if "fp32" in hist:
        out["fp32_mode_vs_fp64_rel_l2"] = rel_l2(hist["fp32"][0], ref)
    out.update({
            "horizon": {"steps": n, "histories": "all bodies; deflection = theta (torsional) or tip "
                                                 "displacement (flag)",
                        "envelope": "FP64 vs FP64 with the initial deflection scaled by 1 + 1e-13",
                        "fsi_iterations_max": int(ref[:, :, 5].max()),
                        "wall_s": {k: v[1] for k, v in hist.items()},
                        "inverse_rebuilds": {k: v[2] for k, v in hist.items()}}})
    return out


def run_reference(args, w):
    """The reference arm: the FP64 oracle as it stands on the host cores, on the same workload and metric.  Each
    step is the bounded sample of oracle_level_sample (a pair of dense-DST level solves, extrapolated to the
    step); as many of the K steps as fit in about a minute are run (at least one)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pairs = w["n_levels"] + 1
    ts, t_start = [], time.perf_counter()
    for _ in range(max(1, args.steps)):
        ts.append(pairs * _level_pair_seconds(w, w["nx"], w["ny"]))
        if time.perf_counter() - t_start > 60.0:
            break
    step_s = statistics.mean(ts)
    value = cells_per_step(w) / step_s
    cores = os.cpu_count()
    sample = ("%d steps, each one pair of level solves (A_w^-1, Lap^-1; naive dense DST, numpy FP64) on one %d x %d "
              "level of %s extrapolated to %d pairs; advection, FSI and B0 columns not counted (an upper bound on "
              "the oracle's rate); all %d host cores" % (len(ts), w["nx"], w["ny"], w["name"], pairs, cores))
    line = {"metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w["name"], "cells_per_step": cells_per_step(w)},
            "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.oracle_worker:
        _oracle_worker(args.oracle_worker, args.oracle_budget)
        return
    w = workload()
    if args.oracle_level:
        nx, ny = (int(v) for v in args.oracle_level.split(","))
        print(_level_pair_seconds(w, nx, ny), flush=True)
        return
    if args.offline:
        run_offline()
        return
    if args.serving > 0:
        run_serving(args.serving)
        return
    if args.profile_steps > 0:
        from paper_2103_06415_gb300 import workloads as wl
        from paper_2103_06415_gb300 import build as _b
        _b.build()
        import paper_2103_06415_gb300 as lib
        from runners import gpu_context
        wr = {"flag": wl.flag_512x256_3lvl_reduced_omega0, "tandem_full": wl.tandem_1536x768_5lvl,
              "tandem": wl.tandem_1536x768_reduced}[args.profile_case]()
        c = gpu_context(wr, precision={"mixed": lib.FSI_PREC_MIXED, "fp32": lib.FSI_PREC_FP32,
                                       "fp64": lib.FSI_PREC_FP64}[args.precision],
                        use_graph=False, dst_method=1 if args.profile_dst == "gemm" else 0)
        c.advance(args.profile_steps)
        c.sync()
        print(json.dumps({"profile_case": wr["name"], "steps": args.profile_steps, "stats": c.stats()}))
        return
    if args.impl == "reference":
        run_reference(args, w)
        return
    if args.comparator_only:
        import torch
        from paper_2103_06415_gb300 import build as _b
        _b.build()

        def timed_steps(c, stream, k):
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
            torch.cuda.synchronize()
            for e0, e1 in evs:
                e0.record(stream)
                c.advance(1)
                e1.record(stream)
            c.sync()
            torch.cuda.synchronize()
            return [e0.elapsed_time(e1) for e0, e1 in evs]

        print(json.dumps({"true_e_comparator": run_comparator(args, timed_steps)}), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # CPU baseline first, before any GPU call (rank 0, N = 1 only)
    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = oracle_level_sample(w)

    import numpy as np
    import torch
    from paper_2103_06415_gb300 import build as _b
    _b.build()
    import paper_2103_06415_gb300 as lib
    from runners import gpu_context

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    prec = {"mixed": lib.FSI_PREC_MIXED, "fp32": lib.FSI_PREC_FP32, "fp64": lib.FSI_PREC_FP64}[args.precision]

    def make(p, wk_override=None):
        wk = wk_override or w
        st = torch.cuda.Stream()
        t0 = time.perf_counter()
        c = gpu_context(wk, precision=p, precompute=False, stream=st.cuda_stream)
        c.precompute(wk.get("drop_tol", 0.0))
        return c, st, time.perf_counter() - t0

    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def timed_steps(c, stream, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        for e0, e1 in evs:
            # the L2 flush runs on the run's own stream: while the GPU executes it, the host enqueues the
            # start event, the step's graph and the end event, so the events bracket device work only
            with torch.cuda.stream(stream):
                flush.zero_()
            e0.record(stream)
            c.advance(1)
            e1.record(stream)
        c.sync()
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in evs]

    ctx, stream, b0_s = make(prec)
    ctx.advance(args.warmup)
    ctx.sync()
    clk = Clocks(local)
    times = timed_steps(ctx, stream, args.steps)
    clocks = clk.stop()
    cells = cells_per_step(w)
    total_ms, value = aggregate_replicas(sum(times), cells * args.steps, world)
    stats = ctx.stats()
    # the FSI kernel's phase timers for a separate pass after the timed steps (they are off while timing)
    n_phase = 50
    ctx.set_phase_timing(True)
    ctx.advance(n_phase)
    ctx.sync()
    phases = {k: v / n_phase for k, v in ctx.phase_times().items()}
    ctx.set_phase_timing(False)

    extra = {}
    if prec != lib.FSI_PREC_FP64 and rank == 0:
        # the plain FP64 path on the same workload and steps
        ctx64, stream64, _ = make(lib.FSI_PREC_FP64)
        ctx64.advance(args.warmup)
        t64 = timed_steps(ctx64, stream64, args.steps)
        extra["fp64_path"] = {"value": cells * args.steps / (sum(t64) * 1e-3), "unit": "cell-steps/s",
                              "ms_per_step": statistics.mean(t64), "p50_ms": statistics.median(t64),
                              "p99_ms": float(np.percentile(t64, 99))}
        ctx64.close()
        # the timed path against FP64 over the workload's whole horizon, beside the FP64 envelope
        horizon = w["steps"] if args.horizon_steps < 0 else args.horizon_steps
        if horizon > 0:
            extra.update(mixed_vs_fp64_horizon(w, horizon, make, lib, prec))
        # the 3-level 512 x 256 flag: its own step time and its 2000-step precision check
        w2 = secondary_workload()
        c2, st2, _ = make(prec, w2)
        c2.advance(args.warmup)
        t2 = timed_steps(c2, st2, args.steps)
        sec = {"workload": w2["name"], "value": cells_per_step(w2) * args.steps / (sum(t2) * 1e-3),
               "unit": "cell-steps/s", "ms_per_step": statistics.mean(t2), "p50_ms": statistics.median(t2)}
        c2.close()
        sec.update(mixed_vs_fp64_horizon(w2, w2["steps"], make, lib, prec))
        extra[w2["name"]] = sec

    if rank == 0 and not args.no_comparator:
        extra["true_e_comparator"] = run_comparator(args, timed_steps)

    # dominant-kernel roofline: live CUDA-event timing of each launch of the class on the context stream
    roof = None
    if rank == 0:
        roof = roofline(ctx, w, lib, torch, local)

    # end to end through the public API: the whole job of the workload -- build the run from host descriptors,
    # the offline stage, every step followed by a read-back of every body's outputs to page-locked host memory
    # (fsi_read_outputs_async: enqueued behind the step, the GPU does not wait for the host), the final sync,
    # destroy.  The same job with a synchronising read after every step (fsi_get_forces) is reported beside it.
    e2e = None
    if rank == 0:
        ke = w["steps"]
        nbody = len(w["bodies"])
        outs = torch.zeros((ke, 5 * nbody), dtype=torch.float64, pin_memory=True)
        row = 5 * nbody * 8
        t0 = time.perf_counter()
        ce = gpu_context(w, precision=prec, precompute=False)
        ce.precompute(w.get("drop_tol", 0.0))
        t1 = time.perf_counter()
        for k in range(ke):
            ce.advance(1)
            ce.read_outputs_async(outs.data_ptr() + k * row, 5 * nbody)
        ce.sync()
        t2 = time.perf_counter()
        last = [ce.forces(b) for b in range(nbody)]
        ce.close()
        el = time.perf_counter() - t0
        got = outs.numpy()
        assert all(tuple(got[-1, 5 * b:5 * b + 3]) == last[b] for b in range(nbody))
        # the previous form: a synchronising forces read after every step
        t3 = time.perf_counter()
        cs = gpu_context(w, precision=prec, precompute=False)
        cs.precompute(w.get("drop_tol", 0.0))
        for _ in range(ke):
            cs.advance(1)
            cs.forces(0)
        cs.close()
        el_sync = time.perf_counter() - t3
        e2e = {"value": cells * ke / el, "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": 5 * 8 * nbody, "steps": ke,
               "setup_s": t1 - t0, "steps_s": t2 - t1,
               "sync_each_step": {"value": cells * ke / el_sync, "unit": "cell-steps/s",
                                  "d2h_bytes_per_step": 96 + 4},
               "note": "the whole job through the C ABI: wall clock of context creation from host descriptors, "
                       "the offline stage (setup_s), the workload's %d steps each followed by an asynchronous "
                       "read-back of every body's forces and deflections into page-locked host memory "
                       "(fsi_read_outputs_async), the final sync (steps_s), and destroy; there are no per-step "
                       "host inputs.  sync_each_step: the same job with a synchronising fsi_get_forces after "
                       "every step" % ke}

    if rank == 0:
        n2 = 2 * stats["n_sd"]
        side = 2 * stats["b0_window"] + 1
        line = {"metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "p50_ms": statistics.median(times), "p99_ms": float(np.percentile(times, 99)),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {lib.FSI_PREC_FP32: "f32", lib.FSI_PREC_FP64: "f64"}.get(prec, "f32 transforms / f64 fields"),
                "data": "synthetic",
                "config": {"workload": w["name"] + " (three torsional plates in tandem and a clamped flag, each "
                                                   "in its own Omega_0 box)",
                           "levels": w["n_levels"], "nx": w["nx"], "ny": w["ny"], "cells_per_step": cells,
                           "body_points": sum(b["n_pts"] for b in w["bodies"]), "nf": stats["nf"],
                           "n_sd": stats["n_sd"], "b0": {"drop_tol": w.get("drop_tol", 0.0),
                                                         "window_half_width": stats["b0_window"],
                                                         "kept_entries": stats["b0_nnz"],
                                                         "bytes": n2 * 2 * side * side * 8,
                                                         "dense_bytes": n2 * n2 * 8},
                           "offline_s": b0_s, "l2": "flushed between timed steps (512 MiB write)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "gpu_launches": stats["launches_per_step"] * args.steps,
                "fsi_solver": {"iterations_last_step": stats["last_iters"], "solves_last_step": stats["last_solves"],
                               "inverse_rebuilds": stats["inverse_rebuilds"], "steps_run": stats["steps_done"],
                               "phase_ms_per_step": phases},
                "clocks": clocks, "roofline": roof, "e2e": e2e}
        line.update(extra)
        if base is not None:
            line["cpu_baseline"] = {k: base[k] for k in ("value", "unit", "cores", "kind", "sample", "one_thread")
                                    if k in base}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def roofline(ctx, w, lib, torch, local):
    """The dominant kernel's roofline from live per-launch CUDA-event times (fsi_profile_kernel), with the
    transform passes' HBM fractions beside it."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    shares = {}
    for name in ("ysolve", "xf", "xi", "fsi", "rhs", "src", "ring"):
        ms, nl = ctx.profile_kernel(name, 8)
        shares[name] = (ms, nl / 8.0)
    per_step = {k: v[0] * v[1] for k, v in shares.items()}
    st = ctx.stats()
    nf, G = st["nf"], w["n_levels"]
    nxi, nyi = w["nx"] - 1, w["ny"] - 1
    # transform passes (float transforms): algorithmic bytes per launch, one level
    passes = {}
    for name, words in (("ysolve", 3), ("xi", 4), ("xf", 2)):
        ms = shares[name][0]
        b = words * nxi * nyi * 4 * (G if name == "xf" and shares[name][1] < 2 * G else 1)
        if name == "xf":   # one launch transforms every predictor level, the other the corrector's level
            b = words * nxi * nyi * 4 * (G + 1) / max(shares[name][1], 1)
        passes[name] = {"achieved_gbs": b / (ms * 1e-3) / 1e9, "frac": b / (ms * 1e-3) / 1e9 / hbm,
                        "algorithmic_bytes_per_launch": b, "avg_launch_ms": ms}
    # k_fsi: the FSI-iteration kernel (one launch per step); flops per launch from the solver counters.  Its
    # arithmetic is mostly FP64 (ncu: FP64 pipe 24 % busy against 2.7 % for the FP32 FMA pipe), so the roofline
    # is the FP64 pipe at its measured FMA rate (the class the hot-path table gives the small-system kernels);
    # the FP32 part is reported beside it against the measured FP32 FMA rate.
    iters = max(st["last_iters"], 1)
    solves = max(st["last_solves"], iters)
    refreshes = st.get("last_refreshes", 0)
    per_body = [2 * b["n_pts"] for b in w["bodies"]]
    blk3 = sum(n ** 3 for n in per_body)
    n_el = sum(b["n_pts"] - 1 for b in w["bodies"] if b["kind"] == "deformable")
    coupled = sum(n * n for n in per_body)      # entries of K that bodies of separate boxes leave non-zero
    fp64_flops = (iters * 16 * 2 * coupled       # P B0' P^T of the coupled entries (16 multiply-adds each)
                  + solves * 2 * coupled          # double residual rows over the coupled blocks
                  + iters * n_el * 250)           # the flag's element forces
    fp32_flops = (refreshes * 2 * 2 * 2 * blk3   # one Newton-Schulz step: two block GEMMs
                  + solves * 2 * sum(n * n for n in per_body)  # d = X r on the blocks
                  + iters * n_el * (100 + (2 + 2 * n_el) * 54))  # J_d and the structural solves
    fsi_ms = shares["fsi"][0]
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    fma64 = lib.fma_rate(lib.FSI_PREC_FP64) / 1e12
    fma32 = lib.fma_rate(lib.FSI_PREC_FP32) / 1e12
    fp32_derived = sm_count * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = fp64_flops / (fsi_ms * 1e-3) / 1e12
    a32 = fp32_flops / (fsi_ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "k_fsi (FSI iteration, distributed block-inverse solver for nf = %d: "
                                      "P B0' P^T, block Newton-Schulz, double refinement; latency bound)" % nf,
            "pipe": "fp64",
            "achieved": achieved, "peak": fma64, "unit": "TFLOP/s", "frac": achieved / fma64,
            "peak_source": "measured: project-written FP64 fused multiply-add loop on all SMs (fsi_op_fma_rate)",
            "fp32_part": {"achieved": a32, "peak": fma32, "frac": a32 / fma32,
                          "frac_of_derived_peak": a32 / fp32_derived, "derived_peak": fp32_derived,
                          "peak_source": "measured FP32 FMA loop; derived: SMs x 128 lanes x 2 x max SM clock"},
            # dram__bytes_read.sum + dram__bytes_write.sum of one launch, from an ncu capture of the same kernel
            # on the two-level variant of this workload (same nf, bodies, B0' window half-width 13), whose
            # launch does the same per-step work
            "traffic": 16719616 + 232192 if nf == 1608 else None,
            "traffic_note": "ncu capture of k_fsi<BIG> on tandem_1536x768_reduced (nf = 1608, window 13): the "
                            "launch's units (body points, owned rows, window columns) equal this workload's",
            "algorithmic_flops_per_launch": {"fp64": fp64_flops, "fp32": fp32_flops}, "avg_launch_ms": fsi_ms,
            "per_step_kernel_ms": per_step, "dominant": max(per_step, key=per_step.get),
            "transform_passes_hbm": passes, "hbm_peak_gbs": hbm}

if __name__ == "__main__":
    main()
