"""Throughput of the GRPrec ADER step on GB300: FP64 cell-updates/s.

Workload (default): the batched case -- 65,536 independent transmissive Euler
domains, cell counts log-uniform in [4, 512] (seed 2602), half smooth density
waves, half Riemann problems with density/pressure ratios log-uniform in
[1e-3, 1e3], GRPrec degree M = 2, CFL 0.9.  One bench step = one time step of
every domain (the whole hot path: CFL reduction, reconstruction, GRP, update,
repair, write-back).  The state (~0.8 GB) is larger than L2, so no flush is
needed between steps.

The headline value is the batched form with the learned Newton guess (network
trained first, on interfaces harvested from another seed).  Beside it:
  plain        the same domains advanced one domain per solver, direct kernel
               launches, PVRS start: the method without batching and learning
               (a bounded sample of domains);
  batched_pvrs the batched form with the PVRS start (what the learned guess adds);
  equal_error  the largest relative difference between the final states of the
               three forms on the plain sample: the same scheme, so the same L1
               error, up to round-off.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the only reference this build has) on a
bounded sample of the same workload, on the host cores.
"""
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

METRIC = "FP64 cell-updates/s at fixed L1 error, plain vs batched+learned p* guess, 1 GB300"
UNIT = "cell-updates/s"

# Algorithmic FP64 flops per cell-update of the reconstruction + GRP phase (the
# work of the flux kernel), counted by the op-counting build of the CPU oracle
# (oracle/opcount.py) on a sample of each workload: every +, -, *, /, sqrt and
# pow touching the state counts one.  Leading Riemann problems whose traces
# agree to rounding (equal data, every smooth interface of the interpolating
# degrees 2 and 4) count the 19 flops of resolving them as the constant state,
# not the oracle's Newton iterations: that is the algorithm the kernel runs.
FLUX_FLOPS_PER_UPDATE = {("batched", 1): 398.4, ("batched", 2): 646.3, ("batched", 3): 1143.5,
                         ("batched", 4): 1607.8}
# ... and of the whole step (CFL reduction + reconstruction/GRP + update and
# repair), the work of the persistent batched kernel
STEP_FLOPS_PER_UPDATE = {("batched", 2): 718.3}
PROFILE = os.path.join(ROOT, "profiles", "k_flux_batched_m2.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--domains", type=int, default=65536)
    ap.add_argument("--M", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other", action="store_true", help="skip the single-domain workloads")
    ap.add_argument("--launch", default="tune", choices=["tune", "auto", "flat", "fused", "split", "tiled"],
                    help="launch configuration: autotuned (default), library default, or forced")
    ap.add_argument("--guess", default="learned", choices=["learned", "pvrs"])
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: a batch per rank (weak) or one batch split across the ranks (strong)")
    ap.add_argument("--plain-domains", type=int, default=128, help="sample size of the plain form (0: skip)")
    ap.add_argument("--plain-steps", type=int, default=60)
    ap.add_argument("--no-l1", action="store_true", help="skip the L1 errors against exact solutions")
    ap.add_argument("--workload", default="batched", choices=["batched", "sod"],
                    help="the batch (default) or Sod's shock tube on --cells cells (profiling and context)")
    ap.add_argument("--cells", type=int, default=1 << 22)
    ap.add_argument("--recon", default="grprec", choices=["grprec", "nl"])
    ap.add_argument("--solver", default="tt", choices=["tt", "det"])
    ap.add_argument("--dt-hold", type=int, default=1, help="recompute dt every k steps (1: the paper's rule)")
    ap.add_argument("--cfl", type=float, default=0.9)
    ap.add_argument("--tile-cells", type=int, default=512, help="--launch tiled: owned cells per tile")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def source_digest():
    import hashlib
    d = os.path.join(ROOT, "paper_2602_21911_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled(cells, kname):
    """From the committed ncu summary of the dominant kernel (the flux phase):
    DRAM bytes per launch, scaled from its workload to this one by cell count,
    and the executed FP64 flops (dadd + dmul + 2 dfma) per cell-update.  None
    when the kernel source has changed since the capture or the summary is of
    another kernel."""
    if not os.path.exists(PROFILE):
        return None
    kv = {}
    for line in open(PROFILE):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_digest") != source_digest() or kv.get("bench_kernel") != kname:
        return None
    return {"traffic": float(kv["dram_bytes_per_launch"]) * cells / float(kv["cells_per_launch"]),
            "executed_flops_per_cell_update": float(kv["executed_fp64_flops_per_cell_update"])}


def workload(args, rank, world):
    """Weak scaling: every rank advances its own batch (seed 2602 + rank).
    Strong scaling: the ranks split one batch (seed 2602) by longest-first
    balancing of the cell counts."""
    from paper_2602_21911_gb300 import dist as D, inputs as I
    extra = dict(recon=1 if args.recon == "nl" else 0, solver=1 if args.solver == "det" else 0, dt_hold=args.dt_hold)
    if args.workload == "sod":
        prob, avg, lm, lp = I.sod(args.cells, M=args.M, cfl=args.cfl)
        return (dict(prob, **extra), avg, lm, lp)
    if args.scaling == "strong" and world > 1:
        part = D.lpt_partition(I.batched_params(args.domains, 2602)["n"], world)[rank]
        prob, avg, lm, lp = I.batched(args.domains, seed=2602, M=args.M, domains=part)
    else:
        prob, avg, lm, lp = I.batched(args.domains, seed=2602 + rank, M=args.M, cfl=args.cfl)
    return (dict(prob, **extra), avg, lm, lp)


def train_guess(args, device):
    """Harvest interfaces from another seed of the batch (and a shock tube),
    train the network with the library's kernels; returns (weights, box, info)."""
    from paper_2602_21911_gb300 import inputs as I, learned
    t0 = time.perf_counter()
    # the shock tube on 2^16 cells (about t = 0.2) and the batch of another
    # seed: every strong-data Riemann problem with a shock of the flux kernel
    # and of the repair rounds
    runs = [(*I.sod(1 << 16, M=args.M), 30000)]
    runs += [(*I.batched(args.domains, seed=sd, M=args.M), 1500) for sd in (2603, 2605, 2607, 2609)]
    rec = learned.harvest(runs, capacity=12_000_000, log2_stride=0, device=device)
    t1 = time.perf_counter()
    w, box, info = learned.fit_from_records(rec, max_records=12_000_000, batch=4096, max_steps=60_000)
    return w, box, {"records": int(rec.shape[0]), "trained_on": info["n_train"], "val_rms": info["val_rms"],
                    "target_std": float(rec[:, 6].std().item()), "harvest_seconds": t1 - t0,
                    "train_seconds": time.perf_counter() - t1,
                    "harvest": "Sod 2^16 cells x 30000 steps + batched seeds 2603, 2605, 2607, 2609 x 1500 "
                               "steps, flux kernel and repair rounds"}


def plain_arm(args, device, stream, w, box):
    """The plain GPU form on an evenly spread sample of the domains: one
    solver per domain, direct launches, PVRS start.  Also runs the sample
    through the batched forms and returns the largest relative difference of
    the final states (equal error)."""
    import torch
    from paper_2602_21911_gb300 import grprec, inputs as I
    ids = np.unique(np.linspace(0, args.domains - 1, args.plain_domains).astype(np.int64))
    prob, avg, lm, lp = I.batched(args.domains, seed=2602, M=args.M, domains=ids)
    doms = I.split_domains(prob, avg, lm, lp)
    solvers = []
    for pj, aj, mj, qj in doms:
        sj = grprec.Solver(pj, device=device, stream=stream.cuda_stream)
        sj.set_launch(grprec.GRP_LAUNCH_FLAT)
        sj.set_graph(0)
        sj.set_initial(aj, mj, qj)
        sj.step(3)
        solvers.append(sj)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sj in solvers:
        sj.step(args.plain_steps)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    upd = float(prob["n_cells"].sum()) * args.plain_steps
    plain_state = np.concatenate([sj.get_state()[0] for sj in solvers], axis=1)
    for sj in solvers:
        sj.close()
    # the same plain form with each solver's steps replayed from CUDA graphs
    # (launch overhead removed; still one small domain per launch sequence)
    solvers = []
    for pj, aj, mj, qj in doms:
        sj = grprec.Solver(pj, device=device, stream=stream.cuda_stream)
        sj.set_launch(grprec.GRP_LAUNCH_FLAT)
        sj.set_graph(args.plain_steps)
        sj.set_initial(aj, mj, qj)
        sj.step(args.plain_steps)                     # captures the graph of plain_steps steps
        sj.set_initial(aj, mj, qj)
        solvers.append(sj)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sj in solvers:
        sj.step(args.plain_steps)
    torch.cuda.synchronize()
    el_g = time.perf_counter() - t0
    for sj in solvers:
        sj.close()
    # the batched forms on the same sample, same number of steps
    diffs = {}
    forms = [("batched_pvrs", grprec.GRP_GUESS_PVRS)]
    if w is not None:
        forms.append(("batched_learned", grprec.GRP_GUESS_MLP))
    for name, guess in forms:
        sb = grprec.Solver(prob, device=device, stream=stream.cuda_stream, guess=guess)
        if guess == grprec.GRP_GUESS_MLP:
            sb.set_guess_model(w, box)
        sb.set_initial(avg, lm, lp)
        sb.step(3 + args.plain_steps)
        a = sb.get_state()[0]
        sb.close()
        diffs[name] = float((np.abs(a - plain_state).max(axis=1) / np.abs(plain_state).max(axis=1)).max())
    return {"value": upd / el, "unit": UNIT,
            "sample": "%d domains evenly spread over the batch (%d cells) x %d steps, one solver per domain, "
                      "flat kernels, direct launches, PVRS start" % (len(ids), int(prob["n_cells"].sum()),
                                                                     args.plain_steps),
            "graphs": {"value": float(prob["n_cells"].sum()) * args.plain_steps / el_g, "unit": UNIT,
                       "note": "the same, each solver's steps replayed from one CUDA graph"},
            "note": "one small domain per launch sequence: bound by launch and kernel latency, not by the "
                    "method's arithmetic"}, diffs


def other_workloads(local, stream):
    """Throughput of the other configurations (context beside the batched
    headline): the smooth Euler density wave at N = 8192 for M = 1..4 (plain
    single-domain path; launch-latency bound at this size), its L1 density
    error at t = 1 for M = 2, the shock tube at 2^22 cells (M = 2), the batch
    and the shock tube with the GRPrecNL reconstruction and with the DET
    solver, and the advection sine at N = 100 (M = 2) to t = 1."""
    import torch
    from paper_2602_21911_gb300 import grprec, inputs as I
    out = {}

    def timed(s, n):
        s.step(8)
        s.get_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(n)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    for M in (1, 2, 3, 4):
        prob, avg, lm, lp = I.euler_wave(8192, M)
        s = grprec.Solver(prob, device=local, stream=stream.cuda_stream)
        s.set_initial(avg, lm, lp)
        ms = timed(s, 256)
        out["euler_wave_N8192_M%d" % M] = {"cell_updates_per_s": 8192 / (ms * 1e-3), "ms_per_step": ms}
        if M == 2:
            s.set_initial(avg, lm, lp)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.advance_to(1.0)
            e1.record(stream)
            torch.cuda.synchronize()
            l1, _, _ = s.error_norms(np.ascontiguousarray(I.euler_wave_exact(8192, 1.0)[0]))
            stats, _ = s.get_stats()
            out["euler_wave_N8192_M2"].update({"t_end": 1.0, "steps": int(stats[0, 0]),
                                               "seconds_to_t_end": e0.elapsed_time(e1) * 1e-3,
                                               "l1_rho": float(l1[0])})
        s.close()
    prob, avg, lm, lp = I.sod(1 << 22, M=2)
    s = grprec.Solver(prob, device=local, stream=stream.cuda_stream)
    s.set_initial(avg, lm, lp)
    ms = timed(s, 64)
    out["sod_N4194304_M2"] = {"cell_updates_per_s": (1 << 22) / (ms * 1e-3), "ms_per_step": ms,
                              "window": "steps 9..72 of t_end = 0.2"}
    s.close()
    # temporal blocking: dt held over 4 steps (C = 0.6, so that the held step
    # stays below the Courant limit while the shock forms), the flat form and
    # the tiled form (tiles of 512 cells in shared memory, 4 steps per launch:
    # the same results)
    for name, tiled in (("sod_N4194304_M2_C0.6_dthold4_flat", False), ("sod_N4194304_M2_C0.6_dthold4_tiled", True)):
        s = grprec.Solver(dict(prob, dt_hold=4, cfl=0.6), device=local, stream=stream.cuda_stream)
        if tiled:
            s.set_launch(grprec.GRP_LAUNCH_TILED, 128, 512, 4)
        else:
            s.set_launch(grprec.GRP_LAUNCH_FLAT)
        s.set_initial(avg, lm, lp)
        ms = timed(s, 64)
        out[name] = {"cell_updates_per_s": (1 << 22) / (ms * 1e-3), "ms_per_step": ms,
                     "launch": s.get_launch(), "window": "steps 9..72"}
        s.close()
    # GRPrecNL (Sections 3.3-3.4): the batch and the shock tube
    prob, avg, lm, lp = I.batched(65536, seed=2602, M=2)
    s = grprec.Solver(dict(prob, recon=grprec.GRP_RECON_GRPRECNL), device=local, stream=stream.cuda_stream)
    s.set_launch(grprec.GRP_LAUNCH_FLAT)
    s.set_initial(avg, lm, lp)
    ms = timed(s, 32)
    cells = int(prob["n_cells"].sum())
    out["batched_grprecnl_M2"] = {"cell_updates_per_s": cells / (ms * 1e-3), "ms_per_step": ms,
                                  "launch": "flat", "window": "steps 9..40"}
    s.close()
    prob, avg, lm, lp = I.sod(1 << 22, M=2)
    s = grprec.Solver(dict(prob, recon=grprec.GRP_RECON_GRPRECNL), device=local, stream=stream.cuda_stream)
    s.set_initial(avg, lm, lp)
    ms = timed(s, 32)
    out["sod_N4194304_M2_grprecnl"] = {"cell_updates_per_s": (1 << 22) / (ms * 1e-3), "ms_per_step": ms}
    s.close()
    # DET solver (the paper's GRP solver): the batch and the shock tube
    prob, avg, lm, lp = I.batched(65536, seed=2602, M=2)
    s = grprec.Solver(dict(prob, solver=grprec.GRP_SOLVER_DET), device=local, stream=stream.cuda_stream)
    s.set_initial(avg, lm, lp)
    ms = timed(s, 32)
    out["batched_det_M2"] = {"cell_updates_per_s": cells / (ms * 1e-3), "ms_per_step": ms,
                             "launch": "flat", "window": "steps 9..40"}
    s.close()
    prob, avg, lm, lp = I.sod(1 << 22, M=2)
    s = grprec.Solver(dict(prob, solver=grprec.GRP_SOLVER_DET), device=local, stream=stream.cuda_stream)
    s.set_initial(avg, lm, lp)
    ms = timed(s, 32)
    out["sod_N4194304_M2_det"] = {"cell_updates_per_s": (1 << 22) / (ms * 1e-3), "ms_per_step": ms}
    s.close()
    prob, avg, lm, lp = I.advection_sine(100, M=2)
    s = grprec.Solver(prob, device=local, stream=stream.cuda_stream)
    s.set_initial(avg, lm, lp)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.advance_to(1.0)
    e1.record(stream)
    torch.cuda.synchronize()
    l1, _, _ = s.error_norms(np.ascontiguousarray(I.advection_sine_exact(100, 1.0)[0]))
    out["advection_sine_N100_M2"] = {"seconds_to_t_end": e0.elapsed_time(e1) * 1e-3, "l1": float(l1[0])}
    s.close()
    return out


# ---------------------------------------------------------------------------
# Exact solutions for the L1 errors of the measurement (host, numpy): the
# textbook ideal-gas Riemann solution (pressure function, Newton on the star
# pressure, self-similar sampling), vectorised over problems and points.  A
# reference for error norms, not the scheme: nothing here feeds the kernels.
# ---------------------------------------------------------------------------
def _pressure_fn(p, rho, pk, c, g):
    A, B = 2.0 / ((g + 1.0) * rho), (g - 1.0) / (g + 1.0) * pk
    shock = p > pk
    sq = np.sqrt(A / (p + B))
    f = np.where(shock, (p - pk) * sq, 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0))
    df = np.where(shock, sq * (1.0 - 0.5 * (p - pk) / (p + B)), (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * c))
    return f, df


def exact_riemann_density(WL, WR, xi, g=1.4):
    """Density of the exact Riemann solution of primitive states WL | WR (each
    a tuple of arrays of shape (n,)) at the rays xi (shape (n, k)); also
    returns the largest wave speed of each problem.  No vacuum data."""
    rl, ul, pl = [np.asarray(v, dtype=np.float64)[:, None] for v in WL]
    rr, ur, pr = [np.asarray(v, dtype=np.float64)[:, None] for v in WR]
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    p = np.maximum(p, 1e-12 * np.maximum(pl, pr))
    for _ in range(80):
        fl, dfl = _pressure_fn(p, rl, pl, cl, g)
        fr, dfr = _pressure_fn(p, rr, pr, cr, g)
        p = np.maximum(p - (fl + fr + ur - ul) / (dfl + dfr), 1e-3 * p)
    fl, _ = _pressure_fn(p, rl, pl, cl, g)
    fr, _ = _pressure_fn(p, rr, pr, cr, g)
    us = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    gm = (g - 1.0) / (g + 1.0)
    # left wave
    sl_shock = ul - cl * np.sqrt((g + 1.0) / (2.0 * g) * p / pl + z)
    rl_star = np.where(p > pl, rl * (p / pl + gm) / (gm * p / pl + 1.0), rl * (p / pl) ** (1.0 / g))
    cl_star = cl * (p / pl) ** z
    # right wave
    sr_shock = ur + cr * np.sqrt((g + 1.0) / (2.0 * g) * p / pr + z)
    rr_star = np.where(p > pr, rr * (p / pr + gm) / (gm * p / pr + 1.0), rr * (p / pr) ** (1.0 / g))
    cr_star = cr * (p / pr) ** z
    x = np.asarray(xi, dtype=np.float64)
    with np.errstate(invalid="ignore"):            # the fan formulas outside their fans are not selected
        left_fan = rl * (2.0 / (g + 1.0) + gm / cl * (ul - x)) ** (2.0 / (g - 1.0))
        right_fan = rr * (2.0 / (g + 1.0) - gm / cr * (ur - x)) ** (2.0 / (g - 1.0))
    rho_left = np.where(p > pl, np.where(x < sl_shock, rl, rl_star),
                        np.where(x < ul - cl, rl, np.where(x < us - cl_star, left_fan, rl_star)))
    rho_right = np.where(p > pr, np.where(x > sr_shock, rr, rr_star),
                         np.where(x > ur + cr, rr, np.where(x > us + cr_star, right_fan, rr_star)))
    rho = np.where(x < us, rho_left, rho_right)
    smax = np.maximum(np.abs(np.where(p > pl, sl_shock, ul - cl)), np.abs(np.where(p > pr, sr_shock, ur + cr)))
    return rho, smax[:, 0]


def exact_riemann_averages(WL, WR, xc, t, edges, g=1.4, n_gauss=16):
    """Cell averages of the exact density at time t, 16-point Gauss per cell;
    edges (n, N + 1) per problem."""
    s, w = np.polynomial.legendre.leggauss(n_gauss)
    e = np.asarray(edges, dtype=np.float64)
    dx = e[:, 1:] - e[:, :-1]
    x = 0.5 * (e[:, :-1] + e[:, 1:])[:, :, None] + 0.5 * dx[:, :, None] * s[None, None, :]
    n, N = dx.shape
    rho, _ = exact_riemann_density(WL, WR, ((x - xc) / t).reshape(n, -1), g)
    return (rho.reshape(n, N, n_gauss) * (0.5 * w)).sum(axis=2)


def l1_measurements(args, device, stream, w, box):
    """L1 density errors against exact solutions, the 'fixed L1 error' of the
    metric: (a) the batch's Riemann-problem domains of the plain sample at a
    common time before their waves reach the ends, advanced by the plain form
    (one solver per domain), the batched form and the batched form with the
    learned guess: the three L1 errors agree; (b) Sod's shock tube
    (x_c = 0.5) at t = 0.2 on 2^16, 2^17 and 2^18 cells, with the observed
    order."""
    import torch
    from paper_2602_21911_gb300 import grprec, inputs as I
    out = {}
    t_l1 = 0.01
    ids = np.unique(np.linspace(0, args.domains - 1, args.plain_domains).astype(np.int64))
    par = I.batched_params(args.domains, 2602)
    rp = [int(d) for d in ids if not par["smooth"][d]]
    WL = (np.ones(len(rp)), par["uL"][rp], np.ones(len(rp)))
    WR = (par["r_rho"][rp], par["uR"][rp], par["r_p"][rp])
    _, smax = exact_riemann_density(WL, WR, np.zeros((len(rp), 1)))
    keep = [d for d, sm in zip(rp, smax) if 0.45 / sm >= t_l1]
    prob, avg, lm, lp = I.batched(args.domains, seed=2602, M=args.M, domains=keep)
    co = I.cell_offsets(prob)
    exact = np.zeros(int(prob["n_cells"].sum()))
    for k, d in enumerate(keep):
        N = int(prob["n_cells"][k])
        e = np.linspace(0.0, 1.0, N + 1)[None, :]
        exact[co[k]:co[k + 1]] = exact_riemann_averages((np.ones(1), par["uL"][[d]], np.ones(1)),
                                                        (par["r_rho"][[d]], par["uR"][[d]], par["r_p"][[d]]),
                                                        0.5, t_l1, e)[0]
    res = {}
    for name, guess in (("batched_pvrs", grprec.GRP_GUESS_PVRS), ("batched_learned", grprec.GRP_GUESS_MLP)):
        if guess == grprec.GRP_GUESS_MLP and w is None:
            continue
        sb = grprec.Solver(prob, device=device, stream=stream.cuda_stream, guess=guess)
        if guess == grprec.GRP_GUESS_MLP:
            sb.set_guess_model(w, box)
        sb.set_initial(avg, lm, lp)
        sb.advance_to(t_l1)
        l1, _, _ = sb.error_norms(exact)
        res[name] = l1
        sb.close()
    l1p = np.zeros(len(keep))
    for k, (pj, aj, mj, qj) in enumerate(I.split_domains(prob, avg, lm, lp)):
        sj = grprec.Solver(pj, device=device, stream=stream.cuda_stream)
        sj.set_launch(grprec.GRP_LAUNCH_FLAT)
        sj.set_graph(0)
        sj.set_initial(aj, mj, qj)
        sj.advance_to(t_l1)
        l1p[k] = sj.error_norms(np.ascontiguousarray(exact[co[k]:co[k + 1]]))[0][0]
        sj.close()
    res["plain"] = l1p
    out["batch_riemann_domains"] = {
        "t": t_l1, "domains": len(keep), "of_riemann_domains_in_sample": len(rp),
        "selection": "Riemann-problem domains of the plain sample whose fastest wave stays 0.05 from the ends",
        "mean_l1_rho": {k: float(v.mean()) for k, v in res.items()},
        "max_rel_diff_of_l1_vs_plain": {k: float(np.max(np.abs(v - l1p) / l1p)) for k, v in res.items()
                                        if k != "plain"}}
    sod = []
    for N in (1 << 16, 1 << 17, 1 << 18):
        prob, avg, lm, lp = I.sod(N, M=args.M)
        s = grprec.Solver(prob, device=device, stream=stream.cuda_stream)
        s.set_initial(avg, lm, lp)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.advance_to(0.2)
        e1.record(stream)
        torch.cuda.synchronize()
        stats, status = s.get_stats()
        ex = exact_riemann_averages((np.ones(1), np.zeros(1), np.ones(1)), (np.full(1, 0.125), np.zeros(1),
                                    np.full(1, 0.1)), 0.5, 0.2, np.linspace(0.0, 1.0, N + 1)[None, :])[0]
        l1, _, _ = s.error_norms(ex)
        sec = e0.elapsed_time(e1) * 1e-3
        sod.append({"N": N, "steps": int(stats[0, 0]), "l1_rho": float(l1[0]), "seconds": sec,
                    "cell_updates_per_s": N * int(stats[0, 0]) / sec})
        s.close()
    for a, b in zip(sod[:-1], sod[1:]):
        b["order"] = float(np.log2(a["l1_rho"] / b["l1_rho"]))
    out["sod_t0.2"] = sod
    # the time step held over 4 steps at C = 0.6 (the tiled form's reading; its
    # results equal the flat form's with the same dt_hold): L1 beside the above
    N = 1 << 18
    prob, avg, lm, lp = I.sod(N, M=args.M, cfl=0.6)
    s = grprec.Solver(dict(prob, dt_hold=4), device=device, stream=stream.cuda_stream)
    s.set_initial(avg, lm, lp)
    s.advance_to(0.2)
    ex = exact_riemann_averages((np.ones(1), np.zeros(1), np.ones(1)), (np.full(1, 0.125), np.zeros(1),
                                np.full(1, 0.1)), 0.5, 0.2, np.linspace(0.0, 1.0, N + 1)[None, :])[0]
    out["sod_t0.2_C0.6_dthold4_N262144"] = {"l1_rho": float(s.error_norms(ex)[0][0]),
                                       "steps": int(s.get_stats()[0][0, 0])}
    s.close()
    return out


def cpu_baseline(args, steps=100, stride=4):
    """The oracle as it stands, OpenMP over domains, on a bounded sample."""
    import oracle as O
    from paper_2602_21911_gb300 import inputs as I
    ids = np.arange(0, args.domains, stride)
    prob, avg, lm, lp = I.batched(args.domains, seed=2602, M=args.M, domains=ids)
    st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
    S = O.State(prob, avg, g)
    threads = O.cpu_threads()
    t0 = time.perf_counter()
    O.run(prob, S, steps, n_threads=threads)
    el = time.perf_counter() - t0
    upd = float((S.stats[:, O.ST_STEPS] * prob["n_cells"]).sum())
    return {"value": upd / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "every %dth domain (%d domains, %d cells) x %d steps, %.1f s" % (
                stride, len(ids), int(prob["n_cells"].sum()), steps, el)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each step: a bounded sample of the workload through the oracle
    import oracle as O
    from paper_2602_21911_gb300 import inputs as I
    ids = np.arange(0, args.domains, 64)
    prob, avg, lm, lp = I.batched(args.domains, seed=2602, M=args.M, domains=ids)
    st, g = O.init_iface(O.EULER, 1.0, 1.4, lm, lp)
    S = O.State(prob, avg, g)
    threads = O.cpu_threads()
    O.run(prob, S, args.warmup, n_threads=threads)
    s0 = S.stats[:, O.ST_STEPS].copy()
    t0 = time.perf_counter()
    O.run(prob, S, args.steps, n_threads=threads)
    el = time.perf_counter() - t0
    upd = float(((S.stats[:, O.ST_STEPS] - s0) * prob["n_cells"]).sum())
    v = upd / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "batched Euler, 65536 domains x 4..512 cells, M=%d (oracle sample: "
                                   "every 64th domain)" % args.M, "seed": 2602},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "every 64th domain (%d domains) per step" % len(ids)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2602_21911_gb300 import grprec
    prob, avg, lm, lp = workload(args, rank, world)
    peak = grprec.grp_probe_fp64_peak(local)
    stream = torch.cuda.Stream()
    learned = args.guess == "learned"
    w = box = None
    guess_info = None
    if learned:
        w, box, guess_info = train_guess(args, local)
    s = grprec.Solver(prob, device=local, stream=stream.cuda_stream,
                      guess=grprec.GRP_GUESS_MLP if learned else grprec.GRP_GUESS_PVRS)
    if learned:
        s.set_guess_model(w, box)
    if args.launch == "tune":
        from paper_2602_21911_gb300 import autotune
        autotune.tune(prob, avg, lm, lp, device=local, use_cache=False, solver=s)
    elif args.launch == "flat":
        s.set_launch(grprec.GRP_LAUNCH_FLAT)
    elif args.launch == "fused":
        s.set_launch(grprec.GRP_LAUNCH_FUSED)
    elif args.launch == "split":
        s.set_launch(grprec.GRP_LAUNCH_SPLIT)
    elif args.launch == "tiled":
        s.set_launch(grprec.GRP_LAUNCH_TILED, 128, args.tile_cells, args.dt_hold)
    launch = s.get_launch()
    # CUDA graphs of exactly W steps, with the flux kernel's timing events, so
    # that the W warm-up steps capture and instantiate the graph (a one-time
    # set-up) and the K timed steps replay it
    s.set_graph(max(1, args.warmup))
    s.set_kernel_timing(True)
    s.set_initial(avg, lm, lp)
    s.step(args.warmup)
    stats0, _ = s.get_stats()
    launches0 = s.launch_count()
    s.kernel_timing()                                  # drains the warm-up's events
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")            # ncu --nvtx-include timed/ selects these launches
        ev0.record(stream)
        s.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    flux_ms, flux_n = s.kernel_timing()
    s.set_kernel_timing(False)
    ms = ev0.elapsed_time(ev1)
    launches = s.launch_count() - launches0
    stats1, status = s.get_stats()
    upd = float(((stats1[:, 0] - stats0[:, 0]).astype(np.float64) * prob["n_cells"]).sum())
    from paper_2602_21911_gb300 import dist as D
    tmax, upd = D.reduce_time_and_work(ms, upd, device="cuda")
    value = upd / (tmax * 1e-3)

    # end to end through the public API with pinned host buffers
    h_avg = torch.from_numpy(np.ascontiguousarray(avg)).pin_memory()
    h_lm = torch.from_numpy(np.ascontiguousarray(lm)).pin_memory()
    h_lp = torch.from_numpy(np.ascontiguousarray(lp)).pin_memory()
    o_avg = torch.empty_like(h_avg).pin_memory()
    o_if = torch.empty((s.C, s.nif), dtype=torch.float64).pin_memory()
    o_t = torch.empty(s.D, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    s.set_initial(h_avg, h_lm, h_lp)
    s.step(args.warmup + args.steps)
    s.get_state(o_avg, o_if, o_t)
    e2e_s = time.perf_counter() - t0
    st_e2e, _ = s.get_stats()
    upd_e2e = float((st_e2e[:, 0].astype(np.float64) * prob["n_cells"]).sum())
    e2e_ms, upd_e2e = D.reduce_time_and_work(1e3 * e2e_s, upd_e2e, device="cuda")
    e2e_s = 1e-3 * e2e_ms
    nsteps_e2e = args.warmup + args.steps
    guess_stats = {"network_starts": int(st_e2e[:, grprec.STAT_GUESS_USED].sum()),
                   "rejected": int(st_e2e[:, grprec.STAT_GUESS_REJECTED].sum()),
                   "riemann_solves": int(st_e2e[:, grprec.STAT_RS_CALLS].sum()),
                   "newton_iterations": int(st_e2e[:, grprec.STAT_NEWTON_SUM].sum())}

    # the batched form with the PVRS start, same launch configuration (ablation)
    pv_value = None
    if learned:
        sp = grprec.Solver(prob, device=local, stream=stream.cuda_stream, guess=grprec.GRP_GUESS_PVRS)
        sp.set_launch(launch["form"], launch["threads"], launch["cells_per_block"], launch["steps_per_launch"])
        sp.set_graph(max(1, args.warmup))
        sp.set_initial(avg, lm, lp)
        sp.step(args.warmup)
        st0, _ = sp.get_stats()
        torch.cuda.synchronize()
        ev0.record(stream)
        sp.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        st1, _ = sp.get_stats()
        pv_upd = float(((st1[:, 0] - st0[:, 0]).astype(np.float64) * prob["n_cells"]).sum())
        pv_ms, pv_upd = D.reduce_time_and_work(ev0.elapsed_time(ev1), pv_upd, device="cuda")
        pv_value = pv_upd / (pv_ms * 1e-3)
        sp.close()
    plain, equal = plain_arm(args, local, stream, w, box) if rank == 0 and args.plain_domains > 0 else (None, None)
    h2d = 8 * (h_avg.numel() + h_lm.numel() + h_lp.numel())
    d2h = 8 * (o_avg.numel() + o_if.numel() + o_t.numel())
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / max(args.steps, 1), "higher_is_better": True,
            "scaling": args.scaling, "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": ("batched Euler: %d domains x log-uniform 4..512 cells, M=%d, CFL 0.9, "
                                    "transmissive, %s" % (args.domains, args.M,
                                                          "learned p* guess" if learned else "PVRS p* guess")
                                    if args.workload == "batched" else
                                    "Sod shock tube, %d cells, M=%d, CFL %g, transmissive" % (args.cells, args.M,
                                                                                               args.cfl))
                                   + ("" if args.recon == "grprec" else ", GRPrecNL")
                                   + ("" if args.solver == "tt" else ", DET solver")
                                   + ("" if args.dt_hold == 1 else ", dt held over %d steps" % args.dt_hold),
                       "seed": 2602, "cells": int(prob["n_cells"].sum()), "launch": launch,
                       "l2": "state larger than L2 (no flush needed)"},
            "e2e": {"value": upd_e2e / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": h2d / nsteps_e2e, "d2h_bytes_per_step": d2h / nsteps_e2e},
            "gpu_launches": launches, "clocks": clk.summary(),
            "dominant_kernel": {"ms_total": flux_ms, "launches": flux_n,
                                "share_of_timed_region": flux_ms / ms if ms > 0 else None},
            "frozen_domains": int((status != 0).sum()),
            "plain": plain, "batched_pvrs": {"value": pv_value, "unit": UNIT} if pv_value else None,
            "equal_error": {"max_rel_diff_vs_plain": equal,
                            "note": "final averages of the plain sample vs the batched forms on the same "
                                    "domains and steps"} if equal else None,
            "learned_guess": dict(guess_info or {}, **guess_stats) if learned else None}
    default_path = (args.workload == "batched" and args.recon == "grprec" and args.solver == "tt" and args.dt_hold == 1
                    and args.cfl == 0.9)
    if not default_path:
        flops, kname, per_launch_updates = None, None, None     # the op counts are of the default path
    elif launch["form"] == grprec.GRP_LAUNCH_FUSED:
        flops = STEP_FLOPS_PER_UPDATE.get(("batched", args.M))
        kname = "k_batch<Euler,M=%d> (%d steps per launch)" % (args.M, launch["steps_per_launch"])
        per_launch_updates = (upd / world) / args.steps * launch["steps_per_launch"]
    else:
        flops = FLUX_FLOPS_PER_UPDATE.get(("batched", args.M))
        kname = "k_flux + k_flux_hard<Euler,M=%d>" % args.M
        per_launch_updates = (upd / world) / args.steps
    if flops and flux_n:
        dur = flux_ms / flux_n * 1e-3                 # one flux phase (both passes), CUDA events
        alg = flops * per_launch_updates / dur
        prof = profiled(int(prob["n_cells"].sum()), kname)
        if prof:
            ex_flops = prof["executed_flops_per_cell_update"]
            ach, basis = ex_flops * per_launch_updates / dur, "executed"
        else:
            ex_flops, ach, basis = None, alg, "algorithmic"
        line["roofline"] = {"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                            "frac": ach / peak,
                            "traffic": prof["traffic"] if prof else None,
                            "kernel": kname,
                            "peak_source": "measured FP64 FMA-chain probe (grp_probe_fp64_peak), this GPU",
                            "basis": basis,
                            "flops_per_cell_update": ex_flops if prof else flops,
                            "flops_note": "executed = the kernels' own FP64 flops per cell-update (dadd + dmul + "
                                          "2 dfma, ncu, committed summary of the same source) over the live "
                                          "CUDA-event duration of the flux phase; algorithmic = the CPU "
                                          "oracle's operation count, a costlier formulation of the same "
                                          "arithmetic (an upper bound)",
                            "algorithmic": {"flops_per_cell_update": flops, "achieved": alg / 1e12,
                                            "frac": alg / peak}}
    if not args.no_l1 and args.plain_domains > 0:
        line["l1"] = l1_measurements(args, local, stream, w, box)
    if not args.no_other:
        line["workloads"] = other_workloads(local, stream)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
