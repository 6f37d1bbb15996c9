"""Benchmark: converged columns/s of the 1.5D MALI hot path on GB300.

Workload: 256x256 = 65536 synthetic chromospheric columns of 82 heights
(seeded; a stand-in for the paper's 3D MHD snapshot), hydrogen-like 5-level +
continuum atom, 608 wavelengths, 5 angles; every column iterated from the
learned initial guess to max|dn/n| < 1e-3 with Ng acceleration, columns that
do not converge re-run from LTE with collisional-radiative switching; FP32
formal solution and rates, FP64 rate equations and Ng; device work queue over
resident blocks.  The network is trained before the timed region on a
disjoint 256x256 cube that the same GPU MALI converged (from LTE).
One step = one full solve of all columns (inputs resident in HBM).

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rh_synth  # noqa: E402

NX = NY = 256
NDEP = 82
TOL = 1e-3
MAXITER = 500
TRAIN_SEED = 4321          # training cube (disjoint from the evaluated cube, seed 1234 + rank)
TRAIN_EPOCHS = 10
METRIC = "converged columns/s to max|dn/n|<1e-3"
# FP32 operations per formal-solver point (one depth x lambda x mu, both
# sweep directions): thread-level FP32 operations of the column kernel
# (2 x FFMA + FADD + FMUL, predicated-on threads) counted by ncu on 608 cube
# columns x 12 iterations (about the iterations a column takes from the
# learned guess), divided by their points; re-counted whenever the kernel
# changes
FLOP_PER_PT = 180.3
# DRAM bytes (read + write) per column-iteration of the column kernel, from
# the same ncu capture (12.75 GB for 608 x 12): the line-profile cache read
# back every iteration (1.57 MB), its build once per column and the column's
# inputs and results
DRAM_BYTES_PER_COLUMN_ITERATION = (11.522290e9 + 1.232291e9) / (608 * 12)
# warp instructions per column-iteration, same capture: the issue-slot view of
# the same kernel (4 schedulers per SM, one warp instruction per cycle each)
WARP_INST_PER_COLUMN_ITERATION = 15918287990 / (608 * 12)


def algorithmic_flop_per_pt(atom, nu):
    """Algorithmic FP32 operations per formal-solver point of the mixed-
    precision column kernel, counted from its source in the units of the ncu
    count (2 x FMA + ADD + MUL; the MUFU exponentials and reciprocals are
    counted apart), for the transitions actually active at each wavelength
    (no padding lanes, no inactive slots of a tile's union) and the
    optically thick branch of the SC weights (one exponential per step; the
    Taylor branch of thin steps is an accuracy choice).  Per depth, ray and
    direction, with n_l lines and n_c continua active (K = n_l + n_c):
      depth terms (x, e^-x, 1-e^-x, chi_bg, B, eta_bg)     11 + 2 n_l + 7 n_c,
          shared by the two angles of a pass (5 angles: 3 passes);
      opacities of the ray (chi, eta)                      1 + 6 n_l + 1 n_c;
      SC step (dtau, weights, I, I_eff, Psi*, S)            19;
      rate terms per active line (continuum)               10 (9) + (K - 1)
          (+ 2 + (K - 1) cross terms when K > 1, + (2 + (K - 1)) sums into
          the pass's registers for the second angle of a pass);
      warp reduce-scatter of P = 2^ceil(log2 K(K+1)) values  P - 1 + 5 - log2 P
          per pass.
    Both directions count once per point."""
    h, c, k = 6.62607015e-34, 2.99792458e8, 1.380649e-23
    E = np.asarray(atom["E_J"])
    vD = np.sqrt(2 * k * atom["T_ref"] / (atom["mass_amu"] * 1.66053906660e-27))
    ranges = []
    for l, u, q in zip(atom["line_l"], atom["line_u"], atom["line_qwing"]):
        nu0 = (E[u] - E[l]) / h
        ranges.append((nu0 * (1 - q * vD / c), nu0 * (1 + q * vD / c), 0))
    for l, r in zip(atom["cont_l"], atom["cont_ratio"]):
        nue = (E[-1] - E[l]) / h
        ranges.append((nue, r * nue, 1))
    nmu = atom["nmu"]
    npass = (nmu + 1) // 2
    share = npass / nmu                      # depth terms and reductions per ray
    second = (nmu - npass) / nmu             # rays that sum into a pass's registers
    tot = 0.0
    mufu = 0.0
    for f in nu:
        act = [kind for lo, hi, kind in ranges if lo * (1 - 1e-13) <= f <= hi * (1 + 1e-13)]
        nl = act.count(0)
        nc = act.count(1)
        K = max(nl + nc, 1)
        P = 1 << int(np.ceil(np.log2(K * (K + 1))))
        dc = (11 + 2 * nl + 7 * nc) * share
        av = 1 + 6 * nl + nc
        st = 19
        ct = 10 * nl + 9 * nc + K * (K - 1) + (K * (2 + (K - 1)) if K > 1 else 0) + K * (2 + (K - 1)) * second
        fl = (P - 1 + 5 - np.log2(P)) * share
        tot += 2 * (dc + av + st + ct + fl)
        mufu += 2 * (2 * share + 3)          # e^-x, rcp(1 - e^-x); rcp(chi), e^-dtau, rcp(dtau)
    return tot / len(nu), mufu / len(nu)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, p in rows:
            for nm, val in zip(names, p[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---- multi-GPU: independent replicas (weak scaling).  Columns are independent
# (Sect. 2.2, 3.1): each rank solves its own cube, no collective touches the
# data path; only the timings are combined.
def rank_seeds(rank):
    """Seeds of the inputs of one rank: its evaluated cube, its training cube
    and its magnetic field, disjoint across ranks."""
    return {"cube": 1234 + rank, "train": TRAIN_SEED + 7919 * rank, "field": 2024 + rank, "big": 5678 + rank}


def max_over_ranks(x, dist=None, device="cpu"):
    """The slowest rank's time (x on every rank), via all_reduce(MAX)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, steps, seconds):
    """Units all ranks processed per second of the slowest rank."""
    return ws * units_per_rank * steps / seconds


def cpu_baseline(cube, seconds_target=15.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample."""
    import oracle
    atom = rh_synth.hydrogen_like_atom()
    cores = os.cpu_count() or 1
    o = oracle.Oracle()
    o.setup_atom(atom)
    rng = np.random.default_rng(99)
    n0 = 2 * cores
    idx = rng.choice(cube["T"].shape[0], n0, replace=False)
    o.load_columns(rh_synth.subset(cube, idx))
    t0 = time.perf_counter()
    o.iterate(maxiter=MAXITER, tol=TOL, nthreads=cores)
    dt0 = time.perf_counter() - t0
    n1 = int(max(n0, min(4096, n0 * seconds_target / max(dt0, 1e-3))))
    idx = rng.choice(cube["T"].shape[0], n1, replace=False)
    t0 = time.perf_counter()
    conv = oracle_two_pass(o, rh_synth.subset(cube, idx), cores)
    dt = time.perf_counter() - t0
    return {"value": n1 / dt, "unit": "columns/s", "cores": cores, "kind": "oracle",
            "sample": "%d random columns of the 256x256 cube (seed 99), LTE start, tol 1e-3, same re-run "
                      "strategy, %d threads, %.1f s; %d converged" % (n1, cores, dt, conv)}


def true_error(cube, n_gpu, nsample=32, seed=2024):
    """The headline solve's error against the oracle's tight fixed point on
    a seeded sample of columns: the 1e-3 stopping criterion does not bound
    the true error when the iteration's spectral radius is near one."""
    import oracle
    cores = os.cpu_count() or 1
    idx = np.sort(np.random.default_rng(seed).choice(cube["T"].shape[0], nsample, replace=False))
    o = oracle.Oracle()
    o.setup_atom(rh_synth.hydrogen_like_atom())
    o.load_columns(rh_synth.subset(cube, idx))
    t0 = time.perf_counter()
    o.iterate(maxiter=2000, tol=1e-9, nthreads=cores)
    no, _, sto, _ = o.populations()
    ok = sto == oracle.ST_CONV
    d = np.abs(n_gpu[idx] / no - 1).max(axis=(1, 2))[ok]
    return {"max_rel_dn": float(d.max()) if d.size else None, "median_rel_dn": float(np.median(d)) if d.size else None,
            "columns_above_1e-3": int((d > 1e-3).sum()), "columns": int(ok.sum()),
            "reference": "oracle (FP64) converged to max|dn/n| < 1e-9 on %d seeded columns, %d threads, %.1f s"
                         % (nsample, cores, time.perf_counter() - t0)}


def measured_peaks(rh, local):
    """FP32 and FP64 FMA rates of this GPU (rh_fma_peak), each with the
    median SM clock sampled while it ran."""
    out = {}
    for name, prec in (("fp32", 1), ("fp64", 0)):
        rh.fma_peak(local, prec, 0.05)                      # warm-up
        with ClockSampler(local) as clk:
            r = rh.fma_peak(local, prec, 1.0)
        c = clk.summary()
        out[name] = {"tflops": r["flop_s"] / 1e12, "seconds": r["seconds"], "sm_mhz": c.get("sm_mhz"),
                     "reasons": c.get("reasons")}
    return out


def oracle_two_pass(o, cols, cores):
    """The oracle with the same two passes as the GPU run; returns converged count."""
    import oracle
    o.load_columns(cols)
    o.iterate(maxiter=MAXITER, tol=TOL, nthreads=cores)
    n, it, st, _ = o.populations()
    conv = int((st == oracle.ST_CONV).sum())
    for f0 in (1e3, 1e5, 1e7):
        bad = np.where(st != oracle.ST_CONV)[0]
        if not bad.size:
            break
        o2 = oracle.Oracle()
        o2.setup_atom(rh_synth.hydrogen_like_atom())
        cols = rh_synth.subset(cols, bad)
        o2.load_columns(cols)
        o2.iterate(maxiter=MAXITER, tol=TOL, ng_order=0, crsw_init=f0, nthreads=cores)
        st = o2.populations()[2]
        conv += int((st == oracle.ST_CONV).sum())
    return conv


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    cube = rh_synth.chromosphere_cube(NX, NY, NDEP, seed=1234)
    import oracle
    cores = os.cpu_count() or 1
    atom = rh_synth.hydrogen_like_atom()
    o = oracle.Oracle()
    o.setup_atom(atom)
    ncol = 2 * cores
    rng = np.random.default_rng(7)
    times = []
    for step in range(args.warmup + args.steps):
        idx = rng.choice(NX * NY, ncol, replace=False)
        t0 = time.perf_counter()
        oracle_two_pass(o, rh_synth.subset(cube, idx), cores)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = ncol * len(times) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": "columns/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "256x256 synthetic chromosphere cube, 82 heights, H-like 5+1 atom, "
                                   "608 wavelengths, 5 mu; each step a random sample of %d columns" % ncol,
                       "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": "columns/s", "cores": cores, "kind": "oracle",
                             "sample": "%d random columns per step, %d threads" % (ncol, cores)},
            "e2e": {"value": value, "unit": "columns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_full_config(rh, torch, local, stream, ncol, train_cols, seed=5678, fp64_columns=0, oracle_columns=0,
                    hybrid=1, save_sample=0, sample_path=None):
    """The full-run configuration: 512x512 columns of 128 heights (the
    first ncol of that cube), Lyman alpha and beta in PRD with 200
    frequencies each (880 wavelengths) -- R_II-A angle-averaged in the frame
    of the moving gas (the hybrid scheme, hybrid=1; the columns move at up
    to 10 km/s) or in the static frame (hybrid=0) -- solved from the learned
    guess in mixed precision (a network trained on train_cols CRD-converged
    columns of a disjoint 128-height cube), then the FP32 Zeeman Stokes
    spectrum of H alpha (400 wavelengths, mu = 1, seeded field).  One step
    each, timed on the device."""
    t_all = time.perf_counter()
    patom = rh_synth.hydrogen_like_atom(prd_lines=((1, 2), (1, 3)), prd_nlambda=200)
    catom = dict(patom)
    catom["line_prd"] = patom["line_prd"] * 0
    nd = 128
    c = rh.Context(local, stream=stream.cuda_stream)
    c.setup_atom(catom)
    train = rh_synth.chromosphere_cube(256, 256, nd, seed=TRAIN_SEED + 17)
    if train_cols < 65536:
        train = rh_synth.subset(train, slice(0, train_cols))
    c.load_columns(train)
    c.solve(precision=1)
    c.surrogate_init(hidden=512, nhidden=3, seed=0)
    tr = c.surrogate_train(epochs=TRAIN_EPOCHS, batch=512, lr=2e-3, seed=1)
    state = c.surrogate_state()
    del c
    full = rh_synth.chromosphere_cube(512, 512, nd, seed=seed)
    cube = full if ncol >= 512 * 512 else rh_synth.subset(full, slice(0, ncol))
    del full
    dev = {k: torch.from_numpy(v).to("cuda") for k, v in cube.items()}
    p = rh.Context(local, stream=stream.cuda_stream)
    p.setup_atom(patom)
    p.load_columns(dev, on_device=True)
    p.surrogate_init(hidden=512, nhidden=3, seed=0)
    p.surrogate_set_state(state)
    opts = dict(maxiter=MAXITER, tol=TOL, precision=1, start=1, prd_eps0=0.05, prd_hybrid=hybrid)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s = p.solve(**opts)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n_gpu = p.populations()[0]
    # Stokes H alpha after convergence
    rng_f = np.random.default_rng(seed + 1)
    Bc, thc, chc = rng_f.uniform(0.0, 0.2, ncol), np.arccos(rng_f.uniform(-1.0, 1.0, ncol)), rng_f.uniform(0, 2 * np.pi, ncol)
    fld = [torch.from_numpy(np.repeat(x[:, None], nd, axis=1)).to("cuda") for x in (Bc, thc, chc)]
    ha = [i for i, (l, u) in enumerate(zip(patom["line_l"], patom["line_u"])) if (l, u) == (1, 2)][0]
    nu_ha = (patom["E_J"][2] - patom["E_J"][1]) / 6.62607015e-34
    lam = 2.99792458e8 / nu_ha + np.linspace(-2e-10, 2e-10, 400)
    iquv = torch.empty((ncol, lam.size, 4), dtype=torch.float64, device="cuda")
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    p.emergent_stokes(ha, 1.5, *fld, lam, precision=1, out=iquv)
    s1.record(stream)
    torch.cuda.synchronize()
    st_ms = s0.elapsed_time(s1)
    conv_cols = torch.from_numpy(np.where(p.populations()[2] == 0)[0]).to("cuda")
    vi = (iquv[..., 3].abs() / iquv[..., 0]).amax(dim=1)
    st_all = p.populations()[2]
    out = {"workload": "%d columns of the 512x512 synthetic chromosphere cube (seed %d), 128 heights, H-like atom "
                       "with Lyman alpha and beta in PRD (R_II-A, %s, 200 frequencies each; 880 "
                       "wavelengths), learned start, mixed precision, tol 1e-3; then the FP32 H alpha Zeeman "
                       "Stokes spectrum (400 wavelengths)"
                       % (ncol, seed, "angle-averaged in the frame of the moving gas (hybrid)" if hybrid
                          else "angle-averaged in the static frame"),
           "columns": ncol, "value": ncol / ((ms + st_ms) / 1e3), "unit": "columns/s",
           "solve": {"ms": ms, "converged": s["n_converged"], "iterations_per_column": s["iterations_total"] / ncol,
                     "rerun_columns": s["rerun_columns"], "pass_columns": s["pass_columns"],
                     "not_converged": {"maxiter": int((st_all == 1).sum()), "non_finite": int((st_all == 2).sum()),
                                       "singular": int((st_all == 3).sum())},
                     "columns_per_s": ncol / (ms / 1e3)},
           "stokes": {"ms": st_ms, "columns_per_s": ncol / (st_ms / 1e3),
                      "max_abs_V_over_I_converged": float(vi[conv_cols].max()) if conv_cols.numel() else None,
                      "columns_with_abs_V_above_I": int((vi > 1).sum())},
           "learned_start": {"train_columns": train_cols, "loss_last_epoch": tr["loss_last_epoch"],
                             "trained_on": "CRD-converged 128-height columns of a disjoint cube"}}
    if fp64_columns > 0:
        idx = np.sort(np.random.default_rng(99).choice(ncol, min(fp64_columns, ncol), replace=False))
        q = rh.Context(local, stream=stream.cuda_stream)
        q.setup_atom(patom)
        q.load_columns(rh_synth.subset(cube, idx))
        t0 = time.perf_counter()
        sq = q.iterate(maxiter=3 * MAXITER, tol=TOL, precision=0, prd_eps0=0.05, prd_hybrid=hybrid)
        dt = time.perf_counter() - t0
        out["lte_start_fp64"] = {"value": sq["n_converged"] / dt, "unit": "columns/s", "columns": len(idx),
                                 "converged": sq["n_converged"], "iterations_per_column": sq["iterations_total"] / len(idx),
                                 "seconds": dt, "sample": "plain FP64 GPU MALI from LTE, one pass of up to %d "
                                                          "iterations" % (3 * MAXITER)}
    if save_sample > 0 and sample_path:
        # seeded columns' GPU results, for the oracle comparison on a host
        # (--full-run-compare): the oracle's 200-point kernels take minutes
        # per column to build
        idx = np.sort(np.random.default_rng(2024).choice(ncol, min(save_sample, ncol), replace=False))
        p_all = p.populations()
        np.savez(sample_path, idx=idx, n=p_all[0][idx], status=p_all[2][idx], iters=p_all[1][idx], seed=seed,
                 ncol=ncol, hybrid=hybrid)
        out["saved_sample"] = {"path": sample_path, "columns": int(len(idx))}
    if oracle_columns > 0:
        import oracle
        idx = np.sort(np.random.default_rng(2024).choice(ncol, min(oracle_columns, ncol), replace=False))
        o = oracle.Oracle()
        o.setup_atom(patom)
        o.load_columns(rh_synth.subset(cube, idx))
        t0 = time.perf_counter()
        o.iterate(maxiter=3000, tol=1e-8, prd_eps0=0.05, prd_hybrid=hybrid, nthreads=os.cpu_count() or 1)
        no, _, sto, _ = o.populations()
        ok = sto == oracle.ST_CONV
        d = np.abs(n_gpu[idx] / no - 1).max(axis=(1, 2))[ok]
        out["true_error"] = {"max_rel_dn": float(d.max()) if d.size else None,
                             "median_rel_dn": float(np.median(d)) if d.size else None, "columns": int(ok.sum()),
                             "reference": "oracle converged to 1e-8 on %d seeded columns, %.0f s"
                                          % (len(idx), time.perf_counter() - t0)}
    out["wall_s"] = time.perf_counter() - t_all
    return out


def run_gpu(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1411_1079_gb300 as rh

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    seeds = rank_seeds(rank)
    cube = rh_synth.chromosphere_cube(NX, NY, NDEP, seed=seeds["cube"])
    ncol = NX * NY
    stream = torch.cuda.current_stream()
    ctx = rh.Context(local, stream=stream.cuda_stream)
    atom = rh_synth.hydrogen_like_atom()
    ctx.setup_atom(atom)
    alg_flop, alg_mufu = algorithmic_flop_per_pt(atom, ctx.grid())
    # learned initial guess: converge a disjoint cube from LTE, train on it (untimed)
    t0 = time.perf_counter()
    ctx.load_columns(rh_synth.chromosphere_cube(NX, NY, NDEP, seed=seeds["train"]))
    tr_solve = ctx.solve(maxiter=MAXITER, tol=TOL, precision=1)
    ctx.surrogate_init(hidden=512, nhidden=3, seed=0)
    tr = ctx.surrogate_train(epochs=TRAIN_EPOCHS, batch=512, lr=2e-3, seed=1)
    train_info = {"train_columns": ncol, "train_converged": tr_solve["n_converged"],
                  "epochs": TRAIN_EPOCHS, "loss_first_epoch": tr["loss_first_epoch"],
                  "loss_last_epoch": tr["loss_last_epoch"], "train_seconds": tr["seconds"],
                  "data_generation_seconds": time.perf_counter() - t0 - tr["seconds"]}
    peaks_meas = measured_peaks(rh, local)
    dev = {k: torch.from_numpy(v).to("cuda") for k, v in cube.items()}
    ctx.load_columns(dev, on_device=True)
    opts = dict(maxiter=MAXITER, tol=TOL, precision=1, persistent=1, start=1)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    for _ in range(args.warmup):
        s = ctx.solve(**opts)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kern_s = 0.0
    pts = 0.0
    iters = 0
    conv = 0
    launches = 0
    rescued = 0
    with ClockSampler(local) as clk:
        # profiler range = the timed region (no effect without a profiler;
        # ncu --profile-from-start off lists exactly these launches)
        torch.cuda.profiler.start()
        e0.record(stream)
        for _ in range(args.steps):
            s = ctx.solve(**opts)
            kern_s += s["seconds"]
            pts += s["pts"]
            iters += s["iterations_total"]
            conv += s["n_converged"]
            launches += s["launches"]
            rescued += s["rerun_columns"]
        e1.record(stream)
        barrier()
        torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1)
    n_headline = ctx.populations()[0] if rank == 0 and not args.no_cpu_baseline else None
    # the same solve from LTE, for comparison (one step)
    lte_opts = dict(opts, start=0)
    barrier()
    t_l = time.perf_counter()
    s_l = ctx.solve(**lte_opts)
    barrier()
    lte_s = time.perf_counter() - t_l
    lte_iters = s_l["iterations_total"] / ncol
    # the paper's other start solutions (Sect. 2.3), one step each
    other = {}
    for name, kind in (("zero_radiation", 3), ("escape_probability", 4)):
        barrier()
        t_o = time.perf_counter()
        s_o = ctx.solve(**dict(opts, start=kind))
        barrier()
        dt_o = time.perf_counter() - t_o
        other[name] = {"value": ncol / dt_o, "unit": "columns/s",
                       "iterations_per_column": s_o["iterations_total"] / ncol,
                       "converged": s_o["n_converged"]}
    ms = max_over_ranks(ms, dist, "cuda")
    clocks = clk.summary()
    value = whole_job_rate(ncol, ws, args.steps, ms / 1e3)

    # end to end through the C ABI with pinned host buffers
    pin = {k: torch.from_numpy(v).pin_memory() for k, v in cube.items()}
    out = torch.empty((ncol, atom["nlev"], NDEP), dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * 8 for v in pin.values())
    d2h = out.numel() * 8
    ctx.load_columns(pin)
    ctx.solve(**opts)
    ctx.populations(out=out)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.load_columns(pin)
        ctx.solve(**opts)
        ctx.populations(out=out)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e = {"value": whole_job_rate(ncol, ws, args.steps, e2e_s), "unit": "columns/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h + ncol * (4 + 1 + 8)}

    # the 512 x 512 cube (82 heights, seed disjoint from the training and
    # evaluated cubes) from the learned guess, one step: the full-size target
    big = None
    if args.cube512:
        cube512 = rh_synth.chromosphere_cube(512, 512, NDEP, seed=seeds["big"])
        dev512 = {k: torch.from_numpy(v).to("cuda") for k, v in cube512.items()}
        del cube512
        ctx.load_columns(dev512, on_device=True)
        ctx.solve(**dict(opts, maxiter=2))                 # graph capture for this size
        ctx.load_columns(dev512, on_device=True)
        barrier()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        s_b = ctx.solve(**opts)
        b1.record(stream)
        barrier()
        big_ms = max_over_ranks(b0.elapsed_time(b1), dist, "cuda")
        nb = 512 * 512
        big = {"value": whole_job_rate(nb, ws, 1, big_ms / 1e3), "unit": "columns/s", "columns": nb,
               "converged": s_b["n_converged"], "iterations_per_column": s_b["iterations_total"] / nb,
               "ms": big_ms, "workload": "512x512 synthetic chromosphere cube, 82 heights, learned start, one step"}
        del dev512

    # Zeeman Stokes spectra of H alpha after convergence (FP32, mu = 1, 400
    # wavelengths over +-2 A; per column |B| ~ U(0, 2 kG), cos(theta) ~ U(-1, 1),
    # chi ~ U(0, 2 pi), constant with height)
    stokes = None
    if args.stokes:
        ctx.load_columns(dev, on_device=True)
        ctx.solve(**opts)
        rng_f = np.random.default_rng(seeds["field"])
        Bc = rng_f.uniform(0.0, 0.2, ncol)
        thc = np.arccos(rng_f.uniform(-1.0, 1.0, ncol))
        chc = rng_f.uniform(0.0, 2 * np.pi, ncol)
        fld = [torch.from_numpy(np.repeat(x[:, None], NDEP, axis=1)).to("cuda") for x in (Bc, thc, chc)]
        ha = [i for i, (l, u) in enumerate(zip(atom["line_l"], atom["line_u"])) if (l, u) == (1, 2)][0]
        nu_ha = (atom["E_J"][2] - atom["E_J"][1]) / 6.62607015e-34
        lam = 2.99792458e8 / nu_ha + np.linspace(-2e-10, 2e-10, 400)
        iquv = torch.empty((ncol, lam.size, 4), dtype=torch.float64, device="cuda")
        ctx.emergent_stokes(ha, 1.5, *fld, lam, precision=1, out=iquv)      # warm-up
        barrier()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        ctx.emergent_stokes(ha, 1.5, *fld, lam, precision=1, out=iquv)
        s1.record(stream)
        barrier()
        st_ms = s0.elapsed_time(s1)
        vmax = float((iquv[..., 3].abs() / iquv[..., 0]).max())
        stokes = {"value": ncol / (st_ms / 1e3), "unit": "columns/s", "nlambda": int(lam.size),
                  "ms": st_ms, "line": "H alpha (n=2-3), g_eff 1.5", "precision": "fp32 profiles and DELO solver",
                  "max_abs_V_over_I": vmax}

    # angle-averaged PRD in Lyman alpha and beta (LTE start, FP32), on the
    # first PRD_COLUMNS columns of the cube: a separate context and atom
    prd = None
    if args.prd_columns > 0:
        pctx = rh.Context(local, stream=stream.cuda_stream)
        patom = rh_synth.hydrogen_like_atom(prd_lines=((1, 2), (1, 3)))
        pctx.setup_atom(patom)
        psub = rh_synth.subset(cube, slice(0, min(args.prd_columns, ncol)))
        pctx.load_columns(psub)
        pctx.solve(maxiter=MAXITER, tol=TOL, precision=1, prd_eps0=0.05)      # warm-up, tuning
        pctx.load_columns(psub)
        barrier()
        t_p = time.perf_counter()
        s_p = pctx.solve(maxiter=MAXITER, tol=TOL, precision=1, prd_eps0=0.05)
        barrier()
        dt_p = time.perf_counter() - t_p
        npc = len(psub["T"])
        prd = {"value": npc / dt_p, "unit": "columns/s", "columns": npc, "converged": s_p["n_converged"],
               "iterations_per_column": s_p["iterations_total"] / npc,
               "lines": "Lyman alpha and beta, 64 wavelengths each, R_II-A in the static frame, PRD switching "
                        "eps0 = 0.05",
               "precision": "fp32 formal solution/rates/redistribution, fp64 rate equations/Ng"}
        # the same columns with the redistribution in the frame of the moving gas
        pctx.load_columns(psub)
        pctx.solve(maxiter=MAXITER, tol=TOL, precision=1, prd_eps0=0.05, prd_hybrid=1)
        pctx.load_columns(psub)
        barrier()
        t_p = time.perf_counter()
        s_h = pctx.solve(maxiter=MAXITER, tol=TOL, precision=1, prd_eps0=0.05, prd_hybrid=1)
        barrier()
        dt_h = time.perf_counter() - t_p
        prd["hybrid"] = {"value": npc / dt_h, "unit": "columns/s", "converged": s_h["n_converged"],
                         "iterations_per_column": s_h["iterations_total"] / npc,
                         "scheme": "R_II-A angle-averaged in the frame of the moving gas (hybrid)"}

    # plain FP64 MALI from LTE on a random sample of the cube (FP64 arithmetic is
    # slow on this part: one column per SM keeps the run under a minute)
    fp64 = None
    nsm_dev = torch.cuda.get_device_properties(local).multi_processor_count
    if args.fp64_columns_per_sm > 0:
        rng = np.random.default_rng(99)
        idx = np.sort(rng.choice(ncol, size=min(args.fp64_columns_per_sm * nsm_dev, ncol), replace=False))
        ctx.load_columns(rh_synth.subset(cube, idx))
        barrier()
        t_f = time.perf_counter()
        s_f = ctx.iterate(maxiter=MAXITER, tol=TOL, precision=0, persistent=1)
        barrier()
        f_s = time.perf_counter() - t_f
        fp64 = {"value": s_f["n_converged"] / f_s, "unit": "columns/s", "columns": len(idx),
                "converged": s_f["n_converged"], "seconds": f_s,
                "iterations_per_column": s_f["iterations_total"] / len(idx),
                "formal_solver_pts_per_s": s_f["pts"] / s_f["seconds"],
                "roofline": {"bound": "alu", "achieved": s_f["pts"] * alg_flop / s_f["seconds"] / 1e12,
                             "peak": peaks_meas["fp64"]["tflops"], "unit": "TFLOP/s",
                             "frac": s_f["pts"] * alg_flop / s_f["seconds"] / 1e12
                                     / peaks_meas["fp64"]["tflops"],
                             "flop_per_pt": alg_flop,
                             "peak_note": "measured FP64 FMA rate (rh_fma_peak) of this GPU; the same "
                                          "algorithmic operation count as the FP32 sweep (FP64 exponentials, "
                                          "divisions and reciprocals run as FMA sequences on top); ncu: FP64 "
                                          "pipe 80 % busy (profiles/mali_kernel_fp64_152col.md)"},
                "sample": "%d random columns of the cube (%d per SM), LTE start, FP64 throughout, one pass"
                          % (len(idx), len(idx) // nsm_dev)}

    full_run = None
    if args.full_run_columns > 0:
        full_run = run_full_config(rh, torch, local, stream, args.full_run_columns, args.full_run_train,
                                   oracle_columns=0 if args.no_cpu_baseline else args.full_run_oracle)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = _peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    nsm = nsm_dev
    # measured FP32 FMA rate, scaled from the clock it ran at to the median
    # clock of the timed region
    p32 = peaks_meas["fp32"]
    peak_tflops = p32["tflops"] * (sm_mhz / p32["sm_mhz"] if p32.get("sm_mhz") else 1.0)
    achieved = pts * alg_flop / kern_s / 1e12
    achieved_exec = pts * FLOP_PER_PT / kern_s / 1e12
    pts_s = pts / kern_s
    line = {
        "metric": METRIC, "value": value, "unit": "columns/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "256x256 synthetic chromosphere cube (65536 columns), 82 heights, "
                               "H-like 5-level+continuum atom, 608 wavelengths, 5 mu, tol 1e-3, "
                               "learned initial guess (MLP 328-512-512-512-492, BF16, trained on a disjoint "
                               "GPU-converged cube)",
                   "ncol_per_gpu": ncol, "ndep": NDEP, "nlambda": ctx.nlambda, "nmu": atom["nmu"],
                   "precision": "fp32 formal solution/rates, fp64 rate equations/Ng",
                   "scheduling": "device work queue (pool mode); columns not converged are re-run "
                                 "from LTE with collisional-radiative switching x1e3/x1e5/x1e7, no Ng",
                   "l2": "working set 2 GB > L2 (inputs larger than L2)",
                   "parallelism": "dp%d (independent columns)" % ws},
        "formal_solver_pts_per_s": pts_s,
        "iterations_per_column": iters / (ncol * args.steps),
        "lte_start": {"value": ncol / lte_s, "unit": "columns/s", "iterations_per_column": lte_iters,
                      "precision": "fp32 formal solution/rates, fp64 rate equations/Ng"},
        "lte_start_fp64": fp64,
        "other_starts": other,
        "cube_512": big,
        "full_run": full_run,
        "stokes": stokes,
        "prd": prd,
        "surrogate": train_info,
        "launch": {"block_warps": s["block_warps"], "ctas_per_sm": s["ctas_per_sm"],
                   "cuda_graph_replayed": s["graph_replayed"], "kernels_per_step": s["launches"],
                   "shape_from": "rh_autotune on the loaded cube"},
        "converged_fraction": conv / (ncol * args.steps),
        "rerun_columns_per_step": rescued / args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops,
                     "flop_per_pt": alg_flop,
                     "flop_note": "algorithmic FP32 operations per point (2 x FMA + ADD + MUL) counted from the "
                                  "sweep's source for the transitions active at each wavelength, thick-layer SC "
                                  "branch (bench.algorithmic_flop_per_pt); plus %.1f MUFU operations" % alg_mufu,
                     "executed": {"flop_per_pt": FLOP_PER_PT, "achieved": achieved_exec,
                                  "frac": achieved_exec / peak_tflops,
                                  "note": "thread-level FP32 operations executed (ncu, 608 columns x 12 "
                                          "iterations): padding, both SC branches where a warp diverges, inactive "
                                          "slots of a tile's transition union, the profile build"},
                     "traffic": DRAM_BYTES_PER_COLUMN_ITERATION * iters / args.steps,
                     "traffic_note": "bytes per launch: ncu DRAM bytes per column-iteration on the "
                                     "608-column x 12-iteration case x column-iterations of one launch",
                     "kernel": "mali_kernel<float, CRD, cached profiles> (column-resident MALI, FP32 sweep)",
                     "issue_slots": {"achieved": WARP_INST_PER_COLUMN_ITERATION * iters / kern_s,
                                     "peak": nsm * 4 * sm_mhz * 1e6, "unit": "warp instructions/s",
                                     "frac": WARP_INST_PER_COLUMN_ITERATION * iters / kern_s
                                             / (nsm * 4 * sm_mhz * 1e6)},
                     "peak_note": "measured FP32 FMA rate (rh_fma_peak: %.1f TFLOP/s at %s MHz) scaled to the "
                                  "median SM clock of the timed region (%.0f MHz); nominal 152 x 128 x 2 x clock "
                                  "= %.1f TFLOP/s" % (p32["tflops"], p32.get("sm_mhz"), sm_mhz,
                                                      nsm * 256 * sm_mhz * 1e-6)},
        "measured_peaks": peaks_meas,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["true_error"] = true_error(cube, n_headline)
        line["cpu_baseline"] = cpu_baseline(cube)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_full(args):
    """The full-run configuration on the whole 512x512 cube (one step),
    with the plain FP64 GPU MALI timed on a sample beside it and sampled
    columns compared with the oracle; one JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1411_1079_gb300 as rh
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    with ClockSampler(0) as clk:
        r = run_full_config(rh, torch, 0, stream, 512 * 512, args.full_run_train,
                            fp64_columns=args.full_run_fp64, oracle_columns=args.full_run_oracle,
                            save_sample=args.full_run_save, sample_path=args.full_run_sample_path)
    line = {"metric": METRIC, "value": r["value"], "unit": "columns/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": r["solve"]["ms"] + r["stokes"]["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": r["workload"], "ndep": 128, "nlambda": 880, "nmu": 5,
                       "l2": "working set > L2 (inputs larger than L2)", "parallelism": "dp1 (independent columns)"},
            "full_run": r, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_full_compare(args):
    """True error of a full run's saved columns (--full-run-save) against
    the oracle converged to 1e-8 on this host's cores; one JSON line."""
    import oracle
    z = np.load(args.full_run_compare)
    idx, ncol, seed, hyb = z["idx"], int(z["ncol"]), int(z["seed"]), int(z["hybrid"])
    patom = rh_synth.hydrogen_like_atom(prd_lines=((1, 2), (1, 3)), prd_nlambda=200)
    full = rh_synth.chromosphere_cube(512, 512, 128, seed=seed)
    cube = full if ncol >= 512 * 512 else rh_synth.subset(full, slice(0, ncol))
    o = oracle.Oracle()
    o.setup_atom(patom)
    o.load_columns(rh_synth.subset(cube, idx))
    t0 = time.perf_counter()
    o.iterate(maxiter=3000, tol=1e-8, prd_eps0=0.05, prd_hybrid=hyb, nthreads=os.cpu_count() or 1)
    no, ito, sto, _ = o.populations()
    ok = (sto == oracle.ST_CONV) & (z["status"] == 0)
    d = np.abs(z["n"] / no - 1).max(axis=(1, 2))
    print(json.dumps({"true_error": {"max_rel_dn": float(d[ok].max()) if ok.any() else None,
                                     "median_rel_dn": float(np.median(d[ok])) if ok.any() else None,
                                     "per_column": [float(x) for x in d], "columns": [int(i) for i in idx],
                                     "oracle_iterations": [int(i) for i in ito],
                                     "gpu_iterations": [int(i) for i in z["iters"]],
                                     "reference": "oracle converged to 1e-8, %.0f s on %d host threads"
                                                  % (time.perf_counter() - t0, os.cpu_count() or 1)}}), flush=True)


def run_ncu_case(args):
    """Small fixed cases for ncu captures (columns of the 256x256 cube):
    crd -- the column kernel, --ncu-iters iterations from LTE;
    prd -- the same with Lyman alpha and beta in PRD (64 points each;
           --ncu-prd-hybrid: the hybrid scheme);
    stokes -- the H alpha Zeeman Stokes spectrum (400 wavelengths) after a
              few iterations;
    mlp -- one training epoch of the learned-guess network (BF16 GEMMs)."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_1411_1079_gb300 as rh
    cube = rh_synth.chromosphere_cube(NX, NY, NDEP, seed=1234)
    sub = rh_synth.subset(cube, slice(0, args.ncu_columns))
    ctx = rh.Context(0)
    kind = args.ncu_kind
    atom = rh_synth.hydrogen_like_atom(prd_lines=((1, 2), (1, 3))) if kind == "prd" else \
        rh_synth.hydrogen_like_atom()
    ctx.setup_atom(atom)
    ctx.load_columns(sub)
    out = {"ncu_case": kind, "columns": args.ncu_columns, "precision": args.ncu_precision,
           "prd_hybrid": int(args.ncu_prd_hybrid), "formal": args.ncu_formal}
    if kind in ("crd", "prd"):
        s = ctx.iterate(maxiter=args.ncu_iters, tol=0.0, precision=args.ncu_precision,
                        prd_eps0=0.05 if kind == "prd" else 0.0,
                        prd_hybrid=int(args.ncu_prd_hybrid) if kind == "prd" else 0, formal=args.ncu_formal)
        out.update(iterations=args.ncu_iters, seconds=s["seconds"], pts=s["pts"])
    elif kind == "stokes":
        ctx.iterate(maxiter=args.ncu_iters, tol=0.0, precision=1)
        ncol = args.ncu_columns
        rng = np.random.default_rng(2024)
        fld = [np.repeat(x[:, None], NDEP, axis=1) for x in
               (rng.uniform(0.0, 0.2, ncol), np.arccos(rng.uniform(-1.0, 1.0, ncol)), rng.uniform(0, 2 * np.pi, ncol))]
        ha = [i for i, (l, u) in enumerate(zip(atom["line_l"], atom["line_u"])) if (l, u) == (1, 2)][0]
        nu_ha = (atom["E_J"][2] - atom["E_J"][1]) / 6.62607015e-34
        lam = 2.99792458e8 / nu_ha + np.linspace(-2e-10, 2e-10, 400)
        t0 = time.perf_counter()
        ctx.emergent_stokes(ha, 1.5, *fld, lam, precision=args.ncu_precision)
        out.update(nlambda=400, seconds=time.perf_counter() - t0)
    elif kind == "mlp":
        ctx.solve(precision=1)                    # converged columns to learn from
        ctx.surrogate_init(hidden=512, nhidden=3, seed=0)
        t = ctx.surrogate_train(epochs=1, batch=512, lr=2e-3, seed=1)
        out.update(seconds=t["seconds"])
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ncu-case", action="store_true", help="small fixed case for profiler captures")
    ap.add_argument("--no-stokes", dest="stokes", action="store_false",
                    help="skip the Zeeman Stokes spectrum timing")
    ap.add_argument("--no-cube512", dest="cube512", action="store_false",
                    help="skip the one-step 512x512 cube measurement")
    ap.add_argument("--prd-columns", type=int, default=4096,
                    help="columns of the partial-redistribution timing (0: skip)")
    ap.add_argument("--full-run-columns", type=int, default=1216,
                    help="columns of the full-run configuration (512x512 x 128 heights, PRD Lyman alpha/beta at "
                         "200 frequencies, Stokes) to solve; 262144 = the whole cube (0: skip)")
    ap.add_argument("--full-run", action="store_true",
                    help="only the full-run configuration on the whole 512x512 cube (tens of minutes)")
    ap.add_argument("--full-run-fp64", type=int, default=152,
                    help="columns of the plain FP64 comparison in --full-run")
    ap.add_argument("--full-run-train", type=int, default=8192,
                    help="CRD-converged 128-height columns the full run's network is trained on")
    ap.add_argument("--full-run-oracle", type=int, default=0,
                    help="full-run columns compared with the oracle (its 200-point PRD kernels take minutes "
                         "per column to build on the host; 0: skip)")
    ap.add_argument("--full-run-save", type=int, default=0,
                    help="seeded full-run columns whose GPU results --full-run writes to --full-run-sample-path")
    ap.add_argument("--full-run-sample-path", default="full_run_sample.npz")
    ap.add_argument("--full-run-compare", default=None,
                    help="a saved full-run sample: compare it with the oracle on this host (no GPU)")
    ap.add_argument("--fp64-columns-per-sm", type=int, default=3,
                    help="columns per SM of the plain FP64 LTE-start comparison (0: skip)")
    ap.add_argument("--ncu-columns", type=int, default=608)
    ap.add_argument("--ncu-kind", default="crd", choices=["crd", "prd", "stokes", "mlp"])
    ap.add_argument("--ncu-precision", type=int, default=1)
    ap.add_argument("--ncu-iters", type=int, default=3)
    ap.add_argument("--ncu-prd-hybrid", action="store_true")
    ap.add_argument("--ncu-formal", type=int, default=0, choices=[0, 1])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.full_run_compare:
        run_full_compare(args)
    elif args.ncu_case:
        run_ncu_case(args)
    elif args.full_run:
        run_full(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
