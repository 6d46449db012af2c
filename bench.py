"""Benchmark: cell-steps/s of the compressible fast-Eulerian PISO step at 256^3.

Default workload ``hit256``: 256^3 periodic box, barotropic (gamma 1.4),
r.m.s. Mach 0.2, spectrum peak k0 = 8, nu = 0.001, one dust class (tau_p 0.05,
Y 0.01), CFL 0.5 adaptive step, 2 PISO correctors, pressure residual 1e-8;
synthetic spectral initial field (seed 0, one per rank).  One bench "step" is
one PISO time step of the whole box.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
                    [--impl ours|reference]

Prints one JSON line (rank 0).  ``value`` is device-timed throughput with the
state resident in HBM; ``e2e`` repeats the measurement through the public API
with the state copied from and back to pinned host buffers every step.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
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

WORKLOAD = "hit256"
METRIC = "cell-steps/s at 256^3 (learned vs plain solve, same residual); % of HBM peak"
UNIT = "cell-steps/s"

# Algorithmic words per cell (one N^3 array element read or written once) per
# launch of each kernel, barotropic closure, nd dust classes.  Mixed precision:
# the right-hand side also writes the first inner right-hand side and reads
# D^{-1} (it starts the refined solve); the corrector reads neither psi nor b.
def alg_words(kernel, nd, mixed=False, poly=False):
    if poly and kernel in ("cg_dirmatvec", "cg_rupdate", "cg_start", "rhs", "refine"):
        # Neumann-polynomial CG: z, pd_old, psi, x read, q, pd_new, x written | r, q, D^-1, psi read, z and r
        # written | r, D^-1, psi read, z written; the right-hand side and the refinement boundary do not
        # read D^-1 (the solve's first z has its own pass)
        return {"cg_dirmatvec": 7, "cg_rupdate": 6, "cg_start": 4, "rhs": 12, "refine": 10}[kernel]
    table = {
        "dt": 3, "div": 4, "pred": 21, "fluxn": 7 + 2 * nd, "asm": 18, "rhs": 13 if mixed else 11,
        "cg_init": 5, "cg_matvec": 3, "cg_update": 7, "cg_dir": 4,
        "cg_dirmatvec": 8, "cg_rupdate": 4, "cg_xfinal": 3, "corr": 19 if mixed else 21, "accel": 9,
        "dust": 8 + 4 * nd + 2,  # last corrector adds u reads and p write; averaged over 2 correctors
        "bicg_p": 4, "bicg_v": 4, "bicg_s": 3, "bicg_t": 3, "bicg_x": 8, "true_res": 3,
        # refinement (field word = 4 bytes; x64 counts as two words)
        "mix_residual": 6, "mix_accum": 5, "mix_finish": 3, "commit": 0,
        # fused refinement: pairs read and written, x, pd, b, psi, dinv read, r and the FP32 solution written
        "refine": 11, "cg_start": 4,
    }
    return table[kernel]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from profiles/traffic_<workload>.txt (an
    ncu capture), or None when absent or when the kernel sources changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_%s.txt" % workload)
    srcs = [os.path.join(ROOT, "paper_1404_0959_gb300", "csrc", f)
            for f in ("krylov_kernels.cu", "zbulk.cuh", "fe_internal.cuh")]
    try:
        h = hashlib.sha256()
        for f in srcs:
            with open(f, "rb") as fh:
                h.update(fh.read())
        digest = h.hexdigest()[:16]
        with open(path) as fh:
            for line in fh:
                parts = line.split()
                if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel:
                    return float(parts[1]) if parts[2] == digest else None
    except OSError:
        return None
    return None


# ---- multi-rank aggregation (replicas: one box per rank, no data-path collective) ----
def rank_box(cfg, rank):
    """The box of one rank: the workload's parameters with seed + rank (independent replicas)."""
    return dict(N=cfg["N"], nu=cfg["nu"], tau_p=list(cfg["tau_p"]), Y0=list(cfg["Y0"]), mach_rms=cfg["mach_rms"],
                k0=cfg["k0"], seed=cfg["seed"] + rank)


def max_over_ranks(t, world, device="cuda"):
    """The slowest rank's time (every rank returns it); t itself on one rank."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(cells_per_rank, steps, world, t):
    """Whole-job throughput: the cells all ranks stepped over the slowest rank's time."""
    return cells_per_rank * steps * world / t


class Clocks:
    """nvidia-smi sampler (every 25 ms) running across the timed region.

    Each sample carries nvidia-smi's own timestamp; ``begin()`` and ``end()``
    mark the timed region on the same wall clock, and only the samples taken
    between the two marks are summarised (the sampler is already producing
    samples when ``start()`` returns, so a short region still gets some)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 25

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        deadline = time.time() + 5.0  # until the first samples are on disk
        while time.time() < deadline and self.proc.poll() is None:
            with open(self.path) as f:
                if sum(1 for _ in f) >= 2:
                    break
            time.sleep(0.02)

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text):
        from datetime import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.strptime(text, fmt).timestamp()
            except ValueError:
                pass
        return None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(2.0 * self.PERIOD_MS / 1e3)  # the sample that closes the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        inside = rows
        if self.t0 is not None and self.t1 is not None:
            stamped = [(self._stamp(r[0]), r) for r in rows]
            inside = [r for ts, r in stamped if ts is not None and self.t0 <= ts <= self.t1]
        num = lambda v: v.replace(".", "", 1).isdigit()
        sm = [float(r[2]) for r in inside if num(r[2])]
        mx = [float(r[3]) for r in rows if num(r[3])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "period_ms": self.PERIOD_MS,
                "region_s": (self.t1 - self.t0) if self.t0 is not None and self.t1 is not None else None}


def oracle_sample(N, steps, cfg):
    """Time `steps` oracle steps of the workload physics on an N^3 box (spectral IC)."""
    from oracle import piso
    prm = piso.Params(N=N, closure=cfg["closure"], nu=cfg["nu"], tau_p=list(cfg["tau_p"]), Y0=list(cfg["Y0"]),
                      mach_rms=cfg["mach_rms"], k0=cfg["k0"], seed=cfg["seed"], cfl=cfg["cfl"],
                      p_tol=cfg["p_tol"])
    st = piso.initial_state(prm)
    t0 = time.perf_counter()
    for _ in range(steps):
        st, _info = piso.step(prm, st)
    return time.perf_counter() - t0


def host_cpu():
    """CPU model and logical core count of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def _oracle_worker(args):
    N, cfg = args
    return oracle_sample(N, 1, cfg)


def oracle_all_cores(N, cfg, procs):
    """Wall time of `procs` independent one-step oracle samples run at once in
    spawned processes (one per core): the oracle as it stands, replicated."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_worker, [(8, cfg)] * procs)  # start-up (imports) outside the timed region
        t0 = time.perf_counter()
        pool.map(_oracle_worker, [(N, cfg)] * procs)
        return time.perf_counter() - t0


def run_reference(args, cfg, rank):
    if rank != 0:
        return
    N = args.ref_n
    times = []
    for i in range(args.warmup + args.steps):
        t = oracle_sample(N, 1, cfg)
        if i >= args.warmup:
            times.append(t)
    total = sum(times)
    value = N ** 3 * len(times) / total
    cpu = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_N": N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "cpu_model": cpu["model"], "nproc": cpu["nproc"],
                             "sample": "each step: one oracle PISO step of the %s physics on a %d^3 box "
                                       "(single-threaded numpy)" % (WORKLOAD, N)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_path(fe, box, cfg, precision, solver, args, stream, learned_every=0, weights=None):
    """Steps/s of one solver path on the same workload (untimed set-up excluded).
    Learned paths train the network on this run's own pressure pairs first
    (or take `weights` from an earlier path); the trained weights are returned."""
    import torch
    from paper_1404_0959_gb300 import learned
    N = box["N"]
    s = fe.Solver([box], precision=precision, closure=cfg["closure"], cfl=cfg["cfl"], p_tol=cfg["p_tol"],
                  p_maxit=1000, solver=solver, learned_every=learned_every, stream=stream.cuda_stream)
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    out = {"precision": "fp64" if precision == fe.FE_FP64 else "mixed",
           "solver": "jacobi-pcg" if solver == fe.FE_PCG_JACOBI else "neumann1-pcg" if solver == fe.FE_PCG_POLY else
           ("fcg, learned direction every iteration" if learned_every == 1 else
            "fcg, learned first direction of each corrector")}
    if solver == fe.FE_FCG_LEARNED:
        if weights is None:
            fe.fe_load_preconditioner(s.ctx, learned.he_init(0))
            bank = learned.PairBank(s, 6 * args.learn_steps)
            bank.harvest(s, args.learn_steps)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hist = learned.train(s, bank, args.learn_iters, lr=1e-3)
            torch.cuda.synchronize()
            out.update(train_pairs=bank.n, train_iters=args.learn_iters, train_s=time.perf_counter() - t0,
                       loss_first=hist[0], loss_last=hist[-1])
            weights = fe.fe_get_preconditioner(s.ctx)
            s.init_state(0, fe.FE_INIT_SPECTRAL)
        else:
            fe.fe_load_preconditioner(s.ctx, weights)
        s.profile_start("unet")
        s.step(1)
        prof = s.profile_stop()
        out["net_ms_per_apply"] = prof["target_ms"] / max(prof["target_launches"], 1)
        out["net_applies_per_step"] = prof["target_launches"]
    s.autotune(1)
    s.use_graphs(not args.no_graphs)
    code, _ = s.step(args.warmup)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    K = max(2, args.steps // 2)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    code, info = s.step(K)
    ev1.record(stream)
    torch.cuda.synchronize()
    assert code == fe.FE_OK, fe.fe_strerror(code)
    t = ev0.elapsed_time(ev1) / 1e3
    out.update(steps=K, ms_per_step=1e3 * t / K, value=float(N) ** 3 * K / t, krylov_iters_last_step=info[0]["iters"],
               rel_res_last_step=info[0]["rel_res"])
    s.close()
    return out, weights


def time_les(fe, box, cfg, args, stream, m=2):
    """CUDA-event time of the a-priori LES analysis (fe_les_apriori) on the
    workload's spectral state in FP32; roofline from its 74 algorithmic words
    per cell (x pass 4 read + 10 written, y and z passes 10 + 10 each, Favre
    velocity 4 + 3, statistics 13 read)."""
    import torch
    N = box["N"]
    s = fe.Solver([box], precision=fe.FE_FP32_MIXED, closure=cfg["closure"], p_tol=cfg["p_tol"],
                  stream=stream.cuda_stream)
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    for _ in range(max(args.warmup, 3)):
        st = fe.fe_les_apriori(s.ctx, 0, m, 0.17)
    K = max(3, args.steps)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(K):
        st = fe.fe_les_apriori(s.ctx, 0, m, 0.17)
    ev1.record(stream)
    torch.cuda.synchronize()
    s.close()
    ms = ev0.elapsed_time(ev1) / K
    hbm, kind = peaks()
    gbs = 74 * 4 * float(N) ** 3 / (ms / 1e3) / 1e9
    return {"N": N, "m": m, "ms_per_call": ms, "alg_bytes": 74 * 4 * N ** 3, "achieved_gbs": gbs, "peak": hbm,
            "frac": gbs / hbm, "note": "includes the host read of the block partial sums", "stats": st}


# FLOPs of one network application at N^3 (2 x MACs; 27-tap convolutions over
# the padded channel counts the kernels compute): e1a, e1b, out at N (16 -> 16),
# d1 (N/2, 16 -> 32), e2 (N/2, 32 -> 32), d2 (N/4, 32 -> 64), e3 (N/4, 64 -> 64),
# u2 (N/2, 96 -> 32), u1 (N, 48 -> 16).
def unet_flops(N):
    n0, n1, n2 = N ** 3, (N // 2) ** 3, (N // 4) ** 3
    macs = 27 * (3 * n0 * 16 * 16 + n1 * 16 * 32 + n1 * 32 * 32 + n2 * 32 * 64 + n2 * 64 * 64 +
                 n1 * 96 * 32 + n0 * 48 * 16)
    return 2.0 * macs


def solver_id(fe, args):
    """The pressure solver of the FP32 paths: CG with the first-order Neumann polynomial preconditioner
    (Jacobi-PCG where the planes are not streamed), or Jacobi-PCG."""
    return fe.FE_PCG_POLY if args.solver == "poly" else fe.FE_PCG_JACOBI


def time_ensemble(fe, args, compare=False):
    """The 64-box ensemble of uneven boxes (N in {32, 48, 64, 96}, FP32 fields, barotropic) in one context:
    one launch per stage over every box, CUDA-graph steps, autotuned tiles; with compare, the same boxes
    each in a context of its own stepped one after the other (same steps, same state)."""
    import torch
    from paper_1404_0959_gb300.inputs import ensemble64_boxes
    boxes = ensemble64_boxes(64)
    cells = float(sum(b["N"] ** 3 for b in boxes))
    K, W = max(args.steps, 3), max(args.warmup, 3)

    def timed(solver_boxes):
        s = fe.Solver(solver_boxes, precision=fe.FE_FP32_MIXED, p_tol=1e-8, solver=solver_id(fe, args))
        s.init_state(-1, fe.FE_INIT_SPECTRAL)
        s.autotune(2)
        s.use_graphs(True)
        code, _ = s.step(W)
        assert code == fe.FE_OK, fe.fe_strerror(code)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        code, _ = s.step(K)
        ev1.record()
        torch.cuda.synchronize()
        assert code == fe.FE_OK, fe.fe_strerror(code)
        s.close()
        return ev0.elapsed_time(ev1) / 1e3

    t_ens = timed(boxes)
    out = {"boxes": len(boxes), "cells": int(cells), "steps": K, "ms_per_step": 1e3 * t_ens / K,
           "value": cells * K / t_ens, "unit": "cell-steps/s"}
    if compare:
        t_one = sum(timed([b]) for b in boxes)
        out["per_box_contexts"] = {"value": cells * K / t_one, "ms_per_step": 1e3 * t_one / K}
    return out


def ensemble_only(args):
    """--ensemble: the 64-box ensemble of uneven boxes (N in {32, 48, 64, 96}, FP32 fields) stepped in
    one context -- one launch per stage over every box, CUDA graph, autotuned tiles -- against the
    same boxes each in a context of its own stepped one after the other (same steps, same state)."""
    import torch
    from paper_1404_0959_gb300 import build, fe
    from paper_1404_0959_gb300.inputs import ensemble64_boxes
    build.build()
    boxes = ensemble64_boxes(64)
    cells = float(sum(b["N"] ** 3 for b in boxes))
    K, W = args.steps, args.warmup

    def timed(solver_boxes):
        s = fe.Solver(solver_boxes, precision=fe.FE_FP32_MIXED, p_tol=1e-8, solver=solver_id(fe, args))
        s.init_state(-1, fe.FE_INIT_SPECTRAL)
        s.autotune(2)
        s.use_graphs(True)
        code, _ = s.step(W)
        assert code == fe.FE_OK, fe.fe_strerror(code)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        code, _ = s.step(K)
        ev1.record()
        torch.cuda.synchronize()
        assert code == fe.FE_OK, fe.fe_strerror(code)
        s.close()
        return ev0.elapsed_time(ev1) / 1e3

    t_ens = timed(boxes)
    t_one = sum(timed([b]) for b in boxes)
    line = {"metric": "cell-steps/s, 64-box ensemble of uneven boxes (one context vs one context per box)",
            "value": cells * K / t_ens, "unit": "cell-steps/s", "n_gpus": 1, "steps": K, "warmup": W,
            "ms_per_step": 1e3 * t_ens / K, "higher_is_better": True,
            "dtype": "f32 fields, FP64-class float-pair reductions and refinement",
            "data": "synthetic spectral HIT boxes (seed = box index), no dataset",
            "config": {"workload": "ensemble64", "boxes": len(boxes), "cells": int(cells), "p_tol": 1e-8,
                       "cuda_graphs": True},
            "per_box_contexts": {"value": cells * K / t_one, "ms_per_step": 1e3 * t_one / K}}
    print(json.dumps(line), flush=True)


def part_only(args):
    """--part les|twofluid|twoway|fourier|iso: one of the scope table's further rows alone at --N (FP32 fields,
    the benchmark workload's physics), CUDA-event timed, one JSON line."""
    import torch
    from paper_1404_0959_gb300 import build, fe
    from paper_1404_0959_gb300.inputs import WORKLOADS
    build.build()
    cfg = dict(WORKLOADS[WORKLOAD])
    N = args.N
    box = dict(N=N, nu=cfg["nu"], tau_p=cfg["tau_p"], Y0=cfg["Y0"], mach_rms=cfg["mach_rms"], k0=cfg["k0"], seed=0)
    stream = torch.cuda.current_stream()
    hbm, kind = peaks()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"part": args.part, "N": N, "dtype": "f32 fields", "data": "synthetic spectral HIT field", "peak": hbm,
           "solver": "neumann1-pcg" if args.solver == "poly" else "jacobi-pcg",
           "peak_kind": kind}
    if args.part == "les":
        out.update(time_les(fe, box, cfg, args, stream))
    elif args.part == "twofluid":
        res = {}
        for model in (fe.FE_DUST_EQUILIBRIUM, fe.FE_DUST_TWO_FLUID):
            s = fe.Solver([box], precision=fe.FE_FP32_MIXED, closure=cfg["closure"], p_tol=cfg["p_tol"], p_maxit=1000,
                          dust_model=model, solver=solver_id(fe, args), stream=stream.cuda_stream)
            s.init_state(0, fe.FE_INIT_SPECTRAL)
            s.autotune(1)
            s.use_graphs(True)
            code, _ = s.step(args.warmup)
            assert code == fe.FE_OK, fe.fe_strerror(code)
            torch.cuda.synchronize()
            ev0.record(stream)
            code, _ = s.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            assert code == fe.FE_OK, fe.fe_strerror(code)
            name = "two_fluid" if model == fe.FE_DUST_TWO_FLUID else "equilibrium"
            res[name] = {"ms_per_step": ev0.elapsed_time(ev1) / args.steps}
            if model == fe.FE_DUST_TWO_FLUID:
                s.use_graphs(False)
                nd = len(cfg["tau_p"])
                for k, words in (("tf_pred", 23 * nd), ("tf_corr", 24 * nd)):
                    s.profile_start(k)
                    s.step(args.steps)
                    p = s.profile_stop()
                    ms = p["target_ms"] / max(p["target_launches"], 1)
                    gbs = words * 4 * float(N) ** 3 / (ms / 1e3) / 1e9
                    res[k] = {"ms_per_launch": ms, "alg_words_per_cell": words, "achieved_gbs": gbs,
                              "frac": gbs / hbm}
            s.close()
        out.update(res)
    elif args.part == "twoway":
        # the benchmark workload's physics with the dust's reaction on the gas (one class, Y = 0.01)
        res = {}
        for coupling in (fe.FE_COUPLING_ONE_WAY, fe.FE_COUPLING_TWO_WAY):
            s = fe.Solver([box], precision=fe.FE_FP32_MIXED, closure=cfg["closure"], p_tol=cfg["p_tol"],
                          p_maxit=1000, coupling=coupling, solver=solver_id(fe, args), stream=stream.cuda_stream)
            s.init_state(0, fe.FE_INIT_SPECTRAL)
            s.autotune(1)
            s.use_graphs(True)
            code, _ = s.step(args.warmup)
            assert code == fe.FE_OK, fe.fe_strerror(code)
            torch.cuda.synchronize()
            ev0.record(stream)
            code, info = s.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            assert code == fe.FE_OK, fe.fe_strerror(code)
            two = coupling == fe.FE_COUPLING_TWO_WAY
            r = {"ms_per_step": ev0.elapsed_time(ev1) / args.steps, "krylov_iters_last_step": info[0]["iters"]}
            s.use_graphs(False)
            nd = len(cfg["tau_p"])
            # two-way adds Ysum to the predictor and Du/Dt, Ysum and Du/Dt to the assembly
            for k, extra in (("pred", 1), ("asm", 4), ("accel", 1)):
                words = alg_words(k, nd, True) + (extra if two else 0)
                s.profile_start(k)
                s.step(args.steps)
                pr = s.profile_stop()
                ms = pr["target_ms"] / max(pr["target_launches"], 1)
                gbs = words * 4 * float(N) ** 3 / (ms / 1e3) / 1e9
                r[k] = {"ms_per_launch": ms, "alg_words_per_cell": words, "achieved_gbs": gbs, "frac": gbs / hbm}
            res["two_way" if two else "one_way"] = r
            s.close()
        out.update(res)
    elif args.part == "fourier":
        # the Fourier-closure workloads: 128^3 (one class) and 512^3 (three classes), FP32 fields
        res = {}
        for name, n_ in [(w_, n_) for w_, n_ in (("hit128f", 128), ("hit512f", 512))
                         if str(n_) in args.fourier_sizes.split(",")]:
            w = WORKLOADS[name]
            bx_ = dict(N=n_, nu=w["nu"], tau_p=w["tau_p"], Y0=w["Y0"], mach_rms=w["mach_rms"], k0=w["k0"], seed=0)
            s = fe.Solver([bx_], precision=fe.FE_FP32_MIXED, closure=w["closure"], p_tol=w["p_tol"], p_maxit=1000,
                          solver=solver_id(fe, args), stream=stream.cuda_stream)
            s.init_state(0, fe.FE_INIT_SPECTRAL)
            s.autotune(1)
            s.use_graphs(True)
            code, _ = s.step(args.warmup)
            assert code == fe.FE_OK, fe.fe_strerror(code)
            torch.cuda.synchronize()
            ev0.record(stream)
            code, info = s.step(args.steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            assert code == fe.FE_OK, fe.fe_strerror(code)
            ms = ev0.elapsed_time(ev1) / args.steps
            r = {"N": n_, "classes": len(w["tau_p"]), "ms_per_step": ms, "value": float(n_) ** 3 / (ms / 1e3),
                 "unit": "cell-steps/s", "krylov_iters_last_step": info[0]["iters"]}
            s.use_graphs(False)
            for k in ("fe_cell", "fe_face", "fluxn", "dust"):
                s.profile_start(k)
                s.step(2)
                pr = s.profile_stop()
                r[k + "_ms_per_step"] = pr["target_ms"] / 2
            res[name] = r
            s.close()
        out.update(res)
    elif args.part == "iso":
        s = fe.Solver([box], precision=fe.FE_FP32_MIXED, closure=cfg["closure"], p_tol=cfg["p_tol"],
                      stream=stream.cuda_stream)
        s.init_state(0, fe.FE_INIT_SPECTRAL)
        q = s.q_criterion(0)
        iso = 0.5 * s.diagnostics(0)["enstrophy"]
        n, area = fe.fe_isosurface(s.ctx, 0, q.data_ptr(), iso)
        tri = torch.empty((n, 9), dtype=torch.float64, device="cuda")
        W = args.width
        depth = torch.empty((W, W), dtype=torch.float32, device="cuda")
        h = 2 * math.pi / N
        for _ in range(args.warmup):
            fe.fe_isosurface(s.ctx, 0, q.data_ptr(), iso, tri.data_ptr(), n)
            fe.fe_raster_depth(s.ctx, tri.data_ptr(), n, W, (N + 1) * h, depth.data_ptr())
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            fe.fe_isosurface(s.ctx, 0, q.data_ptr(), iso, tri.data_ptr(), n)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_ext = ev0.elapsed_time(ev1) / args.steps
        ev0.record(stream)
        for _ in range(args.steps):
            fe.fe_raster_depth(s.ctx, tri.data_ptr(), n, W, (N + 1) * h, depth.data_ptr())
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_ras = ev0.elapsed_time(ev1) / args.steps
        # extraction traffic: the field read by the count and the emit pass, the per-cube counts
        # written and read, the triangles written (72 bytes each)
        alg = 2 * 4 * N ** 3 + 2 * 4 * N ** 3 + 72 * n
        gbs = alg / (ms_ext / 1e3) / 1e9
        covered = int(torch.isfinite(depth).sum().item())
        out.update(iso=iso, triangles=n, area=area, extract_ms=ms_ext, extract_alg_bytes=alg, extract_gbs=gbs,
                   extract_frac=gbs / hbm, raster_width=W, raster_ms=ms_ras, covered_pixels=covered,
                   note="extraction includes two host reads (block totals, block areas)")
        s.close()
    print(json.dumps(out), flush=True)


def unet_only(args):
    """--unet: CUDA-event time of fe_precond_apply on a random residual (He-initialised weights)."""
    import torch
    from paper_1404_0959_gb300 import fe, learned
    from paper_1404_0959_gb300.inputs import WORKLOADS
    fe.load_library()
    w = WORKLOADS[WORKLOAD]
    N = args.N
    box = dict(N=N, nu=w["nu"], tau_p=w["tau_p"], Y0=w["Y0"], mach_rms=w["mach_rms"], k0=w["k0"], seed=0)
    s = fe.Solver([box], precision=fe.FE_FP32_MIXED, solver=fe.FE_FCG_LEARNED, p_tol=1e-8)
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    fe.fe_load_preconditioner(s.ctx, learned.he_init(0, zero_last=False))
    g = torch.Generator(device="cuda").manual_seed(0)
    r = torch.randn(N, N, N, device="cuda", generator=g)
    z = torch.empty_like(r)
    for _ in range(args.warmup):
        fe.fe_precond_apply(s.ctx, 0, r.data_ptr(), 0.01, z.data_ptr())
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fe.fe_precond_apply(s.ctx, 0, r.data_ptr(), 0.01, z.data_ptr())
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    fl = unet_flops(N)
    print(json.dumps({"metric": "learned-preconditioner network applications/s at %d^3" % N, "value": 1e3 / ms,
                      "unit": "applications/s", "ms_per_apply": ms, "tflops": fl / ms / 1e9,
                      "flops_per_apply": fl, "steps": args.steps, "warmup": args.warmup,
                      "note": "includes the host read of the error flag after every application"}))
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--solver", default="poly", choices=["jacobi", "poly"],
                    help="pressure CG preconditioner: Jacobi, or the first-order Neumann polynomial")
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--ref-n", type=int, default=64)
    ap.add_argument("--cpu-n", type=int, default=128)
    ap.add_argument("--cpu-procs", type=int, default=16, help="oracle processes of the all-cores CPU baseline")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kernel", default=None, help="kernel timed live for the roofline (default: largest share)")
    ap.add_argument("--no-breakdown", action="store_true", help="skip the untimed per-kernel pass")
    ap.add_argument("--no-tune", action="store_true", help="keep the default tile depth")
    ap.add_argument("--tile", type=int, default=0, help="fixed tile depth (no autotuning)")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 and learned comparison paths")
    ap.add_argument("--no-graphs", action="store_true", help="host-driven steps in the headline region")
    ap.add_argument("--learn-steps", type=int, default=4, help="steps harvested for training (learned path)")
    ap.add_argument("--learn-iters", type=int, default=120, help="training iterations (learned path)")
    ap.add_argument("--ensemble", action="store_true",
                    help="time the 64-box ensemble in one context against one context per box")
    ap.add_argument("--unet", action="store_true",
                    help="time only the learned preconditioner's network pass (K applications at N^3)")
    ap.add_argument("--part", default=None, choices=["les", "twofluid", "twoway", "fourier", "iso"],
                    help="time one further row alone: a-priori LES, two-fluid dust step, two-way coupled step, "
                         "Fourier-closure workloads, Q iso-surface + raster")
    ap.add_argument("--width", type=int, default=2048, help="depth image width for --part iso")
    ap.add_argument("--fourier-sizes", default="128,512", help="box sizes of --part fourier (128, 512)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.unet:
        return unet_only(args)
    if args.part:
        return part_only(args)
    if args.ensemble:
        return ensemble_only(args)

    from paper_1404_0959_gb300.inputs import WORKLOADS
    cfg = dict(WORKLOADS[WORKLOAD])
    cfg["N"] = args.N

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, cfg, rank)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1404_0959_gb300 import build, fe
    if rank == 0:
        build.build()
    barrier()

    precision = fe.FE_FP64 if args.precision == "fp64" else fe.FE_FP32_MIXED
    N = cfg["N"]
    nd = len(cfg["tau_p"])
    box = rank_box(cfg, rank)
    stream = torch.cuda.current_stream()
    solver = solver_id(fe, args)
    poly = solver == fe.FE_PCG_POLY and precision == fe.FE_FP32_MIXED
    s = fe.Solver([box], precision=precision, closure=cfg["closure"], cfl=cfg["cfl"], p_tol=cfg["p_tol"],
                  p_maxit=1000, solver=solver, stream=stream.cuda_stream)
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    if args.tile > 0:
        s.set_tiling(args.tile)
        tz = args.tile
    else:
        tz = s.autotune(2) if not args.no_tune else 0
    code, _ = s.step(args.warmup)
    assert code == fe.FE_OK, fe.fe_strerror(code)

    # Every measurement below starts from the state after the warm-up steps
    # (device copies of all state fields and the clock, restored before each
    # pass), so the breakdown, the kernel-level region, the headline region and
    # the end-to-end region all step the same flow through the same Krylov work
    # whichever optional passes run.
    state_ids = [fe.FE_RHO, fe.FE_UX, fe.FE_UY, fe.FE_UZ, fe.FE_P, fe.FE_PHIX, fe.FE_PHIY, fe.FE_PHIZ] + \
                [fe.FE_Y0 + j for j in range(nd)] + ([fe.FE_T] if cfg["closure"] == fe.FE_FOURIER else [])
    snap = {f: s.get_field(0, f, device=True) for f in state_ids}
    snap_clock = s.diagnostics(0)

    def restore():
        fe.fe_set_fields(s.ctx, 0, state_ids, [snap[f].data_ptr() for f in state_ids], 1)
        fe.fe_set_clock(s.ctx, 0, snap_clock["t"], snap_clock["dt_prev"])
        torch.cuda.synchronize()

    # untimed pass: per-kernel device time over one step, one kernel id at a time
    names = ["dt", "div", "pred", "fluxn", "asm", "rhs", "cg_init", "cg_matvec", "cg_update", "cg_dir",
             "cg_dirmatvec", "cg_rupdate", "cg_start", "cg_xfinal", "corr", "accel", "dust", "mix_residual",
             "mix_accum", "refine", "mix_finish", "commit"]
    share = {}
    for k in ([] if args.no_breakdown else names):
        restore()
        s.profile_start(k)
        s.step(1)
        p = s.profile_stop()
        share[k] = (p["target_ms"], p["target_launches"])
    kernel = args.kernel or (max(share, key=lambda k: share[k][0]) if share else "cg_dirmatvec")

    # kernel-level timed region: host-driven steps with CUDA events around
    # every launch of the dominant kernel, and the launch count
    restore()
    s.profile_start(kernel)
    torch.cuda.synchronize()
    code, _ = s.step(args.steps)
    prof = s.profile_stop()
    assert code == fe.FE_OK, fe.fe_strerror(code)

    # headline timed region: each step one CUDA graph (solver loops on the device)
    if not args.no_graphs:
        s.use_graphs(True)
        code, _ = s.step(1)  # builds the graphs of both state parities
        code, _ = s.step(1)
        assert code == fe.FE_OK, fe.fe_strerror(code)
    restore()
    clocks = Clocks(local)
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    clocks.begin()
    ev0.record(stream)
    code, info = s.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    barrier()
    ck = clocks.stop()
    assert code == fe.FE_OK, fe.fe_strerror(code)
    t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world)
    cells = float(N) ** 3
    value = job_rate(cells, args.steps, world, t)
    w = 8 if precision == fe.FE_FP64 else 4
    hbm, peak_kind = peaks()
    per_launch_ms = prof["target_ms"] / max(prof["target_launches"], 1)
    mixed = precision == fe.FE_FP32_MIXED
    alg_bytes = alg_words(kernel, nd, mixed, poly) * w * cells
    # whole step: algorithmic bytes of every launch of the breakdown step over the headline step time
    step_bytes = sum(n * alg_words(k, nd, mixed, poly) * w * cells for k, (_, n) in share.items()) if share else None
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9 if per_launch_ms > 0 else 0.0
    iters = info[0]["iters"]

    # end to end through the public API: state from pinned host, step, state back
    e2e = None
    if not args.no_e2e:
        fields = [fe.FE_RHO, fe.FE_UX, fe.FE_UY, fe.FE_UZ, fe.FE_P, fe.FE_PHIX, fe.FE_PHIY, fe.FE_PHIZ] + \
                 [fe.FE_Y0 + j for j in range(nd)]
        dt_ = torch.float64 if w == 8 else torch.float32
        host = {f: torch.empty((N, N, N), dtype=dt_, pin_memory=True) for f in fields}
        restore()
        for f in fields:
            fe.fe_get_field(s.ctx, 0, f, host[f].data_ptr(), 0)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        ptrs = [host[f].data_ptr() for f in fields]
        for _ in range(args.steps):
            fe.fe_set_fields(s.ctx, 0, fields, ptrs, 0)
            code, _ = s.step(1)
            fe.fe_get_fields(s.ctx, 0, fields, ptrs, 0)
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world)
        nbytes = len(fields) * cells * w
        e2e = {"value": job_rate(cells, args.steps, world, te), "unit": UNIT, "h2d_bytes_per_step": int(nbytes),
               "d2h_bytes_per_step": int(nbytes)}

    s.close()

    # the same workload on the other two solver paths of the metric: plain FP64
    # Jacobi-PCG, and FP32 steps whose pressure solve starts from the learned
    # network's direction (trained first on this run's own pressure pairs)
    extra = {}
    if not args.no_compare:
        extra["plain_fp64"], _ = time_path(fe, box, cfg, fe.FE_FP64, fe.FE_PCG_JACOBI, args, stream)
        other = fe.FE_PCG_JACOBI if solver == fe.FE_PCG_POLY else fe.FE_PCG_POLY
        extra["jacobi_fp32" if other == fe.FE_PCG_JACOBI else "neumann1_fp32"], _ = time_path(
            fe, box, cfg, fe.FE_FP32_MIXED, other, args, stream)
        extra["learned_fp32"], wts = time_path(fe, box, cfg, fe.FE_FP32_MIXED, fe.FE_FCG_LEARNED, args, stream, 0)
        extra["learned_fp32_every_iteration"], _ = time_path(fe, box, cfg, fe.FE_FP32_MIXED, fe.FE_FCG_LEARNED, args,
                                                             stream, 1, wts)
        extra["les_apriori_fp32"] = time_les(fe, box, cfg, args, stream)
        extra["ensemble64_fp32"] = time_ensemble(fe, args)
        # break-even: a network application against the CG iterations it would have to save
        if share:
            per = lambda k: share[k][0] / share[k][1] if share.get(k, (0, 0))[1] else 0.0
            cg_ms = per("cg_dirmatvec") + per("cg_rupdate")
            net_ms = extra["learned_fp32"].get("net_ms_per_apply")
            extra["break_even"] = {"cg_iteration_ms": cg_ms, "net_ms_per_apply": net_ms,
                                   "cg_iterations_one_application_must_save": (net_ms / cg_ms) if cg_ms and net_ms
                                   else None}

    cpu = None
    if rank == 0 and not args.no_cpu:
        host = host_cpu()
        tc = oracle_sample(args.cpu_n, 1, cfg)
        procs = max(1, min(host["nproc"] or 1, args.cpu_procs))
        tp = oracle_all_cores(args.cpu_n, cfg, procs) if procs > 1 else tc
        cpu = {"value": procs * args.cpu_n ** 3 / tp, "unit": UNIT, "cores": procs, "kind": "oracle",
               "cpu_model": host["model"], "nproc": host["nproc"],
               "sample": "%d independent one-step FP64 oracle runs of the %s physics on %d^3 boxes (spectral IC, "
                         "same seed), one spawned single-threaded process per core, run at once"
                         % (procs, WORKLOAD, args.cpu_n),
               "single_core": {"value": args.cpu_n ** 3 / tc, "unit": UNIT, "cores": 1,
                               "sample": "one oracle step on a %d^3 box in this process" % args.cpu_n}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if w == 8 else "f32 fields, FP64-class float-pair reductions and refinement",
                "data": "synthetic spectral HIT field (seed per rank), no dataset",
                "config": {"workload": WORKLOAD, "N": N, "closure": "barotropic", "mach_rms": cfg["mach_rms"],
                           "k0": cfg["k0"], "nu": cfg["nu"], "tau_p": cfg["tau_p"], "Y0": cfg["Y0"],
                           "p_tol": cfg["p_tol"], "precision": args.precision,
                           "solver": "neumann1-pcg" if poly else "jacobi-pcg",
                           "n_corr": 2, "krylov_iters_last_step": iters, "tile": "32x8x%d" % tz if tz else "default",
                           "cuda_graphs": not args.no_graphs,
                           "timed_from": "state after the warm-up steps, restored before every measured pass",
                           "l2": "state of %.1f GB >> 126 MB L2, no flush needed" % (
                               (40 + 4 * nd) * cells * w / 1e9),
                           "parallelism": "replicas" if world > 1 else "single box"},
                "step_roofline": None if step_bytes is None else {
                    "alg_bytes_per_step": step_bytes, "achieved": step_bytes / t * args.steps / 1e9, "peak": hbm,
                    "unit": "GB/s", "frac": step_bytes / t * args.steps / 1e9 / hbm},
                "roofline": {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "peak_kind": peak_kind,
                             "traffic": recorded_traffic(kernel + ("@neumann1" if poly and kernel in (
                                 "cg_dirmatvec", "cg_rupdate", "cg_start") else ""), WORKLOAD) if N == 256 else None,
                             "alg_bytes_per_launch": alg_bytes, "launches": prof["target_launches"],
                             "ms_per_launch": per_launch_ms},
                "kernel_ms_per_step": {k: round(v[0], 4) for k, v in share.items() if v[1] > 0},
                "kernel_launches_per_step": {k: v[1] for k, v in share.items() if v[1] > 0},
                "paths": extra,
                "gpu_launches": prof["launches"],
                "gpu_launches_note": "kernel launches of %d host-driven steps (the graph steps run the same kernels "
                                     "plus one loop-condition kernel per solver iteration)" % args.steps,
                "clocks": ck, "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
