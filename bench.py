#!/usr/bin/env python
"""Benchmark: ensemble CG sample-solves/s on the 64^3-cell KL diffusion workload.

One step = the whole hot path over one batch of 1024 samples: per-mesh set-up
(CRS graph, KL tables, mode matrices), then for each ensemble of s samples the
ensemble assembly and the ensemble CG solve to relative residual 1e-8.  Inputs
(the KL variables of all samples) are resident on the GPU before the timed
region; every step's working set (matrix values of 1.8 GB per s=32 ensemble)
is far larger than the 129 MB L2, so no L2 flush is needed between steps.

Also reported: the roofline of the dominant kernel (the CG SpMV, timed with
CUDA events inside the library on its launch stream, on the first ensemble of
every step: the CG of that ensemble polls its convergence word from the host
after each graph replay, the others loop on the device), the per-sample (s = 1)
GPU path on a subset, the end-to-end number through host buffers, and the CPU
oracle on the host cores (`cpu_baseline`).  `--impl reference` times the CPU
oracle alone (the reference arm of this workload).
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_MESH, M_KL, SIGMA, KAPPA0, L_CORR, TOL = 64, 10, 0.1, 1.0, 1.0, 1e-8
BATCH = 1024
METRIC = "ensemble CG sample-solves/s and ens_spmv HBM GB/s (% peak) vs per-sample, 1 GB300"
UNIT = "sample-solves/s"
WORKLOAD = "KL diffusion, 64^3 hex Q1 mesh (274,625 rows, 7,189,057 nnz), M=10, 1024 samples, CG to 1e-8"


def spmv_bytes(n, nnz, s, vbytes=8):
    """Algorithmic bytes of one fused CG SpMV: values + columns once, row map,
    p read once, q written once (the paper's ensemble byte model made exact)."""
    return nnz * (vbytes * s + 4) + 4 * (n + 1) + 2 * 8 * n * s


def kernel_source_hash():
    """Hash of the sources the CG's SpMV kernel is built from: a committed
    DRAM-traffic figure is used only while it still describes this kernel."""
    h = hashlib.sha256()
    for f in ("ens_spmv.cuh", "ens_cg_kernels.cuh", "ens_cg.cu", "ens_internal.cuh", "ens_cg_k1.cuh",
              "ens_cg_k1_s32.cu"):
        h.update(open(os.path.join(ROOT, "paper_1511_03703_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(s, mode="f64"):
    """DRAM bytes per launch of the CG SpMV from the committed ncu summary (a
    48^3 capture scaled to the 64^3 launch by its algorithmic bytes), if that
    summary was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "cg_spmv_dram_48cubed_s32.txt")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"kernel_source_sha256_16:\s*(\w+)", txt)
    if not m or m.group(1) != kernel_source_hash():
        return None
    m = re.search(rf"traffic_bytes_per_launch_{mode}_s{s}:\s*([0-9.eE+]+)", txt)
    return float(m.group(1)) if m else None


def fp64_alu_peak_tflops(sm_mhz=2070.0):
    """FP64 FMA pipe: 2 DFMA per cycle per SM (ncu peak_sustained), 152 SMs."""
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


def spmv_sweep(torch, device, s_list=(1, 4, 8, 16, 32), iters=24):
    """CG SpMV (K1) launch time per ensemble size and arithmetic form, from
    fixed-iteration CGs (tol 0) on the 64^3 mesh with CUDA events per launch:
    each form at its fastest chunks-per-CTA mapping (`chunks`), with the
    one-chunk mapping's time beside it."""
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import autotune, inputs
    mesh = E.Mesh(N_MESH, M_KL, device=device)
    peak, _ = measured_peaks()
    out = {}
    for s in s_list:
        xs = inputs.kl_samples(inputs.SEED_SCALE, 0, s, M_KL)
        vals, b = mesh.assemble(s, torch.from_numpy(inputs.ensemble_layout(xs)).to(device))
        t = autotune.time_spmv_mappings(mesh, s, iters=iters, vals=vals, b=b)
        row = {}
        for name in FORMS:
            c, ms = min(((c, v) for (f, c), v in t.items() if f == name), key=lambda cv: cv[1])
            gbs = spmv_bytes(mesh.n, mesh.nnz, s) / (ms * 1e-3) / 1e9
            row[name] = {"ms": ms, "gbs": gbs, "hbm_frac": gbs / peak, "k1_mapping": c,
                         "ms_one_chunk": t[(name, 1)],
                         "fp64_tflops": 2 * mesh.nnz * s / (ms * 1e-3) / 1e12}
        out[str(s)] = row
        del vals, b
    return out


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class OracleJobs:
    """Oracle solves (plain FP64 C, OpenMP over samples) on background host
    threads, so that the CPU-side checks of the extension workloads overlap
    their GPU work (ctypes releases the GIL during the call).  Never used
    inside a timed region's CPU measurement."""

    def __init__(self, workers=4):
        import concurrent.futures
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=workers)

    def solve(self, N, xs, tol, max_iter=20000):
        """Future of (x[num_samples, n], iterations, seconds)."""
        xs = np.array(xs, dtype=np.float64, copy=True)

        def job():
            import oracle
            t0 = time.perf_counter()
            x, it, rr, st = oracle.solve_samples(N, M_KL, xs, tol, max_iter, nthreads=len(xs), want_x=True)
            if any(int(v) for v in st):
                raise RuntimeError(f"oracle status {list(st)}")
            return x, it, time.perf_counter() - t0
        return self.pool.submit(job)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- the solver
FORMS = ("f64", "df", "split", "dfv")


def form_flag(form):
    """ens_cg flags of an SpMV form (dfv: ens_cg_df with the pre-split copy)."""
    import paper_1511_03703_gb300 as E
    return {"f64": 0, "df": E.CG_DF64, "split": E.CG_SPLIT64, "dfv": 0}[form]


def make_batch(rank, s, batch):
    from paper_1511_03703_gb300 import inputs
    first = rank * batch
    return inputs.kl_samples(inputs.SEED_SCALE, first, batch, M_KL)


class Runner:
    """Holds device buffers for one batch; run_step() is one timed step.
    k1_chunks: the SpMV's chunks of 32 rows per CTA (None: the default).
    time_spmv: the SpMV launches of the first ensemble of every step are timed
    with CUDA events (ENS_CG_TIME_SPMV, host-polled graph replays); the other
    ensembles run the device-side convergence loop."""

    def __init__(self, torch, s, batch, device, time_spmv=True, df="f64", k1_chunks=None):
        import paper_1511_03703_gb300 as E
        from paper_1511_03703_gb300 import inputs
        self.torch, self.E, self.s, self.batch = torch, E, s, batch
        self.dev = device
        self.nens = batch // s
        self.time_spmv = time_spmv
        self.df = df
        self.k1_flags = E.cg_k1_chunks(k1_chunks)
        n, nnz, _ = E.mesh_sizes(N_MESH)
        self.n, self.nnz = n, nnz
        T = torch
        self.row_map = T.empty(n + 1, dtype=T.int32, device=device)
        self.col = T.empty(nnz, dtype=T.int32, device=device)
        self.bmask = T.empty(n, dtype=T.uint8, device=device)
        self.kl = T.empty(E.kl_table_size(N_MESH, M_KL), dtype=T.float64, device=device)
        self.modes = T.empty((M_KL + 1) * nnz, dtype=T.float64, device=device)
        self.load = T.empty(n, dtype=T.float64, device=device)
        self.values = T.empty(nnz * s, dtype=T.float64, device=device)
        # pre-split double-float copy of the values (dfv form only)
        self.vdf = T.empty(2 * nnz * s, dtype=T.float32, device=device) if df == "dfv" else None
        self.b = T.empty(n * s, dtype=T.float64, device=device)
        self.x = T.empty((self.nens, n * s), dtype=T.float64, device=device)
        self.work = T.empty(E.cg_workspace_size(n, s), dtype=T.uint8, device=device)
        self.graph = E.Graph(self.row_map, self.col)
        self.xi_host = np.stack([inputs.ensemble_layout(b) for b in make_batch(0, s, batch).reshape(self.nens, s, M_KL)])
        self.xi = T.from_numpy(self.xi_host).to(device)
        self.reset_stats()

    def reset_stats(self):
        self.iters = []
        self.spmv_ms = 0.0
        self.spmv_launches = 0
        self.launches = 0
        self.status_bad = 0

    def setup_mesh(self):
        E = self.E
        E.graph_build(N_MESH, self.row_map, self.col, None, self.bmask)
        E.kl_setup(N_MESH, M_KL, L_CORR, self.kl, want_host=False)
        E.mode_matrices(N_MESH, self.graph, M_KL, self.kl, self.modes, self.load)
        self.launches += 5

    def solve_ensemble(self, g, xi=None):
        E = self.E
        # dfv: double-float assembly that also writes the pre-split copy
        E.assemble(self.graph, self.bmask, self.s, M_KL, self.modes, self.load,
                   self.xi[g] if xi is None else xi, SIGMA, KAPPA0, self.values, self.b,
                   values_df=self.vdf, kl_table=self.kl)
        x = self.x[g]
        x.zero_()
        timed = self.time_spmv and g == 0
        flags = ((E.CG_TIME_SPMV if timed else 0) | form_flag(self.df) | E.CG_X0_ZERO | E.CG_GRAPH
                 | self.k1_flags)
        it, rr, st, stats = E.cg(self.graph, self.s, self.values, self.b, x, TOL, 10000, self.work,
                                 flags=flags, check_every=8, values_df=self.vdf)
        self.launches += 2 + stats.kernel_launches
        self.iters.extend(it)
        self.status_bad += sum(1 for v in st if v != 0)
        self.spmv_ms += stats.spmv_ms
        self.spmv_launches += stats.spmv_launches
        return x

    def run_step(self):
        self.setup_mesh()
        for g in range(self.nens):
            self.solve_ensemble(g)


def per_sample_baseline(torch, device, nsamp=32, df="f64"):
    """The s = 1 path (samples one after another), as in the paper's speed-up
    (s * T1 / Ts, Sect. 4): every SpMV form at its autotuned mapping is timed
    and the fastest reported."""
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import autotune
    mesh = E.Mesh(N_MESH, M_KL, device=device)
    best = None
    for form in FORMS:
        c = autotune.best_mapping(mesh, 1, candidates=(form,))["k1_chunks"]
        res = _per_sample_form(torch, device, nsamp, form, c)
        if best is None or res["value"] > best["value"]:
            best = res
    return best


def _per_sample_form(torch, device, nsamp, df, k1_chunks=None):
    r = Runner(torch, 1, nsamp, device, time_spmv=True, df=df, k1_chunks=k1_chunks)
    r.setup_mesh()
    r.solve_ensemble(0)  # warm-up
    r.reset_stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in range(r.nens):
        r.solve_ensemble(g)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": nsamp / dt, "unit": UNIT, "samples": nsamp, "spmv": df, "k1_mapping": k1_chunks,
            "mean_iters": float(np.mean(r.iters)),
            "spmv_gbs": spmv_bytes(r.n, r.nnz, 1) * r.spmv_launches / (r.spmv_ms * 1e-3) / 1e9
            if r.spmv_ms > 0 else None}


def ensemble_size_sweep(torch, device, nsamp=128):
    """Sample-solves/s (assembly + CG) at the smaller ensemble sizes on the
    64^3 workload: nsamp samples each, in the SpMV form and mapping the
    autotuner finds fastest at that size (the s = 32 figure is the headline's
    value)."""
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import autotune
    mesh = E.Mesh(N_MESH, M_KL, device=device)
    out = {}
    for s in (4, 8, 16):
        m = autotune.best_mapping(mesh, s)
        form = m["form"]
        r = Runner(torch, s, nsamp, device, time_spmv=False, df=form, k1_chunks=m["k1_chunks"])
        r.setup_mesh()
        r.solve_ensemble(0)  # warm-up
        r.reset_stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g in range(r.nens):
            r.solve_ensemble(g)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[str(s)] = {"value": nsamp / dt, "unit": UNIT, "samples": nsamp, "spmv": form,
                       "k1_mapping": m["k1_chunks"],
                       "mean_iters": float(np.mean(r.iters)), "failed_members": r.status_bad}
        del r
    return out


def assembly_rate(torch, r, peak, reps=10):
    """Per-ensemble assembly (values, their pre-split copy in the dfv form,
    right-hand side) timed with CUDA events on the headline's buffers: the
    assembly kernels alone, without the coefficient check (which the timed
    step runs once per ensemble and which synchronises)."""
    E = r.E
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        E.assemble(r.graph, r.bmask, r.s, M_KL, r.modes, r.load, r.xi[0], SIGMA, KAPPA0, r.values, r.b,
                   values_df=r.vdf)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    vbytes = 16 if r.vdf is not None else 8
    byt = 8 * (M_KL + 1) * r.nnz + vbytes * r.nnz * r.s + 8 * r.n * r.s
    return {"ms": ms, "bytes": byt, "gbs": byt / (ms * 1e-3) / 1e9, "hbm_frac": byt / (ms * 1e-3) / 1e9 / peak,
            "form": "double-float KL terms, values + pre-split copy" if r.vdf is not None else "FP64",
            "bound": "instruction issue and the FP64 pipe (ncu), not HBM"}


def cpu_baseline_run(nsamples=None, nthreads=None):
    import oracle
    cores = nthreads or oracle.max_threads()
    ns = nsamples or max(2, cores)
    xi = make_batch(0, 1, BATCH)[:ns]
    t0 = time.perf_counter()
    _, it, rr, st = oracle.solve_samples(N_MESH, M_KL, xi, TOL, 10000, nthreads=cores, L=L_CORR,
                                         sigma=SIGMA, kappa0=KAPPA0)
    dt = time.perf_counter() - t0
    return {"value": ns / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{ns} samples of the 64^3 workload (sample indices 0..{ns - 1}), "
                      f"per-sample FP64 assembly + CG, OpenMP over samples on {cores} threads",
            "mean_iters": float(np.mean(it)), "seconds": dt}


def e2e_run(torch, r, steps):
    """Same metric through the library with host buffers: per step the KL
    variables are copied from pinned host memory, and every ensemble's solution
    is copied back to pinned host memory on a second stream while the next
    ensemble computes."""
    T = torch
    xi_pinned = T.from_numpy(r.xi_host).pin_memory()
    x_host = T.empty((r.nens, r.n * r.s), dtype=T.float64).pin_memory()
    copy_stream = T.cuda.Stream(device=r.dev)
    main = T.cuda.current_stream(r.dev)
    T.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        r.xi.copy_(xi_pinned, non_blocking=True)
        r.setup_mesh()
        for g in range(r.nens):
            x = r.solve_ensemble(g)
            ev = T.cuda.Event()
            ev.record(main)
            copy_stream.wait_event(ev)
            with T.cuda.stream(copy_stream):
                x_host[g].copy_(x, non_blocking=True)
        copy_stream.synchronize()
    T.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": steps * r.batch / dt, "unit": UNIT, "ms": 1e3 * dt, "samples": steps * r.batch,
            "h2d_bytes_per_step": int(r.xi_host.nbytes),
            "d2h_bytes_per_step": int(r.nens * r.n * r.s * 8)}


def extensions(args):
    """The extension workloads in compact form, for the default line (after
    the headline's timed region, N = 1 only): A7 mixed precision at 128^3
    (2 ensembles of 16), A8 batched (all 2048 samples), A9 learned guess
    (full training, 1024 test samples), NEXT-3 MG-PCG at 64^3 (2 ensembles).
    Each carries its error against oracle solves of two samples, computed on
    background host threads while the GPU runs the next workload."""
    jobs = OracleJobs()
    pending = {}
    t0 = time.perf_counter()
    for name, fn in (("mixed_128cubed", run_mixed), ("batched_16to64cubed", run_batched),
                     ("learned_guess_64cubed", run_guess), ("mg_pcg_64cubed", run_mg)):
        t1 = time.perf_counter()
        res, fut, finish = fn(args, compact=True, oracle_jobs=jobs)
        res["wall_seconds"] = time.perf_counter() - t1
        pending[name] = (res, fut, finish)
    t_gpu = time.perf_counter() - t0
    out = {}
    for name, (res, fut, finish) in pending.items():
        finish(fut.result())
        out[name] = res
    out["seconds"] = {"gpu_side": t_gpu, "total_with_oracle_checks": time.perf_counter() - t0}
    return out


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_first_sample(rank, per_rank):
    """Weak scaling: rank r solves samples [r*per_rank, (r+1)*per_rank)."""
    return rank * per_rank


def rank_xi(rank, per_rank, s):
    """The KL variables of rank r's shard, one row per ensemble in the
    commuted layout (per_rank / s ensembles of s members)."""
    from paper_1511_03703_gb300 import inputs
    xs = inputs.kl_samples(inputs.SEED_SCALE, shard_first_sample(rank, per_rank), per_rank, M_KL)
    return np.stack([inputs.ensemble_layout(b) for b in xs.reshape(per_rank // s, s, M_KL)])


def max_over_ranks(ms, world, device="cpu"):
    """Timed-region length of the slowest rank (all-reduce MAX; barrier after)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_throughput(world, steps, per_rank, ms):
    """Whole-job samples per second: every rank's samples over the slowest rank's time."""
    return world * steps * per_rank / (ms * 1e-3)


def main_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device(f"cuda:{local}")
    torch.cuda.set_device(device)
    import paper_1511_03703_gb300 as E
    E.lib()
    s = args.s
    df = args.spmv
    r = Runner(torch, s, BATCH, device, time_spmv=True, df=df)
    if world > 1:  # shard: this rank's own 1024 samples
        r.xi_host = rank_xi(rank, BATCH, s)
        r.xi = torch.from_numpy(r.xi_host).to(device)
    for _ in range(args.warmup):
        r.run_step()
    torch.cuda.synchronize()
    r.reset_stats()
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    stream = torch.cuda.current_stream(device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        r.run_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, device)
    value = job_throughput(world, args.steps, BATCH, ms)
    peak, peak_kind = measured_peaks()
    avg_spmv_ms = r.spmv_ms / max(r.spmv_launches, 1)
    bytes_launch = spmv_bytes(r.n, r.nnz, s)
    achieved = bytes_launch / (avg_spmv_ms * 1e-3) / 1e9
    flops = 2.0 * r.nnz * s / (avg_spmv_ms * 1e-3) / 1e12
    traffic = profiled_traffic(s, args.spmv)
    gpu_launches = r.launches
    spmv_launches_timed = r.spmv_launches  # before e2e_run adds its own steps' launches
    iters = r.iters
    bad = r.status_bad
    # end to end through the API on every rank (host buffers), slowest rank's time
    e2e = e2e_run(torch, r, max(1, min(args.steps, 2)))
    e2e_ms = max_over_ranks(e2e.pop("ms"), world, device)
    e2e["value"] = world * e2e.pop("samples") / (e2e_ms * 1e-3)
    out = None
    if rank == 0:
        sm_mhz = clk.get("sm_mhz") or 2070.0
        if df != "f64":
            roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"}
        else:
            alu = fp64_alu_peak_tflops(sm_mhz)
            roof = {"bound": "alu", "achieved": flops, "peak": alu, "unit": "TFLOP/s",
                    "frac": flops / alu, "traffic": traffic,
                    "peak_source": "FP64 FMA pipe: 152 SMs x 2 DFMA/cycle x 2 flop x median SM clock "
                                   "under load (derived; probe measured 0.596 TFMA/s at 2.07 GHz)",
                    "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                            "peak_source": f"{peak_kind} hbm_gbs"}}
        roof.update({"kernel": f"cg_spmv_kernel<{s},{df}> (q = A p fused with per-member p.q)",
                     "bytes_per_launch": bytes_launch, "avg_launch_ms": avg_spmv_ms,
                     "launches_timed": spmv_launches_timed,
                     "timed_on": "CUDA events around every SpMV launch of the first ensemble of each timed step"})
        # the single-GPU comparisons (per-sample CG, other SpMV forms, the
        # sweep, the CPU oracle) only at N = 1
        solo = world == 1
        per = per_sample_baseline(torch, device, df=df) if solo else None
        ens_speedup = value / world / per["value"] if solo else None
        others = {}
        if solo and not args.quick:
            for form in FORMS:
                if form == df:
                    continue
                r2 = Runner(torch, s, BATCH, device, time_spmv=True, df=form)
                r2.xi = r.xi
                r2.run_step()
                torch.cuda.synchronize()
                r2.reset_stats()
                t0 = time.perf_counter()
                r2.run_step()
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                ms2 = r2.spmv_ms / max(r2.spmv_launches, 1)
                others[form] = {"value": BATCH / dt, "unit": UNIT, "steps": 1,
                                "spmv_gbs": bytes_launch / (ms2 * 1e-3) / 1e9,
                                "spmv_hbm_frac": bytes_launch / (ms2 * 1e-3) / 1e9 / peak,
                                "mean_iters": float(np.mean(r2.iters)), "failed_members": r2.status_bad}
                del r2
        sweep = None if (args.quick or not solo) else spmv_sweep(torch, device)
        asm = assembly_rate(torch, r, peak) if solo else None
        ssweep = None if (args.quick or not solo) else ensemble_size_sweep(torch, device)
        cpu = cpu_baseline_run() if (solo and not args.no_cpu_baseline) else None
        ext = None if (args.quick or args.no_extensions or not solo) else extensions(args)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"f64": "f64",
                      "df": "f64 (SpMV products and sums in double-float 2xf32, all else f64)",
                      "split": "f64 (SpMV: even entries FP64 FMA, odd entries double-float 2xf32; all else f64)",
                      "dfv": "f64 (SpMV in double-float 2xf32 from values pre-split once per ensemble, "
                             "bitwise the df form; all else f64)"}[df],
            "data": "synthetic",
            "config": headline_config(args, world),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "per_sample_gpu": per,
            "ensemble_speedup_vs_per_sample": ens_speedup,
            "other_spmv_forms": others,
            "spmv_sweep_64cubed": sweep,
            "ensemble_size_sweep_64cubed": ssweep,
            "assembly": asm,
            "extensions": ext,
            "cg_iterations": {"mean": float(np.mean(iters)), "min": int(min(iters)),
                              "max": int(max(iters)), "failed_members": bad},
            "gpu_launches": gpu_launches,
            "clocks": clk,
        }
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def headline_config(args, world):
    """The headline workload's config (both arms report the same one)."""
    return {"workload": WORKLOAD, "ensemble_size": args.s, "batch_samples": BATCH,
            "ensembles_per_step": BATCH // args.s, "tol": TOL, "kl_terms": M_KL,
            "sigma": SIGMA, "corr_length": L_CORR, "spmv": args.spmv,
            "l2": "inputs larger than L2 (1.8 GB values per ensemble)",
            "parallelism": f"replica per GPU, {world} GPU(s), samples sharded by rank"}


def main_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return None
    import oracle
    cores = oracle.max_threads()
    ns = max(2, cores)
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; a first run would only repeat the same work
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline_run(ns, cores))
    t = sum(v["seconds"] for v in vals)
    value = args.steps * ns / t
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": headline_config(args, world),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": vals[0]["sample"] + f"; {ns} of the workload's samples per step "
                                      "(a bounded sample: the oracle is per sample, no ensembles)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return out


# ------------------------------------------------ mixed-precision workload
MIX_N, MIX_S, MIX_BATCH, MIX_TOL = 128, 16, 256, 1e-10
MIX_WORKLOAD = ("KL diffusion, 128^3 hex Q1 mesh (2,146,689 rows, 57,066,625 nnz), M=10, "
                "256 samples as 16 ensembles of s=16, true residual 1e-10")


def run_mixed(args, compact=False, oracle_jobs=None):
    """FP64 ensemble CG vs FP64-refined FP32 / BF16 inner CG on the 128^3 workload.
    One step = set-up + the ensembles (assembly, value conversion, solve); the
    full workload is 16 ensembles of s = 16, the compact one (for the default
    bench line) 2.  Returns the result dict; the error of two samples against
    FP64 oracle solves (tol 1e-12) is filled in when the oracle job ends."""
    import torch
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import inputs
    dev = torch.device("cuda:0")
    E.lib()
    N, M, s = MIX_N, M_KL, MIX_S
    batch = 2 * s if compact else MIX_BATCH
    nens = batch // s
    steps, warmup = (1, 1) if compact else (args.steps, args.warmup)
    xs_all = inputs.kl_samples(inputs.SEED_MIXED, 0, batch, M)
    nref = 2
    jobs = oracle_jobs or OracleJobs()
    fut = jobs.solve(N, xs_all[:nref], 1e-12)
    xi = torch.from_numpy(np.stack([inputs.ensemble_layout(b) for b in xs_all.reshape(nens, s, M)])).to(dev)
    mesh = E.Mesh(N, M, device=dev)
    vals = torch.empty(mesh.nnz * s, dtype=torch.float64, device=dev)
    b = torch.empty(mesh.n * s, dtype=torch.float64, device=dev)
    X = torch.empty((nens, mesh.n * s), dtype=torch.float64, device=dev)
    v32 = torch.empty(mesh.nnz * s, dtype=torch.float32, device=dev)
    vbf = torch.empty(mesh.nnz * s, dtype=torch.bfloat16, device=dev)
    diag = torch.empty(mesh.n * s, dtype=torch.float32, device=dev)
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=dev)  # FP64 comparator: dfv form
    wcg = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=dev)
    wmx = torch.empty(E.cg_mixed_workspace_size(mesh.n, s), dtype=torch.uint8, device=dev)
    peak, _ = measured_peaks()
    n, nnz = mesh.n, mesh.nnz

    def run(form, stats):
        mesh.assemble(s, xi[0], values=vals, b=b)  # warm the set-up path
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        E.graph_build(N, mesh.row_map, mesh.col_entry, None, mesh.bmask)
        E.kl_setup(N, M, L_CORR, mesh.kl_table, want_host=False)
        E.mode_matrices(N, mesh.graph, M, mesh.kl_table, mesh.modes, mesh.load)
        for g in range(nens):
            if form != "f64":
                mesh.assemble(s, xi[g], values=vals, b=b)
            x = X[g]
            x.zero_()
            if form == "f64":
                mesh.assemble(s, xi[g], values=vals, b=b, values_df=vdf)  # double-float assembly + split
                it, rr, st, cs = E.cg(mesh.graph, s, vals, b, x, MIX_TOL, 10000, wcg,
                                      flags=E.CG_TIME_SPMV | E.CG_X0_ZERO, check_every=32, values_df=vdf)
                stats["outer"].extend([1] * s)
                stats["inner"].extend(it)
                vb = 8
            else:
                lo = v32 if form == "f32" else vbf
                dg = diag if form == "bf16" else None
                E.convert_values(mesh.graph, s, vals, lo, dg)
                oi, ii, rr, st, cs = E.cg_mixed(mesh.graph, s, vals, lo, b, x, MIX_TOL, wmx, diag_lo=dg,
                                                inner_tol=1e-2 if form == "bf16" else 1e-4,
                                                max_inner=5000, check_every=32, flags=E.CG_TIME_SPMV)
                stats["outer"].extend(oi)
                stats["inner"].extend(ii)
                vb = 4 if form == "f32" else 2
            stats["bad"] += sum(1 for v in st if v != 0)
            stats["relres"].extend(rr)
            stats["spmv_ms"] += cs.spmv_ms
            stats["spmv_n"] += cs.spmv_launches
            stats["vb"] = vb
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3

    out, xg = {}, {}
    for form in ("f64", "f32", "bf16"):
        for _ in range(warmup):
            run(form, {"outer": [], "inner": [], "relres": [], "bad": 0, "spmv_ms": 0.0, "spmv_n": 0})
        st = {"outer": [], "inner": [], "relres": [], "bad": 0, "spmv_ms": 0.0, "spmv_n": 0}
        tt = sum(run(form, st) for _ in range(steps))
        vb = st["vb"]
        if form == "f64":
            sb = spmv_bytes(n, nnz, s)
        else:  # low-precision values, float x gather and q write, (bf16) FP32 diagonal
            sb = nnz * (vb * s + 4) + 4 * (n + 1) + 2 * 4 * n * s + (4 * n * s if form == "bf16" else 0)
        ms = st["spmv_ms"] / max(st["spmv_n"], 1)
        out[form] = {"value": steps * batch / tt, "unit": UNIT,
                     "spmv": "f64 (dfv: pre-split double-float)" if form == "f64"
                     else f"{form} values, f32 accumulation",
                     "spmv_gbs": sb / (ms * 1e-3) / 1e9, "spmv_hbm_frac": sb / (ms * 1e-3) / 1e9 / peak,
                     "outer_mean": float(np.mean(st["outer"])), "inner_mean": float(np.mean(st["inner"])),
                     "max_relres": float(max(st["relres"])), "failed": st["bad"]}
        xg[form] = X[0].view(-1, s)[:, :nref].cpu().numpy().copy()   # last step's first two members
    del vals, b, X, v32, vbf, diag, vdf, wcg, wmx, mesh
    torch.cuda.empty_cache()
    res = {"metric": "ensemble CG sample-solves/s, FP64 vs mixed precision (FP32 / BF16 values, FP64 refinement)",
           "value": out["f32"]["value"], "unit": UNIT, "n_gpus": 1, "steps": steps,
           "warmup": warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 inner (f32 values), f64 residual and update", "data": "synthetic",
           "config": {"workload": MIX_WORKLOAD if not compact else
                      MIX_WORKLOAD.replace("256 samples as 16 ensembles", "32 samples as 2 ensembles"),
                      "ensemble_size": s, "batch_samples": batch,
                      "inner_tol": {"f32": 1e-4, "bf16": 1e-2}, "bf16_diagonal": "fp32, row-sum compensated",
                      "l2": "inputs larger than L2"},
           "forms": out}

    def finish(oracle_result):
        xo, ito, sec = oracle_result
        for form in out:
            out[form]["rel_err_vs_fp64_oracle"] = [
                float(np.linalg.norm(xg[form][:, j] - xo[j]) / np.linalg.norm(xo[j])) for j in range(nref)]
        res["oracle"] = {"samples": f"sample indices 0..{nref - 1} of the 128^3 workload", "tol": 1e-12,
                         "iters": [int(v) for v in ito], "seconds": sec, "threads": nref}
    return res, fut, finish


def main_mixed(args):
    res, fut, finish = run_mixed(args)
    finish(fut.result())
    print(json.dumps(res))


# ------------------------------------------------------- batched workload
BAT_MESHES, BAT_WIDTHS, BAT_GROUP = (16, 32, 48, 64), (4, 8, 16, 32), 128
BAT_WORKLOAD = ("KL diffusion, hex Q1 meshes 16^3, 32^3, 48^3, 64^3 x ensemble widths 4, 8, 16, 32, "
                "128 samples per (mesh, width) group, 2048 samples, M=10, CG to 1e-8")


def run_batched(args, compact=False, oracle_jobs=None):
    """16 groups of 128 samples solved (a) one ens_cg call per ensemble and
    (b) one ens_cg_batched call for all 240 ensembles, with knobs from the
    autotuner (SpMV form per (mesh, s); graph length for the batch).  compact:
    one warm-up and one timed step.  The first sample of the 16^3 and of the
    32^3 group at s = 4 are checked against oracle solves (tol 1e-12)."""
    import torch
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import autotune, inputs
    dev = torch.device("cuda:0")
    E.lib()
    steps, warmup = (1, 1) if compact else (args.steps, args.warmup)
    jobs = oracle_jobs or OracleJobs()
    # group g = (mesh index) * 4 + (width index); (16^3, s=4) is group 0, (32^3, s=4) group 4
    checks = [(16, 0), (32, 4)]
    futs = [jobs.solve(N, inputs.kl_samples(inputs.SEED_BATCHED, g * BAT_GROUP, 1, M_KL), 1e-12)
            for N, g in checks]
    meshes = {N: E.Mesh(N, M_KL, device=dev) for N in BAT_MESHES}
    items, groups = [], []
    g = 0
    for N in BAT_MESHES:
        for s in BAT_WIDTHS:
            xs = inputs.kl_samples(inputs.SEED_BATCHED, g * BAT_GROUP, BAT_GROUP, M_KL)
            for k in range(BAT_GROUP // s):
                xi = torch.from_numpy(inputs.ensemble_layout(xs[k * s:(k + 1) * s])).to(dev)
                vdf = torch.empty(2 * meshes[N].nnz * s, dtype=torch.float32, device=dev)
                vals, b = meshes[N].assemble(s, xi, values_df=vdf)
                x = torch.zeros(meshes[N].n * s, dtype=torch.float64, device=dev)
                items.append({"N": N, "s": s, "xi": xi, "vals": vals, "vdf": vdf, "b": b, "x": x, "group": g})
            groups.append((N, s))
            g += 1
    t0 = time.perf_counter()
    # every item carries its pre-split values (written by the double-float
    # assembly), so all four SpMV forms are candidates; each (mesh, s) gets its
    # own (form, chunks per SpMV CTA) for the separate launches
    mappings = {(N, s): autotune.best_mapping(meshes[N], s) for N in BAT_MESHES for s in BAT_WIDTHS}
    forms = {key: m["form"] for key, m in mappings.items()}
    works = {}
    for it in items:
        key = (it["N"], it["s"])
        if key not in works:
            works[key] = torch.empty(E.cg_workspace_size(meshes[it["N"]].n, it["s"]), dtype=torch.uint8, device=dev)
    # batch-wide form: the one most groups chose, weighted by their bytes
    votes = {}
    for it in items:
        f = forms[(it["N"], it["s"])]
        votes[f] = votes.get(f, 0) + meshes[it["N"]].nnz * it["s"]
    bform = max(votes, key=votes.get)
    batch = E.Batch([(meshes[it["N"]].graph, it["s"], it["vals"], it["b"], it["x"])
                     + ((it["vdf"],) if bform == "dfv" else ()) for it in items])
    bwork = torch.empty(batch.workspace_size(), dtype=torch.uint8, device=dev)
    bflags = autotune.FORMS[bform] | autotune.best_batch_k1(batch, bwork, autotune.FORMS[bform],
                                                            tag=f"batched-16^3-64^3-{bform}")
    ce = autotune.best_check_every(batch, bwork, bflags, tag=f"batched-16^3-64^3-{bform}")
    tune_s = time.perf_counter() - t0

    def reassemble():
        for N in BAT_MESHES:
            mesh = meshes[N]
            E.graph_build(N, mesh.row_map, mesh.col_entry, None, mesh.bmask)
            E.kl_setup(N, M_KL, L_CORR, mesh.kl_table, want_host=False)
            E.mode_matrices(N, mesh.graph, M_KL, mesh.kl_table, mesh.modes, mesh.load)
        for it in items:
            meshes[it["N"]].assemble(it["s"], it["xi"], values=it["vals"], b=it["b"], values_df=it["vdf"])
            it["x"].zero_()

    def separate():
        iters = []
        for it in items:
            mesh = meshes[it["N"]]
            m = mappings[(it["N"], it["s"])]
            i, r, st, _ = E.cg(mesh.graph, it["s"], it["vals"], it["b"], it["x"], TOL, 10000,
                               works[(it["N"], it["s"])], flags=autotune.mapping_flags(m), check_every=16,
                               values_df=it["vdf"] if m["form"] == "dfv" else None)
            iters.append(i)
        return iters

    def batched():
        i, r, st, stats = batch.solve(TOL, 10000, bwork, flags=bflags | E.CG_GRAPH, check_every=ce)
        return i

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        reassemble()
        res = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, res

    total = len(items) and sum(it["s"] for it in items)
    for _ in range(warmup):
        timed(separate)
        timed(batched)
    ts = tb = 0.0
    for _ in range(steps):
        t, it_sep = timed(separate)
        ts += t
        t, it_bat = timed(batched)
        tb += t
    same = all(a == b for a, b in zip(it_sep, it_bat))
    per_group = {}
    for it, its in zip(items, it_bat):
        per_group.setdefault(f"{it['N']}^3,s={it['s']}", []).extend(its)
    # the batched solutions of the checked samples (member 0 of each group's first ensemble)
    xg = [next(it for it in items if it["group"] == g)["x"].view(-1, 4)[:, 0].cpu().numpy().copy()
          for _, g in checks]
    line = {"metric": "batched ensemble CG sample-solves/s: one launch per CG phase vs separate launches",
            "value": steps * total / tb, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": BAT_WORKLOAD, "ensembles": len(items), "samples": total,
                       "batch_spmv_form": bform, "graph_check_every": ce,
                       "batch_spmv_cta_threads": 1024 if bflags & E.CG_BATCH_K1_WIDE else 512,
                       "per_group_mapping": {f"{N}^3,s={s}": {"form": mappings[(N, s)]["form"],
                                                              "k1_mapping": mappings[(N, s)]["k1_chunks"]}
                                             for (N, s) in groups},
                       "tuning_seconds": tune_s, "step": "mesh set-up + assembly of every ensemble + solve"},
            "separate_launches": {"value": steps * total / ts, "unit": UNIT},
            "speedup_batched_vs_separate": ts / tb,
            "iterations_identical": same,
            "mean_iterations_per_group": {k: float(np.mean(v)) for k, v in per_group.items()}}
    del items, batch, bwork, works
    torch.cuda.empty_cache()

    class _Futs:
        def result(self):
            return [f.result() for f in futs]

    def finish(results):
        errs, its = [], []
        for (xo, ito, _), x in zip(results, xg):
            errs.append(float(np.linalg.norm(x - xo[0]) / np.linalg.norm(xo[0])))
            its.append(int(ito[0]))
        line["rel_err_vs_fp64_oracle"] = errs
        line["oracle"] = {"samples": "first sample of the 16^3 and of the 32^3 group at s = 4", "tol": 1e-12,
                          "iters": its}
    return line, _Futs(), finish


def main_batched(args):
    res, fut, finish = run_batched(args)
    finish(fut.result())
    print(json.dumps(res))


# ------------------------------------------------- learned-guess workload
GUESS_TRAIN, GUESS_TEST, GUESS_EPOCHS, GUESS_K, GUESS_L = 4096, 1024, 2000, 64, 80
GUESS_WORKLOAD = ("KL diffusion, 64^3 hex Q1 mesh, M=10: MLP 10-256-256-64 (GELU, FP32) -> 64 POD "
                  "coefficients, trained on 4096 solved samples, tested on 1024 fresh samples, CG to 1e-8")


def run_guess(args, compact=False, oracle_jobs=None):
    """Zero-guess ensemble CG vs CG from the learned guess on 1024 fresh
    samples (s = 32), both to ||r|| <= 1e-8 ||b||; training (solves, POD,
    MLP epochs) timed separately.  compact: one warm-up and one timed step.
    Test samples 0 and 1 (solved from the learned guess) are checked against
    oracle solves (tol 1e-12)."""
    import torch
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import inputs
    from paper_1511_03703_gb300.learned import LearnedGuess, collect
    dev = torch.device("cuda:0")
    E.lib()
    s = 32
    steps, warmup = (1, 1) if compact else (args.steps, args.warmup)
    nref = 2
    jobs = oracle_jobs or OracleJobs()
    fut = jobs.solve(N_MESH, inputs.kl_samples(inputs.SEED_GUESS_TEST, 0, nref, M_KL), 1e-12)
    flags = E.CG_GRAPH
    mesh = E.Mesh(N_MESH, M_KL, device=dev)

    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    xtr = inputs.kl_samples(inputs.SEED_GUESS_TRAIN, 0, GUESS_TRAIN, M_KL)
    t_solve, (X, it_train) = wall(lambda: collect(mesh, xtr, s=s, tol=TOL))
    g = LearnedGuess(mesh.n, GUESS_K)
    t_pod, T = wall(lambda: g.fit_basis(X, l=GUESS_L, power_iters=1))
    del X
    torch.cuda.empty_cache()
    g.init_params()
    t_train, losses = wall(lambda: g.train(xtr, T, epochs=GUESS_EPOCHS))
    sig = g.sigma.cpu().numpy()

    xte = inputs.kl_samples(inputs.SEED_GUESS_TEST, 0, GUESS_TEST, M_KL)
    xis = [torch.from_numpy(inputs.ensemble_layout(xte[j:j + s])).to(dev) for j in range(0, GUESS_TEST, s)]
    vals = torch.empty(mesh.nnz * s, dtype=torch.float64, device=dev)
    b = torch.empty(mesh.n * s, dtype=torch.float64, device=dev)
    x = torch.empty(mesh.n * s, dtype=torch.float64, device=dev)
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=dev)
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=dev)

    first = {}

    def run(learned):
        iters, fb, launches = [], 0, 0
        for gi, xi in enumerate(xis):
            mesh.assemble(s, xi, values=vals, b=b, values_df=vdf)
            launches += 2
            if learned:
                g.predict(xi, s, x)
                launches += 5
            else:
                x.zero_()
            it, rr, st, stats = E.cg(mesh.graph, s, vals, b, x, TOL, 10000, work,
                                     flags=flags | (E.CG_GUESS_FALLBACK if learned else E.CG_X0_ZERO),
                                     check_every=8, values_df=vdf)
            if any(st):
                raise RuntimeError(f"CG status {st}")
            iters += it
            fb += stats.guess_fallbacks
            launches += stats.kernel_launches
            if gi == 0 and learned:
                first["x"] = x.view(-1, s)[:, :nref].clone()
        return iters, fb, launches

    def timed(learned):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = run(learned)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, res

    for _ in range(warmup):
        timed(False)
        timed(True)
    tz = tl = 0.0
    for _ in range(steps):
        t, (iz, _, lz) = timed(False)
        tz += t
        t, (il, fb, ll) = timed(True)
        tl += t
    xg = first["x"].cpu().numpy()
    line = {"metric": "ensemble CG sample-solves/s from the learned initial guess vs from zero, 1 GB300",
            "value": steps * GUESS_TEST / tl, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": 1e3 * tl / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 CG, f32 network", "data": "synthetic",
            "config": {"workload": GUESS_WORKLOAD, "ensemble_size": s, "spmv": "dfv",
                       "step": "assembly + guess + CG of all 1024 test samples",
                       "pod_modes": GUESS_K, "pod_oversampled": GUESS_L, "epochs": GUESS_EPOCHS,
                       "batch": 256},
            "zero_guess": {"value": steps * GUESS_TEST / tz, "unit": UNIT,
                           "mean_iterations": float(np.mean(iz)), "max_iterations": int(np.max(iz))},
            "learned_guess": {"mean_iterations": float(np.mean(il)), "max_iterations": int(np.max(il)),
                              "min_iterations": int(np.min(il)), "fallback_rate": fb / GUESS_TEST},
            "speedup_vs_zero_guess": tz / tl,
            "training": {"solve_seconds": t_solve, "train_mean_iterations": float(np.mean(it_train)),
                         "pod_seconds": t_pod, "mlp_seconds": t_train,
                         "mlp_steps": GUESS_EPOCHS * GUESS_TRAIN // 256,
                         "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1]),
                         "sigma_1": float(sig[0]), "sigma_64_over_sigma_1": float(sig[-1] / sig[0])},
            "gpu_launches": ll}
    del vals, b, x, vdf, work, g, mesh
    torch.cuda.empty_cache()

    def finish(oracle_result):
        xo, ito, sec = oracle_result
        line["rel_err_vs_fp64_oracle"] = [float(np.linalg.norm(xg[:, j] - xo[j]) / np.linalg.norm(xo[j]))
                                          for j in range(nref)]
        line["oracle"] = {"samples": "test samples 0 and 1 (solved from the learned guess)", "tol": 1e-12,
                          "iters": [int(v) for v in ito]}
    return line, fut, finish


def main_guess(args):
    res, fut, finish = run_guess(args)
    finish(fut.result())
    print(json.dumps(res))


# ------------------------------------------------ coupled CG (Sects. 3.4, 3.7)
CPL_SAMPLES = 256
CPL_WORKLOAD = ("KL diffusion, 64^3 hex Q1 mesh, M=10, 256 samples as ensembles of s = 4, 8, 16, 32, "
                "CG to 1e-8: coupled (member-summed dots) vs per-member")


def main_coupled(args):
    """Iteration growth of the paper's coupled ensemble CG with s, and what
    grouping similar samples recovers, against the per-member CG."""
    import torch
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import inputs
    dev = torch.device("cuda:0")
    E.lib()
    mesh = E.Mesh(N_MESH, M_KL, device=dev)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, CPL_SAMPLES, M_KL)
    smax = 32
    vals = torch.empty(mesh.nnz * smax, dtype=torch.float64, device=dev)
    vdf = torch.empty(2 * mesh.nnz * smax, dtype=torch.float32, device=dev)
    b = torch.empty(mesh.n * smax, dtype=torch.float64, device=dev)
    x = torch.empty(mesh.n * smax, dtype=torch.float64, device=dev)
    work = torch.empty(E.cg_workspace_size(mesh.n, smax), dtype=torch.uint8, device=dev)

    def solve_all(order, s, coupled):
        """Iterations per sample (in sample order) and seconds for all samples."""
        its = np.zeros(CPL_SAMPLES, dtype=np.int64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g in range(CPL_SAMPLES // s):
            idx = order[g * s:(g + 1) * s]
            xi = torch.from_numpy(inputs.ensemble_layout(xs[idx])).to(dev)
            v, bb = vals[:mesh.nnz * s], b[:mesh.n * s]
            vd = vdf[:2 * mesh.nnz * s]
            mesh.assemble(s, xi, values=v, b=bb, values_df=vd)
            xx = x[:mesh.n * s]
            xx.zero_()
            it, rr, st, _ = E.cg(mesh.graph, s, v, bb, xx, TOL, 10000, work,
                                 flags=E.CG_GRAPH | E.CG_X0_ZERO | (E.CG_COUPLED if coupled else 0),
                                 check_every=8, values_df=vd)
            if any(st):
                raise RuntimeError(f"CG status {st}")
            its[idx] = it
        torch.cuda.synchronize()
        return its, time.perf_counter() - t0

    natural = np.arange(CPL_SAMPLES)
    for _ in range(max(1, args.warmup)):
        solve_all(natural, 32, True)
    member_its, _ = solve_all(natural, 32, False)      # per-member counts do not depend on s
    by_iters = np.argsort(member_its, kind="stable")
    by_xi1 = np.argsort(xs[:, 0], kind="stable")
    rows = {}
    for s in (4, 8, 16, 32):
        r = {}
        for name, order, coupled in (("per_member", natural, False), ("coupled", natural, True),
                                     ("coupled_grouped_by_xi1", by_xi1, True),
                                     ("coupled_grouped_by_iterations", by_iters, True)):
            its, sec = solve_all(order, s, coupled)
            r[name] = {"mean_iterations": float(its.mean()), "max_iterations": int(its.max()),
                       "sample_solves_per_s": CPL_SAMPLES / sec}
        r["coupled_iteration_growth"] = r["coupled"]["mean_iterations"] / r["per_member"]["mean_iterations"]
        rows[str(s)] = r
    line = {"metric": "coupled ensemble CG (Sects. 3.4, 3.7) iterations and sample-solves/s vs per-member CG, 1 GB300",
            "value": rows["32"]["coupled"]["sample_solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (dfv SpMV)", "data": "synthetic",
            "config": {"workload": CPL_WORKLOAD, "grouping": "natural order; sorted by xi_1; sorted by the "
                       "per-member iteration count (best case)"},
            "per_member_iterations": {"mean": float(member_its.mean()), "min": int(member_its.min()),
                                      "max": int(member_its.max())},
            "by_ensemble_size": rows}
    print(json.dumps(line))


# --------------------------------------------- preconditioned CG (NEXT-2)
PCG_SAMPLES = 256
PCG_WORKLOAD = ("KL diffusion, 64^3 hex Q1 mesh, M=10, 256 samples as 8 ensembles of s=32, CG to 1e-8: "
                "plain vs Jacobi- and Chebyshev-preconditioned ensemble CG (FP64 SpMV form)")


def main_pcg(args):
    """Iterations, SpMVs per solve and sample-solves/s of the preconditioned
    ensemble CG against the plain one, all in the FP64 SpMV form (the
    preconditioned solver is FP64 throughout); the pre-split plain CG is
    reported for reference."""
    import torch
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import inputs
    dev = torch.device("cuda:0")
    E.lib()
    s = 32
    mesh = E.Mesh(N_MESH, M_KL, device=dev)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, PCG_SAMPLES, M_KL)
    xis = [torch.from_numpy(inputs.ensemble_layout(xs[j:j + s])).to(dev) for j in range(0, PCG_SAMPLES, s)]
    vals = torch.empty(mesh.nnz * s, dtype=torch.float64, device=dev)
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=dev)
    b = torch.empty(mesh.n * s, dtype=torch.float64, device=dev)
    x = torch.empty(mesh.n * s, dtype=torch.float64, device=dev)
    wcg = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=dev)
    wpc = torch.empty(E.pcg_workspace_size(mesh.n, s), dtype=torch.uint8, device=dev)
    v0 = torch.from_numpy(np.stack([inputs.random_vector(500 + e, mesh.n) for e in range(s)], axis=1)
                          .reshape(-1)).to(dev)
    forms = [("cg_f64", None, 0), ("cg_dfv", None, 0), ("pcg_jacobi", E.PC_JACOBI, 0)] + \
        [(f"pcg_chebyshev{d}", E.PC_CHEBYSHEV, d) for d in (2, 3, 4)]

    def run(name, pc, deg):
        its, lams = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for xi in xis:
            mesh.assemble(s, xi, values=vals, b=b, values_df=vdf if name == "cg_dfv" else None)
            x.zero_()
            fl = E.CG_GRAPH | E.CG_X0_ZERO
            if pc is None:
                it, rr, st, _ = E.cg(mesh.graph, s, vals, b, x, TOL, 10000, wcg, flags=fl, check_every=8,
                                     values_df=vdf if name == "cg_dfv" else None)
            else:
                it, rr, st, lam, _ = E.pcg(mesh.graph, s, vals, b, x, TOL, 10000, wpc, precond=pc,
                                           degree=max(deg, 1), power_iters=10, power_start=v0, flags=fl,
                                           check_every=8)
                lams += lam
            if any(st):
                raise RuntimeError(f"{name}: status {st}")
            its += it
        torch.cuda.synchronize()
        return its, time.perf_counter() - t0, lams

    out = {}
    for name, pc, deg in forms:
        for _ in range(args.warmup):
            run(name, pc, deg)
        its, sec, lams = run(name, pc, deg)
        spmv = 1 + (deg - 1 if deg >= 2 else 0)
        out[name] = {"mean_iterations": float(np.mean(its)), "max_iterations": int(np.max(its)),
                     "spmv_per_iteration": spmv, "mean_spmv_per_solve": float(np.mean(its)) * spmv,
                     "sample_solves_per_s": PCG_SAMPLES / sec}
        if lams:
            out[name]["lambda_max_D^-1A_mean"] = float(np.mean(lams))
    line = {"metric": "preconditioned ensemble CG sample-solves/s and iterations vs plain ensemble CG, 1 GB300",
            "value": max(v["sample_solves_per_s"] for k, v in out.items() if k.startswith("pcg")), "unit": UNIT,
            "n_gpus": 1, "steps": 1, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": PCG_WORKLOAD, "chebyshev": "interval [lam/30, lam], lam = 1.1 x a 10-step "
                       "power estimate of the largest eigenvalue of D^-1 A"},
            "forms": out}
    print(json.dumps(line))


# ----------------------------------- multigrid-preconditioned CG (NEXT-3)
MG_SAMPLES = 256
MG_LANCZOS_STEPS = 5   # the *_lanczos forms' steps (ENS_PC_LANCZOS)
MG_WORKLOAD = ("KL diffusion, 64^3 hex Q1 mesh, M=10, 256 samples as 8 ensembles of s=32, CG to 1e-8: "
               "multigrid-preconditioned ensemble CG (V-cycle over 64^3..4^3, Chebyshev-2 smoothers, "
               "direct coarse solve; mg: the SpMVs in double-float from pre-split values on every level, "
               "mg_f64: all FP64) vs plain ensemble CG")


def run_mg(args, compact=False, oracle_jobs=None):
    """The paper's solver form (Sect. 3.5): MG-PCG on the nested meshes
    against the plain CG, same samples and tolerance; each step assembles
    every level of every ensemble and solves.  compact: 64 samples (2
    ensembles), one warm-up.  Samples 0 and 1 of the MG-PCG solve (the
    default, pre-split form) are checked against oracle CG solves (tol 1e-12)."""
    import torch
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import inputs
    dev = torch.device("cuda:0")
    E.lib()
    s = 32
    nsamp = 2 * s if compact else MG_SAMPLES
    warmup = 1 if compact else args.warmup
    nref = 2
    jobs = oracle_jobs or OracleJobs()
    fut = jobs.solve(N_MESH, inputs.kl_samples(inputs.SEED_SCALE, 0, nref, M_KL), 1e-12)
    t0 = time.perf_counter()
    mg = E.Multigrid(N_MESH, M_KL, device=dev)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, nsamp, M_KL)
    xis = [torch.from_numpy(inputs.ensemble_layout(xs[j:j + s])).to(dev) for j in range(0, nsamp, s)]
    starts = [torch.from_numpy(np.stack([inputs.random_vector(600 + 100 * l + e, m.n) for e in range(s)],
                                        axis=1).reshape(-1)).to(dev) for l, m in enumerate(mg.meshes)]
    mesh = mg.meshes[0]
    first = {}
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=dev)
    # mg: every level's SpMVs from pre-split values (level 0's buffer shared with cg_dfv)
    vdfs = [vdf] + [torch.empty(2 * m.nnz * s, dtype=torch.float32, device=dev) for m in mg.meshes[1:]]
    wcg = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=dev)
    x = torch.empty(mesh.n * s, dtype=torch.float64, device=dev)
    vals0, _ = mg.assemble(s, xis[0], values_df=vdfs)
    v32s = mg.to_f32(s, vals0)
    wmg = torch.empty(max(mg.workspace_size(s, vals0, starts, vdfs),
                          mg.workspace_size(s, vals0, starts, [vdf], v32s)), dtype=torch.uint8, device=dev)
    del vals0

    def run(form_name):
        # *_lanczos: the smoothers' eigenvalue bound from MG_LANCZOS_STEPS Lanczos steps
        lanczos = form_name.endswith("_lanczos")
        form = form_name[:-len("_lanczos")] if lanczos else form_name
        eig = dict(flags=E.PC_LANCZOS, power_iters=MG_LANCZOS_STEPS) if lanczos else dict(flags=0, power_iters=10)
        its = []
        torch.cuda.synchronize()
        t = time.perf_counter()
        for gi, xi in enumerate(xis):
            x.zero_()
            if form in ("mg", "mg_f64", "mg_fp32_vcycle"):
                # mg: K1 and every level's V-cycle SpMVs from pre-split values;
                # mg_fp32_vcycle: K1 pre-split, the V-cycle in FP32
                pre = vdfs if form == "mg" else ([vdf] if form == "mg_fp32_vcycle" else None)
                # (mg_fp32_vcycle: K1 pre-split; the V-cycle and its eigenvalue bound in FP32)
                vals, b = mg.assemble(s, xi, df=True, values_df=pre)
                v32 = mg.to_f32(s, vals, out=v32s) if form == "mg_fp32_vcycle" else None
                it, rr, st, _ = mg.solve(s, vals, b, x, TOL, 500, wmg, starts,
                                         flags=E.CG_GRAPH | E.CG_X0_ZERO | eig["flags"],
                                         power_iters=eig["power_iters"], check_every=4, values_df=pre,
                                         values_f32=v32)
            else:
                vals, b = mesh.assemble(s, xi, values_df=vdf if form == "cg_dfv" else None)
                it, rr, st, _ = E.cg(mesh.graph, s, vals, b, x, TOL, 10000, wcg,
                                     flags=E.CG_GRAPH | E.CG_X0_ZERO, check_every=8,
                                     values_df=vdf if form == "cg_dfv" else None)
            if any(st):
                raise RuntimeError(f"{form}: status {st}")
            its += it
            if gi == 0 and form_name == "mg":
                first["x"] = x.view(-1, s)[:, :nref].clone()
        torch.cuda.synchronize()
        return its, time.perf_counter() - t

    out = {}
    forms = ("cg_dfv", "mg", "mg_lanczos", "mg_fp32_vcycle") if compact else (
        "cg_f64", "cg_dfv", "mg_f64", "mg", "mg_lanczos", "mg_fp32_vcycle", "mg_fp32_vcycle_lanczos")
    for form in forms:
        for _ in range(warmup):
            run(form)
        its, sec = run(form)
        out[form] = {"mean_iterations": float(np.mean(its)), "max_iterations": int(np.max(its)),
                     "sample_solves_per_s": nsamp / sec}
    xg = first["x"].cpu().numpy()
    line = {"metric": "multigrid-preconditioned ensemble CG sample-solves/s vs plain ensemble CG, 1 GB300",
            "value": out["mg"]["sample_solves_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": MG_WORKLOAD if not compact else
                       MG_WORKLOAD.replace("256 samples as 8 ensembles", "64 samples as 2 ensembles"),
                       "levels": mg.sizes, "smoother": "Chebyshev degree 2 on "
                       "[lam/5, 1.1 lam], 10 power steps (*_lanczos forms: %d Lanczos steps)" % MG_LANCZOS_STEPS,
                       "mesh_setup_seconds": t_setup,
                       "step": "assembly of every level + solve, per ensemble"},
            "forms": out, "speedup_vs_plain_cg_dfv": out["mg"]["sample_solves_per_s"] /
            out["cg_dfv"]["sample_solves_per_s"]}
    del mg, x, vdf, vdfs, wcg, wmg, v32s, starts, xis
    torch.cuda.empty_cache()

    def finish(oracle_result):
        xo, ito, sec = oracle_result
        line["rel_err_vs_fp64_oracle"] = [float(np.linalg.norm(xg[:, j] - xo[j]) / np.linalg.norm(xo[j]))
                                          for j in range(nref)]
        line["oracle"] = {"samples": "samples 0 and 1 of the 64^3 workload (MG-PCG, pre-split form)",
                          "tol": 1e-12, "iters": [int(v) for v in ito]}
    return line, fut, finish


def main_mg(args):
    res, fut, finish = run_mg(args)
    finish(fut.result())
    print(json.dumps(res))


# ------------------------------------------ nonlinear advection-diffusion
NL_SAMPLES = 256
NL_ALPHA, NL_BETA, NL_V = 1.0, 10.0, (1.0, 1.0, 1.0)
NL_TOL, NL_LIN_TOL = 1e-8, 1e-6
NL_WORKLOAD = ("nonlinear advection-diffusion -div(kappa grad u) + alpha v.grad u + beta u^2 = 1, 64^3 hex Q1 "
               "mesh, M=10, alpha=1, v=(1,1,1), beta=10, 256 samples as 8 ensembles of s=32: Newton to "
               "||F|| <= 1e-8 ||F(0)||, GMRES(30) to 1e-6 ||F_k|| per step, right-preconditioned by the V-cycle "
               "of the diffusion operator (pre-split values on every level)")


def main_nonlinear(args):
    """NEXT-4: Newton-GMRES for the nonlinear problem (Sect. 4, Eq. 7 with
    alpha, beta != 0; Eq. 10); each step assembles every level of every
    ensemble and solves from u = 0."""
    import torch
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import inputs
    dev = torch.device("cuda:0")
    E.lib()
    s = 32
    t0 = time.perf_counter()
    nl = E.Nonlinear(N_MESH, M_KL, v=NL_V, precond=E.NL_PRECOND_MG, device=dev)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, NL_SAMPLES, M_KL)
    xis = [torch.from_numpy(inputs.ensemble_layout(xs[j:j + s])).to(dev) for j in range(0, NL_SAMPLES, s)]
    starts = [torch.from_numpy(np.stack([inputs.random_vector(600 + 100 * l + e, m.n) for e in range(s)],
                                        axis=1).reshape(-1)).to(dev) for l, m in enumerate(nl.meshes)]
    p = nl.params(NL_ALPHA, NL_BETA, tol=NL_TOL, lin_tol=NL_LIN_TOL, restart=30, max_lin=300, max_newton=20)
    # the V-cycle's eigenvalue bounds by Lanczos steps (ENS_PC_LANCZOS)
    p_lz = nl.params(NL_ALPHA, NL_BETA, tol=NL_TOL, lin_tol=NL_LIN_TOL, restart=30, max_lin=300, max_newton=20,
                     power_iters=MG_LANCZOS_STEPS, flags=E.PC_LANCZOS)
    u = torch.empty(nl.mesh.n * s, dtype=torch.float64, device=dev)
    # every level pre-split (the V-cycle's SpMVs; level 0's also makes the GMRES SpMV pre-split)
    vdf = [torch.empty(2 * m.nnz * s, dtype=torch.float32, device=dev) for m in nl.meshes]
    vals0, _ = nl.assemble(s, xis[0], values_df=vdf)
    work = torch.empty(nl.workspace_size(s, vals0, starts, p, vdf), dtype=torch.uint8, device=dev)
    v32 = nl.mg.to_f32(s, vals0)
    work32 = torch.empty(nl.workspace_size(s, vals0, starts, p, vdf, v32), dtype=torch.uint8, device=dev)
    del vals0

    def run(f32=False, lanczos=False):
        newton, lin, launches = [], [], 0
        pp = p_lz if lanczos else p
        torch.cuda.synchronize()
        t = time.perf_counter()
        for xi in xis:
            u.zero_()
            vals, b = nl.assemble(s, xi, values_df=vdf)
            if f32:  # the V-cycle in FP32 (mixed-precision preconditioner; flexible GMRES)
                nl.mg.to_f32(s, vals, out=v32)
                ni, li, rr, st, stats = nl.solve(s, vals, b, u, work32, starts, pp, values_df=vdf, values_f32=v32)
            else:
                ni, li, rr, st, stats = nl.solve(s, vals, b, u, work, starts, pp, values_df=vdf)
            if any(st):
                raise RuntimeError(f"nonlinear: status {st}")
            newton += ni
            lin += li
            launches += stats.kernel_launches
        torch.cuda.synchronize()
        return newton, lin, launches, time.perf_counter() - t

    for _ in range(args.warmup):
        run()
        run(True)
        run(lanczos=True)
    newton, lin, launches, sec = run()
    newton32, lin32, _, sec32 = run(True)
    newton_lz, lin_lz, _, sec_lz = run(lanczos=True)
    line = {"metric": "nonlinear advection-diffusion Newton-GMRES sample-solves/s, 1 GB300",
            "value": NL_SAMPLES / sec, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": NL_WORKLOAD, "levels": nl.mg.sizes, "smoother": "Chebyshev degree 2 on "
                       "[lam/5, 1.1 lam], 10 power steps", "mesh_setup_seconds": t_setup,
                       "step": "assembly of every level + Newton solve, per ensemble"},
            "newton_steps": {"mean": float(np.mean(newton)), "max": int(np.max(newton))},
            "gmres_steps_per_solve": {"mean": float(np.mean(lin)), "max": int(np.max(lin))},
            "gmres_steps_per_newton_step": float(np.sum(lin)) / float(np.sum(newton)),
            "fp32_vcycle": {"sample_solves_per_s": NL_SAMPLES / sec32,
                            "newton_steps_mean": float(np.mean(newton32)),
                            "gmres_steps_per_solve_mean": float(np.mean(lin32))},
            "lanczos_bound": {"sample_solves_per_s": NL_SAMPLES / sec_lz, "steps": MG_LANCZOS_STEPS,
                              "newton_steps_mean": float(np.mean(newton_lz)),
                              "gmres_steps_per_solve_mean": float(np.mean(lin_lz))},
            "gpu_launches": launches}
    print(json.dumps(line))



def main_profile_cg(args):
    """Profiling driver: one ensemble CG with a fixed iteration count on an
    N^3 mesh (M = 10, seed of the 64^3 workload), so that an ncu capture
    (`ncu --clock-control none -k regex:cg_spmv_kernel -s 1 -c 1 ...`, after
    the same command has exited 0 without ncu) sees a steady-state launch.  The SpMV
    form is --spmv (dfv: double-float assembly writing the pre-split copy,
    then ens_cg_df, as in the headline).  Tolerance 0, so exactly --iters
    iterations run."""
    import torch
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import inputs
    N, s, iters, form = args.N, args.s, args.iters, args.spmv
    dev = torch.device("cuda:0")
    mesh = E.Mesh(N, M_KL, device=dev)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, s, M_KL)
    xi = torch.from_numpy(inputs.ensemble_layout(xs)).to(dev)
    vdf = torch.empty(2 * mesh.nnz * s, dtype=torch.float32, device=dev) if form == "dfv" else None
    vals, b = mesh.assemble(s, xi, values_df=vdf)
    x = torch.zeros(mesh.n * s, dtype=torch.float64, device=dev)
    work = torch.empty(E.cg_workspace_size(mesh.n, s), dtype=torch.uint8, device=dev)
    it, rr, st, stats = E.cg(mesh.graph, s, vals, b, x, 0.0, iters, work,
                             flags=form_flag(form) | E.cg_k1_chunks(args.k1_chunks),
                             check_every=iters, values_df=vdf)
    torch.cuda.synchronize()
    print("N", N, "s", s, "iters", it[:2], "status", st[:2], "nnz", mesh.nnz, "rows", mesh.n)


def _profile_starts(torch, meshes, s, dev):
    from paper_1511_03703_gb300 import inputs
    return [torch.from_numpy(np.stack([inputs.random_vector(600 + 100 * l + e, m.n) for e in range(s)],
                                      axis=1).reshape(-1)).to(dev) for l, m in enumerate(meshes)]


def main_profile_mg(args):
    """Profiling driver: multigrid-preconditioned ensemble CG on an N^3 mesh.
    --reps times: assemble every level of one ensemble of s samples
    (double-float assembly, M = 10, seed of the 64^3 workload) and solve to
    1e-8 (graph replay of 4 iterations), printing the wall time of each part.
    --mode presplit: every level also writes its pre-split values (the
    V-cycle's SpMVs in double-float, as in the benchmark); --mode f32: the
    finest level writes its pre-split values and every level an FP32 copy for
    the FP32 V-cycle.  --lanczos: the smoothers' eigenvalue bounds by
    MG_LANCZOS_STEPS Lanczos steps instead of 10 power steps."""
    import torch
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import inputs
    N, s, reps = args.N, args.s, args.reps
    presplit, f32 = args.mode == "presplit", args.mode == "f32"
    dev = torch.device("cuda:0")
    mg = E.Multigrid(N, M_KL, device=dev)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, s, M_KL)
    xi = torch.from_numpy(inputs.ensemble_layout(xs)).to(dev)
    starts = _profile_starts(torch, mg.meshes, s, dev)
    x = torch.zeros(mg.meshes[0].n * s, dtype=torch.float64, device=dev)
    split_levels = mg.meshes if presplit else (mg.meshes[:1] if f32 else [])
    pre = [torch.empty(2 * m.nnz * s, dtype=torch.float32, device=dev) for m in split_levels] or None
    vals, b = mg.assemble(s, xi, df=True, values_df=pre)
    v32 = mg.to_f32(s, vals) if f32 else None
    work = torch.empty(mg.workspace_size(s, vals, starts, pre, v32), dtype=torch.uint8, device=dev)
    for rep in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x.zero_()
        vals, b = mg.assemble(s, xi, df=True, values_df=pre)
        if f32:
            mg.to_f32(s, vals, out=v32)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        eig = dict(flags=E.PC_LANCZOS, power_iters=MG_LANCZOS_STEPS) if args.lanczos else dict(flags=0,
                                                                                             power_iters=10)
        it, rr, st, stats = mg.solve(s, vals, b, x, 1e-8, 500, work, starts,
                                     flags=E.CG_GRAPH | E.CG_X0_ZERO | eig["flags"], power_iters=eig["power_iters"],
                                     check_every=4, values_df=pre, values_f32=v32)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        print(f"rep {rep}: assemble {1e3 * (t1 - t0):.2f} ms, solve {1e3 * (t2 - t1):.2f} ms, "
              f"iterations {max(it)}, status {sorted(set(st))}")


def main_profile_nl(args):
    """Profiling driver: Newton-GMRES for the nonlinear advection-diffusion
    problem on an N^3 mesh (v = (1, 1, 1), alpha = 1, beta = 10, tol 1e-8,
    GMRES(30) to 1e-6 per step, V-cycle right preconditioner, every level
    pre-split).  --reps times: assemble every level of one ensemble of s
    samples and solve from u = 0, printing the wall time of each part."""
    import torch
    import paper_1511_03703_gb300 as E
    from paper_1511_03703_gb300 import inputs
    N, s, reps = args.N, args.s, args.reps
    dev = torch.device("cuda:0")
    nl = E.Nonlinear(N, M_KL, v=(1.0, 1.0, 1.0), precond=E.NL_PRECOND_MG, device=dev)
    xs = inputs.kl_samples(inputs.SEED_SCALE, 0, s, M_KL)
    xi = torch.from_numpy(inputs.ensemble_layout(xs)).to(dev)
    starts = _profile_starts(torch, nl.meshes, s, dev)
    p = nl.params(1.0, 10.0, tol=1e-8, lin_tol=1e-6, restart=30, max_lin=300, max_newton=20)
    u = torch.zeros(nl.mesh.n * s, dtype=torch.float64, device=dev)
    vdf = [torch.empty(2 * m.nnz * s, dtype=torch.float32, device=dev) for m in nl.meshes]
    vals, b = nl.assemble(s, xi, values_df=vdf)
    work = torch.empty(nl.workspace_size(s, vals, starts, p, vdf), dtype=torch.uint8, device=dev)
    for rep in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u.zero_()
        vals, b = nl.assemble(s, xi, values_df=vdf)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ni, li, rr, st, stats = nl.solve(s, vals, b, u, work, starts, p, values_df=vdf)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        print(f"rep {rep}: assemble {1e3 * (t1 - t0):.2f} ms, solve {1e3 * (t2 - t1):.2f} ms, "
              f"newton {max(ni)}, gmres {max(li)}, status {sorted(set(st))}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--s", type=int, default=32, choices=[1, 4, 8, 16, 32])
    ap.add_argument("--spmv", default="dfv", choices=list(FORMS),
                    help="CG SpMV arithmetic: native FP64 FMA, double-float on the FP32 pipe, "
                         "alternate entries on each (split), or double-float reading values "
                         "pre-split once per ensemble (dfv)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the other-form run, the s sweep and the "
                                                          "extension workloads")
    ap.add_argument("--no-extensions", action="store_true",
                    help="skip the compact extension workloads (A7, A8, A9, MG-PCG) of the default line")
    ap.add_argument("--workload", default="scale", choices=["scale", "mixed", "batched", "guess", "coupled", "pcg", "mg",
                                                             "nonlinear", "profile-cg", "profile-mg", "profile-nl"],
                    help="scale: 64^3 ensemble CG (default line); mixed: 128^3 mixed precision; "
                         "batched: 16^3..64^3 x s=4..32 in one batch; guess: learned initial guess; "
                         "coupled: the paper's coupled CG vs per-member CG; pcg: preconditioned CG; "
                         "mg: multigrid-preconditioned CG; nonlinear: Newton-GMRES for the "
                         "advection-diffusion problem; profile-cg / profile-mg / profile-nl: one solve on "
                         "an --N mesh for ncu captures (no JSON line)")
    ap.add_argument("--N", type=int, default=64, help="profile-*: cells per side")
    ap.add_argument("--iters", type=int, default=8, help="profile-cg: fixed CG iteration count")
    ap.add_argument("--k1-chunks", type=int, default=0, choices=[0, 1, 2, 4, 8],
                    help="profile-cg: chunks of 32 rows per SpMV CTA (0: the library's default)")
    ap.add_argument("--reps", type=int, default=2, help="profile-mg / profile-nl: repetitions")
    ap.add_argument("--lanczos", action="store_true", help="profile-mg: eigenvalue bounds by Lanczos steps")
    ap.add_argument("--mode", default="presplit", choices=["", "presplit", "f32"],
                    help="profile-mg: which levels are pre-split / FP32")
    args = ap.parse_args()
    profile = {"profile-cg": main_profile_cg, "profile-mg": main_profile_mg, "profile-nl": main_profile_nl}
    if args.workload in profile:
        profile[args.workload](args)
        return
    if args.workload == "mixed" and args.impl != "reference":
        main_mixed(args)
        return
    if args.workload == "batched" and args.impl != "reference":
        main_batched(args)
        return
    if args.workload == "guess" and args.impl != "reference":
        main_guess(args)
        return
    if args.workload == "coupled" and args.impl != "reference":
        main_coupled(args)
        return
    if args.workload == "pcg" and args.impl != "reference":
        main_pcg(args)
        return
    if args.workload == "mg" and args.impl != "reference":
        main_mg(args)
        return
    if args.workload == "nonlinear" and args.impl != "reference":
        main_nonlinear(args)
        return
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
