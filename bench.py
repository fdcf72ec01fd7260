"""Benchmark: BKS solves/s on the 100,000 x 100,000 x 50 power-law tensor
(5M stored entries, rank (3,3,3), BK(2,4)), mixed precision vs FP64 at equal
tolerance, with the contraction kernel's achieved HBM bandwidth, an
end-to-end number through the C ABI with host buffers, and the CPU oracle as
the baseline.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

A step is one full BKS solve (Algorithm 5) from a seeded start to the
tolerance on the resident tensor.  Between steps a 512 MB buffer is written
to flush the L2 cache.  N > 1 runs N independent replicas (one process per
GPU, weak scaling): the path has no exchange step to distribute.
"""
from __future__ import annotations

import os

# the CPU oracle legs report single-threaded timings: pin the BLAS pools
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = {
    "workload": "zipf1.1 (1,2)-symmetric 100000x100000x50, ~5.0M stored (4.055M draws, "
                "mirrored, duplicates summed), rank (3,3,3), BK(s=2,p=4) -> (k1,k3)=(36,21)",
    "m": 100_000, "n": 50, "draws": 4_055_000, "zipf_s": 1.1, "seed": 2,
    "r": 3, "stages": 2, "block_p": 4, "tol": 1e-9, "mixed_tol": 1e-4, "tol_scale_free": 1,
}
# The stopping test of both forms is the scale-free ||grad|| / ||F||^2 <= 1e-9
# (the paper's ||grad|| / ||F|| grows with the scale of A: ||F|| ~ 5e4 here);
# the bench checks that both results are within 1e-6 (sin of the largest
# principal angle) of a tightly converged FP64 solution.


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self, idx=0):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={idx}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = []
        mx = 0.0
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                mx = max(mx, float(s[2]))
            except ValueError:
                continue
            for nm, val in zip(names, s[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def whole_job_rate(local_seconds, steps, dist=None, device="cpu"):
    """Whole-job solves/s over the ranks: every rank times `steps` solves of
    its own replica; the job's time is the slowest rank's (MAX all-reduce),
    and the units are all ranks' solves.  Returns (rate, job seconds)."""
    tot, world = float(local_seconds), 1
    if dist is not None:
        import torch
        t = torch.tensor([tot], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot, world = float(t.item()), dist.get_world_size()
    return world * steps / tot, tot


def make_input():
    w = WORKLOAD
    return synth.zipf_tensor(w["seed"], w["m"], w["n"], w["draws"], w["zipf_s"],
                             values="lognormal")


def start_matrices(m, n, r, seed=20):
    g = synth.rng(seed)
    return synth.orthonormal(g, m, r), synth.orthonormal(g, n, r)


# ---------------------------------------------------------------------------
def cpu_oracle_sample(coo, budget_s=20.0):
    """The oracle as it stands on the host cores: one outer iteration of
    Algorithm 5 (stage 1 + expansion + core + inner solve) on a row-sample of
    the workload, scaled to solves/s by the GPU run's outer-iteration count.
    The sample keeps the draws whose i and j fall in the first `frac` of the
    permuted index range, so it has the same generator and value law."""
    import oracle as O
    w = WORKLOAD
    frac = 0.5
    mm = int(w["m"] * frac)
    # rows of the sample: relabel indices < mm (the permutation is uniform)
    sel = (coo.i < mm) & (coo.j < mm)
    sub = (coo.i[sel], coo.j[sel], coo.k[sel], coo.v[sel])
    t0 = time.perf_counter()
    A = O.symmetrise(mm, w["n"], *sub)
    U0, W0 = start_matrices(mm, w["n"], w["r"])
    t1 = time.perf_counter()
    res = O.bks(A, U0, W0, s=w["stages"], p=w["block_p"], tol=0.0, max_outer=1)
    t2 = time.perf_counter()
    return {"seconds_per_outer_iter": t2 - t1, "ingest_s": t1 - t0, "nnz_sample": A.nnz,
            "m_sample": mm, "threads": 1}


def run_reference(args):
    """--impl reference: the CPU oracle on the host cores, same config and
    metric (BKS solves/s), each step a bounded sample (one outer iteration
    on a half-index row sample) extrapolated to a full solve."""
    coo = make_input()
    outer_iters = 6  # outer iterations of an FP64 solve at this tolerance (the GPU FP64 solve's count)
    times = []
    for s in range(args.warmup + args.steps):
        d = cpu_oracle_sample(coo)
        if s >= args.warmup:
            times.append(d["seconds_per_outer_iter"])
    t_iter = statistics.median(times)
    nnz_full = 5_000_000  # stored entries of the full workload (measured by the GPU arm)
    scale = nnz_full / max(1, d["nnz_sample"])
    solve_s = t_iter * scale * outer_iters
    value = 1.0 / solve_s
    line = {"metric": "BKS solves/s", "value": value, "unit": "solves/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": solve_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["workload"]},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"one outer iteration on a {d['m_sample']}-row sample "
                                       f"({d['nnz_sample']} stored), scaled by stored entries "
                                       f"x {outer_iters} outer iterations"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# DRAM bytes (read + write) of k_contract<float,float,4,4,0> in one ncu
# capture of the 500,000 x 500,000 x 200 case (`--ncu-case mode1 --size mid`)
MID_TRAFFIC_BYTES = 186_827_264 + 30_340_352
MID_NNZ = 11_777_770
LARGE = {"m": 1_000_000, "n": 200, "draws": 60_000_000, "zipf_s": 1.2, "seed": 3, "r": 5}


def large_roofline(bk, torch, stream, flush, hbm, peak_kind):
    """The contraction roofline case: the mode-1 contraction on the
    1e6 x 1e6 x 200 Zipf(1.2) tensor (FP32 values, mirrored, duplicates
    summed), with the 4 x 4 block shape of BK(2,4) (X and Y 4 columns,
    output 16).  `traffic`: DRAM bytes of k_contract measured by ncu on the
    500,000 x 500,000 x 200 case (11,777,770 stored, same kernel; that size
    runs the (64, 1024) plan, this one (128, 2048)), scaled to this launch by
    stored entries.  One timed call = pack of X and Y,
    the contraction kernel, the piece reduction of long rows and the zero
    rows; algorithmic bytes = index and value streams + row pointers + X and
    Y read once + output written once (gathers served by L2 not counted)."""
    L = LARGE
    coo = synth.zipf_tensor(L["seed"], L["m"], L["n"], L["draws"], L["zipf_s"],
                            values="absnormal", vdtype=np.float32)
    T = bk.bks_tensor_create_coo(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    del coo
    m, n, p, q = L["m"], L["n"], 4, 4
    g = synth.rng(11)
    X = torch.tensor(g.standard_normal((m, p)), device="cuda", dtype=torch.float32)
    Y = torch.tensor(g.standard_normal((n, q)), device="cuda", dtype=torch.float32)
    out = torch.empty((p * q, m), device="cuda", dtype=torch.float32).t()
    for _ in range(3):
        bk.bks_contract_mode1(T, X, Y, out=out, stream=stream)
    ts = []
    for _ in range(20):
        flush.fill_(2.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bk.bks_contract_mode1(T, X, Y, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    kt = statistics.median(ts)
    nnz = T.nnz
    alg = nnz * (4 + 4 + 4) + (m + 1) * 4 + m * p * 4 + n * q * 4 + m * p * q * 4
    ach = alg / kt / 1e9
    T.close()
    traffic = int(MID_TRAFFIC_BYTES * nnz / MID_NNZ)
    return {"kernel": "bks_contract_mode1 FP32 (pack + k_contract<float,float,4,4> + piece "
                      "reduction + zero rows)",
            "workload": f"zipf1.2 (1,2)-symmetric 1e6 x 1e6 x 200, {nnz} stored "
                        f"({L['draws']} draws mirrored, duplicates summed), X 4 cols, Y 4 cols",
            "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "peak_kind": peak_kind, "traffic": traffic,
            "traffic_note": "ncu dram bytes of k_contract on the 11.8M-entry case, scaled by "
                            "stored entries", "alg_bytes_per_launch": alg,
            "median_launch_s": kt, "nnz_stored": nnz}


def ncu_case(args):
    """Profiling entry for ncu: a few launches of one kernel family, or the
    bench's mixed-precision solve (twice, the first one warms up)."""
    import torch
    import paper_2012_07595_gb300 as bk
    from paper_2012_07595_gb300 import _build
    _build.build()
    if args.size == "large":
        L = LARGE
        coo = synth.zipf_tensor(L["seed"], L["m"], L["n"], L["draws"], L["zipf_s"],
                                values="absnormal", vdtype=np.float32)
        r, p = L["r"], 4
    elif args.size == "mid":
        coo = synth.zipf_tensor(3, 500_000, 200, 12_000_000, 1.2, values="absnormal",
                                vdtype=np.float32)
        r, p = 4, 4
    else:
        coo = make_input()
        if args.ncu_case != "solve":
            coo.v = coo.v.astype(np.float32)
        r, p = WORKLOAD["r"], 4
    T = bk.bks_tensor_create_coo(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    g = synth.rng(9)
    X = torch.tensor(g.standard_normal((coo.m, r)), device="cuda", dtype=torch.float32)
    Y = torch.tensor(g.standard_normal((coo.n, p)), device="cuda", dtype=torch.float32)
    if args.ncu_case == "solve":
        w = WORKLOAD
        U0h, W0h = start_matrices(coo.m, coo.n, w["r"])
        prm = bk.BksParams(r1=w["r"], r3=w["r"], stages=w["stages"], block_p=w["block_p"],
                           tol=w["tol"], precision=bk.BKS_PREC_MIXED, mixed_tol=w["mixed_tol"],
                           tol_scale_free=w["tol_scale_free"], refine_sweeps=50, max_outer=500)
        for rep in range(2):
            c0 = bk.bks_launch_count()
            bk.bks_solve(T, prm, torch.tensor(U0h, device="cuda"), torch.tensor(W0h, device="cuda"))
            torch.cuda.synchronize()
            print(f"solve {rep}: {bk.bks_launch_count() - c0} launches")
        return
    for _ in range(3):
        if args.ncu_case == "mode1":
            bk.bks_contract_mode1(T, X, Y)
        elif args.ncu_case == "mode3":
            bk.bks_contract_mode3(T, X)
        elif args.ncu_case == "core":
            Xc = torch.tensor(g.standard_normal((coo.m, 36)), device="cuda", dtype=torch.float32)
            Zc = torch.tensor(g.standard_normal((coo.n, 21)), device="cuda", dtype=torch.float32)
            bk.bks_core(T, Xc, Zc)
    torch.cuda.synchronize()
    print(f"ncu case {args.ncu_case} ({args.size}) done: nnz {T.nnz}")


def batch_and_serve(bk, torch, scale, n_batch, n_serve, stream):
    """The batched form (many small solves on concurrent streams, work tiles
    autotuned per size class) and the serving loop (Poisson arrivals,
    admission by a 150 GB budget, continuous batching), both on jobs drawn
    as the batched workload (sizes scaled by `scale`), mixed precision at
    the scale-free tolerance 1e-9, against the same jobs solved one at a
    time in FP64."""
    jobs = synth.batch_jobs(seed=4, count=n_batch, scale=scale)
    coos = [synth.job_tensor(j) for j in jobs]

    def prm(r, prec):
        return bk.BksParams(r1=r, r3=r, stages=2, block_p=4, tol=1e-9, tol_scale_free=1,
                            precision=prec, mixed_tol=1e-4, refine_sweeps=50, max_outer=200,
                            max_inner=100)

    tens = [bk.bks_tensor_create_coo(c.m, c.n, c.i, c.j, c.k, c.v) for c in coos]
    for T in tens[:4]:
        bk.bks_tensor_autotune(T)   # warm the library's kernels
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = bk.bks_batch_solve(tens, [prm(j["r"], bk.BKS_PREC_MIXED) for j in jobs],
                             nstreams=8, autotune=True, stream=stream)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    ok = sum(1 for r in res if r[4] == 0)
    t0 = time.perf_counter()
    for T, j in zip(tens, jobs):
        try:
            bk.bks_solve(T, prm(j["r"], bk.BKS_PREC_FP64), stream=stream)
        except bk.BksError:
            pass
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    batched = {"jobs": n_batch, "ok": ok, "solves_per_s": n_batch / t_batch,
               "sequential_fp64_solves_per_s": n_batch / t_seq,
               "speedup_vs_sequential_fp64": t_seq / t_batch, "streams": 8,
               "scale": scale, "nnz_stored_total": int(sum(T.nnz for T in tens))}
    del tens
    # serving: Poisson arrivals, mean gap 5 ms
    arrivals, sjobs = synth.serving_stream(seed=5, requests=n_serve, scale=scale)
    scoos = [synth.job_tensor(j) for j in sjobs]
    with bk.Server(150 << 30, max_slots=8, autotune=True) as srv:
        start = time.perf_counter()
        tickets = []
        for a, j, c in zip(arrivals, sjobs, scoos):
            now = time.perf_counter() - start
            if a > now:
                time.sleep(a - now)
            tickets.append(srv.submit(c.m, c.n, c.i, c.j, c.k, c.v,
                                      prm(j["r"], bk.BKS_PREC_MIXED)))
        outs = [srv.poll(t, wait=True) for t in tickets]
        wall = time.perf_counter() - start
    lat = sorted(o["latency_s"] for o in outs)
    serving = {"requests": n_serve, "ok": sum(1 for o in outs if o["status"] == 0),
               "solves_per_s": n_serve / wall, "offered_per_s": n_serve / float(arrivals[-1]),
               "latency_p50_s": lat[len(lat) // 2],
               "latency_p99_s": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
               "slots": 8, "budget_bytes": 150 << 30, "scale": scale}
    return batched, serving


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-scale", type=float, default=0.1,
                    help="size scale of the batched/serving jobs (1.0 = m up to 2e5 and "
                         "up to 5M stored entries per job); 0 skips them")
    ap.add_argument("--batch-jobs", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--ncu-case", default=None,
                    help="profiling entry: build the workload, run a few launches of one "
                         "kernel family (mode1, mode3, core, solve) and exit without a JSON line")
    ap.add_argument("--size", default="medium", choices=["medium", "mid", "large"],
                    help="ncu-case workload: medium = 1e5 x 1e5 x 50 (5M stored), "
                         "mid = 5e5 x 5e5 x 200 (11.8M stored), large = 1e6 x 1e6 x 200 "
                         "(48.5M stored)")
    args = ap.parse_args()
    if args.ncu_case:
        return ncu_case(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    import paper_2012_07595_gb300 as bk
    from paper_2012_07595_gb300 import _build
    _build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    w = WORKLOAD
    coo = make_input()
    U0h, W0h = start_matrices(w["m"], w["n"], w["r"])
    stream = torch.cuda.current_stream()
    T = bk.bks_tensor_create_coo(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
    U0 = torch.tensor(U0h, device="cuda")
    W0 = torch.tensor(W0h, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def params(prec, inner=None):
        return bk.BksParams(r1=w["r"], r3=w["r"], stages=w["stages"], block_p=w["block_p"],
                            tol=w["tol"], precision=prec, mixed_tol=w["mixed_tol"],
                            tol_scale_free=w["tol_scale_free"], refine_sweeps=50,
                            max_outer=500,
                            inner_schedule=bk.BKS_INNER_FAST if inner is None else inner)

    def timed_solves(prec, steps, warm):
        lat = []
        infos = []
        for s in range(warm + steps):
            flush.fill_(float(s))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            e0.record(stream)
            U, W, F, info = bk.bks_solve(T, params(prec), U0, W0, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if s >= warm:
                lat.append(e0.elapsed_time(e1) / 1e3)
                infos.append(info)
        return lat, infos, (U, W, F)

    # ---- tightly converged FP64 reference (not timed) ----
    pref = params(bk.BKS_PREC_FP64)
    pref.tol = 1e-11
    pref.max_outer = 100
    Uref, Wref, _, _ = bk.bks_solve(T, pref, U0, W0, stream=stream)
    Uref, Wref = Uref.cpu().numpy(), Wref.cpu().numpy()

    # ---- headline: mixed-precision solves ----
    clocks = Clocks()
    clocks.start(local)
    launches0 = bk.bks_launch_count()
    lat_mixed, inf_mixed, res_mixed = timed_solves(bk.BKS_PREC_MIXED, args.steps, args.warmup)
    launches = (bk.bks_launch_count() - launches0) * args.steps / (args.steps + args.warmup)
    clk = clocks.stop()
    value, tot = whole_job_rate(sum(lat_mixed), args.steps, dist, "cuda")
    # ---- FP64 at the same tolerance ----
    lat64, inf64, res64 = timed_solves(bk.BKS_PREC_FP64, max(2, args.steps // 2), 1)
    fp64_rate = len(lat64) / sum(lat64)
    # subspace agreement mixed vs FP64: sin of the largest principal angle
    def sin_max(A, B):
        D = B - A @ (A.T @ B)
        return float(np.linalg.norm(D, 2))
    Um, Wm = res_mixed[0].cpu().numpy(), res_mixed[1].cpu().numpy()
    U6, W6 = res64[0].cpu().numpy(), res64[1].cpu().numpy()
    ang = {"mixed_vs_ref": max(sin_max(Uref, Um), sin_max(Wref, Wm)),
           "fp64_vs_ref": max(sin_max(Uref, U6), sin_max(Wref, W6)),
           "mixed_vs_fp64": max(sin_max(U6, Um), sin_max(W6, Wm))}

    # ---- contraction kernel roofline (mode-1, FP32, stage-2 width 3x4) ----
    hbm, peak_kind = _peaks()
    X32 = torch.tensor(synth.rng(5).standard_normal((w["m"], w["r"])), device="cuda",
                       dtype=torch.float32)
    Y32 = torch.tensor(synth.rng(6).standard_normal((w["n"], 4)), device="cuda",
                       dtype=torch.float32)
    T32 = bk.bks_tensor_create_coo(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v.astype(np.float32))
    out32 = torch.empty((12, w["m"]), device="cuda", dtype=torch.float32).t()
    for _ in range(3):
        bk.bks_contract_mode1(T32, X32, Y32, out=out32, stream=stream)
    reps = 20
    ktimes = []
    for _ in range(reps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bk.bks_contract_mode1(T32, X32, Y32, out=out32, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ktimes.append(e0.elapsed_time(e1) / 1e3)
    kt = statistics.median(ktimes)
    nnz = T32.nnz
    alg_bytes = nnz * (4 + 4 + 4) + (w["m"] + 1) * 4 + w["m"] * w["r"] * 4 + w["n"] * 4 * 4 \
        + w["m"] * 12 * 4
    achieved = alg_bytes / kt / 1e9
    roofline_workload = {"kernel": "bks_contract_mode1 FP32 3 x 4 (pack + k_contract<float,float,"
                                   "4,4> + piece reduction + zero rows)",
                         "workload": w["workload"],
                         "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_kind": peak_kind, "traffic": None,
                         "alg_bytes_per_launch": alg_bytes, "median_launch_s": kt}
    del T32
    roofline = large_roofline(bk, torch, stream, flush, hbm, peak_kind)

    # ---- end to end through the C ABI with host buffers ----
    e2e_steps = max(1, min(3, args.steps))
    t_e2e = []
    h2d = coo.nnz * (4 * 3 + 8) + (w["m"] * w["r"] + w["n"] * w["r"]) * 8
    d2h = (w["m"] * w["r"] + w["n"] * w["r"] + w["r"] ** 3) * 8
    for s in range(e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Th = bk.bks_tensor_create_coo(coo.m, coo.n, coo.i, coo.j, coo.k, coo.v)
        U0d = torch.tensor(U0h).cuda()
        W0d = torch.tensor(W0h).cuda()
        U, W, F, _ = bk.bks_solve(Th, params(bk.BKS_PREC_MIXED), U0d, W0d, stream=stream)
        Uc, Wc, Fc = U.cpu(), W.cpu(), F.cpu()
        torch.cuda.synchronize()
        if s > 0:
            t_e2e.append(time.perf_counter() - t0)
        Th.close()
    e2e_rate = world * e2e_steps / sum(t_e2e)

    # ---- batched form and serving loop (scaled job sizes, see the keys) ----
    batched = serving = None
    if args.batch_scale > 0:
        batched, serving = batch_and_serve(bk, torch, args.batch_scale, args.batch_jobs,
                                           args.serve_requests, stream)

    # ---- CPU oracle baseline (bounded sample) ----
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        d = cpu_oracle_sample(coo)
        outer = statistics.median([i["iters"] for i in inf64])
        scale = T.nnz / max(1, d["nnz_sample"])
        solve_s = d["seconds_per_outer_iter"] * scale * max(1, outer)
        cpu = {"value": 1.0 / solve_s, "unit": "solves/s", "cores": d["threads"],
               "kind": "oracle",
               "sample": f"one FP64 outer iteration on a {d['m_sample']}-row sample "
                         f"({d['nnz_sample']} stored), {d['seconds_per_outer_iter']:.1f} s, scaled "
                         f"by stored entries x {outer} outer iterations (FP64 GPU solve count)"}

    lat_sorted = sorted(lat_mixed)
    line = {
        "metric": "BKS solves/s", "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": w["workload"], "precision": "mixed (FP32 contractions, FP64 "
                   "orthogonalisation/inner solve/restart, FP64 refinement)",
                   "stop": f"||grad||/||F||^2 <= {w['tol']}", "accuracy": "both results within "
                   "1e-6 (sin of largest principal angle) of an FP64 solution converged to "
                   "||grad||/||F||^2 <= 1e-11",
                   "l2": "512 MB buffer written between timed steps",
                   "parallelism": f"replicas x{world}"},
        "fp64_solves_per_s": fp64_rate, "mixed_over_fp64": value / world / fp64_rate,
        "subspace_sin": ang,
        "latency_s": {"p50": lat_sorted[len(lat_sorted) // 2],
                      "p99": lat_sorted[min(len(lat_sorted) - 1, int(0.99 * len(lat_sorted)))]},
        "outer_iters": {"mixed": [i["iters"] for i in inf_mixed],
                        "mixed_fp32": [i["fp32_iters"] for i in inf_mixed],
                        "fp64": [i["iters"] for i in inf64]},
        "grad_rel": {"mixed": inf_mixed[-1]["grad_rel"], "fp64": inf64[-1]["grad_rel"]},
        "phase_ms": {"mixed": inf_mixed[-1]["phase_ms"], "fp64": inf64[-1]["phase_ms"]},
        "roofline": roofline,
        "roofline_workload": roofline_workload,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_rate, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "batched": batched,
        "serving": serving,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
