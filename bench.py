#!/usr/bin/env python
"""Benchmark of the sector Hamiltonian-vector product at N_s = 15, half filling.

One step = one matrix-free H*v (the hot path's core; every Lanczos and
Green's-function step is one of these plus vector updates) on the three-orbital
Kanamori impurity with 12 bath sites, sector (N_up, N_dn) = (7, 8),
dim 6435^2 = 41,409,225, seeded random bath (synthetic; the paper's LDA baths
are not available).  Inputs are larger than L2 (x is 331 MB), so no flush is
needed between steps.

Prints one JSON line (rank 0).  Replicas only: with --gpus N under torchrun each
rank runs the same workload on its own GPU, no collective on the data path
(weak scaling); value = sum over ranks of bytes / max-over-ranks time.

--impl reference times the CPU oracle (the reference arm: the paper has no
code to run) on a bounded row sample of the same workload on the host cores.

Other workloads (--workload): sectors12 (all 169 sectors of N_s = 12, batched),
solve15 (ground state, G(i w_n), spectral function, set-up, stored CSR),
serve (a stream of impurity solves through the request server), lowest8
(eight lowest states, full basis vs thick restart), dmft (ED/DMFT of the
square-lattice Hubbard model).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "H*v GB/s (% of HBM peak) at N_s=15; solves/s, p99 latency vs plain FP64"
NS, NUP, NDN = 15, 7, 8
SEED = 0


def args_parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default="df64", choices=["df64", "fp64", "fp32"])
    p.add_argument("--e2e-steps", type=int, default=12)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the FP64 / FP32 side measurements")
    p.add_argument("--no-autotune", action="store_true", help="time the untuned default H*v variant")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--workload", default="hv15", choices=["hv15", "sectors12", "serve", "solve15", "lowest8", "dmft"],
                   help="hv15: H*v at N_s=15 (default); sectors12: 8 lowest states of all 169 sectors at N_s=12; "
                        "serve: Poisson stream of impurity solves, N_s in 10..16; "
                        "solve15: N_s=15 ground state + G(i w_n) per vector format, and the stored-CSR H*v")
    p.add_argument("--requests", type=int, default=40)
    p.add_argument("--serve-requests", type=int, default=16, help="requests of the serve block in the default line")
    p.add_argument("--serve-tol", type=float, default=1e-8)
    p.add_argument("--sectors-tol", type=float, default=1e-8, help="tolerance of every format in --workload sectors12")
    p.add_argument("--sectors-formats", default="fp64,fp32,df64", help="vector formats of --workload sectors12")
    p.add_argument("--sectors-max-iter", type=int, default=400, help="Lanczos steps at most in --workload sectors12")
    p.add_argument("--no-one-at-a-time", action="store_true",
                   help="--workload sectors12 without the one-sector-at-a-time FP64 baseline")
    p.add_argument("--no-serve", action="store_true", help="skip the serve block of the default line")
    return p.parse_args(argv)


def workload_config(prec, dim):
    eb = 4 if prec == "fp32" else 8
    return {"workload": f"three-orbital Kanamori impurity, N_s=15 (3 impurity + 12 bath), sector (7,8), "
                        f"dim {dim}, matrix-free H*v",
            "n_s": NS, "sector": [NUP, NDN], "dim": dim, "vector_format": prec,
            "l2": f"inputs larger than L2 (x = {dim * eb / 1e6:.0f} MB, L2 ~126 MB): no flush",
            "model": "kanamori U=2.3 J=0.4 U'=U-2J J'=J, eps_k~U[-1.5,1.5], V~U[0.1,0.4], seed 0"}


# Arithmetic ceiling of one H*v.  Multiply-adds per element: the off-diagonal
# entries of the row plus two for the diagonal (e_dn + W and e_up).  A
# double-float multiply-add is 12 FP32 instructions; float vectors take one FP32
# FMA per multiply-add (natural-order kernel, float sums); FP64 rows take one
# DFMA.  FP32 peak from the unit counts at the 2.07 GHz maximum SM clock (152
# SMs x 128 FP32 lanes).  The FP64 peak is the measured DFMA rate on this GPU
# (a dependent-FMA probe on every SM: 0.50 T DFMA/s, about 1.6 per SM per clock),
# since GB300's FP64 pipe does not reach a unit-count figure.
FP32_PEAK = 152 * 128 * 2.07e9
DFMA_PEAK = 0.50e12


def alu_roofline(prec, dim, nnz_per_row, launch_ms):
    macs = dim * (nnz_per_row + 1.0)
    if prec == "fp64":
        ops, peak, unit = macs, DFMA_PEAK, "T DFMA/s"
    else:
        ops, peak, unit = macs * (12 if prec == "df64" else 1), FP32_PEAK, "T FP32 instructions/s"
    achieved = ops / (launch_ms * 1e-3)
    return {"bound": "alu", "achieved": round(achieved / 1e12, 3), "peak": round(peak / 1e12, 3), "unit": unit,
            "frac": round(achieved / peak, 4), "ops_per_launch": ops, "macs_per_element": nnz_per_row + 1.0,
            "peak_source": ("measured DFMA rate (probe)" if prec == "fp64"
                            else "unit counts x 2.07 GHz maximum SM clock")}


def ranks_max(vals, dist, device):
    """Each timing (ms) maximised over ranks, so that whole-job rates are set by
    the slowest rank; identity on one rank."""
    if dist is None:
        return [float(v) for v in vals]
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_gbs(world, bytes_per_rank, ms):
    """Whole-job rate in GB/s: every rank moves bytes_per_rank per step of ms."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


def alg_bytes(prec, dim):
    """Compulsory traffic of one H*v: read x once, write y once."""
    return 2 * dim * (4 if prec == "fp32" else 8)


# ----------------------------------------------------------- clock sampler
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle leg
def oracle_rows_rate(model, x, seconds, rng):
    """Oracle H*v on sampled rows (literal operator application); returns
    (rows per second, rows done, seconds)."""
    from oracle import sector as osec
    dim = len(x)
    done, t0 = 0, time.perf_counter()
    chunk = 50_000
    while True:
        rows = np.sort(rng.integers(0, dim, chunk))
        osec.apply_rows(model, NUP, NDN, rows, x)
        done += chunk
        el = time.perf_counter() - t0
        if el >= seconds:
            return done / el, done, el


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":", 1)[0].strip().lower()
            if k in ("model name", "cpu part", "hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_csr_block(model, n_up, n_dn, row0, nrows):
    """Rows [row0, row0 + nrows) of the sector CSR, built by the oracle (literal
    operator products applied to each row state)."""
    import scipy.sparse as sp
    from oracle import sector as osec
    rows = np.arange(row0, row0 + nrows, dtype=np.int64)
    ptr, cols, vals = osec.row_entries(model, n_up, n_dn, rows)
    dim = W_sector_dim(model.n_s, n_up, n_dn)
    return sp.csr_matrix((vals, cols.astype(np.int32), ptr), shape=(nrows, dim))


def W_sector_dim(n_s, n_up, n_dn):
    import workloads as W
    return W.sector_dim(n_s, n_up, n_dn)


def time_loop(f, seconds, min_reps=3):
    f()
    reps, t0 = 0, time.perf_counter()
    while True:
        f()
        reps += 1
        el = time.perf_counter() - t0
        if reps >= min_reps and el >= seconds:
            return el / reps, reps


def cpu_baseline(model, x, prec, seconds, legs=True):
    """The CPU oracle timed on this host: its sector H*v (SciPy CSR product over
    the oracle-built matrix) on a contiguous block of rows of the same sector,
    one core (the reported value); the same CSR through torch on every core; the
    oracle's literal-operator product on random rows; and the oracle's
    eigensolver wall-clock at the C0 and C1 sizes."""
    eb = 4 if prec == "fp32" else 8
    cores = cpu_cores()
    D_dn = W_sector_dim(NS, 0, NDN)
    nrows = D_dn * 96                                       # 96 up strings, ~1.5% of the sector's rows
    row0 = D_dn * (W_sector_dim(NS, NUP, 0) // 2)           # from the middle of the row order
    t0 = time.perf_counter()
    A = oracle_csr_block(model, NUP, NDN, row0, nrows)
    t_build = time.perf_counter() - t0
    x64 = np.asarray(x, dtype=np.float64)
    per, reps = time_loop(lambda: A @ x64, seconds / 2)
    rows_per_s = nrows / per
    out = {"value": rows_per_s * 2 * eb / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"rows {row0}..{row0 + nrows - 1} ({nrows} rows, {A.nnz} stored entries) of the (7,8) "
                     f"sector's CSR built by the oracle (literal operator products, {t_build:.1f} s), SciPy CSR "
                     f"matvec on 1 core, {reps} products of {per * 1e3:.2f} ms; GB/s = rows/s x {2 * eb} B "
                     f"(the metric's compulsory bytes per row)",
           "cpu_model": cpu_model(), "host_cores": cores}
    if not legs:
        return out
    out["legs"] = {}
    try:
        import torch
        nt = torch.get_num_threads()
        torch.set_num_threads(cores)
        At = torch.sparse_csr_tensor(torch.from_numpy(A.indptr.astype(np.int64)),
                                     torch.from_numpy(A.indices.astype(np.int64)),
                                     torch.from_numpy(A.data), size=A.shape, check_invariants=False)
        xt = torch.from_numpy(x64)
        pt, rt = time_loop(lambda: At @ xt, seconds / 4)
        torch.set_num_threads(nt)
        out["legs"]["torch_sparse_csr_all_cores"] = {
            "GB/s": nrows / pt * 2 * eb / 1e9, "threads": cores, "ms_per_product": pt * 1e3, "reps": rt,
            "rows": nrows}
    except Exception as e:  # torch without sparse CSR matmul on this host
        out["legs"]["torch_sparse_csr_all_cores"] = {"unavailable": str(e)[:200]}
    rng = np.random.default_rng(123)
    rate, done, el = oracle_rows_rate(model, x64, seconds / 4, rng)
    out["legs"]["literal_operator_rows_1_core"] = {"GB/s": rate * 2 * eb / 1e9, "rows": done, "seconds": el}
    out["legs"]["oracle_eigensolver"] = oracle_eigsh_times()
    return out


def oracle_eigsh_times():
    """Oracle lowest eigenvalue wall-clock (sector CSR built by the oracle, then
    dense eigh up to dim 4900 or ARPACK eigsh): C0, the AIM N_s=6 (3,3) (dim
    400), and C1, the Kanamori N_s=12 (6,6) (dim 853,776), ground state."""
    import workloads as W
    from oracle import sector as osec, spectrum
    res = {}
    for name, m, nu, nd in (("C0 AIM N_s=6 (3,3)", W.aim(6, seed=0), 3, 3),
                            ("C1 Kanamori N_s=12 (6,6)", W.kanamori(12, seed=0), 6, 6)):
        t0 = time.perf_counter()
        H = osec.build_csr(m, nu, nd)
        t1 = time.perf_counter()
        w = spectrum.lowest(H, 1)
        t2 = time.perf_counter()
        res[name] = {"dim": int(H.shape[0]), "build_s": t1 - t0, "eigensolve_s": t2 - t1, "E0": float(w[0])}
    return res


def row_kernel(prec):
    """The fast row kernel that ed_apply_h launches, untuned, for this vector format."""
    return "k_apply_nat" if prec == "fp32" else "k_apply_win"


def row_kernel_of(kernel_id):
    """Kernel name of an ed_sector_info / ed_tune_result kernel id."""
    return {2: "k_apply_win", 3: "k_apply_pair", 4: "k_apply_nat"}.get(kernel_id, f"generic_{kernel_id}")


def traffic_for(kernel_src_sha, prec, kernel=None):
    """DRAM bytes per launch of the row kernel from the committed ncu summary,
    only if it was captured from the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"{kernel or row_kernel(prec)}_{prec}_n15_traffic.txt")
    try:
        kv = dict(line.split(":", 1) for line in open(p) if ":" in line)
    except Exception:
        return None
    if kv.get("apply_src_sha", "").strip() != kernel_src_sha:
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def src_sha():
    h = hashlib.sha256()
    for f in ("apply_fast.cu", "apply_nat.cu", "ed_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1004_3354_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ ours
def run_ours(a):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1004_3354_gb300 as ed
    import workloads as W
    if not os.path.exists(ed.LIB_PATH):
        from paper_1004_3354_gb300 import _build
        _build.build()

    model = W.kanamori(NS, seed=SEED)
    dim = W.sector_dim(NS, NUP, NDN)
    x64 = W.random_vector(dim, seed=1)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(model, x64, a.prec, a.cpu_seconds)

    ctx = ed.ed_ctx_create(local)
    sec = ed.ed_sector_create(ctx, model, NUP, NDN, a.prec)
    tuned = None
    if not a.no_autotune:
        r = ed.ed_sector_autotune(sec, reps=5)
        tuned = {"chosen": r.chosen, "candidates": [
            {"kernel": row_kernel_of(r.kernel[i]), "block": r.block[i], "min_blocks_per_sm": r.min_blocks[i],
             "ms": round(r.ms[i], 5) if r.ms[i] > 0 else None} for i in range(r.n_candidates)]}
    variant = ed.ed_sector_get_variant(sec)
    kernel_name = row_kernel_of(ed.ed_sector_get_info(sec).kernel)
    p = ed.PREC_NAMES[a.prec]
    epv = ed.elems_per_value(p)
    tdt = ed.torch_dtype(p)
    x64d = torch.from_numpy(x64).cuda()
    x = torch.empty(dim * epv, dtype=tdt, device="cuda")
    ed.ed_convert(x64d, ed.ED_PREC_FP64, x, p, dim)
    del x64d
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, a.warmup)):
        ed.ed_apply_h(sec, x, y, stream)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(a.steps):
        evs[i][0].record(stream)
        ed.ed_apply_h(sec, x, y, stream)
        evs[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = [s.elapsed_time(e) for s, e in evs]
    ms_step = total_ms / a.steps
    nbytes = alg_bytes(a.prec, dim)

    # end to end through the C ABI with host buffers: ed_apply_h_host takes
    # e2e_steps vectors in pinned host memory, copies each in, applies H and
    # copies each result out, pipelined on its internal streams (the copy-in of
    # step i+1 and the copy-out of step i-1 overlap H*v of step i)
    h2d = d2h = dim * (4 if a.prec == "fp32" else 8)
    n_e2e = max(4, a.e2e_steps // world)   # pinned host memory: 2 x n_e2e vectors per rank
    xh1 = x.cpu()
    hx = torch.empty(n_e2e * xh1.numel(), dtype=tdt).pin_memory()
    for i in range(n_e2e):
        hx[i * xh1.numel():(i + 1) * xh1.numel()].copy_(xh1)
    hy = torch.empty_like(hx).pin_memory()
    # warm-up over every vector: makes the transfer buffers and touches every
    # pinned page once (the first DMA to a page costs more on these hosts)
    ed.ed_apply_h_host(sec, n_e2e, hx, hy, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_runs = []
    for _ in range(3):   # the host link is shared with the machine's other tenants: median of three calls
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ed.ed_apply_h_host(sec, n_e2e, hx, hy, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_runs.append(e0.elapsed_time(e1) / n_e2e)
    e2e_ms = statistics.median(e2e_runs)
    del hx, hy
    ms_step, e2e_ms = ranks_max([ms_step, e2e_ms], dist, "cuda")
    value = whole_job_gbs(world, nbytes, ms_step)
    e2e = {"value": whole_job_gbs(world, nbytes, e2e_ms), "unit": "GB/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": n_e2e,
           "ms_per_step_runs": [round(v, 4) for v in e2e_runs],
           "what": "ed_apply_h_host C-ABI calls on e2e_steps vectors in pinned host memory (median of three "
                   "calls): every step's x copied host -> device and y device -> host inside the call, pipelined "
                   "on the library's internal streams with the applies"}

    extras = {}
    if not a.no_extras and rank == 0:
        for q in ("fp64", "fp32", "df64"):
            if q == a.prec:
                continue
            s2 = ed.ed_sector_create(ctx, model, NUP, NDN, q)
            if not a.no_autotune:
                ed.ed_sector_autotune(s2, reps=3)
            qp = ed.PREC_NAMES[q]
            xq = torch.empty(dim * ed.elems_per_value(qp), dtype=ed.torch_dtype(qp), device="cuda")
            ed.ed_convert(x, p, xq, qp, dim)
            yq = torch.empty_like(xq)
            for _ in range(3):
                ed.ed_apply_h(s2, xq, yq, stream)
            n_q = 10 if q != "fp64" else 5
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(n_q):
                ed.ed_apply_h(s2, xq, yq, stream)
            s1.record(stream)
            torch.cuda.synchronize()
            msq = s0.elapsed_time(s1) / n_q
            extras[q] = {"ms_per_apply": msq, "GB/s": alg_bytes(q, dim) / (msq * 1e-3) / 1e9,
                         "kernel": row_kernel_of(ed.ed_sector_get_info(s2).kernel),
                         "variant": ed.ed_sector_get_variant(s2)}
            del xq, yq
            ed.ed_sector_destroy(s2)

    # the serving half of the metric (solves/s and p99 latency vs plain FP64),
    # a bounded run of the request stream on rank 0 of a one-GPU job
    serve = None
    if not a.no_serve and rank == 0 and world == 1:
        serve = serve_bench(ed, ctx, torch, n_req=a.serve_requests, k=4, tol=a.serve_tol, precs=("fp32",))

    info = ed.ed_sector_get_info(sec)
    peak, src = peaks()
    avg_launch = statistics.mean(launch_ms)
    achieved = nbytes / (avg_launch * 1e-3) / 1e9
    sha = src_sha()
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"df64": "df64 (f32 hi+lo pairs)", "fp64": "f64", "fp32": "f32 (df64 accumulate)"}[a.prec],
        "data": "synthetic (seeded random bath)", "config": workload_config(a.prec, dim),
        "pct_hbm_peak": round(100 * value / world / peak, 2),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic_for(sha, a.prec, kernel_name),
                     "kernel": kernel_name, "variant": variant, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)",
                     "alg_bytes_per_launch": nbytes, "median_launch_ms": statistics.median(launch_ms),
                     "apply_src_sha": sha},
        "alu_roofline": alu_roofline(a.prec, dim, info.nnz_per_row, statistics.mean(launch_ms)),
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": a.steps,
        "clocks": clk, "nnz_per_row": round(info.nnz_per_row, 3), "other_formats": extras, "autotune": tuned,
        "serve": serve,
    }
    ed.ed_sector_destroy(sec)
    ed.ed_ctx_destroy(ctx)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_reference(a):
    """The reference arm: the CPU oracle's sector H*v (SciPy CSR product over the
    oracle-built matrix, one core) on a block of rows of the same N_s=15 (7,8)
    sector, one product per step; rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as W
    model = W.kanamori(NS, seed=SEED)
    dim = W.sector_dim(NS, NUP, NDN)
    x = W.random_vector(dim, seed=1)
    D_dn = W_sector_dim(NS, 0, NDN)
    nrows = D_dn * 96
    row0 = D_dn * (W_sector_dim(NS, NUP, 0) // 2)
    t0 = time.perf_counter()
    A = oracle_csr_block(model, NUP, NDN, row0, nrows)
    t_build = time.perf_counter() - t0
    for _ in range(max(1, a.warmup)):
        A @ x
    t0 = time.perf_counter()
    for _ in range(a.steps):
        A @ x
    el = time.perf_counter() - t0
    eb = 4 if a.prec == "fp32" else 8
    value = nrows * a.steps / el * 2 * eb / 1e9
    sample = (f"{a.steps} products over rows {row0}..{row0 + nrows - 1} ({nrows} rows, {A.nnz} stored entries) of "
              f"the (7,8) sector's CSR built by the oracle ({t_build:.1f} s, not timed), SciPy CSR matvec, 1 core; "
              f"GB/s = rows/s x {2 * eb} B")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": 0,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * el / a.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded random bath)",
           "config": workload_config(a.prec, dim),
           "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample,
                            "cpu_model": cpu_model(), "host_cores": cpu_cores()},
           "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_sectors12(a):
    """All 169 (N_up, N_dn) sectors of the N_s=12 three-orbital Kanamori model,
    8 lowest states each: one batched solve (one CUDA-graph replay per Lanczos
    step over every sector) in each vector format against the same sectors
    solved one at a time in FP64, all at one tolerance.  Only sectors that
    converged count towards solves/s."""
    import torch
    import paper_1004_3354_gb300 as ed
    import workloads as W
    if not os.path.exists(ed.LIB_PATH):
        from paper_1004_3354_gb300 import _build
        _build.build()
    torch.cuda.set_device(0)
    model = W.kanamori(12, seed=0)
    secs = [(u, d) for u in range(13) for d in range(13)]
    dims = [W.sector_dim(12, u, d) for (u, d) in secs]
    tol, max_iter, k = a.sectors_tol, a.sectors_max_iter, 8
    ctx = ed.ed_ctx_create(0)
    out = {"metric": "converged sector solves/s (all 169 sectors of N_s=12, 8 lowest each)",
           "unit": "sector solves/s", "higher_is_better": True, "n_gpus": 1, "data": "synthetic (seeded random bath)",
           "config": {"workload": f"three-orbital Kanamori N_s=12, all 169 sectors, k={k}, tol {tol} in every "
                                  f"format, full CGS2, max_iter {max_iter}"},
           "results": {}}

    def converged(iters):
        # a sector that stopped before max_iter met tol (or exhausted its Krylov space)
        return [bool(it < max_iter or dims[i] <= it + 1) for i, it in enumerate(iters)]

    for prec in [f.strip() for f in a.sectors_formats.split(",") if f.strip()]:
        b = ed.ed_batch_create(ctx, model, secs, prec)
        tune = None
        if not a.no_autotune:
            r = ed.ed_batch_autotune(b, steps=16)
            tune = {"chosen_chunk": r.chunk[r.chosen], "ms_per_step": {
                str(r.chunk[i]): round(r.ms_per_step[i], 4) for i in range(r.n_candidates)}}
        ed.ed_batch_lanczos(b, len(secs), k=k, tol=tol, max_iter=max_iter, allow_not_converged=True)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, it, info, st = ed.ed_batch_lanczos(b, len(secs), k=k, tol=tol, max_iter=max_iter,
                                               allow_not_converged=True)
        el = time.perf_counter() - t0
        ed.ed_batch_destroy(b)
        conv = converged(it)
        out["results"][f"batched_{prec}"] = {
            "seconds": el, "converged_sectors": int(sum(conv)), "solves_per_s": sum(conv) / el,
            "steps": info.steps, "graph_replays": info.graph_replays, "max_iters": int(max(it)), "status": int(st),
            "ground_energy_66": float(ev[6 * 13 + 6, 0]), "packing": tune}
    if a.no_one_at_a_time:
        ed.ed_ctx_destroy(ctx)
        print(json.dumps(out), flush=True)
        return
    # one sector at a time, FP64, no batching or graphs
    t0 = time.perf_counter()
    e66, n_conv = None, 0
    for (u, d) in secs:
        s_ = ed.ed_sector_create(ctx, model, u, d, "fp64")
        ev, info, st = ed.ed_lanczos(s_, k=k, tol=tol, max_iter=max_iter, allow_not_converged=True)
        n_conv += int(st == 0)
        if (u, d) == (6, 6):
            e66 = float(ev[0])
        ed.ed_sector_destroy(s_)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    out["results"]["one_at_a_time_fp64"] = {"seconds": el, "converged_sectors": n_conv, "solves_per_s": n_conv / el,
                                            "ground_energy_66": e66}
    for prec in ("fp32", "df64"):
        if f"batched_{prec}" in out["results"]:
            out["results"][f"batched_{prec}"]["rel_E0_66_diff_vs_fp64"] = abs(
                out["results"][f"batched_{prec}"]["ground_energy_66"] - e66) / abs(e66)
    if "batched_fp64" in out["results"]:
        out["value"] = out["results"]["batched_fp64"]["solves_per_s"]
        out["speedup_batched_fp64_vs_one_at_a_time"] = out["value"] / out["results"]["one_at_a_time_fp64"]["solves_per_s"]
    ed.ed_ctx_destroy(ctx)
    print(json.dumps(out), flush=True)


def tr_basis(k):
    """Thick-restart basis the request server uses for a k > 1 request."""
    return min(max(4 * k + 8, 20), 64)


def fifo_latencies_ms(service, arrivals):
    """Latencies (ms) of requests served one at a time, first come first served:
    request i starts when it has arrived and request i - 1 has finished."""
    fin, lat = 0.0, []
    for s_, a_ in zip(service, arrivals):
        fin = max(fin, a_) + s_
        lat.append((fin - a_) * 1e3)
    return lat


def serve_golden():
    try:
        with open(os.path.join(ROOT, "tests", "golden", "serve_stream.json")) as f:
            g = json.load(f)
        return {r["id"]: r for r in g["requests"]}, g["greens"]["n"]
    except (OSError, KeyError, ValueError):
        return {}, []


def oracle_errors(results, golden, pts, k, stream):
    """Max relative error of the k lowest energies and max |G - G_oracle| over
    the requests the oracle solved (tests/golden/serve_stream.json), matched on
    the request's model seed, N_s and sector."""
    e_err, g_err, n = 0.0, 0.0, 0
    for q, res in results.items():
        g = golden.get(q)
        r = stream[q]
        if g is None or res["E"] is None or (g["n_s"], g["model_seed"], g["sector"]) != (
                r["n_s"], r["model_seed"], [r["n_up"], r["n_dn"]]):
            continue
        ref = np.array(g["E"][:k])
        E = np.array(res["E"][:len(ref)])
        e_err = max(e_err, float(np.max(np.abs(E - ref) / np.abs(ref))))
        if res["G"] is not None and pts:
            Gr = np.array(g["G_re"]) + 1j * np.array(g["G_im"])
            g_err = max(g_err, float(np.max(np.abs(res["G"][pts] - Gr))))
        n += 1
    return {"requests_checked": n, "max_rel_E_err_vs_oracle": e_err if n else None,
            "max_abs_G_err_vs_oracle": g_err if n else None}


PACK_DIM = 250_000   # served requests with at most this many states are solved in packs (N_s <= 11 here)


def serve_saturation(ed, ctx, stream, models, k, tol, prec, pack_dim, max_active=16, depth=100, nw=1024, beta=40.0):
    """All requests submitted at t = 0; returns (seconds, failures, max active)."""
    srv = ed.ed_server_create(ctx, hbm_budget=200 * 1024 ** 3, max_active=max_active, prec=prec, tol=tol,
                              max_iter=3000, cf_depth=depth, n_w=nw, beta=beta, pack_dim=pack_dim)
    t0 = time.perf_counter()
    tickets = [ed.ed_submit(srv, m, r["n_up"], r["n_dn"], k=k) for r, m in zip(stream, models)]
    done, fails = set(), 0
    while len(done) < len(tickets):
        for t in tickets:
            if t in done:
                continue
            d, res, G = ed.ed_poll(srv, t)
            if d:
                done.add(t)
                fails += int(res.status != 0)
        time.sleep(0.0005)
    el = time.perf_counter() - t0
    mx = ed.ed_server_get_stats(srv).max_active_seen
    ed.ed_server_destroy(srv)
    return el, fails, mx


def small_requests_bench(ed, ctx, n_req=32, k=4, tol=1e-8, prec="fp32"):
    """Small impurity solves (N_s 8..11, the same request shape as the serving
    stream) served one request per stream against packs of them (one batched
    Lanczos over all their sectors per step)."""
    import workloads as W
    stream = W.serving_stream(n_req, seed=1, rate=1.0, ns_range=(8, 11))
    models = [W.kanamori(r["n_s"], seed=r["model_seed"]) for r in stream]
    out = {"requests": n_req, "k": k, "tol": tol, "prec": prec, "n_s": "8..11", "pack_dim": PACK_DIM}
    for label, pd in (("one_stream_per_request", 0), ("packs", PACK_DIM)):
        serve_saturation(ed, ctx, stream[:4], models[:4], k, tol, prec, pd)      # warm-up
        el, fails, mx = serve_saturation(ed, ctx, stream, models, k, tol, prec, pd)
        out[label] = {"solves_per_s": n_req / el, "seconds": el, "failed": fails, "max_active_seen": mx}
    out["speedup_packs"] = out["packs"]["solves_per_s"] / out["one_stream_per_request"]["solves_per_s"]
    return out


def serve_bench(ed, ctx, torch, n_req=16, k=4, tol=1e-8, precs=("fp32",), modes=("saturation", "poisson"),
                served_fp64=False, max_active=16, pack_dim=PACK_DIM):
    """Impurity-solve requests (three-orbital Kanamori, N_s uniform in 10..16,
    sector ((N+1)/2, N/2), k lowest states and G(i w_n) of orbital 0 spin up
    from them, Boltzmann weights at beta = 40, 1024 Matsubara points, CF depth
    100) through the request server, against the same library's plain FP64
    path solving them one at a time (default kernels, the same thick-restart
    solver and tolerance, no server, no concurrency).  The plain path's Poisson
    latencies are those of a first-come-first-served queue over its measured
    service times at the same arrival times."""
    import workloads as W
    beta, nw, depth = 40.0, 1024, 100
    stream = W.serving_stream(n_req, seed=0, rate=1.0, ns_range=(10, 16))
    models = [W.kanamori(r["n_s"], seed=r["model_seed"]) for r in stream]
    golden, pts = serve_golden()
    m_b = tr_basis(k)
    # plain FP64, one request at a time
    service, base = [], {}
    t_all = time.perf_counter()
    for q, (r, m) in enumerate(zip(stream, models)):
        t0 = time.perf_counter()
        sec = ed.ed_sector_create(ctx, m, r["n_up"], r["n_dn"], "fp64")
        dim = ed.ed_sector_get_info(sec).dim
        kk = min(k, dim)
        vecs = torch.empty(kk * dim, dtype=torch.float64, device="cuda")
        ev, info, st = ed.ed_lanczos_tr(sec, k=kk, tol=tol, max_basis=min(m_b, dim), keep=0, max_iter=3000,
                                        check_every=4, evecs=vecs, allow_not_converged=True)
        states = [(r["n_up"], r["n_dn"], float(ev[j]), vecs[j * dim:(j + 1) * dim]) for j in range(kk)]
        G = ed.ed_greens_cf(ctx, m, "fp64", states, beta, nw, orbital=m.orb0, spin=0, depth=depth)
        torch.cuda.synchronize()
        ed.ed_sector_destroy(sec)
        del vecs, states
        service.append(time.perf_counter() - t0)
        base[q] = {"E": [float(e) for e in ev], "G": G, "status": st, "iters": int(info.iters)}
    base_total = time.perf_counter() - t_all
    base_rate = n_req / base_total
    rate = 0.8 * base_rate                      # open-loop arrivals at 0.8x plain capacity
    arrivals = [r["t_arrive"] / rate for r in stream]
    lat_sat = fifo_latencies_ms(service, [0.0] * n_req)
    lat_poi = fifo_latencies_ms(service, arrivals)
    out = {"requests": n_req, "k": k, "tol": tol, "cf_depth": depth, "n_w": nw, "beta": beta,
           "thick_restart_basis": m_b, "pack_dim": pack_dim,
           "workload": f"{n_req} requests, three-orbital Kanamori N_s~U{{10..16}}, sector ((N+1)/2, N/2), "
                       f"k={k} lowest + G(i w_n) from them",
           "plain_fp64_one_at_a_time": {
               "solves_per_s": base_rate, "seconds": base_total,
               "saturation": {"p50_ms": float(np.percentile(lat_sat, 50)), "p99_ms": float(np.percentile(lat_sat, 99))},
               "poisson": {"p50_ms": float(np.percentile(lat_poi, 50)), "p99_ms": float(np.percentile(lat_poi, 99)),
                           "arrival_rate_per_s": rate},
               "not_converged": sum(1 for v in base.values() if v["status"] != 0),
               "mean_iters": float(np.mean([v["iters"] for v in base.values()])),
               "max_iters": max(v["iters"] for v in base.values()),
               **oracle_errors(base, golden, pts, k, stream)}}
    budget = 200 * 1024 ** 3
    for prec in list(precs) + (["fp64"] if served_fp64 else []):
        for mode in modes:
            srv = ed.ed_server_create(ctx, hbm_budget=budget, max_active=max_active, prec=prec, tol=tol,
                                      max_iter=3000, cf_depth=depth, n_w=nw, beta=beta, pack_dim=pack_dim)
            arr = [0.0] * n_req if mode == "saturation" else arrivals
            tickets, results = [None] * n_req, {}
            t0 = time.perf_counter()
            i = 0
            while len(results) < n_req:
                now = time.perf_counter() - t0
                while i < n_req and arr[i] <= now:
                    tickets[i] = ed.ed_submit(srv, models[i], stream[i]["n_up"], stream[i]["n_dn"], k=k)
                    i += 1
                for q in range(i):
                    if q in results:
                        continue
                    done, res, G = ed.ed_poll(srv, tickets[q])
                    if done:
                        results[q] = {"status": res.status, "E": [res.E[j] for j in range(res.n_E)], "G": G,
                                      "lat": res.latency_ms, "iters": res.iters,
                                      "error": ed.last_error() if res.status != 0 else None}
                time.sleep(0.0005)
            el = time.perf_counter() - t0
            stats = ed.ed_server_get_stats(srv)
            ed.ed_server_destroy(srv)
            lat = [results[q]["lat"] for q in range(n_req)]
            e_vs_plain = max(abs(results[q]["E"][0] - base[q]["E"][0]) / abs(base[q]["E"][0]) for q in range(n_req))
            out[f"served_{prec}_{mode}"] = {
                "solves_per_s": n_req / el, "seconds": el, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "failed": stats.failed,
                "server_stats_ms": {"latency_p50": stats.latency_p50_ms, "latency_p99": stats.latency_p99_ms,
                                    "queue_p50": stats.queue_p50_ms, "queue_p99": stats.queue_p99_ms},
                "not_converged": sum(1 for q in results if results[q]["status"] == ed.ED_ERR_NOT_CONVERGED),
                "errors": sorted({f"{stream[q]['n_s']}: {results[q]['status']} {results[q]['error']}"
                                  for q in results if results[q]["status"] != 0})[:8],
                "max_iters": max(results[q]["iters"] for q in results),
                "mean_iters": float(np.mean([results[q]["iters"] for q in results])),
                "max_active_seen": stats.max_active_seen, "arrival_rate_per_s": None if mode == "saturation" else rate,
                "max_rel_E0_diff_vs_plain_fp64": e_vs_plain, **oracle_errors(results, golden, pts, k, stream)}
    if "served_fp32_saturation" in out:
        out["speedup_served_fp32_vs_plain_fp64"] = out["served_fp32_saturation"]["solves_per_s"] / base_rate
    out["small_requests"] = small_requests_bench(ed, ctx, k=k, tol=tol, prec=precs[0])
    return out


def run_serve(a):
    """The request stream of the serving configuration (N_s 10..16, k = 4 lowest
    states + G per request) through the request server in every vector format,
    saturation and Poisson arrivals, against the plain FP64 path one at a time."""
    import torch
    import paper_1004_3354_gb300 as ed
    if not os.path.exists(ed.LIB_PATH):
        from paper_1004_3354_gb300 import _build
        _build.build()
    torch.cuda.set_device(0)
    ctx = ed.ed_ctx_create(0)
    r = serve_bench(ed, ctx, torch, n_req=a.requests, k=4, tol=a.serve_tol, precs=("fp32", "df64"),
                    served_fp64=True)
    ed.ed_ctx_destroy(ctx)
    out = {"metric": "impurity solves/s served (N_s 10..16, 4 lowest states + G(i w_n))", "unit": "solves/s",
           "higher_is_better": True, "n_gpus": 1, "data": "synthetic (seeded random baths, Poisson arrivals)",
           "config": {"workload": r["workload"], "tol": a.serve_tol}, **r}
    out["value"] = r["served_fp32_saturation"]["solves_per_s"]
    print(json.dumps(out), flush=True)


def run_solve15(a):
    """The N_s=15 (7,8) sector: ground state (three-vector Lanczos), the
    continued-fraction G(i w_n) on 1024 Matsubara points at beta = 40 and the
    spectral function A(w) on 2001 real frequencies, in FP64, DF64 and FP32
    vectors; the stored-CSR H*v (FP64) beside the matrix-free one."""
    import torch
    import paper_1004_3354_gb300 as ed
    import workloads as W
    if not os.path.exists(ed.LIB_PATH):
        from paper_1004_3354_gb300 import _build
        _build.build()
    torch.cuda.set_device(0)
    m = W.kanamori(NS, seed=SEED)
    dim = W.sector_dim(NS, NUP, NDN)
    ctx = ed.ed_ctx_create(0)
    out = {"metric": "N_s=15 ground state + G(i w_n): time and error per vector format", "n_gpus": 1,
           "data": "synthetic (seeded random bath)", "config": workload_config("fp64", dim), "results": {}}
    ref_E, ref_G, ref_A = None, None, None
    for prec in ("fp64", "df64", "fp32"):
        p = ed.PREC_NAMES[prec]
        sec = ed.ed_sector_create(ctx, m, NUP, NDN, prec)
        psi = torch.empty(dim * ed.elems_per_value(p), dtype=ed.torch_dtype(p), device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, info, st = ed.ed_lanczos(sec, k=1, tol=1e-10 if prec != "fp32" else 1e-7, max_iter=500, reorth=False,
                                     evecs=psi, allow_not_converged=True)
        t1 = time.perf_counter()
        G = ed.ed_greens_cf(ctx, m, prec, [(NUP, NDN, float(ev[0]), psi)], 40.0, 1024, orbital=m.orb0, spin=0,
                            depth=150)
        t2 = time.perf_counter()
        # spectral function on the real axis: A(w) = -Im G(w + i 0.05) / pi, 2001 points in [-8, 8]
        zr = np.linspace(-8.0, 8.0, 2001) + 0.05j
        Gr = ed.ed_greens_cf_z(ctx, m, prec, [(NUP, NDN, float(ev[0]), psi)], zr, 40.0, orbital=m.orb0, spin=0,
                               depth=150)
        t3 = time.perf_counter()
        A = -Gr.imag / np.pi
        ed.ed_sector_destroy(sec)
        del psi
        r = {"E0": float(ev[0]), "lanczos_steps": info.iters, "ground_state_s": t1 - t0,
             "apply_ms_total": info.apply_ms, "greens_s": t2 - t1, "spectral_real_axis_s": t3 - t2,
             "spectral_weight_in_window": float(np.trapezoid(A, zr.real) if hasattr(np, "trapezoid")
                                                else np.trapz(A, zr.real)),
             "status": st}
        if prec == "fp64":
            ref_E, ref_G, ref_A = float(ev[0]), G, A
        else:
            r["rel_E0_err_vs_fp64"] = abs(float(ev[0]) - ref_E) / abs(ref_E)
            r["max_abs_G_err_vs_fp64"] = float(np.max(np.abs(G - ref_G)))
            r["max_abs_A_err_vs_fp64"] = float(np.max(np.abs(A - ref_A)))
        out["results"][prec] = r
    # set-up (the T_setup of Table 1): sector tables, fast row-kernel tables, stored CSR
    setup = {}
    for ns, nu, nd in ((15, 7, 8), (16, 8, 8)):
        mm = W.kanamori(ns, seed=SEED)
        for label, flags in (("tables", ed.ED_SECTOR_GENERIC), ("tables+fast", 0)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sx = ed.ed_sector_create(ctx, mm, nu, nd, "df64", flags)
            torch.cuda.synchronize()
            setup[f"ns{ns}_{label}_s"] = time.perf_counter() - t0
            ed.ed_sector_destroy(sx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sec = ed.ed_sector_create(ctx, m, NUP, NDN, "fp64", ed.ED_SECTOR_CSR)
    torch.cuda.synchronize()
    setup["ns15_tables+fast+csr_s"] = time.perf_counter() - t0
    out["setup"] = setup
    # stored CSR vs matrix-free, FP64
    info = ed.ed_sector_get_info(sec)
    x = torch.from_numpy(W.random_vector(dim, seed=1)).cuda()
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    for f in (ed.ed_apply_h_csr, ed.ed_apply_h):
        f(sec, x, y1)
    torch.cuda.synchronize()
    res = {}
    for name, f, y in (("csr", ed.ed_apply_h_csr, y1), ("matrix_free", ed.ed_apply_h, y2)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            f(sec, x, y)
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / 10
    csr_bytes = info.csr_nnz * 12 + (dim + 1) * 8 + 2 * dim * 8
    out["csr_vs_matrix_free_fp64"] = {
        "csr_nnz": info.csr_nnz, "csr_ms": res["csr"], "matrix_free_ms": res["matrix_free"],
        "csr_GB_per_s_of_its_bytes": csr_bytes / (res["csr"] * 1e-3) / 1e9,
        "csr_bytes_per_apply": csr_bytes, "max_abs_diff": float((y1 - y2).abs().max())}
    ed.ed_sector_destroy(sec)
    ed.ed_ctx_destroy(ctx)
    print(json.dumps(out), flush=True)


def dmft_loop(ed, ctx, torch, n_s, U=2.0, t=0.5, beta=40.0, n_w=512, n_fit=64, n_iter=20, prec="df64",
              tol=1e-10, conv=1e-5, n_k=256, neighbours=True, depth=150, log=None):
    """ED/DMFT for the one-band Hubbard model on the square lattice at half
    filling (Sec. 3.2: U = 2, t = 0.5): each iteration builds the AIM of the
    current bath, finds the ground state of the half-filled sector (and of its
    four neighbours, weighted by Boltzmann factors), forms G(i w_n) by
    continued fractions and updates the bath with ed_dmft_update.  Stops when
    G changes by less than `conv` on every frequency.  Every step runs in the
    library; this function only passes data between its calls."""
    import workloads as W
    mu = U / 2.0
    eps_d = -mu
    e, w = W.square_lattice_energies(t, n_k)
    eps, V = W.dmft_initial_bath(n_s - 1, half_width=2 * t, v=0.3)
    half = n_s // 2
    sectors = [(half, half)]
    if neighbours:
        sectors += [(half + 1, half), (half, half + 1), (half - 1, half), (half, half - 1)]
    G_prev, hist = None, []
    p = ed.PREC_NAMES[prec]
    for it in range(n_iter):
        t0 = time.perf_counter()
        m = W.aim_bath(eps_d, U, eps, V)
        states = []
        for nu, nd in sectors:
            sec = ed.ed_sector_create(ctx, m, nu, nd, prec)
            dim = ed.ed_sector_get_info(sec).dim
            psi = torch.empty(dim * ed.elems_per_value(p), dtype=ed.torch_dtype(p), device="cuda")
            ev, info, st = ed.ed_lanczos(sec, k=1, tol=tol, max_iter=600, reorth=False, evecs=psi,
                                         allow_not_converged=True)
            states.append((nu, nd, float(ev[0]), psi))
            ed.ed_sector_destroy(sec)
        t1 = time.perf_counter()
        G = ed.ed_greens_cf(ctx, m, prec, states, beta, n_w, orbital=m.orb0, spin=0, depth=depth)
        t2 = time.perf_counter()
        eps, V, c2, sig, gl, dn = ed.ed_dmft_update(ctx, G, beta, eps_d, mu, eps, V, e, w, n_fit)
        t3 = time.perf_counter()
        dG = None if G_prev is None else float(np.max(np.abs(G - G_prev)))
        E = [s_[2] for s_ in states]
        rec = {"iter": it, "dG": dG, "chi2": c2, "E0": min(E), "ground_sector": list(sectors[int(np.argmin(E))]),
               "solve_s": t1 - t0, "greens_s": t2 - t1, "update_s": t3 - t2, "total_s": t3 - t0}
        hist.append(rec)
        if log:
            log(rec)
        G_prev = G
        del states
        if dG is not None and dG < conv:
            break
    wn = np.pi / beta
    Z = 1.0 / (1.0 - sig[0].imag / wn)  # quasiparticle weight estimate from the lowest Matsubara point
    return {"history": hist, "G": G, "Sigma": sig, "G_loc": gl, "eps": eps, "V": V, "Z": Z,
            "converged": bool(hist[-1]["dG"] is not None and hist[-1]["dG"] < conv)}


def run_dmft(a):
    """ED/DMFT of the one-band Hubbard model on the square lattice at half
    filling, U = 2, t = 0.5 (Sec. 3.2), beta = 40: the N_s = 8 loop to
    self-consistency, and the time of one ED/DMFT iteration at N_s = 16 (the
    unit of the paper's Table 1, there 382-602 s on 256-512 CPU cores)."""
    import torch
    import paper_1004_3354_gb300 as ed
    if not os.path.exists(ed.LIB_PATH):
        from paper_1004_3354_gb300 import _build
        _build.build()
    torch.cuda.set_device(0)
    ctx = ed.ed_ctx_create(0)
    out = {"metric": "ED/DMFT: iterations to self-consistency (N_s=8) and seconds per iteration (N_s=16)",
           "n_gpus": 1, "data": "square-lattice Hubbard model, U=2, t=0.5, beta=40, half filling",
           "vector_format": "df64", "results": {}}
    r8 = dmft_loop(ed, ctx, torch, 8, n_iter=40)
    out["results"]["ns8_loop"] = {
        "iterations": len(r8["history"]), "converged": r8["converged"], "final_dG": r8["history"][-1]["dG"],
        "final_chi2": r8["history"][-1]["chi2"], "Z": r8["Z"], "seconds_per_iteration":
            float(np.mean([h["total_s"] for h in r8["history"]])),
        "max_abs_re_G": float(np.max(np.abs(r8["G"].real))), "bath_eps": r8["eps"].tolist(),
        "bath_V": r8["V"].tolist()}
    r16 = dmft_loop(ed, ctx, torch, 16, n_iter=2)
    h = r16["history"]
    out["results"]["ns16_iteration"] = {
        "iterations_run": len(h), "seconds": [x["total_s"] for x in h],
        "solve_s": [x["solve_s"] for x in h], "greens_s": [x["greens_s"] for x in h],
        "update_s": [x["update_s"] for x in h], "E0": [x["E0"] for x in h],
        "sectors": "(8,8) and its four neighbours, ground state each",
        "paper_context": "Table 1: one iteration at N_s=16 took 602 s on 256 and 382 s on 512 CPU cores"}
    ed.ed_ctx_destroy(ctx)
    print(json.dumps(out), flush=True)


def run_lowest8(a):
    """Eight lowest states (k = 8, DF64 vectors, tol 1e-10): the N_s=15 (7,8)
    sector by Lanczos with a full CGS2 basis and by thick-restart Lanczos with a
    40-vector basis; the N_s=16 (8,8) sector (dim 165,636,900, 1.3 GB per
    vector) by thick restart only, whose bounded basis fits in HBM where a full
    basis of a few hundred vectors would not."""
    import torch
    import paper_1004_3354_gb300 as ed
    import workloads as W
    if not os.path.exists(ed.LIB_PATH):
        from paper_1004_3354_gb300 import _build
        _build.build()
    torch.cuda.set_device(0)
    ctx = ed.ed_ctx_create(0)
    out = {"metric": "8 lowest states: time, H*v products and device memory, full basis vs thick restart",
           "n_gpus": 1, "data": "synthetic (seeded random bath)", "vector_format": "df64", "results": {}}
    runs = [(15, 7, 8, "full_basis"), (15, 7, 8, "thick_restart"), (16, 8, 8, "thick_restart")]
    ref = {}
    for ns, nu, nd, how in runs:
        m = W.kanamori(ns, seed=SEED)
        sec = ed.ed_sector_create(ctx, m, nu, nd, "df64")
        dim = W.sector_dim(ns, nu, nd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if how == "full_basis":
            # the full basis is allocated for max_iter + 1 vectors (plus the work vector)
            ev, info, st = ed.ed_lanczos(sec, k=8, tol=1e-10, max_iter=320, check_every=10,
                                         allow_not_converged=True)
            r = {"iters": info.iters, "basis_bytes": (320 + 2) * dim * 8,
                 "basis_bytes_used": (info.iters + 2) * dim * 8}
        else:
            ev, info, st = ed.ed_lanczos_tr(sec, k=8, tol=1e-10, max_basis=40, keep=20, max_iter=3000,
                                            check_every=5, allow_not_converged=True)
            r = {"iters": info.iters, "restarts": info.restarts, "basis_bytes": info.basis_bytes}
        el = time.perf_counter() - t0
        r.update({"n_s": ns, "sector": [nu, nd], "dim": dim, "seconds": el, "apply_ms_total": info.apply_ms,
                  "status": st, "n_converged": info.n_converged, "evals": [float(v) for v in ev],
                  "max_residual": float(max(info.residual[:8]))})
        if ns in ref:
            r["max_abs_eval_diff_vs_full_basis"] = float(np.max(np.abs(np.array(ev) - ref[ns])))
        else:
            ref[ns] = np.array(ev)
        out["results"][f"ns{ns}_{how}"] = r
        ed.ed_sector_destroy(sec)
    ed.ed_ctx_destroy(ctx)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "sectors12":
        run_sectors12(a)
    elif a.workload == "serve":
        run_serve(a)
    elif a.workload == "solve15":
        run_solve15(a)
    elif a.workload == "lowest8":
        run_lowest8(a)
    elif a.workload == "dmft":
        run_dmft(a)
    else:
        run_ours(a)
