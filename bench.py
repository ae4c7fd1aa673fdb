"""Benchmark: thick-restart block Lanczos steps on the 20-m-state 5+5 M-scheme
space (D = 18,600,516), block size q = 32, mixed precision (FP32 vectors
and on-the-fly block product, FP64 projection coefficients, Cholesky QR and
Rayleigh-Ritz), basis of up to 1024 vectors.

One step = one block iteration of the solver: W = H V_k (matrix elements
generated on the fly), full reorthogonalisation against the stored basis
(selective: a pass against the last two blocks, one full classical
Gram-Schmidt pass, a second one when the DGKS norm test asks for it),
Cholesky QR twice, Rayleigh-Ritz on the
projected matrix, and a thick restart when the basis is full.  The
Hamiltonian's tables are built once before timing.

metric: block H.V throughput, GNZ*q/s = structural nonzeros of H * q per
second of step time (nonzeros counted before cancellation: pairs of basis
states linked by any M-allowed term).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank solves its own independent replica
(replicas only; no data-path collective); value = all ranks' work / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "s20_5p5n"
METRIC = "block H·V GNZ·q/s"
UNIT = "GNZ*q/s"


def popcount32(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.uint32)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(x).astype(np.int64)
    x = x - ((x >> 1) & 0x55555555)
    x = (x & 0x33333333) + ((x >> 2) & 0x33333333)
    return ((((x + (x >> 4)) & 0x0F0F0F0F) * 0x01010101) & 0xFFFFFFFF) >> 24


def slab_rows(bitsA, mA, mB, twoM) -> int:
    """R = sum over target A determinants p' of sum over the distinct source
    A determinants p feeding it (like-particle terms: same 2M, at most two
    particles moved; one-body jumps of the factorised cross term: one
    particle moved, any 2M) of N_B(2M - 2M_p): the neutron-slab rows one
    apply must read in the factorised slab model."""
    nbB = {}
    for m in mB:
        nbB[int(m)] = nbB.get(int(m), 0) + 1
    NBp = np.array([nbB.get(twoM - int(m), 0) for m in mA], dtype=np.int64)
    R = 0
    for i in range(len(bitsA)):
        if NBp[i] == 0:
            continue
        pc = popcount32(bitsA ^ bitsA[i])
        src = (pc <= 2) | ((pc <= 4) & (mA == mA[i]))
        R += int(NBp[src].sum())
    return R


def structural_nnz(bitsA, mA, bitsB, mB, blocks) -> int:
    """Pairs (i, j) of basis states linked by an M-allowed term of H: the
    A and B parts together move at most two particles, total 2M equal.
    Counted per (A pair, B pair) class with the block sizes."""
    # For each A determinant p and each A source p (any 2M), the number of
    # moved particles dA; likewise for B.  A pair of product states is
    # linked iff dA + dB <= 2 and both lie in the basis.
    from collections import defaultdict
    idxB = defaultdict(list)
    for j, m in enumerate(mB):
        idxB[int(m)].append(j)
    # count B pairs by (M_B target, M_B source, dB)
    cntB = defaultdict(int)
    for mt, js in idxB.items():
        bt = bitsB[js]
        for ms, ks in idxB.items():
            bs = bitsB[ks]
            for x in bt:
                pc = popcount32(bs ^ x) // 2
                for d in (0, 1, 2):
                    c = int(np.count_nonzero(pc == d))
                    if c:
                        cntB[(mt, ms, d)] += c
    twoM = int(blocks[0][0] + blocks[0][1])
    total = 0
    mA_set = sorted(set(int(m) for m in mA))
    idxA = {m: np.nonzero(mA == m)[0] for m in mA_set}
    for mt in mA_set:
        at = bitsA[idxA[mt]]
        for ms in mA_set:
            as_ = bitsA[idxA[ms]]
            for x in at:
                pc = popcount32(as_ ^ x) // 2
                for d in (0, 1, 2):
                    c = int(np.count_nonzero(pc == d))
                    if not c:
                        continue
                    for dB in range(0, 3 - d):
                        total += c * cntB.get((twoM - mt, twoM - ms, dB), 0)
    return total


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def product_kernel_name(shape, q):
    """The kernel(s) of one block product for a launch shape (kernel, rows per
    work item, blocks per SM) at FP32 rows of q values: the split product is
    two launches, the like-particle grouped kernel then the cross-term
    kernel."""
    kern, rows, bps = shape
    grouped = "apply_grouped_kernel<float, %d, %d>" % {8: (2, 1), 16: (4, 1), 32: (8, 1)}.get(q, (4, 4))
    if kern == 5:
        return "%s + apply_pn_tma_kernel" % grouped
    if kern in (3, 4):
        v = (4, 4, 512, 2) if kern == 4 else ((8, 4, 512, 1) if bps == 1 else (8, 2, 384, 2))
        return "%s + apply_pn_kernel<%d, %d, %d, %d>" % ((grouped,) + v)
    if kern == 2:
        return "apply_grouped_kernel<float, %d, 2>" % {8: 1, 16: 2, 32: 4}.get(q, 4)
    if kern == 1:
        return "apply_fast_kernel<%d, %d, false>" % ({8: 2, 16: 4}.get(q, 8), bps)
    return grouped


def ncu_traffic(kernel, rows_per_item, path=os.path.join(ROOT, "profiles", "apply_traffic.json")):
    """(DRAM bytes per apply launch, kernel name) from a committed ncu summary.
    The bytes are None unless the summary was taken on the same kernel, on its
    source file as it is now (its SHA-256 is stored beside the figure) and
    with the same launch shape (neutron rows per work item)."""
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None, None
    if "apply_pn" in kernel:
        names = ["apply_grouped.cu", "apply_pn.cu"]
    else:
        names = ["apply_fast.cu" if kernel.startswith("apply_fast") else "apply_grouped.cu"]
    shas = {}
    for name in names:
        try:
            shas[name] = hashlib.sha256(open(os.path.join(ROOT, "paper_1902_02064_gb300", "csrc", name),
                                             "rb").read()).hexdigest()
        except OSError:
            shas[name] = None
    stored = d.get("source_sha256")
    if not isinstance(stored, dict):
        stored = {names[0]: stored}
    if d.get("kernel") != kernel or stored != shas or d.get("rows_per_item", 128) != rows_per_item:
        return None, d.get("kernel")
    return d.get("dram_bytes_per_launch_full_size"), d.get("kernel")


# ----------------------------------------------------------------------------
# oracle timing (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------

class _RowGen:
    """Rows of a seeded uniform(-1, 1) D x q block, generated on demand."""

    def __init__(self, q, seed):
        self.q, self.seed = q, seed

    def __getitem__(self, i):
        idx = np.arange(self.q, dtype=np.uint64) + np.uint64(int(i) * self.q) \
            + np.uint64((self.seed & 0xFFFFFFFF) << 32)
        h = synth.splitmix64(idx)
        return ((h >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))) * 2.0 - 1.0


class OracleSample:
    """The oracle's one-row-at-a-time H.V on a sample of rows of the workload."""

    def __init__(self, name, q):
        from oracle import hamiltonian as oh
        self.oh = oh
        w, sa, sb, inter = synth.workload(name)
        self.L = oh.LazyIndex(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
        self.T = oh.TermTables(inter)
        self.V = _RowGen(q, w.seed)
        self.q = q
        self.rng = np.random.default_rng(1234)

    def run(self, seconds):
        """Rows until `seconds` pass; returns (structural nnz * q, elapsed)."""
        t0 = time.perf_counter()
        work = 0
        rows = 0
        while time.perf_counter() - t0 < seconds:
            r = int(self.rng.integers(0, self.L.dim))
            SA, SB = self.L.state(r)
            targets = set()
            acc = np.zeros(self.q)
            for v, A2, B2 in self.oh.column_terms(SA, SB, self.T):
                j = self.L.index(A2, B2)
                acc += v * self.V[j]
                targets.add(j)
            work += len(targets) * self.q
            rows += 1
        return work, time.perf_counter() - t0, rows


def cpu_baseline(name, q, seconds):
    o = OracleSample(name, q)
    work, el, rows = o.run(seconds)
    return {"value": work / el / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d random rows of H.V (q=%d) of the %s workload by the FP64 oracle's "
                      "one-row-at-a-time operator application, %.1f s" % (rows, q, name, el)}


def _spmm_rows(args):
    """Worker: its row block of the oracle's CSR H times V, reps times;
    returns its own elapsed seconds."""
    Hb, V, reps = args
    Hb @ V
    t0 = time.perf_counter()
    for _ in range(reps):
        Hb @ V
    return time.perf_counter() - t0


def _oracle_ttn_child(name, cap_q):
    """Child process (one BLAS thread): the oracle's Lanczos (Alg. 1, full
    reorthogonalisation twice) to the workload's nev at 1e-10 ||H||."""
    from oracle import basis as ob
    from oracle import hamiltonian as oh
    from oracle import lanczos as ol
    w, sa, sb, inter = synth.workload(name)
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    H = oh.assemble(B, inter)
    ev = np.linalg.eigvalsh(H.toarray()) if B.dim <= 4000 else None
    normH = max(abs(ev[0]), abs(ev[-1])) if ev is not None else json.load(
        open(os.path.join(ROOT, "tests", "golden", "eigs_%s.json" % name)))["normH"]
    v1 = synth.random_block(B.dim, 1, 5)[:, 0]
    t0 = time.perf_counter()
    theta, X, res, it = ol.lanczos(lambda x: H @ x, B.dim, w.nev, 1e-10, normH, v1, max_iter=min(B.dim, 3000))
    cap_q.put({"seconds": time.perf_counter() - t0, "iterations": it, "nev": w.nev, "dim": B.dim})


def cpu_oracle_extra(cap_seconds=120.0):
    """The oracle's CSR product H V on the 28,503-dim workload (q = 8) on one
    core and with row blocks over all host cores, and the oracle's time to
    nev eigenpairs (Lanczos, one BLAS thread) on the 640- and 28,503-dim
    workloads, each capped at cap_seconds."""
    import multiprocessing as mp
    from oracle import basis as ob
    from oracle import hamiltonian as oh
    name = "s12_4p4n"
    w, sa, sb, inter = synth.workload(name)
    t0 = time.perf_counter()
    B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
    H = oh.assemble(B, inter).tocsr()
    t_asm = time.perf_counter() - t0
    V = synth.random_block(B.dim, w.q, 1)
    reps = 20
    t1 = _spmm_rows((H, V, reps)) / reps
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    # row blocks of about equal nonzeros
    cuts = np.searchsorted(H.indptr, np.linspace(0, H.nnz, cores + 1)).tolist()
    cuts[0], cuts[-1] = 0, B.dim
    blocks = [H[cuts[i]:cuts[i + 1]] for i in range(cores) if cuts[i + 1] > cuts[i]]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(blocks)) as pool:
        tall = max(pool.map(_spmm_rows, [(b, V, reps) for b in blocks])) / reps
    out = {"csr_spmm": {"workload": name, "dim": B.dim, "nnz": int(H.nnz), "q": w.q,
                        "assembly_s": t_asm,
                        "one_core": {"gnzq_per_s": H.nnz * w.q / t1 / 1e9, "ms": t1 * 1e3},
                        "all_cores": {"cores": len(blocks), "gnzq_per_s": H.nnz * w.q / tall / 1e9,
                                      "ms": tall * 1e3, "sample": "row blocks of equal nonzeros, one per "
                                                                  "spawned process, slowest block's time"}}}
    ttn = {}
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        for nm in ("s12_2p2n", "s12_4p4n"):
            q = ctx.Queue()
            pr = ctx.Process(target=_oracle_ttn_child, args=(nm, q))
            t0 = time.perf_counter()
            pr.start()
            pr.join(cap_seconds)
            if pr.is_alive():
                pr.terminate()
                pr.join()
                ttn[nm] = {"finished": False, "cap_s": cap_seconds}
            else:
                r = q.get() if not q.empty() else {}
                r.update({"finished": bool(r), "wall_s_with_assembly": time.perf_counter() - t0})
                ttn[nm] = r
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    out["time_to_nev"] = {"method": "oracle Lanczos (Alg. 1, full reorthogonalisation twice), FP64, tol 1e-10 "
                                    "||H||, one BLAS thread", "cores": 1, **ttn}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = synth.WORKLOADS[WORKLOAD]
    o = OracleSample(WORKLOAD, w.q)
    per_step = 3.0
    for _ in range(args.warmup):
        o.run(per_step / 3)
    works, times, rows = 0, 0.0, 0
    for _ in range(args.steps):
        wk, el, rw = o.run(per_step)
        works += wk
        times += el
        rows += rw
    value = works / times / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": times / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "dim": 18600516, "q": w.q, "nev": w.nev,
                                        "max_basis": w.max_basis, "precision": "FP64 oracle, one row at a time",
                                        "parallelism": "one host core"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d random rows of H.V per %d steps, FP64 oracle, one core" % (rows, args.steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def max_over_ranks(x, dist=None, device="cpu"):
    """The largest x over all ranks (a replicas job takes as long as its
    slowest replica); x itself on a single process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds, world):
    """Whole-job rate of `world` replicas that each processed
    units_per_rank units, the job taking `seconds` (the slowest rank)."""
    return world * units_per_rank / seconds


def run_ours(args, rank, world):
    import torch
    import paper_1902_02064_gb300 as trbl

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))

    def barrier():
        if dist is not None:
            dist.barrier()

    w, sa, sb, inter = synth.workload(args.workload)
    q = args.q or w.q
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    D = tb.dim
    bitsA, mA, bitsB, mB, blocks = tb.export()
    R = slab_rows(bitsA, mA, mB, w.twoM)
    nnz = structural_nnz(bitsA, mA, bitsB, mB, blocks)
    b_slab = 4 * q * (R + D)  # bytes per apply, FP32

    stream = torch.cuda.current_stream()
    # launch shape of the product: the autotuner times every (kernel, rows per
    # work item, blocks per SM) shape and keeps the fastest (results do not change)
    tune_ms, tune_rows = trbl.apply_autotune(th, q, trbl.TRBL_F32)
    shape = trbl.apply_get_shape(th)
    torch.cuda.empty_cache()

    def steady_solver():
        # a solver in its steady state: taken through its first thick restart
        # (basis filled to max_basis, Ritz vectors kept, refilled) before the
        # warm-up steps, so that the timed steps see the basis fills and the
        # restarts of a long solve; Rayleigh-Ritz at the solver's own adaptive
        # cadence, as in a solve
        s_ = trbl.Solver(th, w.nev, q, w.max_basis, w.tol, precision=trbl.TRBL_PREC_MIXED, seed=w.seed,
                         check_every=0, stream=stream)
        while s_.stats()["restarts"] < 1:
            s_.step()
        return s_

    sv = steady_solver()
    fill0 = sv.fill()
    for _ in range(args.warmup):
        sv.step()
    torch.cuda.synchronize()
    barrier()
    st0 = sv.stats()
    fill1 = sv.fill()
    l0 = trbl.trbl_kernel_launches()
    clocks = ClockSampler(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    # the timed steps are the profiler's range (ncu --profile-from-start off
    # captures exactly them; without a profiler these calls do nothing)
    torch.cuda.profiler.start()
    e0.record(stream)
    for _ in range(args.steps):
        sv.step()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    barrier()
    clk = clocks.stop()
    launches = trbl.trbl_kernel_launches() - l0
    st1 = sv.stats()
    fill2 = sv.fill()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    ms_step = ms / args.steps
    value = job_throughput(nnz * q * args.steps, ms * 1e-3, world) / 1e9
    ms_apply = (st1["ms_apply"] - st0["ms_apply"]) / args.steps
    achieved = b_slab / (ms_apply * 1e-3) / 1e9
    kname = product_kernel_name(shape, q)
    traffic, _ = ncu_traffic(kname, tune_rows)

    # end to end: the same block steps as the device-timed region (a fresh
    # solver through the same set-up and warm-up, whose last step fills the
    # host copy of the block), with V_k supplied from and V_{k+1} returned to
    # page-locked host memory on the GPU's nearest memory node
    # (trbl_host_alloc) through the C ABI (trbl_solver_step_host)
    del sv
    torch.cuda.synchronize()
    sv = steady_solver()
    ptr, nbytes = sv.block()
    host_in = trbl.HostBuffer(nbytes, dev)
    host_out = trbl.HostBuffer(nbytes, dev)
    for _ in range(args.warmup - 1):
        sv.step()
    sv.step_host(None, host_in)
    torch.cuda.synchronize()
    barrier()
    se0 = sv.stats()
    t0 = time.perf_counter()
    copy_out_steps = []
    for k in range(args.steps):
        src, dst = (host_in, host_out) if k % 2 == 0 else (host_out, host_in)
        c0 = sv.stats()["ms_copy_out"]
        sv.step_host(src, dst)
        copy_out_steps.append(round(sv.stats()["ms_copy_out"] - c0, 2))
    torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    se1 = sv.stats()
    e2e_value = job_throughput(nnz * q * args.steps, el, world) / 1e9
    e2e_phase_ms = sum(se1[k] - se0[k] for k in ("ms_apply", "ms_orth", "ms_qr", "ms_ritz", "ms_restart"))
    copy_in_ms = (se1["ms_copy_in"] - se0["ms_copy_in"]) / args.steps
    copy_out_ms = (se1["ms_copy_out"] - se0["ms_copy_out"]) / args.steps
    copy_ms = el * 1e3 - e2e_phase_ms
    numa = host_in.numa_node
    host_in.free()
    host_out.free()

    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "dim": D, "q": q, "nev": w.nev, "max_basis": w.max_basis,
                   "precision": "mixed (FP32 vectors/apply, FP64 coefficients, CholQR2, Ritz)",
                   "reorthogonalisation": "selective (local pass, one full pass, second pass on the DGKS test)",
                   "structural_nnz": nnz,
                   "steps": "steady state: the solver is taken through its first thick restart before the "
                            "warm-up; Rayleigh-Ritz at the solver's adaptive cadence",
                   "basis_fill": {"after_first_restart": fill0, "first_timed_step": fill1, "after_timed_steps": fill2},
                   "restarts_in_timed_region": st1["restarts"] - st0["restarts"],
                   "l2": "inputs larger than L2 (basis %.1f GB, block %.2f GB)"
                         % (D * w.max_basis * 4 / 1e9, D * q * 4 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "apply": {"ms_per_launch": ms_apply, "gnzq_per_s": nnz * q / (ms_apply * 1e-3) / 1e9,
                  "share_of_step": ms_apply / ms_step,
                  "autotune": {"shapes": "(kernel, rows per item, blocks per SM): grouped 16/32/64/128 at 8; "
                                         "fast 16/32/64 at 8; fast 16/32/64 at 6; grouped with two 16-byte "
                                         "chunks per lane 16/32/64 at 8; split 64 at 2; split with four "
                                         "jumps per batch 64 at 2",
                               "ms": tune_ms, "chosen": {"kernel": ["grouped", "fast", "grouped_x2", "split",
                                                                    "split_x4"][shape[0]],
                                                         "rows_per_item": shape[1], "blocks_per_sm": shape[2]}}},
        "phases_ms_per_step": {k: (st1[k] - st0[k]) / args.steps
                               for k in ("ms_apply", "ms_orth", "ms_qr", "ms_ritz", "ms_restart")},
        "second_reorth_passes_in_timed_steps": st1["second_passes"] - st0["second_passes"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kname,
                     "algorithmic_bytes_per_launch": b_slab,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback 6800 GB/s"},
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "ms_per_step": el / args.steps * 1e3,
                "steps": "the device-timed block steps, on a fresh solver",
                "solver_phase_ms_per_step": e2e_phase_ms / args.steps,
                "host_buffers": "trbl_host_alloc (cudaHostAlloc; GPU's nearest host node %d)" % numa,
                "copy_gb_per_s": 2 * nbytes * args.steps / (copy_ms * 1e-3) / 1e9 if copy_ms > 0 else None,
                "copy_in_ms_per_step": copy_in_ms, "copy_out_ms_per_step": copy_out_ms,
                "copy_out_ms_steps": copy_out_steps,
                "ms_beyond_solver_phases_per_step": (el * 1e3 - e2e_phase_ms) / args.steps},
    }
    if rank == 0 and world == 1 and not args.no_proj:
        del sv
        sv = None
        torch.cuda.empty_cache()
        line["projections"] = projections_at(trbl, D, 640, q, peak)
    if rank == 0 and world == 1 and not args.no_ttn:
        ttn = {"s12_4p4n": time_to_nev(trbl)}
        if not args.no_ttn_large:
            # the headline solves: the 48Cr-sized space (nev 200, basis 1024):
            # mixed block q = 16, FP64 block q = 16, FP64 Lanczos q = 1; the
            # 18.6M-dim space (nev 500, basis 1024): mixed q = 32
            ttn["s20_4p4n"] = time_to_nev_large(
                trbl, "s20_4p4n", (("fp64_q16", trbl.TRBL_PREC_F64, 16), ("mixed_q16", trbl.TRBL_PREC_MIXED, 16),
                                   ("fp64_q1", trbl.TRBL_PREC_F64, 1)))
            ttn[args.workload] = time_to_nev_large(trbl, args.workload,
                                                   (("mixed_q%d" % q, trbl.TRBL_PREC_MIXED, q),), th=th)
        line["time_to_nev"] = ttn
    if rank == 0 and world == 1 and not args.no_batch:
        line["gradient_batch"] = gradient_batch(trbl)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, q, args.cpu_seconds)
        line["cpu_baseline"]["oracle_extra"] = cpu_oracle_extra()
    del sv
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def projections_at(trbl, D, m, q, peak, reps=5):
    """The solver's two dense contractions alone at the workload's size, m
    stored vectors (C = B^T W, W -= B C; FP32 data): tensor-core (tcgen05,
    split TF32) and CUDA-core forms, CUDA-event timed, with the fraction of
    the measured HBM bandwidth (bytes 4 D (m + q) and 4 D (m + 2q))."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    B = torch.rand((D, m), generator=g, device="cuda") * 2 - 1
    W = torch.rand((D, q), generator=g, device="cuda") * 2 - 1
    U = (torch.rand((m, q), generator=g, device="cuda", dtype=torch.float64) * 2 - 1) / m
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    calls = {"dot_tensor": (lambda: trbl.block_dot(B, W, tensor_cores=True), 4 * D * (m + q)),
             "dot_cuda_core": (lambda: trbl.block_dot(B, W), 4 * D * (m + q)),
             "update_tensor": (lambda: trbl.block_update(B, U, W, -1.0, 1.0, algo=trbl.TRBL_PROJ_TENSOR),
                               4 * D * (m + 2 * q)),
             "update_cuda_core": (lambda: trbl.block_update(B, U, W, -1.0, 1.0, algo=trbl.TRBL_PROJ_CUDA_CORE),
                                  4 * D * (m + 2 * q))}
    out = {"dim": D, "m": m, "q": q, "inputs": "B %.1f GB (larger than L2)" % (4 * D * m / 1e9),
           "kernels": "block_dot_tc_kernel, rowgemm_tc_kernel (tcgen05 kind::tf32, split operands)",
           "ncu": "profiles/proj_tc_D1M_m640_q32.md"}
    for name, (f, nbytes) in calls.items():
        f()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            f()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "gbs": gbs, "frac_of_hbm": gbs / peak}
    del B, W, U
    torch.cuda.empty_cache()
    return out


def time_to_nev(trbl, name="s12_4p4n"):
    """Full solves of the 12-m-state 4+4 workload (D = 28,503, nev = 100):
    mixed precision q = 8, FP64 q = 8, and plain FP64 Lanczos (q = 1), same
    GPU; eigenvalue errors against the oracle's stored eigenvalues."""
    import torch
    w, sa, sb, inter = synth.workload(name)
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "eigs_%s.json" % name)))
    ref = np.array(gold["evals"][: w.nev])
    normH = gold["normH"]
    out = {"workload": name, "dim": tb.dim, "nev": w.nev, "max_basis": w.max_basis, "normH": normH}
    runs = (("mixed_q8", trbl.TRBL_PREC_MIXED, w.q, 1e-6), ("fp64_q8", trbl.TRBL_PREC_F64, w.q, 1e-10),
            ("fp64_q1", trbl.TRBL_PREC_F64, 1, 1e-10))
    for label, prec, q, tol in runs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, rs, X, st = trbl.solve(th, w.nev, q, w.max_basis, tol, precision=prec, want_vectors=False,
                                   raise_on_noconv=False, max_iter=20000)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        out[label] = {"seconds": el, "tol_rel_normH": tol, "converged": st["converged"], "rc": st["rc"],
                      "iterations": st["iterations"], "restarts": st["restarts"],
                      "max_abs_eig_err_over_normH": float(np.abs(ev - ref).max() / normH),
                      "max_true_resid_over_normH": float(np.nanmax(rs) / normH),
                      "phase_ms": {k: st[k] for k in ("ms_apply", "ms_orth", "ms_qr", "ms_ritz", "ms_restart")}}
    return out


def time_to_nev_large(trbl, name, arms, th=None):
    """Full solves of a large workload to residual 1e-6 ||H|| (no stored
    oracle eigenvalues at this size): each arm's eigenvalues are compared
    with the first arm's, and every arm reports its true residuals (FP64
    apply).  Each timed solve follows a short untimed one (3 block steps),
    so that first-use kernel loading is not counted.  arms: (label,
    precision, q) tuples; th: the workload's Hamiltonian if already built."""
    import torch
    w, sa, sb, inter = synth.workload(name)
    if th is None:
        tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
        th = trbl.Hamiltonian.from_interaction(tb, inter)
    tune_ms, tune_rows = trbl.apply_autotune(th, w.q, trbl.TRBL_F32)
    shape = trbl.apply_get_shape(th)
    torch.cuda.empty_cache()
    out = {"workload": name, "dim": th.basis.dim, "nev": w.nev, "max_basis": w.max_basis, "tol_rel_normH": 1e-6,
           "product_shape": {"kernel": ["grouped", "fast", "grouped_x2", "split", "split_x4", "split_tma"][shape[0]], "rows_per_item": shape[1],
                             "blocks_per_sm": shape[2]}}
    first = None
    for label, prec, q in arms:
        trbl.solve(th, w.nev, q, w.max_basis, 1e-6, precision=prec, want_vectors=False, raise_on_noconv=False,
                   max_iter=3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev, rs, X, st = trbl.solve(th, w.nev, q, w.max_basis, 1e-6, precision=prec, want_vectors=False,
                                   raise_on_noconv=False, max_iter=20000)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        r = {"seconds": el, "q": q, "converged": st["converged"], "rc": st["rc"], "iterations": st["iterations"],
             "restarts": st["restarts"], "second_reorth_passes": st["second_passes"], "normH": st["normH"],
             "max_true_resid_over_normH": float(np.nanmax(rs) / st["normH"]),
             "phase_ms": {k: st[k] for k in ("ms_apply", "ms_orth", "ms_qr", "ms_ritz", "ms_restart")}}
        if first is None:
            first = ev
        else:
            r["max_abs_eig_diff_vs_first_arm_over_normH"] = float(np.abs(ev - first).max() / st["normH"])
        out[label] = r
        print(json.dumps({label: r}), file=sys.stderr, flush=True)
    return out


def gradient_batch(trbl, nset=64):
    """Gradient batch: nset parameter sets (seeds 100..) of the 12-m-state 4+4
    space (D = 28,503), the 20 lowest eigenpairs each (q = 8, basis 256, FP64)
    and the Hellmann-Feynman gradient of every level cluster, solved as one
    batch (trbl_solve_batch) and as nset single solves."""
    import torch
    sp = synth.make_space(synth.SPACE12_SHELLS)
    tb = trbl.Basis(sp, 4, sp, 4, 0)
    inters = [synth.draw_interaction(sp, sp, 100 + k) for k in range(nset)]
    hs = [trbl.Hamiltonian.from_interaction(tb, it) for it in inters]
    nev, q, mb, tol = 20, 8, 256, 1e-10
    ms, rows = trbl.apply_autotune(hs[0], q, trbl.TRBL_F64)
    # untimed warm-up of the solver and gradient paths (kernel loading), so
    # that neither timed leg pays it
    e0, r0, X0, st0 = trbl.solve(hs[0], nev, q, mb, tol)
    trbl.hf_gradient_clusters(hs[0], X0, trbl.clusters_of(e0, 1e-8 * st0["normH"]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev, rs, X, status, st = trbl.solve_batch(hs, nev, q, mb, tol, want_vectors=True, want_resid=False)
    torch.cuda.synchronize()
    t_solve_b = time.perf_counter() - t0
    euler = 0.0
    for k in range(nset):
        cls = trbl.clusters_of(ev[k], 1e-8 * st["normH"])
        for cl, g in zip(cls, trbl.hf_gradient_clusters(hs[k], X[k], cls)):
            euler = max(euler, abs(g @ inters[k].theta - ev[k][cl].sum()) / st["normH"])
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    max_diff = 0.0
    for k in range(nset):
        e1, r1, X1, st1 = trbl.solve(hs[k], nev, q, mb, tol)
        trbl.hf_gradient_clusters(hs[k], X1, trbl.clusters_of(e1, 1e-8 * st1["normH"]))
        max_diff = max(max_diff, float(np.abs(e1 - ev[k]).max()))
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    return {"sets": nset, "dim": tb.dim, "nev": nev, "q": q, "params_per_set": len(inters[0].theta),
            "autotune_ms": ms, "rows_per_item": rows,
            "batched_solve_s": t_solve_b, "batched_solve_plus_gradients_s": t_batch,
            "sequential_solves_plus_gradients_s": t_seq, "speedup": t_seq / t_batch,
            "sets_ok": int(sum(1 for x in status if x == 0)), "graph_steps": st["iterations"],
            "ms_graph_steps": st["ms_apply"], "ms_between_steps": st["ms_ritz"],
            "second_reorth_set_steps": st["second_passes"],
            "max_eig_diff_batch_vs_single_over_normH": max_diff / st["normH"],
            "max_euler_identity_error_over_normH": euler}


def run_proj_only(args):
    """Time the block projection C = B^T W and the update W -= B U alone (FP32
    data; tensor-core and CUDA-core forms) for D, m, q given as "D,m,q"."""
    import torch
    import paper_1902_02064_gb300 as trbl
    D, m, q = (int(x) for x in args.proj_only.split(","))
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    B = torch.rand((D, m), generator=g, device="cuda") * 2 - 1
    W = torch.rand((D, q), generator=g, device="cuda") * 2 - 1
    U = (torch.rand((m, q), generator=g, device="cuda", dtype=torch.float64) * 2 - 1) / m
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    calls = {"dot_tc": lambda: trbl.block_dot(B, W, tensor_cores=True),
             "dot_cc": lambda: trbl.block_dot(B, W),
             "update_tc": lambda: trbl.block_update(B, U, W, -1.0, 1.0, algo=trbl.TRBL_PROJ_TENSOR),
             "update_cc": lambda: trbl.block_update(B, U, W, -1.0, 1.0, algo=trbl.TRBL_PROJ_CUDA_CORE)}
    out = {"D": D, "m": m, "q": q}
    for name, f in calls.items():
        for _ in range(args.warmup):
            f()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            f()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        nbytes = 4 * D * (m + q) if name.startswith("dot") else 4 * D * (m + 2 * q)
        out[name] = {"ms": ms, "gbs": nbytes / (ms * 1e-3) / 1e9}
    print(json.dumps(out), flush=True)


def run_wide_only(args):
    """Time the wide tensor-core GEMM alone (the thick restart's V U and the
    Ritz vectors; Out = In U, FP32 In and Out, FP64 U) for "D,K,n": FLOP
    rate (2 D K n, three split TF32 products counted once) and bytes
    4 D (K + n) against the measured peaks."""
    import torch
    import paper_1902_02064_gb300 as trbl
    D, K, n = (int(x) for x in args.wide_only.split(","))
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    In = torch.rand((D, K), generator=g, device="cuda") * 2 - 1
    U = (torch.rand((K, n), generator=g, device="cuda", dtype=torch.float64) * 2 - 1) / K
    Out = torch.empty((D, (n + 3) // 4 * 4), device="cuda")[:, :n]
    for _ in range(args.warmup):
        trbl.block_update(In, U, Out, 1.0, 0.0, algo=trbl.TRBL_PROJ_TENSOR)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        trbl.block_update(In, U, Out, 1.0, 0.0, algo=trbl.TRBL_PROJ_TENSOR)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    peaks = measured_peaks() or {}
    tf = 2.0 * D * K * n / (ms * 1e-3) / 1e12
    gbs = 4.0 * D * (K + n) / (ms * 1e-3) / 1e9
    print(json.dumps({"D": D, "K": K, "n": n, "ms": ms, "tflops_fp32_products": tf,
                      "tf32_tflops_issued": 3 * tf, "gbs": gbs,
                      "frac_hbm": gbs / peaks["hbm_gbs"] if peaks else None}), flush=True)


def run_apply_only(args):
    """Time the block product alone on one workload (used for kernel profiles)."""
    import torch
    import paper_1902_02064_gb300 as trbl
    w, sa, sb, inter = synth.workload(args.apply_only)
    q = args.q or w.q
    tb = trbl.Basis(sa, w.nA, sb, w.nB, w.twoM)
    th = trbl.Hamiltonian.from_interaction(tb, inter)
    bitsA, mA, bitsB, mB, blocks = tb.export()
    R = slab_rows(bitsA, mA, mB, w.twoM)
    nnz = structural_nnz(bitsA, mA, bitsB, mB, blocks)
    dt = torch.float64 if args.fp64 else torch.float32
    if args.rows:
        tune_ms, tune_rows = None, args.rows
        kern = {"grouped": trbl.TRBL_APPLY_GROUPED, "fast": trbl.TRBL_APPLY_FAST,
                "grouped_x2": trbl.TRBL_APPLY_GROUPED_X2, "split": trbl.TRBL_APPLY_SPLIT,
                "split_x4": trbl.TRBL_APPLY_SPLIT_X4, "split_tma": trbl.TRBL_APPLY_SPLIT_TMA}[args.kernel]
        trbl.apply_set_shape(th, kern, args.rows, args.bps)
        trbl.apply_set_compensated(th, args.comp)
    else:
        tune_ms, tune_rows = trbl.apply_autotune(th, q, trbl.TRBL_F64 if args.fp64 else trbl.TRBL_F32)
    g = torch.Generator(device="cuda")
    g.manual_seed(w.seed)
    V = torch.rand((tb.dim, q), generator=g, device="cuda", dtype=dt) * 2 - 1
    W = torch.empty_like(V)
    for _ in range(args.warmup):
        th.apply(V, W)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        th.apply(V, W)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    b_slab = (8 if args.fp64 else 4) * q * (R + tb.dim)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    print(json.dumps({"workload": args.apply_only, "dim": tb.dim, "q": q, "dtype": str(dt),
                      "ms_per_apply": ms, "gnzq_per_s": nnz * q / (ms * 1e-3) / 1e9,
                      "structural_nnz": nnz, "slab_rows_R": R, "algorithmic_bytes": b_slab,
                      "rows_per_item": tune_rows, "autotune_ms": tune_ms, "shape": trbl.apply_get_shape(th),
                      "compensated": bool(args.comp),
                      "achieved_gbs": b_slab / (ms * 1e-3) / 1e9, "frac_of_measured_hbm": b_slab / (ms * 1e-3) / 1e9 / peak}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttn", action="store_true", help="skip the time-to-nev solves")
    ap.add_argument("--no-ttn-large", action="store_true",
                    help="skip the time-to-nev solves of the 2M- and 18.6M-dim workloads")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-set gradient batch")
    ap.add_argument("--no-proj", action="store_true", help="skip the projection kernels' own timing")
    ap.add_argument("--arms", default=None, metavar="LABEL,...",
                    help="with --ttn-large: run only these arms (fp64_q16, mixed_q16, fp64_q1, mixed_q32)")
    ap.add_argument("--ttn-large", metavar="WORKLOAD", default=None,
                    help="only: time to nev eigenpairs at 1e-6 ||H|| on a large workload (s20_4p4n: mixed, "
                         "FP64 block and FP64 q = 1 arms; s20_5p5n: mixed) and print one JSON line")
    ap.add_argument("--apply-only", default=None, help="time only W = H V on this workload")
    ap.add_argument("--wide-only", default=None, metavar="D,K,n",
                    help="time only the wide tensor-core GEMM Out = In U (restart and Ritz vectors)")
    ap.add_argument("--proj-only", default=None, metavar="D,m,q",
                    help="time only the block projection and update (FP32, both forms) at these sizes")
    ap.add_argument("--workload", default=WORKLOAD, help="workload of the solver steps (default: the 5+5 space)")
    ap.add_argument("--q", type=int, default=0)
    ap.add_argument("--rows", type=int, default=0,
                    help="--apply-only: fixed neutron rows per work item instead of the autotuner's choice")
    ap.add_argument("--kernel", default="fast", choices=["fast", "grouped", "grouped_x2", "split", "split_x4", "split_tma"],
                    help="--apply-only with --rows: the product kernel")
    ap.add_argument("--bps", type=int, default=8, choices=[1, 2, 6, 8],
                    help="--apply-only with --rows: resident blocks per SM of the fast kernel")
    ap.add_argument("--comp", action="store_true",
                    help="--apply-only with --rows: compensated row sums in the fast kernel")
    ap.add_argument("--fp64", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.apply_only:
        run_apply_only(args)
    elif args.wide_only:
        run_wide_only(args)
    elif args.proj_only:
        run_proj_only(args)
    elif args.ttn_large:
        import paper_1902_02064_gb300 as trbl
        w = synth.WORKLOADS[args.ttn_large]
        if args.ttn_large == "s20_5p5n":
            arms = (("mixed_q%d" % w.q, trbl.TRBL_PREC_MIXED, w.q),)
        else:
            arms = (("fp64_q%d" % w.q, trbl.TRBL_PREC_F64, w.q), ("mixed_q%d" % w.q, trbl.TRBL_PREC_MIXED, w.q),
                    ("fp64_q1", trbl.TRBL_PREC_F64, 1))
        if args.arms:
            keep = args.arms.split(",")
            arms = tuple(a for a in arms if a[0] in keep)
            if not arms:
                sys.exit("--arms: none of %s among this workload's arms" % keep)
        print(json.dumps({"time_to_nev": time_to_nev_large(trbl, args.ttn_large, arms)}), flush=True)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
