"""Benchmark of the share-domain iris uniqueness check on GB300.

One step = one pass of the whole hot path over one query batch: query preparation (A2),
the six share-domain ring GEMMs per resident database chunk (A3, three parties x code/mask),
lift + threshold + MSB + in-block OR (A4-A8) per chunk, the rest of the OR tree (A8) and the
copy of the bit components. Workload (default): 100,000 database rows x 32 queries x 31
rotations, 12,800-bit codes, synthetic (seeded), database shares resident on the device.

Prints one JSON line. `value` is comparisons/s of the tcgen05 path (the resident int8 limb
planes widened to fp16 in shared memory, exact, fp32 accumulators in tensor memory) with the
query shares already on the device, timed with CUDA events on the library's control stream;
`e2e` is the same through host (pinned) buffers with the copies inside the timed region, timed
by the host's clock from the first submit to the last fetched result; `int8_mix_path`,
`int8_tensor_only_path` (mma.sync s8 with and without dp4a) and `int32_path` (plain CUDA-core
ring GEMM) run the same workload, and each reports whether its bits equal the headline's. --impl reference times the
CPU oracle (the 3-party simulation of Alg. 3) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "masked-HD comparisons/s, int8-limb TC vs plain int32 path; % of INT8 peak"
UNIT = "comparisons/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-i32", action="store_true")
    ap.add_argument("--cpu-sample-rows", type=int, default=2048)
    ap.add_argument("--kernel", default=None, help="time one kernel alone: a ring-GEMM path (i8mix | i8mma | i32 | tc | tc32), "
                    "compare, overlap (Galois GEMM and comparison alone and on two streams), or fused "
                    "(the fused chunk step against the unfused one)")
    ap.add_argument("--rows", type=int, default=16384, help="database rows of the --kernel case")
    ap.add_argument("--fused-path", default="tcg", choices=["tc", "tcg"], help="sharing of --kernel fused")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--serving", action="store_true",
                    help="serving run: Poisson arrivals of 1..256-query batches at 3 rates (workload c4)")
    ap.add_argument("--requests-per-rate", type=int, default=300)
    ap.add_argument("--rates", default="0.3,0.6,0.9", help="arrival rates as fractions of the measured capacity")
    ap.add_argument("--pool", type=int, default=0, help="serving pool in query slots (0 = library default)")
    ap.add_argument("--capacity-requests", type=int, default=8)
    ap.add_argument("--persons", action="store_true",
                    help="both eyes + inner-batch matching (ipc_check_persons), the paper's deployed query shape")
    ap.add_argument("--persons-rows", type=int, default=262144, help="database rows per eye")
    ap.add_argument("--persons-batch", type=int, default=32)
    ap.add_argument("--persons-path", default="tcg", choices=["tc", "tcg", "i8mix"])
    ap.add_argument("--serving-path", default="tc", choices=["tc", "tcg"],
                    help="tc: replicated-sharing dots; tcg: Galois-ring Shamir dots")
    return ap.parse_args()


def run_compare_kernel(args, w):
    """The comparison phase (A4-A8 with the in-block OR) of one chunk alone: all query columns
    x --rows rows of random dot-product shares, timed with CUDA events. Besides the headline
    MPCLift comparison, the same shape in the other settings of Table 2 (Sec. 6.2): plain masks
    (16-bit MSB), ConstLift and NoLift (32-bit MSB without Lift)."""
    import torch

    import paper_2405_04463_gb300 as ipc
    N, rows = w.Q * w.R, args.rows
    g = torch.Generator(device="cpu").manual_seed(7)
    zc = [torch.randint(-32768, 32768, (N, rows), dtype=torch.int16, generator=g).cuda() for _ in range(3)]
    zm = [torch.randint(0, 12801, (N, rows), dtype=torch.int16, generator=g).cuda() for _ in range(3)]
    zc32 = [torch.randint(-2**31, 2**31 - 1, (N, rows), dtype=torch.int32, generator=g).cuda() for _ in range(3)]
    zm32 = [torch.randint(-2**31, 2**31 - 1, (N, rows), dtype=torch.int32, generator=g).cuda() for _ in range(3)]
    tags = torch.zeros((N, 2), dtype=torch.int32, device="cuda")
    nb = (rows + 1023) // 1024
    roots = torch.zeros((3, N, nb), dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    modes = {
        "mpclift": (lambda: ipc.ipc_compare(zc, zm, rows, N, rows, 0, tags, w.prf_seeds, w.thr_a, 5, roots, nb),
                    12.0, 33 + 61),
        "plain_mask": (lambda: ipc.ipc_compare_plain(zc, zm[0], rows, N, rows, 0, tags, w.prf_seeds, w.thr_a, 5,
                                                     roots, nb), 8.0, 29),
        "constlift": (lambda: ipc.ipc_compare_liftfree(zc, None, zm32, rows, N, rows, 0, tags, w.prf_seeds,
                                                       w.thr_a, 0, 5, roots, nb), 18.0, 61),
        "nolift": (lambda: ipc.ipc_compare_liftfree(None, zc32, zm32, rows, N, rows, 0, tags, w.prf_seeds,
                                                    w.thr_a, 0, 5, roots, nb), 24.0, 61),
    }
    out = {"kernel": "compare", "rows": rows, "cols": N}
    for name, (launch, bpc, ands) in modes.items():
        launch()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.reps):
            launch()
        e1.record(st)
        e1.synchronize()
        ipc.ipc_status()
        ms = e0.elapsed_time(e1) / args.reps
        # bpc: bytes of dot-product components read per comparison (3 parties; ml public for plain)
        out[name] = {"ms_per_launch": ms, "comparisons_per_s": N * rows / (ms * 1e-3), "and_gates": ands,
                     "algorithmic_bytes_per_launch": bpc * N * rows,
                     "achieved_gbs": bpc * N * rows / (ms * 1e-3) / 1e9}
    out.update(out["mpclift"])
    print(json.dumps(out))


def run_overlap(args, w):
    """Can the comparison phase hide behind the dot-product GEMMs on the same GPU? The Galois-ring
    GEMM of one party and vector (K = l) over a chunk of --rows rows and the MPCLift comparison of
    the same chunk are timed alone, then launched together on two streams, interleaved. Overlap
    would show as together < GEMM + comparison; it is what a fused GEMM + comparison kernel
    (Sec. 6.4's dots-then-comparisons split on one device) would have to exploit."""
    import torch

    import paper_2405_04463_gb300 as ipc
    l, N, rows = w.l, w.Q * w.R, args.rows
    n_pad = (N + 127) // 128 * 128
    f16 = lambda t: t.to(torch.float16).view(torch.int16).contiguous()
    xl = torch.randint(-128, 128, (rows, l), dtype=torch.int8, device="cuda")
    xh = torch.randint(-128, 128, (rows, l), dtype=torch.int8, device="cuda")
    bl = f16(torch.randint(-128, 128, (n_pad, l), dtype=torch.int8, device="cuda"))
    bh = f16(torch.randint(-128, 128, (n_pad, l), dtype=torch.int8, device="cuda"))
    tags = torch.zeros((N, 2), dtype=torch.int32, device="cuda")
    z = torch.empty((N, rows), dtype=torch.int16, device="cuda")
    g = torch.Generator(device="cpu").manual_seed(7)
    zc = [torch.randint(-32768, 32768, (N, rows), dtype=torch.int16, generator=g).cuda() for _ in range(3)]
    zm = [torch.randint(0, 12801, (N, rows), dtype=torch.int16, generator=g).cuda() for _ in range(3)]
    nb = (rows + 1023) // 1024
    roots = torch.zeros((3, N, nb), dtype=torch.int32, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def gemm(st):
        ipc.ipc_ring_gemm_tc_galois(256, xl, xh, rows, bl, bh, N, n_pad, l, tags, 1, 2, 0, z, rows, 0, stream=st)

    def cmp(st):
        ipc.ipc_compare(zc, zm, rows, N, rows, 0, tags, w.prf_seeds, w.thr_a, 5, roots, nb, stream=st)

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t)

    reps = max(args.reps, 6)
    for _ in range(2):
        gemm(s1)
        cmp(s2)
    t_gemm = timed(lambda: [gemm(s1) for _ in range(reps)]) / reps
    t_cmp = timed(lambda: [cmp(s2) for _ in range(reps)]) / reps

    def both():
        for _ in range(reps):
            gemm(s1)
            cmp(s2)
    t_both = timed(both) / reps
    ipc.ipc_status()
    print(json.dumps({"kernel": "overlap", "rows": rows, "cols": N, "gemm_ms": t_gemm, "compare_ms": t_cmp,
                      "together_ms": t_both, "sum_ms": t_gemm + t_cmp,
                      "hidden_fraction_of_compare": (t_gemm + t_cmp - t_both) / t_cmp,
                      "note": "per pair of launches, host wall clock around reps launches on two streams"}))


def run_fused(args, w):
    """The chunk step of a context, fused (one gemm_cmp_kernel launch per chunk: the six ring GEMMs
    tile by tile and each tile's comparison phase, then the block join) and unfused (six GEMM
    launches on the party streams and one comparison launch), on the workload's first --rows
    database rows (one resident chunk for --rows <= 65,536), Galois-ring Shamir dots (--path tcg,
    the default) or replicated sharing (tc). Steps timed with CUDA events on the control stream."""
    import torch

    import paper_2405_04463_gb300 as ipc
    from paper_2405_04463_gb300.workload import galois, load_workload, make_ctx, query_shares_gpu

    wr = dataclasses.replace(w, s=args.rows)
    gal = galois(args.fused_path)
    qc, qm = query_shares_gpu(wr, galois_shares=gal)
    out = {"kernel": "fused", "path": args.fused_path, "rows": args.rows, "cols": wr.Q * wr.R}
    bits = {}
    for fused in (False, True):
        ctx = make_ctx(wr, path=args.fused_path, max_queries=wr.Q, max_requests=SLOTS, fused=fused)
        try:
            load_workload(ctx, wr, chunk=16384, galois_shares=gal)
            stream = torch.cuda.ExternalStream(ipc.ipc_ctx_stream(ctx))
            b = np.zeros(wr.Q, np.uint8)

            def steps(k):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                rids = [ipc.submit_queries(ctx, [qc[j] for j in range(3)], [qm[j] for j in range(3)], wr.Q, 1)
                        for _ in range(k)]
                e1.record(stream)
                for r in rids:
                    ipc.fetch_match_bits(ctx, r, b, wr.Q, -1)
                torch.cuda.synchronize()
                return e0.elapsed_time(e1) / k

            steps(1)
            ms = steps(max(1, min(args.reps, SLOTS)))
        finally:
            ipc.ipc_destroy(ctx)
        key = "fused" if fused else "unfused"
        out[key] = {"ms_per_step": ms, "comparisons_per_s": wr.comparisons / (ms * 1e-3)}
        bits[key] = b.copy()
    out["bits_equal"] = bool((bits["fused"] == bits["unfused"]).all())
    print(json.dumps(out))


def run_kernel(args, w):
    """One ring-GEMM launch shape of the workload (all its query columns x --rows rows), random
    operands, timed alone with CUDA events; used for ncu captures on a small case."""
    import torch

    import paper_2405_04463_gb300 as ipc
    if args.kernel == "compare":
        return run_compare_kernel(args, w)
    if args.kernel == "overlap":
        return run_overlap(args, w)
    if args.kernel == "fused":
        return run_fused(args, w)
    l, N = w.l, w.Q * w.R
    n_pad = (N + 127) // 128 * 128
    rows = args.rows
    planes = [torch.randint(-128, 128, (rows, l), dtype=torch.int8, device="cuda") for _ in range(4)]
    blo = torch.randint(-128, 128, (n_pad, 2 * l), dtype=torch.int8, device="cuda")
    bhi = torch.randint(-128, 128, (n_pad, 2 * l), dtype=torch.int8, device="cuda")
    tags = torch.zeros((N, 2), dtype=torch.int32, device="cuda")
    z = torch.empty((N, rows), dtype=torch.int16, device="cuda")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    products = 3.0
    f16 = lambda t: t.to(torch.float16).view(torch.int16).contiguous()
    if args.kernel == "tc32":
        # the Z_2^32 ring product: four int8 database limb planes per component, fp16 query limbs,
        # ten limb products, z as uint32
        x8 = [torch.randint(-128, 128, (rows, l), dtype=torch.int8, device="cuda") for _ in range(8)]
        b4 = [f16(torch.randint(-128, 128, (n_pad, 2 * l), dtype=torch.int8, device="cuda")) for _ in range(4)]
        del planes, blo, bhi
        z = torch.empty((N, rows), dtype=torch.int32, device="cuda")
        products = 10.0

        def launch():
            ipc.ipc_ring_gemm_tc32(2, x8, rows, b4, N, n_pad, l, tags, 1, 2, 0, z, rows, 0)
    elif args.kernel == "tc":
        # int8 database planes, the query limbs as fp16 bit patterns (conversion outside the timing)
        blo, bhi = f16(blo), f16(bhi)

        def launch():
            ipc.ipc_ring_gemm_tc(planes[0:2], planes[2:4], rows, blo, bhi, N, n_pad, l, tags, 1, 2, 0, z, rows, 0)
    else:
        def launch():
            ipc.ipc_ring_gemm(args.kernel, planes[0:2], planes[2:4], rows, blo, bhi, N, n_pad, l, tags, 1, 2, 0, z,
                              rows, 0)
    launch()
    e0.record(st)
    for _ in range(args.reps):
        launch()
    e1.record(st)
    e1.synchronize()
    ipc.ipc_status()
    ms = e0.elapsed_time(e1) / args.reps
    macs = products * N * rows * 2 * l if args.kernel != "i32" else 1.0 * N * rows * 2 * l
    limbs = 4 if args.kernel == "tc32" else 2
    qes = 2 if args.kernel in ("tc", "tc32") else 1   # fp16 query limbs on the tcgen05 paths
    print(json.dumps({"kernel": args.kernel, "rows": rows, "cols": N, "ms_per_launch": ms,
                      "algorithmic_ops_per_launch": 2 * macs, "achieved_tops": 2 * macs / (ms * 1e-3) / 1e12,
                      "operand_bytes_per_launch": 2 * limbs * rows * l + qes * limbs * n_pad * 2 * l,
                      "z_bytes": (4 if args.kernel == "tc32" else 2) * N * rows}))


def max_over_ranks(x: float) -> float:
    """The largest x over all ranks: the job's time is its slowest rank's. The ranks are
    independent replicas, so this bookkeeping goes over a host (gloo) process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units per second of the whole job: every rank processed units_per_rank in (at most) ms."""
    return units_per_rank * world / (ms * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): the 3-party simulation on a bounded sample.
# ------------------------------------------------------------------------------------------

def oracle_sample(w: synth.Workload, rows: int):
    import oracle
    og = oracle.Geom(w.rows, w.cols, w.cell, w.rot_lo, w.R)
    dc, dm = w.db_bits(np.arange(rows))
    qc, qm = w.query_bits()
    dbc, dbm = oracle.encode_share(dc, dm, w.l, w.db_share_seed, 0)
    qsc, qsm = oracle.encode_share(qc[:1], qm[:1], w.l, w.q_share_seed, 1)
    cfg = oracle.mpc_cfg(w.prf_seeds, req=1, thr_a=w.thr_a)

    def step():
        t = time.perf_counter()
        oracle.mpc_match(cfg, og, dbc, dbm, qsc, qsm)
        return time.perf_counter() - t

    return step, rows * w.R, f"1 query x {w.R} rotations x {rows} database rows of the workload"


def plaintext_rate(w: synth.Workload, rows: int, threads: int):
    """Alg. 1 (the plaintext matcher of the oracle, all queries x rotations) on the first `rows`
    database rows with `threads` OpenMP threads: comparisons/s. Context for the share-domain
    numbers (the paper quotes its CPU matcher per core)."""
    import oracle
    og = oracle.Geom(w.rows, w.cols, w.cell, w.rot_lo, w.R)
    dc, dm = w.db_bits(np.arange(rows))
    qc, qm = w.query_bits()
    t = time.perf_counter()
    oracle.plain_match(og, qc, qm, dc, dm, threads=threads)
    secs = time.perf_counter() - t
    return {"value": rows * w.Q * w.R / secs, "unit": UNIT, "cores": threads, "seconds": secs,
            "sample": f"{w.Q} queries x {w.R} rotations x {rows} database rows, plaintext Alg. 1"}


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    step, comps, sample = oracle_sample(w, max(64, args.cpu_sample_rows // 2))
    for _ in range(args.warmup):
        step()
    times = [step() for _ in range(args.steps)]
    total = sum(times)
    value = comps * args.steps / total
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16/u32 ring (C, CPU)",
        "data": "synthetic", "config": {"workload": w.name, "sample": sample},
        "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": value, "unit": UNIT},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def ncu_traffic(kernel: str, src: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    h = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    if not m or not h:
        return None
    return float(m.group(1)) if source_hash(src) == h.group(1) else None


def source_hash(src: str) -> str:
    """SHA-256 of a kernel's .cu file followed by the headers it includes from its own directory,
    depth first in order of first inclusion."""
    seen, order = set(), []

    def visit(path):
        if path in seen:
            return
        seen.add(path)
        order.append(path)
        for inc in re.findall(r'^#include "([^"/]+)"', open(path).read(), re.M):  # same directory only
            dep = os.path.join(os.path.dirname(path), inc)
            if os.path.exists(dep):
                visit(dep)

    visit(src)
    hs = hashlib.sha256()
    for path in order:
        hs.update(open(path, "rb").read())
    return hs.hexdigest()


SLOTS = 2   # request slots of each benchmark context: one request running, the next one queued


def run_ours(args, w):
    import torch

    import paper_2405_04463_gb300 as ipc
    from paper_2405_04463_gb300.workload import (galois, lift_shares, load_workload, make_ctx, plain_mask_u16,
                                                 query_shares_gpu)

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        # replicas only: the data path exchanges nothing; the barrier and the max over ranks of
        # the step time go over gloo on the host
        import torch.distributed as dist
        dist.init_process_group("gloo")
    dev = torch.cuda.current_device()

    # ---- setup (untimed): resident database, query shares, contexts ----
    # headline: the tcgen05 path; beside it the two int8 mma.sync paths and the int32 path
    # plus the paper's deployed Galois-ring Shamir dot products on the same tcgen05 kernels
    # (the other paths' contexts are made one at a time below, each freed after its run)
    ctxs = {"tc": make_ctx(w, path="tc", max_queries=w.Q, max_requests=SLOTS)}
    load_workload(ctxs["tc"], w, chunk=32768)
    qcode, qmask = query_shares_gpu(w)
    gqcode, gqmask = query_shares_gpu(w, galois_shares=True)
    pqmask = plain_mask_u16(w.query_bits()[1], w.l)
    lift_q = {lf: lift_shares(*w.query_bits(), w.l, w.q_share_seed, 1, lift=lf) for lf in ("const", "none")}
    hcode = [qcode[j].cpu().pin_memory() for j in range(3)]
    hmask = [qmask[j].cpu().pin_memory() for j in range(3)]
    torch.cuda.synchronize()
    n_chunks = (w.s + 65535) // 65536
    launches_per_step = 6 + n_chunks * 7 + 2

    def run_steps(ctx, k, host_inputs, gal=False, plain=False, lift=None, alternate=False):
        """k requests of the workload's query batch. Pipelined (default): up to the context's
        request slots in flight, the oldest fetched before the next submit; alternating: each
        request fetched before the next is submitted. Returns (device ms per step from events on
        the control stream, host wall ms per step from the first submit to the last fetched
        result, the opened bits)."""
        stream = torch.cuda.ExternalStream(ipc.ipc_ctx_stream(ctx))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        qc_, qm_ = (gqcode, gqmask) if gal else (qcode, qmask)
        code = hcode if host_inputs else [qc_[j] for j in range(3)]
        mask = hmask if host_inputs else [qm_[j] for j in range(3)]
        if plain:
            mask = [pqmask, None, None]
        if lift:
            code, mask = [lift_q[lift][0][j] for j in range(3)], [lift_q[lift][1][j] for j in range(3)]
        bits = np.zeros(w.Q, np.uint8)
        inflight = []
        depth = 1 if alternate else SLOTS
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(k):
            if len(inflight) == depth:
                ipc.fetch_match_bits(ctx, inflight.pop(0), bits, w.Q, -1)
            inflight.append(ipc.submit_queries(ctx, code, mask, w.Q, 0 if host_inputs else 1))
        e1.record(stream)
        for rid in inflight:
            ipc.fetch_match_bits(ctx, rid, bits, w.Q, -1)
        wall = time.perf_counter() - t0
        e1.synchronize()
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1))
        wall_ms = max_over_ranks(1e3 * wall)
        return ms / k, wall_ms / k, bits.copy()

    main = ctxs["tc"]
    run_steps(main, args.warmup, False)
    clocks = Clocks(dev)
    clocks.start()
    ms_main, wall_main, bits = run_steps(main, args.steps, False)
    clk = clocks.stop()
    run_steps(main, 1, True)
    ms_e2e, wall_e2e, bits_e2e = run_steps(main, args.steps, True)
    # the natural use of the API: submit, fetch, submit, fetch ... (no request overlaps another)
    ms_alt, wall_alt, bits_alt = run_steps(main, args.steps, True, alternate=True)
    # the comparison paths below each load their own copy of the database: free the headline's
    # first, so that the largest workloads fit beside them
    for c in ctxs.values():
        ipc.ipc_destroy(c)
    ctxs.clear()
    torch.cuda.empty_cache()

    def other(path, plain=False, lift=None, fused=False):
        gal = galois(path)
        ctx = make_ctx(w, path=path, max_queries=w.Q, plain_mask=plain, lift=lift or "mpc", max_requests=SLOTS,
                       fused=fused)
        try:
            load_workload(ctx, w, chunk=32768, galois_shares=gal, plain_mask=plain, lift=lift)
            run_steps(ctx, 1, False, gal, plain, lift)
            ms, _, b = run_steps(ctx, args.steps, False, gal, plain, lift)
        except ipc.IpcError as e:   # e.g. a database copy that does not fit beside nothing else
            return {"value": None, "unavailable": str(e)}
        finally:
            ipc.ipc_destroy(ctx)
            torch.cuda.empty_cache()
        return {"value": whole_job_rate(w.comparisons, world, ms), "ms_per_step": ms,
                "bits_equal_to_headline_path": bool((b == bits).all())}

    out_gal = other("tcg")
    # the fused chunk step (six ring GEMMs and the comparison phase in one launch per chunk)
    out_fused_gal = other("tcg", fused=True)
    out_fused = other("tc", fused=True)
    out_plain = other("tc", plain=True)
    out_plain_gal = other("tcg", plain=True)
    out_const = other("tc", lift="const")
    out_nolift = other("tc", lift="none")
    del lift_q
    out_mix = other("i8mix")
    out_mma = other("i8mma")
    out_i32 = other("i32") if not args.no_i32 else None

    # ---- each ring-GEMM kernel alone: one launch over a 65536-row chunk, all query columns ----
    l, N = w.l, w.Q * w.R
    n_pad = (N + 127) // 128 * 128
    rows = min(65536, w.s)
    planes = [torch.randint(-128, 128, (rows, l), dtype=torch.int8, device="cuda") for _ in range(4)]
    blo = torch.randint(-128, 128, (n_pad, 2 * l), dtype=torch.int8, device="cuda")
    bhi = torch.randint(-128, 128, (n_pad, 2 * l), dtype=torch.int8, device="cuda")
    f16 = [t.to(torch.float16).view(torch.int16).contiguous() for t in (blo, bhi)]
    tags = torch.zeros((N, 2), dtype=torch.int32, device="cuda")
    z = torch.empty((N, rows), dtype=torch.int16, device="cuda")
    st = torch.cuda.current_stream()

    x8 = planes + planes
    b4 = [f16[0], f16[1], f16[0], f16[1]]
    z32 = torch.empty((N, rows), dtype=torch.int32, device="cuda")

    def launch(path):
        if path == "tc32":
            ipc.ipc_ring_gemm_tc32(2, x8, rows, b4, N, n_pad, l, tags, 1, 2, 0, z32, rows, 0)
        elif path == "tc":
            ipc.ipc_ring_gemm_tc(planes[0:2], planes[2:4], rows, f16[0], f16[1], N, n_pad, l, tags, 1, 2, 0, z, rows, 0)
        else:
            ipc.ipc_ring_gemm(path, planes[0:2], planes[2:4], rows, blo, bhi, N, n_pad, l, tags, 1, 2, 0, z, rows, 0)

    def gemm_time(path, reps):
        for _ in range(2):
            launch(path)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            launch(path)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    t_tc = gemm_time("tc", 10)
    t_tc32 = gemm_time("tc32", 4)
    t_mix = gemm_time("i8mix", 3)
    t_i8 = gemm_time("i8mma", 3)
    t_i32 = gemm_time("i32", 2) if not args.no_i32 else None
    ipc.ipc_status()
    ops = 2.0 * 3 * N * rows * 2 * l          # 3 limb products per ring multiply-add, 2 ops each
    peaks = measured_peaks()
    bf16_burst, bf16_sust = peaks.get("bf16_tflops"), peaks.get("bf16_tflops_sustained")
    peak_mma = ipc.ipc_measure_peak(0)
    peak_imad = ipc.ipc_measure_peak(1)
    peak_dp4a = ipc.ipc_measure_peak(2)
    achieved = ops / (t_tc * 1e-3) / 1e12
    traffic = ncu_traffic("gemm_tc_kernel", os.path.join(ROOT, "paper_2405_04463_gb300", "csrc", "gemm_tc.cu"))
    # algorithmic bytes of one launch: the two database components' int8 limb planes (the size
    # of their u16 shares), the fp16 query operand and z
    alg_bytes = 2 * 2 * rows * l + 2 * 2 * n_pad * 2 * l + 2 * N * rows
    roofline = {"bound": "tensor",
                "kernel": "gemm_tc_kernel (tcgen05.mma kind::f16; int8 database limbs widened to fp16 in shared "
                          "memory, fp16 query limbs; exact)",
                "achieved": achieved, "peak": bf16_burst, "unit": "TFLOP/s",
                "frac": achieved / bf16_burst if bf16_burst else None, "traffic": traffic,
                "algorithmic_bytes": alg_bytes, "traffic_over_algorithmic": traffic / alg_bytes if traffic else None,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst: the kernel is timed alone, back to back; "
                               "fp16 and bf16 have the same dense tensor rate)",
                "launch_ms": t_tc, "flops_per_launch": ops,
                "int8_kernels": {
                    "gemm_i8_kernel<1> (mma.sync s8 + dp4a)": {
                        "launch_ms": t_mix, "achieved_tops": ops / (t_mix * 1e-3) / 1e12,
                        "frac_of_measured_mma_plus_dp4a": ops / (t_mix * 1e-3) / 1e12 / (peak_mma + peak_dp4a)},
                    "gemm_i8_kernel<0> (mma.sync s8)": {
                        "launch_ms": t_i8, "achieved_tops": ops / (t_i8 * 1e-3) / 1e12,
                        "frac_of_measured_mma": ops / (t_i8 * 1e-3) / 1e12 / peak_mma},
                    "measured_int8_peaks_tops": {"mma_sync_s8": peak_mma, "dp4a": peak_dp4a,
                                                 "source": "register-only loops (ipc_measure_peak)"}}}
    ops32 = 2.0 * 10 * N * rows * 2 * l   # ten limb products per Z_2^32 ring multiply-add
    tc32_kernel = {"kernel": "gemm_tc32_kernel (tcgen05.mma kind::f16, four limbs, Z_2^32)", "bound": "tensor",
                   "achieved": ops32 / (t_tc32 * 1e-3) / 1e12, "peak": bf16_burst, "unit": "TFLOP/s",
                   "frac": ops32 / (t_tc32 * 1e-3) / 1e12 / bf16_burst if bf16_burst else None,
                   "launch_ms": t_tc32, "flops_per_launch": ops32,
                   "traffic": ncu_traffic("gemm_tc32_kernel", os.path.join(ROOT, "paper_2405_04463_gb300", "csrc",
                                                                           "ring32.cu"))}
    i32_kernel = None
    if t_i32:
        imads = 1.0 * N * rows * 2 * l
        i32_kernel = {"kernel": "gemm_i32_kernel", "bound": "alu", "achieved": imads / (t_i32 * 1e-3) / 1e12,
                      "peak": peak_imad, "unit": "T IMAD/s", "frac": imads / (t_i32 * 1e-3) / 1e12 / peak_imad,
                      "launch_ms": t_i32}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        step, comps, sample = oracle_sample(w, args.cpu_sample_rows)
        secs = step()
        cpu = {"value": comps / secs, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample, "seconds": secs,
               "plaintext_alg1": {"one_core": plaintext_rate(w, 512, 1),
                                  "all_cores": plaintext_rate(w, 4096, os.cpu_count() or 1),
                                  "note": "the oracle's plaintext matcher, not the share-domain protocol"}}

    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    value = whole_job_rate(w.comparisons, world, ms_main)
    h2d = 2 * 3 * w.Q * w.l * 2
    flops_per_cmp = 921600.0   # 3 parties x 2 vectors x 2 l x 3 limb products x 2 ops
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_main, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": w.name, "db_rows": w.s, "queries": w.Q, "rotations": w.R, "code_bits": w.l,
                   "planted": w.planted,
                   "path": "tc: int8 limbs as exact fp16 operands of tcgen05.mma (database resident as int8, "
                           "widened in shared memory), fp32 TMEM accumulators re-based every 128 k inside "
                           "[2^23, 2^24] (bit-exact; integer results; no rounding anywhere)",
                   "parallelism": f"replicas x{world}",
                   "sharing": "3-party replicated (ABY3); galois_shamir_path: Galois-ring Shamir dots",
                   "l2": "inputs larger than L2: resident int8 limb planes 12 B x rows x 12800 = "
                         f"{12 * w.s * w.l / 1e9:.1f} GB"},
        "tensor_peak_frac_step": value * flops_per_cmp / (bf16_sust * 1e12) if bf16_sust else None,
        # the metric's "% of INT8 peak" belongs to the integer-only paths: their limb ops per second
        # (921,600 per comparison) against the measured dense INT8 tensor rate of this GPU
        # (mma.sync s8; sm_103a has no integer tcgen05). The headline runs on the fp16 tcgen05
        # tensor cores and is reported against their peak (roofline, tensor_peak_frac_step).
        "int8_peak": {
            "measured_mma_sync_s8_tops": peak_mma, "measured_dp4a_tops": peak_dp4a,
            "int8_tensor_only_path_pct_of_mma_sync": 100.0 * out_mma["value"] * flops_per_cmp / (peak_mma * 1e12)
            if out_mma["value"] else None,
            "int8_mix_path_pct_of_mma_sync_plus_dp4a": 100.0 * out_mix["value"] * flops_per_cmp /
            ((peak_mma + peak_dp4a) * 1e12) if out_mix["value"] else None},
        "galois_shamir_path": dict(out_gal, note="the paper's deployed sharing of the dot products "
                                                 "(Sec. 4.3.2): one length-l GEMM per party and vector "
                                                 "instead of 2l, same tcgen05 kernel, same comparison phase"),
        "fused_step": {
            "galois_shamir": dict(out_fused_gal, unfused_ms_per_step=out_gal.get("ms_per_step")),
            "replicated": dict(out_fused, unfused_ms_per_step=ms_main),
            "note": "Sec. 6.4's dots and comparisons of a chunk in one launch: the six ring GEMMs tile by tile "
                    "(gemm_cmp_kernel), each tile's comparison phase run by its drain warps after the sixth "
                    "GEMM, z read back from L2; then the block join of the part roots"},
        "plain_mask_path": dict(out_plain, galois_shamir=out_plain_gal,
                                note="protocol 1 (Sec. 4, Alg. 2): public masks, ml one plaintext GEMM "
                                     "(K = l) instead of three shared ones, 16-bit comparison (29 ANDs)"),
        "lift_variants": {
            "constlift": out_const, "nolift": out_nolift,
            "note": "Sec. 5.1 / Table 2: ml (ConstLift) or ml and dot (NoLift) computed over Z_2^32 by the "
                    "ten-product tcgen05 ring GEMM, comparison without Lift (61 ANDs); the headline path is "
                    "MPCLift"},
        "int8_mix_path": out_mix,
        "int8_tensor_only_path": out_mma,
        "int32_path": out_i32,
        "ratio_vs_int32": (value / out_i32["value"]) if out_i32 and out_i32["value"] else None,
        "ratio_int8_mix_vs_int32": (out_mix["value"] / out_i32["value"])
        if out_i32 and out_i32["value"] and out_mix["value"] else None,
        "roofline": roofline,
        "int32_kernel": i32_kernel,
        "tc32_kernel": tc32_kernel,
        "cpu_baseline": cpu,
        "e2e": {"value": whole_job_rate(w.comparisons, world, wall_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 3 * w.Q, "wall_ms_per_step": wall_e2e, "device_ms_per_step": ms_e2e,
                "clock": "host wall clock from the first submit_queries to the last fetched result",
                "bits_equal": bool((bits_e2e == bits).all()),
                "alternating": {"value": whole_job_rate(w.comparisons, world, wall_alt), "wall_ms_per_step": wall_alt,
                                "device_ms_per_step": ms_alt, "bits_equal": bool((bits_alt == bits).all()),
                                "note": "submit, fetch, submit, fetch: one request at a time"}},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "match_bits": int(bits.sum()),
        "measured_peaks": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained")},
    }
    print(json.dumps(res), flush=True)


def run_serving(args):
    """Continuous batching on the serving workload: 250,000 resident rows, batches of U{1..256}
    queries x 31 rotations arriving by a seeded Poisson process at fractions of the measured
    capacity (requests/s of a burst of batches of 128 and 129 queries, mean 128.5). Latency =
    completion - submission per request, both taken by the library's own clock."""

    import torch

    import paper_2405_04463_gb300 as ipc
    from paper_2405_04463_gb300.workload import encode_gpu, galois, load_workload, make_ctx

    w = synth.workload("c4")
    torch.cuda.set_device(0)
    path = args.serving_path
    ctx = make_ctx(w, path=path, max_queries=256)
    t_load = time.perf_counter()
    load_workload(ctx, w, chunk=32768, galois_shares=galois(path))
    t_load = time.perf_counter() - t_load
    # 512 query shares on the host; request k takes a window of its batch size
    rng = np.random.default_rng(0x5E7E)
    qc = rng.integers(0, 2**63, size=(512, w.nwords), dtype=np.int64).view(np.uint64)
    qm = rng.integers(0, 2**63, size=(512, w.nwords), dtype=np.int64).view(np.uint64)
    qcode, qmask = encode_gpu(qc, qm, w.l, w.q_share_seed, 1, galois_shares=galois(path))
    hcode = [qcode[j].cpu().numpy() for j in range(3)]
    hmask = [qmask[j].cpu().numpy() for j in range(3)]
    del qcode, qmask
    ipc.ipc_serve_start(ctx, pool_queries=args.pool, variant=ipc.IPC_SERVE_AUTOTUNE)
    tuning = ipc.ipc_serve_tuning(ctx)
    clocks = Clocks(0)
    clocks.start()

    def submit(q, off):
        code = [np.ascontiguousarray(hcode[j][off:off + q]) for j in range(3)]
        mask = [np.ascontiguousarray(hmask[j][off:off + q]) for j in range(3)]
        while True:
            try:
                return ipc.ipc_serve_submit(ctx, code, mask, q)
            except ipc.IpcError as e:
                if e.rc != ipc.IPC_EAGAIN:
                    raise
                time.sleep(0.001)

    def collect(rids, sizes):
        times = []
        for rid, q in zip(rids, sizes):
            sh = np.zeros((3, q), np.uint8)
            ipc.fetch_bit_shares(ctx, rid, sh, q, -1)
            times.append(ipc.ipc_serve_times(ctx, rid))
            ipc.ipc_release(ctx, rid)
        return np.array(times)

    # capacity: a burst of batches of 128 and 129 queries
    st0 = ipc.ipc_serve_stats(ctx)
    sizes = [128 + (k & 1) for k in range(args.capacity_requests)]
    rids = [submit(q, k % 128) for k, q in enumerate(sizes)]
    t = collect(rids, sizes)
    span = t[:, 2].max() - t[:, 0].min()
    capacity = len(sizes) / span
    st1 = ipc.ipc_serve_stats(ctx)
    cap_cmp = (st1["comparisons"] - st0["comparisons"]) / span
    out_rates = []
    for k, frac in enumerate(float(x) for x in args.rates.split(",")):
        lam = frac * capacity
        r = np.random.default_rng(0xA441 + k)
        gaps = r.exponential(1.0 / lam, size=args.requests_per_rate)
        qs = r.integers(1, 257, size=args.requests_per_rate)
        offs = r.integers(0, 256, size=args.requests_per_rate)
        rids = []
        s0 = ipc.ipc_serve_stats(ctx)
        t0 = time.perf_counter()
        at = 0.0
        for g, q, o in zip(gaps, qs, offs):
            at += g
            d = t0 + at - time.perf_counter()
            if d > 0:
                time.sleep(d)
            rids.append(submit(int(q), int(o)))
        t = collect(rids, [int(q) for q in qs])
        s1 = ipc.ipc_serve_stats(ctx)
        lat = t[:, 2] - t[:, 0]
        wait = t[:, 1] - t[:, 0]
        span = t[:, 2].max() - t[:, 0].min()
        out_rates.append({
            "fraction_of_capacity": frac, "offered_req_per_s": lam, "requests": len(rids),
            "achieved_req_per_s": len(rids) / span, "mean_batch": float(qs.mean()),
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(lat.mean()), "max": float(lat.max())},
            "admission_wait_s": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
            "comparisons_per_s": (s1["comparisons"] - s0["comparisons"]) / span,
            "steps": s1["steps"] - s0["steps"],
            "variant_steps": [a - b for a, b in zip(s1["variant_steps"], s0["variant_steps"])],
        })
    clk = clocks.stop()
    stats = ipc.ipc_serve_stats(ctx)
    ipc.ipc_serve_stop(ctx)
    ipc.ipc_destroy(ctx)
    print(json.dumps({
        "metric": "serving: latency p50/p99 and comparisons/s under Poisson arrivals", "unit": "s / comparisons/s",
        "config": {"workload": w.name, "db_rows": w.s, "rotations": w.R, "batch": "U{1..256} queries",
                   "arrivals": "Poisson, seeded", "path": path, "pool_query_slots": stats["pool_queries"],
                   "pool_cols": stats["pool_cols"], "chunks": stats["n_chunks"],
                   "requests_per_rate": args.requests_per_rate},
        "load_s": t_load, "capacity_req_per_s": capacity, "capacity_comparisons_per_s": cap_cmp,
        "rates": out_rates, "tuning": json.loads(tuning) if tuning else None, "clocks": clk,
        "data": "synthetic"}), flush=True)


def run_persons(args):
    """Batches of P persons x 2 eyes x 31 rotations against a database per eye, plus the
    inner-batch matching of each batch (Sec. 5.4), through ipc_check_persons with host inputs:
    each call is synchronous and returns the persons' bit components, so the time per batch is
    host wall time around the call."""
    import torch

    import paper_2405_04463_gb300 as ipc
    from paper_2405_04463_gb300.workload import encode_gpu, galois, load_workload, make_ctx

    torch.cuda.set_device(0)
    path, P, rows = args.persons_path, args.persons_batch, args.persons_rows
    gal = galois(path)
    eyes = [synth.Workload(f"eye {e}: {rows} rows", s=rows, Q=P, seed=0x1A150004 + 16 * e) for e in range(2)]
    seeds = eyes[0].prf_seeds
    ctxs = []
    for w in eyes:
        w.prf_seeds = seeds
        c = make_ctx(w, path=path, max_queries=P)
        load_workload(c, w, chunk=32768, galois_shares=gal)
        ctxs.append(c)
    rng = np.random.default_rng(0x9E75)
    batches = []
    for k in range(args.warmup + args.steps):
        code, mask = [], []
        for e in range(2):
            qc = rng.integers(0, 2**63, size=(P, eyes[e].nwords), dtype=np.int64).view(np.uint64)
            qm = rng.integers(0, 2**63, size=(P, eyes[e].nwords), dtype=np.int64).view(np.uint64)
            c_, m_ = encode_gpu(qc, qm, eyes[e].l, eyes[e].q_share_seed, 1, galois_shares=gal)
            code += [c_[j].cpu().numpy() for j in range(3)]
            mask += [m_[j].cpu().numpy() for j in range(3)]
        batches.append((code, mask))
    for code, mask in batches[:args.warmup]:
        ipc.ipc_check_persons(ctxs, code, mask, P, 0)
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for code, mask in batches[args.warmup:]:
        ipc.ipc_check_persons(ctxs, code, mask, P, 0)
    dt = (time.perf_counter() - t0) / args.steps
    clk = clocks.stop()
    for c in ctxs:
        ipc.ipc_destroy(c)
    R = eyes[0].R
    db_cmp = 2 * P * R * rows
    batch_cmp = 2 * R * P * (P - 1) // 2
    print(json.dumps({
        "metric": "persons: both eyes x 31 rotations against the database + inner-batch matching",
        "value": (db_cmp + batch_cmp) / dt, "unit": "comparisons/s", "ms_per_batch": 1e3 * dt,
        "persons_per_s": P / dt, "steps": args.steps, "warmup": args.warmup,
        "config": {"persons": P, "eyes": 2, "rotations": R, "db_rows_per_eye": rows, "path": path,
                   "comparisons_per_batch": {"database": db_cmp, "inner_batch": batch_cmp},
                   "inputs": "host query shares, copied inside the call (e2e)"},
        "clocks": clk, "data": "synthetic"}), flush=True)


def main():
    args = parse()
    if args.persons:
        run_persons(args)
        return
    if args.serving:
        run_serving(args)
        return
    w = synth.workload(args.workload)
    if args.kernel:
        run_kernel(args, w)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
