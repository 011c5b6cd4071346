"""Benchmark of the Talek server read path on GB300 (one JSON line on rank 0).

Workload (paper scale): a blocked cuckoo table of n = 32768 buckets x d = 4
slots x 1024-byte messages (128 MiB, uniform random bytes, seed 0); one step
serves 32000 simulated users issuing one PIR read each (Bernoulli(0.5)
request vectors), in batches of B = 256 requests per table pass.  Four copies
of the table (512 MiB in all, more than the 126 MB L2) are read in rotation,
so every pass streams its table from HBM.

Reported: reads/s of the step (`value`), per-batch-width legs (B = 1 plain
kernel, 32, 256) with their table-scan GB/s, the end-to-end rate through the
synchronous host-buffer entry point (`e2e`), the oracle and a multi-core CPU
engine timed on the host (`cpu_baseline`), the 64-table uneven workload, the
4 GiB table, writes, serving under a 64 GiB budget at Poisson 5 k and 50 k
reads/s (p50/p99), SM clocks sampled during the timed region, and the
roofline of the dominant kernel.

Multi-GPU: every rank serves its own 32000 reads from its own replica of the
table (the paper's servers each hold a full copy); no data-path collective,
weak scaling.  `--impl reference` times the CPU oracle instead.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_BUCKETS, D_SLOTS, MSG_BYTES = 32768, 4, 1024
USERS = 32000
B_HEAD = 256
LAUNCHES_HEAD = (USERS + B_HEAD - 1) // B_HEAD  # scan launches per headline step
COPIES = 4
HBM_PEAK_FALLBACK = 6800.0
SMS, LOP3_PER_CLK_PER_SM = 152, 64
SMEM_BYTES_PER_CLK_PER_SM = 128  # 32 banks x 4 bytes
# DRAM bytes (read + write) per launch of each kernel on this workload, from
# ncu captures summarised in profiles/ (the batched kernels: mean of three
# launches of one capture; the plain kernel: one launch)
TRAFFIC_BATCHED_B256 = (136.659968e6 + 3.284480e6 + 136.435200e6 + 0.130304e6 + 136.602368e6
                        + 0.338944e6) / 3
TRAFFIC_PLAIN_B1 = 134.240768e6 + 3.548928e6
TRAFFIC_M4RM_B256 = (136.340736e6 + 3.074048e6 + 136.585216e6 + 0.072192e6 + 136.370944e6
                     + 0.116480e6) / 3
TRAFFIC_GF2MMA_B256 = (135.351040e6 + 2.960640e6 + 135.359488e6 + 0.532736e6 + 135.379200e6
                       + 0.106752e6) / 3


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return {}


def smem_peak_tbs(sm_mhz: float) -> float:
    """Shared-memory bandwidth peak: SMs x 128 B/clk x clock."""
    return SMS * SMEM_BYTES_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12


def m4rm_smem_bytes(n: int, row_words: int, B: int) -> float:
    """Shared-memory bytes the Four-Russians kernel must move per launch: per
    group of 8 buckets and 64-word column tile, the 256 combinations written
    once per 256/512-request tile, plus one 256-byte lookup per request."""
    bt = 256 if B <= 256 else 512
    groups, wtiles, btiles = (n + 7) // 8, (row_words + 63) // 64, (B + bt - 1) // bt
    return float(groups) * wtiles * (btiles * 256 * 64 * 4 + B * 64 * 4)


FP4_ISSUE_PFLOPS_2070 = 9.70  # tcgen05.mma kind::mxf4 N=224 K=64, M=128 or a CTA pair's M=256, all SMs at 2070 MHz (tests/test_gpu_mma_rates.py)


def fp4_peak_tflops(peaks: dict) -> tuple[float, str]:
    """Dense fp4 tensor peak: the measured bf16 cuBLAS burst peak (the kernel is
    timed over a sub-second region) x 6, the nominal fp4 / bf16 ratio (13.5 /
    2.25 PFLOP/s)."""
    if "bf16_tflops" in peaks:
        return 6.0 * peaks["bf16_tflops"], "of measured (bf16 burst x 6, the nominal fp4/bf16 ratio)"
    return 6.0 * 1900.0, "of fallback (1.9 PFLOP/s bf16 x 6)"


def gf2_mma_flops(n: int, row_bytes: int, B: int) -> float:
    """Tensor-core work of the GF(2) product as an integer 0/1 product:
    one multiply-add per (request, bucket, table bit)."""
    return 2.0 * B * n * row_bytes * 8


def alu_peak_tops(sm_mhz: float) -> float:
    """LOP3 (32-bit conditional-XOR word op) peak: SMs x lanes/clk x clock."""
    return SMS * LOP3_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 50 ms; stop() keeps the
    samples whose timestamps fall in the timed region (all of the loaded run
    if none do)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self, t_lo: float = 0.0, t_hi: float = 0.0) -> dict:
        import datetime
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            try:
                rows.append((ts, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if r[0] is not None and t_lo <= r[0] <= t_hi]
        window = "timed region"
        if not inside:
            inside, window = rows, "loaded run (warm-up and timed region)"
        reasons = set()
        for r in inside:
            for name, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        sm = [r[1] for r in inside]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(r[2] for r in inside) if inside else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args) -> None:
    """The oracle, as it stands, on the host cores: a bounded sample of the
    same workload (reads of the 128 MiB table) per step."""
    import oracle
    from paper_2001_08250_gb300 import synth
    rank, world, _ = dist_env()
    if rank != 0:
        return
    oracle.build()
    T = synth.table_bytes(N_BUCKETS, D_SLOTS, MSG_BYTES, seed=0)
    R = synth.random_bits(USERS, N_BUCKETS, seed=1)
    per_step = 4
    for s in range(args.warmup):
        oracle.read_batch(T, N_BUCKETS, D_SLOTS, MSG_BYTES, R[s * per_step:(s + 1) * per_step])
    t0 = time.perf_counter()
    for s in range(args.steps):
        i = (args.warmup + s) * per_step % USERS
        oracle.read_batch(T, N_BUCKETS, D_SLOTS, MSG_BYTES, R[i:i + per_step])
    dt = time.perf_counter() - t0
    v = per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": "pir_reads_per_s", "value": v, "unit": "reads/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": v, "unit": "reads/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} reads of the 128 MiB table per step"},
        "e2e": {"value": v, "unit": "reads/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args) -> dict:
    return {"workload": "paper-scale PIR reads: n=32768 buckets, d=4, 1024-byte messages "
                        "(128 MiB table), 32000 Bernoulli(0.5) reads per step, batch width 256",
            "n": N_BUCKETS, "d": D_SLOTS, "msg_bytes": MSG_BYTES, "reads_per_step": USERS,
            "batch": B_HEAD, "parallelism": f"replicas x{args.gpus}",
            "l2": f"{COPIES} rotated table copies ({COPIES * 128} MiB) > L2 per pass"}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--legs", default="head,head_m4rm,head_lop3,plain,b32,masked,sharded,e2e,serve_sweep,cpu,multi,large,getupdates,writes",
                    help="comma list of: head (B=256, timed headline: the automatic choice, the "
                         "tensor-core kernel), head_m4rm / head_lop3 (B=256 on the Four-Russians / "
                         "register-tiled LOP3 kernel), plain (B=1), b32, masked (serialized-PIR "
                         "masked replies at B=256 and B=1), sharded (the table in 4 row shards "
                         "on this GPU, partial replies XOR-combined), getupdates (compressed "
                         "interest-vector deltas), "
                         "e2e (host buffers), cpu (oracle and multi-core CPU baselines), multi "
                         "(64 uneven tables, one graph-captured launch), large (4 GiB table, "
                         "B=1024), writes, serve_sweep (tables filling a 64 GiB budget, Poisson "
                         "arrivals at --sweep-rates for --sweep-seconds each); serve (not "
                         "default: a short run on eight tables at --serve-rate)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the tile-shape autotuner (use the built-in shape choice)")
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--sweep-rates", default="5000,50000",
                    help="read arrival rates of the serve_sweep leg")
    ap.add_argument("--sweep-seconds", type=float, default=10.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    args.legs = set(args.legs.split(","))
    if args.no_serve:
        args.legs.discard("serve")

    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2001_08250_gb300 import build, synth, talekpir
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    L = talekpir.lib()

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    stream = torch.cuda.Stream()
    n, d, z = N_BUCKETS, D_SLOTS, MSG_BYTES
    row = d * z
    T = synth.table_bytes(n, d, z, seed=0)
    dbs = []
    for _ in range(COPIES):
        db = talekpir.DB(n, d, z)
        db.load(T)
        dbs.append(db)
    R = synth.random_bits(USERS, n, seed=1 + rank)
    dR = torch.from_numpy(R.view(np.int64)).cuda()
    dO = torch.empty((USERS, row), dtype=torch.uint8, device="cuda")
    words = R.shape[1]

    # one 32-byte mask seed per read, for the serialized-PIR leg
    dS = torch.from_numpy(synth.mask_seeds(USERS, seed=1 + rank)).cuda()

    def run_step(B, events=None, masked=False):
        for i, b0 in enumerate(range(0, USERS, B)):
            nb = min(B, USERS - b0)
            if events is not None:
                events[i][0].record(stream)
            if masked:
                dbs[i % COPIES].read_batch_masked_async(dR[b0:b0 + nb], nb, dS[b0:b0 + nb],
                                                        dO[b0:b0 + nb], stream)
            else:
                dbs[i % COPIES].read_batch_async(dR[b0:b0 + nb], nb, dO[b0:b0 + nb], stream)
            if events is not None:
                events[i][1].record(stream)

    last_launches = [0]  # library kernel launches in the last timed region

    def timed(B, steps, warmup, with_launch_events=False, clocks=None, masked=False):
        if clocks:
            # the sampler starts while warm-up steps keep the GPU busy (at
            # least 0.4 s of them), so its samples fall in the loaded run
            clocks.start()
        t_warm = time.perf_counter()
        with torch.cuda.stream(stream):
            done = 0
            while done < warmup or (clocks and time.perf_counter() - t_warm < 0.4):
                run_step(B, masked=masked)
                done += 1
                if clocks and done % 4 == 0:
                    stream.synchronize()
        torch.cuda.synchronize()
        nb = (USERS + B - 1) // B
        ev = None
        per_launch = []
        barrier()
        torch.cuda.synchronize()
        t_lo = time.time()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0 = talekpir.kernel_launches()
        start.record(stream)
        for _ in range(steps):
            if with_launch_events:
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(nb)]
            run_step(B, ev, masked=masked)
            if with_launch_events:
                per_launch.append(ev)
        end.record(stream)
        last_launches[0] = talekpir.kernel_launches() - k0
        torch.cuda.synchronize()
        ck = clocks.stop(t_lo, time.time()) if clocks else None
        barrier()
        ms = start.elapsed_time(end) / steps
        durs = [a.elapsed_time(b) for evs in per_launch for a, b in evs]
        return ms, durs, ck

    tune = None
    if not args.no_autotune:
        tune = dbs[0].autotune(B_HEAD, reps=3)
        dbs[0].autotune(32, reps=3)

    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)
    table_bytes = n * row
    algo_bytes_per_read = table_bytes + n / 8 + row  # table + request bits + reply

    # ---- headline: batch width 256, batched kernel
    clocks = ClockSampler(local)
    head_launches = 0
    if "head" in args.legs:
        ms, _, ck = timed(B_HEAD, args.steps, args.warmup, clocks=clocks)
        head_launches = last_launches[0]
    else:
        ms, ck = float("nan"), None
    ms = max_over_ranks(ms)
    value = USERS * world / (ms * 1e-3)
    # average launch duration = the timed region (CUDA events on the
    # launching stream) / launches: events between launches would break their
    # programmatic overlap (the tensor-core kernel is the step's only launch
    # per batch here, per the ncu launch list and the launch count)
    launch_ms = ms / LAUNCHES_HEAD
    ops_per_launch = B_HEAD * n * (row // 4)
    sm_mhz = (ck or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    tc_peak, tc_basis = fp4_peak_tflops(peaks)
    tc_tflops = gf2_mma_flops(n, row, B_HEAD) / (launch_ms * 1e-3) / 1e12
    smem_peak = smem_peak_tbs(sm_mhz)

    # ---- the same step through many-table calls (64 batches per persistent
    # launch): reported beside the headline, which reads batch by batch
    multi_call = None
    if "head" in args.legs:
        mjobs = [(dbs[i % COPIES], min(B_HEAD, USERS - b0), dR[b0:b0 + B_HEAD], dO[b0:b0 + B_HEAD])
                 for i, b0 in enumerate(range(0, USERS, B_HEAD))]

        def multi_step():
            for j0 in range(0, len(mjobs), 64):
                talekpir.read_multi_async(mjobs[j0:j0 + 64], stream)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                multi_step()
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0 = talekpir.kernel_launches()
        e0.record(stream)
        for _ in range(args.steps):
            multi_step()
        e1.record(stream)
        mk = talekpir.kernel_launches() - k0
        torch.cuda.synchronize()
        mms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
        multi_call = {"reads_per_s": USERS * world / (mms * 1e-3), "ms_per_step": mms,
                      "launches_per_step": mk / args.steps,
                      "call": "tpir_read_multi_async, 64 batches per call"}

    # ---- the same batches on the Four-Russians kernel (shared-memory-bound)
    m4 = None
    if "head_m4rm" in args.legs:
        for db in dbs:
            db.set_kernel(4)
        mms, _, _ = timed(B_HEAD, max(3, args.steps // 2), 1)
        for db in dbs:
            db.set_kernel(0)
        mms = max_over_ranks(mms)
        m_launch = mms / LAUNCHES_HEAD
        m_tbs = m4rm_smem_bytes(n, row // 4, B_HEAD) / (m_launch * 1e-3) / 1e12
        m4 = {"reads_per_s": USERS * world / (mms * 1e-3), "ms_per_step": mms, "launch_ms": m_launch,
              "roofline": {"bound": "smem", "achieved": m_tbs, "peak": smem_peak, "unit": "TB/s",
                           "frac": m_tbs / smem_peak, "traffic": TRAFFIC_M4RM_B256,
                           "kernel": "m4rm_scan_kernel",
                           "peak_basis": f"{SMS} SMs x {SMEM_BYTES_PER_CLK_PER_SM} B/clk shared memory x {sm_mhz:.0f} MHz"}}

    # ---- the same batches on the register-tiled LOP3 kernel (ALU-bound)
    lop3 = None
    if "head_lop3" in args.legs:
        for db in dbs:
            db.set_kernel(2)
        lms, _, _ = timed(B_HEAD, max(3, args.steps // 2), 1)
        for db in dbs:
            db.set_kernel(0)
        lms = max_over_ranks(lms)
        l_launch = lms / LAUNCHES_HEAD
        l_tops = ops_per_launch / (l_launch * 1e-3) / 1e12
        lop3 = {"reads_per_s": USERS * world / (lms * 1e-3), "ms_per_step": lms,
                "launch_ms": l_launch,
                "roofline": {"bound": "alu", "achieved": l_tops, "peak": alu_peak_tops(sm_mhz),
                             "unit": "Top/s", "frac": l_tops / alu_peak_tops(sm_mhz),
                             "traffic": TRAFFIC_BATCHED_B256, "kernel": "batched_scan_kernel",
                             "peak_basis": f"{SMS} SMs x {LOP3_PER_CLK_PER_SM} LOP3/clk x {sm_mhz:.0f} MHz"}}

    # ---- legs: plain (B=1) and B=32
    legs = {}
    for B, steps, name in ((1, max(2, args.steps // 4), "plain"), (32, max(3, args.steps // 2), "b32")):
        if name not in args.legs:
            legs[str(B)] = {"reads_per_s": float("nan"), "scan_gbs": float("nan")}
            continue
        bms, bd, _ = timed(B, steps, 1)
        bms = max_over_ranks(bms)
        legs[str(B)] = {"reads_per_s": USERS * world / (bms * 1e-3), "ms_per_step": bms}
        if B == 1:
            # average duration of one read = the timed region / reads (events
            # between launches would break their programmatic overlap)
            pl_ms = bms / USERS
            legs["1"]["scan_gbs"] = algo_bytes_per_read / (pl_ms * 1e-3) / 1e9
            legs["1"]["launch_ms"] = pl_ms
        else:
            legs[str(B)]["scan_gbs"] = (USERS / B) * table_bytes / (bms * 1e-3) / 1e9
    legs[str(B_HEAD)] = {"reads_per_s": value, "ms_per_step": ms,
                         "scan_gbs": (USERS / B_HEAD) * table_bytes / (ms * 1e-3) / 1e9,
                         "launch_ms": launch_ms}
    plain_gbs = legs["1"]["scan_gbs"]

    # ---- serialized PIR (Section 6): the same reads with one-time masks
    masked = None
    if "masked" in args.legs:
        masked = {}
        for B, steps in ((B_HEAD, max(3, args.steps // 2)), (1, max(2, args.steps // 4))):
            mms, _, _ = timed(B, steps, 1, masked=True)
            mms = max_over_ranks(mms)
            base = legs[str(B)].get("ms_per_step")
            masked[str(B)] = {"reads_per_s": USERS * world / (mms * 1e-3), "ms_per_step": mms,
                              "overhead_vs_unmasked": (mms / base - 1.0) if base else None}

    # ---- row shards (Section 9.4 scale-out) emulated on this GPU: the table in
    # SHARDS row shards, each batch read by every shard from the same request
    # rows, partial replies XOR-combined by the exchange's combine kernel
    sharded = None
    if "sharded" in args.legs and rank == 0:
        sharded = sharded_leg(talekpir, torch, stream, T, dR, args, legs)

    # ---- end to end through the host-buffer entry point (pinned host memory)
    hR = torch.from_numpy(R.view(np.int64)).pin_memory().numpy().view(np.uint64)
    hO = torch.empty((USERS, row), dtype=torch.uint8).pin_memory().numpy()

    def e2e_call(c):
        # table copy c serves a quarter of the step's reads through the
        # pipelined host-buffer call (batches of B_HEAD; copies overlap scans)
        q = (USERS + COPIES - 1) // COPIES
        b0, nb = c * q, min(q, USERS - c * q)
        rc = L.tpir_read_batch_pipelined(dbs[c].h, hR[b0:b0 + nb].ctypes.data, nb, B_HEAD,
                                         hO[b0:b0 + nb].ctypes.data)
        assert rc == 0, rc

    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(COPIES)

    def e2e_step():
        # a server answering its tables from one host thread each (one tpir_db
        # per thread, as the API allows): one call's copy-in and copy-out
        # overlap another's scans
        list(pool.map(e2e_call, range(COPIES)))

    def e2e_step_one_thread():
        for c in range(COPIES):
            e2e_call(c)
    e2e = None
    if "e2e" in args.legs:
        e2e_steps = max(2, args.steps // 2)
        times = {}
        for name, step in (("threads", e2e_step), ("one_thread", e2e_step_one_thread)):
            for _ in range(args.warmup):
                step()
            barrier()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                step()
            times[name] = max_over_ranks((time.perf_counter() - t0) / e2e_steps)
        e2e = {"value": USERS * world / times["threads"], "unit": "reads/s",
               "h2d_bytes_per_step": int(USERS * words * 8), "d2h_bytes_per_step": int(USERS * row),
               "host_threads": COPIES, "value_one_thread": USERS * world / times["one_thread"]}
    pool.shutdown()

    # ---- short serve run (continuous batching), rank 0 only
    serve = None
    if "serve" in args.legs and rank == 0:
        serve = serve_leg(talekpir, synth, args.serve_rate, args.serve_seconds)

    # ---- CPU baseline: the oracle on a bounded sample, rank 0 only
    cpu = None
    if rank == 0 and "cpu" in args.legs:
        cpu = cpu_leg(T, R)

    getupdates = getupdates_leg(talekpir, synth, torch, stream) if ("getupdates" in args.legs and rank == 0) else None
    writes = writes_leg(talekpir, synth) if ("writes" in args.legs and rank == 0) else None

    sweep = None
    if "serve_sweep" in args.legs and rank == 0:
        sweep = serve_sweep_leg(talekpir, synth, torch, stream, args)
    multi = multi_leg(talekpir, synth, torch, stream, args) if "multi" in args.legs else None
    large = large_leg(talekpir, synth, torch, stream, args, hbm_peak) if "large" in args.legs else None

    gpu_launches = head_launches  # the library's own kernel launches in the timed region, counted
    if rank == 0:
        line = {
            "metric": "pir_reads_per_s", "value": value, "unit": "reads/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "e2m1 0/1 operands (unit block scales), fp32 exact integer counts (replies u8, bit-exact)",
            "data": "synthetic", "config": workload_config(args),
            "e2e": e2e, "gpu_launches": gpu_launches,
            "clocks": ck,
            "roofline": {"bound": "tensor", "achieved": tc_tflops, "peak": tc_peak,
                         "unit": "TFLOP/s", "frac": tc_tflops / tc_peak,
                         "traffic": TRAFFIC_GF2MMA_B256,
                         "kernel": "gf2_mma_pair_kernel (tcgen05 cta_group::2 kind::mxf4, e2m1 0/1 operands)",
                         "peak_basis": tc_basis,
                         "frac_of_issue_rate": tc_tflops / (FP4_ISSUE_PFLOPS_2070 * 1e3 * sm_mhz / 2070.0),
                         "issue_rate_basis": "back-to-back kind::mxf4 N=224 K=64 MMAs (M=128 per SM, or M=256 per CTA pair) on all SMs, 9.70 PFLOP/s at 2070 MHz (tests/test_gpu_mma_rates.py), scaled to the sampled clock",
                         "lop3_equivalent_tops": ops_per_launch / (launch_ms * 1e-3) / 1e12},
            "head_m4rm": m4,
            "head_lop3": lop3,
            "roofline_plain": {"bound": "hbm", "achieved": plain_gbs, "peak": hbm_peak,
                               "unit": "GB/s", "frac": plain_gbs / hbm_peak,
                               "traffic": TRAFFIC_PLAIN_B1,
                               "kernel": "plain_tma_kernel", "peak_basis": "of measured" if peaks else "of fallback"},
            "legs": legs,
            "head_many_table_calls": multi_call,
            "masked": masked,
            "sharded": sharded,
            "autotune": tune,
            "speedup_batched_vs_plain": value / legs["1"]["reads_per_s"],
            "serve": serve,
            "multi_table": multi,
            "serve_sweep": sweep,
            "getupdates": getupdates,
            "writes": writes,
            "large_table": large,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    for db in dbs:
        db.close()
    if world > 1:
        dist.destroy_process_group()


SHARDS = 4


def cpu_leg(T, R) -> dict:
    """CPU baselines on this host, reported only: the oracle (single-threaded
    C, one pass over the table per read) on 8 reads, and the paper-style
    multi-core engine (Section 9.2's CPU server: one pass over the table per
    batch, buckets split over pthreads on every core) on batches of B_HEAD
    reads of the same table."""
    import oracle
    n, d, z = N_BUCKETS, D_SLOTS, MSG_BYTES
    oracle.build()
    oracle.build_engine()
    nproc = os.cpu_count() or 1
    sample = 8
    t0 = time.perf_counter()
    oracle.read_batch(T, n, d, z, R[:sample])
    cdt = time.perf_counter() - t0
    oracle.engine_read_batch(T, n, d, z, R[:B_HEAD], threads=nproc)   # pages in, warms up
    reps = 3
    t0 = time.perf_counter()
    for r in range(reps):
        oracle.engine_read_batch(T, n, d, z, R[(r + 1) * B_HEAD:(r + 2) * B_HEAD], threads=nproc)
    edt = (time.perf_counter() - t0) / reps
    return {"value": sample / cdt, "unit": "reads/s", "cores": 1, "kind": "oracle",
            "sample": f"{sample} reads of the 128 MiB table (single-threaded C)",
            "host_cores": nproc,
            "multi_core": {"value": B_HEAD / edt, "unit": "reads/s", "cores": nproc,
                           "threads": nproc,
                           "kind": "paper-style batched CPU scan (pthreads, one table pass per batch)",
                           "sample": f"{reps} batches of {B_HEAD} reads of the 128 MiB table"}}


def getupdates_leg(talekpir, synth, torch, stream) -> dict:
    """Compressed GetUpdates: a window of 8 Bloom deltas over m = 2^24 bits,
    131 072 writes x 4 positions per delta (1 M writes in the window), each
    delta and the global interest vector Rice-coded on the device."""
    m, kpos, window, per = 1 << 24, 4, 8, 1 << 17
    db = talekpir.DB(64, 4, 64)
    db.bloom_create(m, kpos, window, per)
    keys = synth.write_keys(window * per, seed=13)
    pos = synth.bloom_positions(keys, m, kpos)
    for i in range(0, len(pos), 1 << 16):
        assert db.bloom_insert_batch(pos[i:i + (1 << 16)]) == talekpir.OK
    out = {"m_bits": m, "k": kpos, "window": window, "writes_per_delta": per,
           "raw_bytes": m // 8}
    _, nb, cnt, k = db.bloom_get_compressed(1)
    out.update({"delta_bits_set": cnt, "delta_compressed_bytes": (nb + 7) // 8, "delta_rice_k": k})
    _, nb, cnt, k = db.bloom_get_compressed(0)
    out.update({"global_bits_set": cnt, "global_compressed_bytes": (nb + 7) // 8, "global_rice_k": k})
    # device time of one delta's encoding (a delta is encoded once and served
    # to every client that asks)
    vec = torch.zeros(m // 64, dtype=torch.int64, device="cuda")
    vec.copy_(torch.from_numpy(db.bloom_get().view(np.int64)))
    cap = m // 4
    dout = torch.empty(cap // 4, dtype=torch.int32, device="cuda")
    res = torch.empty(3, dtype=torch.int64, device="cuda")
    for _ in range(3):
        talekpir.rice_encode_async(vec, m, dout, cap, res, -1, stream.cuda_stream)
    ms = _events_ms(torch, stream, lambda: talekpir.rice_encode_async(vec, m, dout, cap, res, -1,
                                                                       stream.cuda_stream), 10)
    out["global_encode_us"] = ms * 1000
    db.close()
    return out


def writes_leg(talekpir, synth) -> dict:
    """Cuckoo writes (Section 5.3) and interest-vector updates (Section 7) on
    the paper-scale table (n = 32768 x 4 x 1 KiB), collection capacity 95 % of
    the slots (the load of the paper's cost table), at most 500 evictions: the
    table is first filled to 90 %, then 4096 writes are timed in batches of
    256 (tpir_write_batch: host placement, then the slot moves and payloads on
    the device) and 256 more one by one (tpir_write: host time per call, the
    moves and message travelling in the launch), then 256 each followed by a
    wait for its completion (tpir_db_sync) and 256 through tpir_write_noalloc
    (message in a device buffer) each followed by a wait on its stream: the
    medians are the completion latencies; interest vectors of
    m = 2^20 bits, k = 4, 65 536 writes' positions per call.  The calls are
    synchronous: host wall-clock."""
    n, d, z = N_BUCKETS, D_SLOTS, MSG_BYTES
    cap = int(0.95 * n * d)
    fill = int(0.90 * n * d)
    timed_batch, timed_single, per = 4096, 256, 256
    db = talekpir.DB(n, d, z)
    db.set_policy(cap, 500, 11)
    keys = synth.write_keys(fill + timed_batch + 3 * timed_single, seed=12)
    b1, b2 = synth.bucket_pairs(keys, n)
    M = synth.messages(4096, z, seed=12)  # payload bytes do not change the cost
    for i in range(0, fill, 4096):
        j = min(fill, i + 4096)
        db.write_batch(b1[i:j], b2[i:j], M[: j - i])
    ev_total, efull = 0, 0
    t0 = time.perf_counter()
    for i in range(fill, fill + timed_batch, per):
        st, ev = db.write_batch(b1[i:i + per], b2[i:i + per], M[:per])
        ev_total += int(ev.sum())
        efull += int((st != talekpir.OK).sum())
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    for i in range(fill + timed_batch, fill + timed_batch + timed_single):
        rc, ev = db.write(int(b1[i]), int(b2[i]), M[i % 4096])
        ev_total += ev
        efull += int(rc != talekpir.OK)
    db.sync()
    ts = time.perf_counter() - t0
    # completion latency: each write followed by a wait for its moves
    lat = []
    base = fill + timed_batch + timed_single
    for i in range(base, base + timed_single):
        t1 = time.perf_counter()
        rc, ev = db.write(int(b1[i]), int(b2[i]), M[i % 4096])
        db.sync()
        lat.append(time.perf_counter() - t1)
        ev_total += ev
        efull += int(rc != talekpir.OK)
    # the write that allocates nothing: message from a device buffer, moves
    # in the launch, on a caller's stream; completion latency per call
    import torch
    nstream = torch.cuda.Stream()
    dM = torch.from_numpy(M[:timed_single]).cuda()
    lat_na = []
    base += timed_single
    for j, i in enumerate(range(base, base + timed_single)):
        t1 = time.perf_counter()
        ev_na = ctypes.c_uint32(0)
        rc = talekpir.lib().tpir_write_noalloc(db.h, int(b1[i]), int(b2[i]), dM[j].data_ptr(),
                                               ctypes.byref(ev_na), nstream.cuda_stream)
        nstream.synchronize()
        lat_na.append(time.perf_counter() - t1)
        ev_total += ev_na.value
        efull += int(rc != talekpir.OK)
    db.bloom_create(1 << 20, 4, 1, 0)
    pos = synth.bloom_positions(keys[:65536], 1 << 20, 4)
    assert db.bloom_insert_batch(pos) == talekpir.OK
    t0 = time.perf_counter()
    for _ in range(10):
        assert db.bloom_insert_batch(pos) == talekpir.OK
    tbl = (time.perf_counter() - t0) / 10
    db.close()
    return {"table": "n=32768 x 4 x 1024 B, capacity 95 % of slots, filled to 90 %",
            "batched_writes_per_s": timed_batch / tb, "batch": per,
            "batched_us_per_write": tb / timed_batch * 1e6,
            "single_write_us": ts / timed_single * 1e6,
            "single_write_latency_us": statistics.median(lat) * 1e6,
            "noalloc_write_latency_us": statistics.median(lat_na) * 1e6,
            "mean_evictions": ev_total / (timed_batch + 3 * timed_single), "efull": efull,
            "interest_vector_updates_per_s": 65536 / tbl, "interest_vector_m_bits": 1 << 20,
            "interest_vector_k": 4}


def sharded_leg(talekpir, torch, stream, T, dR, args, legs) -> dict:
    """The paper-scale table split into SHARDS row shards on one GPU; every
    batch of B_HEAD requests is read by all shards (full-length request rows)
    and the partial replies XOR-combined.  Against the unsharded B_HEAD step."""
    n, d, z = N_BUCKETS, D_SLOTS, MSG_BYTES
    row = d * z
    # COPIES rotated copies of every shard, as the unsharded step rotates tables
    copies = []
    for _ in range(COPIES):
        shards = []
        for begin, rows in talekpir.shard_plan(n, SHARDS):
            db = talekpir.DB(rows, d, z, shard=(n, begin))
            db.load(T[begin:begin + rows])
            shards.append(db)
        copies.append(shards)
    nb = (USERS + B_HEAD - 1) // B_HEAD
    parts = torch.empty((SHARDS, B_HEAD, row), dtype=torch.uint8, device="cuda")
    out = torch.empty((USERS, row), dtype=torch.uint8, device="cuda")
    views = [parts[i] for i in range(SHARDS)]

    def step(combine=True):
        for i in range(nb):
            b0 = i * B_HEAD
            m = min(B_HEAD, USERS - b0)
            for k, db in enumerate(copies[i % COPIES]):
                db.read_batch_async(dR[b0:b0 + m], m, parts[k, :m], stream)
            if combine:
                talekpir.xor_combine([v[:m] for v in views], m * row, out[b0:b0 + m],
                                     stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    steps = max(3, args.steps // 2)
    ms = _events_ms(torch, stream, step, steps)
    ms_nocomb = _events_ms(torch, stream, lambda: step(False), steps)
    base = legs.get(str(B_HEAD), {}).get("ms_per_step")
    for shards in copies:
        for db in shards:
            db.close()
    return {"shards": SHARDS, "batch": B_HEAD, "reads_per_s": USERS / (ms * 1e-3),
            "ms_per_step": ms, "ms_partials_only": ms_nocomb,
            "combine_ms_per_step": ms - ms_nocomb,
            "overhead_vs_unsharded": (ms / base - 1.0) if base else None}


def _events_ms(torch, stream, fn, reps):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def multi_leg(talekpir, synth, torch, stream, args) -> dict:
    """64 uneven tables (n = 2^U(10,17) buckets, d in {2,4,8}, messages of
    256/1024/4096 bytes, 16..512 reads each): all reads in one captured graph
    holding one persistent launch per kernel kind (LOP3 for batches below 48,
    the tensor-core kernel for the rest, one launch per request-staging
    mode), against 64 separate launches each taking the automatic choice."""
    shapes = synth.multi_table_shapes(64, seed=3)
    jobs, dbs, total_bytes, reads, ops = [], [], 0, 0, 0
    for i, (n, d, z, B) in enumerate(shapes):
        # the same seeded inputs as the parity test of this workload
        db = talekpir.DB(n, d, z)
        T = synth.table_bytes_torch(n, d, z, seed=3, table=i)
        db.load_async(T, stream)
        torch.cuda.synchronize()
        del T
        R = torch.from_numpy(synth.random_bits(B, n, seed=3, table=i).view(np.int64)).cuda()
        O = torch.empty((B, d * z), dtype=torch.uint8, device="cuda")
        jobs.append((db, B, R, O))
        dbs.append(db)
        total_bytes += n * d * z
        reads += B
        ops += B * n * d * z // 4
    def graph_time():
        g = talekpir.MultiGraph(jobs)
        for _ in range(args.warmup):
            g.launch(stream)
        ms = _events_ms(torch, stream, lambda: g.launch(stream), max(3, args.steps))
        g.close()
        return ms

    # the built-in choices first, then the autotuner's: one trial per (row
    # width, batch-size class), on the class's smallest table (larger tables
    # take the plan of the nearest size class)
    graph_ms_builtin = graph_time()
    tuned = 0
    kernels_chosen = {}
    if not args.no_autotune:
        seen = {}
        for (db, B, R, O) in jobs:
            key = (db.row_bytes, max(1, (B - 1).bit_length()))
            if key not in seen or db.n < seen[key][0].n:
                seen[key] = (db, B)
        for db, B in seen.values():
            r = db.autotune(B, reps=2)
            k = {1: "plain", 2: "lop3", 4: "four_russians", 5: "tensor"}.get(r["kernel"], str(r["kernel"]))
            kernels_chosen[k] = kernels_chosen.get(k, 0) + 1
        tuned = len(seen)
    graph_ms = graph_time() if tuned else graph_ms_builtin

    def separate():
        for (db, B, R, O) in jobs:
            db.read_batch_async(R, B, O, stream)
    for _ in range(2):
        separate()
    sep_ms = _events_ms(torch, stream, separate, max(2, args.steps // 2))
    talekpir.tune_clear()
    for db in dbs:
        db.close()
    return {"tables": len(shapes), "table_bytes": total_bytes, "reads": reads,
            "tuned_classes": tuned, "tuned_kernels": kernels_chosen,
            "graph_ms_builtin_choice": graph_ms_builtin,
            "graph_ms": graph_ms, "separate_ms": sep_ms,
            "tuning_gain": graph_ms_builtin / graph_ms - 1.0,
            "reads_per_s_graph": reads / (graph_ms * 1e-3),
            "reads_per_s_separate": reads / (sep_ms * 1e-3),
            # 32-bit XOR-AND operations of the plain product per second (the
            # tensor-core jobs do the product on tensor cores, so this can
            # pass the LOP3 peak) and the product's 0/1 multiply-adds as flops
            # (2 per request bit x table bit), against the tensor-core roofline
            "lop3_equivalent_tops_graph": ops / (graph_ms * 1e-3) / 1e12,
            "product_tflops_graph": 64.0 * ops / (graph_ms * 1e-3) / 1e12}


def large_leg(talekpir, synth, torch, stream, args, hbm_peak) -> dict:
    """n = 2^20 buckets x 4 x 1 KiB (4 GiB): B = 1024 packed request rows in one
    batched pass (the GF(2) product), and single plain reads (HBM stream)."""
    n, d, z, B = 1 << 20, 4, 1024, 1024
    # the same seeded inputs as the parity test of this workload
    db = talekpir.DB(n, d, z)
    T = synth.table_bytes_torch(n, d, z, seed=0, table=4)
    db.load_async(T, stream)
    torch.cuda.synchronize()
    del T
    R = torch.from_numpy(synth.random_bits(B, n, seed=4).view(np.int64)).cuda()
    O = torch.empty((B, d * z), dtype=torch.uint8, device="cuda")
    db.read_batch_async(R, B, O, stream)
    bms = _events_ms(torch, stream, lambda: db.read_batch_async(R, B, O, stream), 3)
    db.set_kernel(4)
    db.read_batch_async(R, B, O, stream)
    mms = _events_ms(torch, stream, lambda: db.read_batch_async(R, B, O, stream), 2)
    db.set_kernel(2)
    db.read_batch_async(R, B, O, stream)
    lms = _events_ms(torch, stream, lambda: db.read_batch_async(R, B, O, stream), 2)
    db.set_kernel(0)
    db.read_batch_async(R[:1], 1, O[:1], stream)
    pms = _events_ms(torch, stream, lambda: db.read_batch_async(R[:1], 1, O[:1], stream), 16)
    db.close()
    ops = B * n * d * z // 4
    tb = n * d * z
    return {"n": n, "d": d, "msg_bytes": z, "B": B, "table_bytes": tb,
            "batched_ms": bms, "batched_reads_per_s": B / (bms * 1e-3),
            "batched_lop3_equivalent_tops": ops / (bms * 1e-3) / 1e12,
            "batched_kernel": "gf2_mma_kernel (automatic choice at B = 1024)",
            "batched_tensor_tflops": gf2_mma_flops(n, d * z, B) / (bms * 1e-3) / 1e12,
            "m4rm_kernel_ms": mms, "m4rm_kernel_reads_per_s": B / (mms * 1e-3),
            "lop3_kernel_ms": lms, "lop3_kernel_reads_per_s": B / (lms * 1e-3),
            "lop3_kernel_frac_at_2070MHz": ops / (lms * 1e-3) / 1e12 / alu_peak_tops(2070.0),
            "m4rm_smem_frac_at_2070MHz": m4rm_smem_bytes(n, d * z // 4, B) / (mms * 1e-3) / 1e12 / smem_peak_tbs(2070.0),
            "plain_ms": pms, "plain_reads_per_s": 1.0 / (pms * 1e-3),
            "plain_scan_gbs": (tb + n / 8 + d * z) / (pms * 1e-3) / 1e9,
            "plain_frac_hbm": (tb + n / 8 + d * z) / (pms * 1e-3) / 1e9 / hbm_peak}


def _drive(srv, talekpir, synth, tids, sizes, reqs, msgs, rate, seconds, seed, m_bits, k):
    """Open-loop Poisson ops at `rate` reads/s plus 10% writes (each with k
    interest-vector positions); latency from each op's scheduled arrival."""
    import threading
    count = int(rate / 0.9 * seconds)
    arr = synth.poisson_arrivals(rate / 0.9, count, seed=seed)
    is_w = synth.op_mix(count, 0.1, seed=seed)
    tsel = (synth.stream(synth.stream_key(seed, 99), count) % np.uint64(len(tids))).astype(np.int64)
    keys = synth.write_keys(count, seed=seed + 1)
    outs = [np.empty(4096, dtype=np.uint8) for _ in range(4096)]
    done = [0]

    def poller():
        while done[0] < count:
            done[0] += len(srv.poll())
            time.sleep(0.0005)

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.monotonic_ns()
    for i in range(count):
        ta = t0 + int(arr[i] * 1e9)
        while time.monotonic_ns() < ta:
            pass
        t = int(tsel[i])
        if is_w[i]:
            b1, b2 = synth.bucket_pairs(keys[i:i + 1], sizes[t])
            pos = synth.bloom_positions(keys[i:i + 1], m_bits, k)[0]
            while srv.submit_write(tids[t], int(b1[0]), int(b2[0]), msgs[i % len(msgs)], i, pos,
                                   ta) == talekpir.EAGAIN:
                time.sleep(0.0001)
        else:
            while srv.submit_read(tids[t], reqs[t][i % len(reqs[t])], outs[i % 4096], i,
                                  ta) == talekpir.EAGAIN:
                time.sleep(0.0001)
    srv.drain()
    th.join()
    return count


def serve_sweep_leg(talekpir, synth, torch, stream, args) -> dict:
    """Serving under a 64 GiB HBM budget: tables of 2^15..2^18 buckets x 4 x
    1 KiB (seeded uniform payload) are added until the budget refuses one;
    then open-loop Poisson reads at each rate of --sweep-rates for
    --sweep-seconds, with 10% writes (max 500 evictions, k = 4 interest-vector
    positions in m = 2^20 bits).  Latency runs from each op's scheduled
    arrival to its completion (no coordinated omission)."""
    m_bits, k = 1 << 20, 4
    srv = talekpir.Server(hbm_budget_bytes=64 << 30, max_batch=256, max_inflight=4)
    sizes, tids = [], []
    cycle = [1 << 15, 1 << 16, 1 << 17, 1 << 18]
    t_fill = time.perf_counter()
    while True:
        n = cycle[len(tids) % 4]
        try:
            tid = srv.add_table(n, 4, 1024)
        except talekpir.TpirError:
            break
        db = srv.table(tid)
        T = synth.table_bytes_torch(n, 4, 1024, seed=5, table=len(tids))   # seeded payload
        db.load_async(T, stream)
        torch.cuda.synchronize()
        del T
        db.bloom_create(m_bits, k, window=4, writes_per_delta=1000)
        sizes.append(n)
        tids.append(tid)
    t_fill = time.perf_counter() - t_fill
    reqs = [synth.random_bits(16, n, seed=7, table=i) for i, n in enumerate(sizes)]
    msgs = synth.messages(64, 1024, seed=8)
    rates = [float(x) for x in args.sweep_rates.split(",") if x]
    res = []
    for rate in rates:
        srv.reset_stats()
        ops = _drive(srv, talekpir, synth, tids, sizes, reqs, msgs, rate, args.sweep_seconds,
                     seed=int(rate), m_bits=m_bits, k=k)
        st = srv.stats()
        res.append({"offered_reads_per_s": rate, "reads_per_s": st.reads_per_s,
                    "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "max_ms": st.max_ms,
                    "reads": st.reads_done, "writes": st.writes_done, "failed": st.failed,
                    "rejected": st.rejected, "launches": st.launches,
                    "mean_batch": st.mean_batch, "ops": ops,
                    "launches_by_kernel": {"plain": st.kernel_launches[1],
                                           "lop3": st.kernel_launches[2],
                                           "four_russians": st.kernel_launches[4],
                                           "tensor": st.kernel_launches[5]}})
    total = int(sum(n * 4096 for n in sizes))
    srv.close()
    return {"tables": len(sizes), "table_bytes": total, "hbm_budget": 64 << 30,
            "fill_s": t_fill, "seconds_per_rate": args.sweep_seconds, "rates": res}


def serve_leg(talekpir, synth, rate: float, seconds: float) -> dict:
    """Open-loop Poisson arrivals (10% writes with k = 4 Bloom positions) over
    eight resident tables of 2^15..2^18 buckets x 4 x 1 KiB; latency is
    measured from each op's scheduled arrival time."""
    import threading
    srv = talekpir.Server(hbm_budget_bytes=64 << 30, max_batch=256, max_inflight=2)
    sizes = [1 << 15, 1 << 16, 1 << 17, 1 << 18, 1 << 15, 1 << 16, 1 << 17, 1 << 15]
    tids = []
    for s in sizes:
        tid = srv.add_table(s, 4, 1024)
        db = srv.table(tid)
        db.bloom_create(1 << 20, 4, window=4, writes_per_delta=1000)
        tids.append(tid)
    count = int(rate * seconds)
    arr = synth.poisson_arrivals(rate, count, seed=5)
    is_w = synth.op_mix(count, 0.1, seed=5)
    tsel = (synth.stream(synth.stream_key(5, 99), count) % np.uint64(len(tids))).astype(np.int64)
    keys = synth.write_keys(count, seed=6)
    reqs = {t: synth.random_bits(64, sizes[t], seed=7, table=t) for t in tids}
    msg = synth.messages(64, 1024, seed=8)
    outs = np.empty((count, 4096), dtype=np.uint8)
    done = [0]

    def poller():
        while done[0] < count:
            done[0] += len(srv.poll())
            time.sleep(0.0005)

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.monotonic_ns()
    for i in range(count):
        ta = t0 + int(arr[i] * 1e9)
        while time.monotonic_ns() < ta:
            pass
        t = int(tsel[i])
        if is_w[i]:
            b1, b2 = synth.bucket_pairs(keys[i:i + 1], sizes[t])
            pos = synth.bloom_positions(keys[i:i + 1], 1 << 20, 4)[0]
            while srv.submit_write(t, int(b1[0]), int(b2[0]), msg[i % 64], i, pos, ta) == talekpir.EAGAIN:
                time.sleep(0.0001)
        else:
            while srv.submit_read(t, reqs[t][i % 64], outs[i], i, ta) == talekpir.EAGAIN:
                time.sleep(0.0001)
    srv.drain()
    th.join()
    st = srv.stats()
    out = {"offered_reads_per_s": rate * 0.9, "reads_per_s": st.reads_per_s, "p50_ms": st.p50_ms,
           "p99_ms": st.p99_ms, "max_ms": st.max_ms, "reads": st.reads_done,
           "writes": st.writes_done, "failed": st.failed, "launches": st.launches,
           "mean_batch": st.mean_batch, "tables": len(tids),
           "table_bytes": int(sum(s * 4096 for s in sizes))}
    srv.close()
    return out


if __name__ == "__main__":
    main()
