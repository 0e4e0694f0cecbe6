"""Benchmark: FP64-accurate GEMM TFLOP/s (2mnk/t) on one GB300, native vs emulated.

Workload (default): square FP64 product C := A*B + C, m = n = k = 8192,
column-major, entries uniform[-1, 1] from the seeded generator; each operand
(512 MB) is larger than L2, so no L2 flush is needed between steps.

A step is one call of the public C ABI (momms_gemm_ex in AUTO mode: the plan
picks the emulated path, whose slice count comes from the data).  The JSON line
carries the device-resident throughput (`value`), the end-to-end throughput with
host buffers (`e2e`), the roofline of the dominant kernel (the tcgen05 slice
product, timed per launch with CUDA events), the native DMMA path measured in
the same run, SM clocks sampled during the timed region, and the CPU oracle
timed on a bounded sample (`cpu_baseline`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--size 8192] [--impl reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU
(replicas; no collective on the data path); value = all ranks' flops / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64-accurate GEMM TFLOP/s (2mnk/t) & % roofline, native vs emulated"

# DRAM bytes (read + write) of one slice-product call (main + tail + fix-up launch) from an ncu
# capture (m=n=k=8192, S=6, member C2, default group), with that call's algorithmic tensor flops;
# other sizes scale it by the tensor flops.  "current" is False once the kernel has changed since
# the capture: `traffic` is then null and the old figure is reported beside it as
# `traffic_last_capture`, until the capture is taken again.
NCU_SLICE_CAPTURE = {"dram_bytes": (27.75e9 + 0.706e9 + 0.087e9) + (1.93e9 + 0.0545e9),
                     "tensor_flops": 21 * 2.0 * 8192 ** 3,
                     "current": False,
                     "source": "ncu DRAM counters of the 8192^3 slice-product call, scaled by tensor flops for "
                               "other sizes; taken before the kernel's current version"}
# The same for the residue-product launch of the modular encoding (m=n=k=8192, 12 moduli): the
# launch of a timed step of this bench (ncu dram__bytes_read.sum 8.929 GB, dram__bytes_write.sum
# 0.802 GB; one-pass metrics, the same command run without ncu first).
NCU_RESIDUE_CAPTURE = {"dram_bytes": 8.9286e9 + 0.8018e9,
                       "tensor_flops": 12 * 2.0 * 8192 ** 3,
                       "current": True,
                       "source": "ncu DRAM counters (read + write) of the 8192^3 residue-product launch (12 moduli) "
                                 "of a timed step, scaled by tensor flops for other sizes"}
UNIT = "TFLOP/s"
SCHEMES = {"auto": 0, "slices": 1, "moduli": 2}  # momms_scheme_t


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--size", type=int, default=8192)
    p.add_argument("--shape", default="square",
                   choices=["square", "rankk", "panel", "backward", "batched", "host", "trsm", "trmm", "syrk"],
                   help="square: m=n=k=size; rankk: m=n=2*size, k=256; panel: m=k=2*size, n=256; "
                        "backward: dA = dC B^T and dB = A^T dC for A 4096x2048, B 2048x4096; "
                        "batched: 2000 problems, m, n, k log-uniform in [32, 2048]; "
                        "host: m=n=k=size with A, B, C in pinned host memory (momms_gemm_host); "
                        "trsm / trmm: lower triangular A size x size, B size x size (momms_trsm / momms_trmm, "
                        "B restored from a copy each step); syrk: C lower += A A^T, A size x size")
    p.add_argument("--block", type=int, default=0, help="momms_gemm_host block size (0 = from the budget)")
    p.add_argument("--host-resident", default="c", choices=["c", "a"],
                   help="momms_gemm_host member at the HBM level: Resident C or Resident A")
    p.add_argument("--host-k", type=int, default=0, help="k of the host shape (0 = size)")
    p.add_argument("--scheme", default="auto", choices=["auto", "slices", "moduli"],
                   help="integer encoding of the emulated product (momms_set_scheme)")
    p.add_argument("--device-gb", type=float, default=0.0, help="momms_gemm_host device budget (0 = half free)")
    p.add_argument("--mode", default="auto", choices=["auto", "native", "emulated"])
    p.add_argument("--member", default="auto", choices=["auto", "C2", "A2", "B2", "A1"])
    p.add_argument("--slices", type=int, default=0, help="emulated slice count (0 = from the data)")
    p.add_argument("--group", type=int, default=0, help="C2 raster group in tile rows (0 = library default)")
    p.add_argument("--ctas", type=int, default=0, help="grid cap of the product launch (0 = library default)")
    p.add_argument("--tile-n", type=int, default=0, choices=[0, 96, 192],
                   help="emulated tile width (momms_set_tile_n; 0 = automatic)")
    p.add_argument("--cta-pairs", default="auto", choices=["auto", "off", "on"],
                   help="residue products on CTA pairs (momms_set_cta_pairs)")
    p.add_argument("--plan", default="device", choices=["device", "host"],
                   help="where the data-driven slice count is chosen (momms_set_plan_on_device)")
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--native-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    return p.parse_args()


def shape_of(args):
    n = args.size
    if args.shape == "rankk":
        return 2 * n, 2 * n, 256
    if args.shape == "panel":
        return 2 * n, 256, 2 * n
    return n, n, n


def workload_name(args):
    m, n, k = shape_of(args)
    kind = {"square": "square", "rankk": "rank-k", "panel": "panel-panel"}.get(args.shape, args.shape)
    return (f"{kind} FP64 GEMM C := A*B + C, m={m} n={n} k={k}, column-major (ld = rows), "
            f"A, B, C uniform[-1,1] (seeded SplitMix64)")


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(mx)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(flops_per_rank, ms_per_step_this_rank, world):
    """Whole-job TFLOP/s: every rank runs the same workload (replicas, weak scaling);
    the time is the slowest rank's."""
    ms = max_over_ranks(ms_per_step_this_rank, world)
    return world * flops_per_rank / (ms * 1e-3) / 1e12, ms


# ----------------------------------------------------------------------------- CPU oracle sample
class OracleSample:
    """The oracle (as it stands) on a column sample of the n^3 workload.

    Column j of C needs all of A and column j of B, so a block of c columns is an
    n x c x n product of the same workload.  The inputs are generated once."""

    def __init__(self, n):
        import oracle
        from paper_1904_05717_gb300 import synthetic as syn
        self.oracle = oracle
        self.n = n
        self.cores = oracle.max_threads()
        self.A = syn.matrix("uniform", n, n, syn.workload_seed(1, "A"))
        # enough columns for the largest sample; column j is column j of the workload
        self.B = syn.matrix("uniform", n, min(n, 4096), syn.workload_seed(1, "B"))
        self.C = syn.matrix("uniform", n, min(n, 4096), syn.workload_seed(1, "C"))
        c = max(self.cores, 8)
        t0 = time.perf_counter()
        self.run(c)
        self.per_col = (time.perf_counter() - t0) / c

    def run(self, cols):
        B = np.asfortranarray(self.B[:, :cols])
        C = np.array(self.C[:, :cols], order="F")  # the oracle updates C in place; keep the workload's C
        t0 = time.perf_counter()
        self.oracle.dgemm(self.A, B, C, 1.0, 1.0)
        return time.perf_counter() - t0

    def columns_for(self, seconds):
        cols = int(max(self.cores, min(self.B.shape[1], seconds / max(self.per_col, 1e-9))))
        return max(self.cores, cols - cols % self.cores)

    def measure(self, seconds):
        cols = self.columns_for(seconds)
        dt = self.run(cols)
        n = self.n
        tflops = 2.0 * n * n * cols / dt / 1e12
        desc = (f"oracle triple loop (p ascending, no FMA, OpenMP over columns) on {cols} of {n} columns "
                f"of the m=n=k={n} product ({2.0 * n * n * cols:.3g} flops, {dt:.2f} s)")
        return tflops, desc


def oracle_error_ratio(A, B, C0, C_gpu, k):
    """max |C_gpu - C_oracle| / bound over the given block of C = A B + C0 (alpha = beta = 1), the
    bound being 4 k u (|A||B| + |C0|)(1 + 4ku) + 2^-1021."""
    import oracle
    A, B, C0 = (np.asfortranarray(x) for x in (A, B, C0))
    Cref = oracle.dgemm(A, B, C0.copy(order="F"), 1.0, 1.0)
    N = oracle.dgemm_abs(A, B)
    u = 2.0 ** -53
    bound = 4.0 * k * u * (N + np.abs(C0)) * (1.0 + 4.0 * k * u) + 2.0 ** -1021
    return float(np.max(np.abs(C_gpu - Cref) / bound))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.size
    sample = OracleSample(n)
    # each step is a bounded sample; the whole run stays within a few minutes
    per_step = max(0.3, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    vals = []
    desc = ""
    for i in range(args.warmup + args.steps):
        v, desc = sample.measure(per_step)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.median(vals) if vals else 0.0
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": sample.cores, "kind": "oracle",
                         "sample": desc + f"; median of {len(vals)} samples"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_side_workload(args):
    """The backward and batched workloads: one step = one momms_gemm_backward (both
    products) or one momms_gemm_batched call on device-resident inputs, CUDA-event timed."""
    import torch

    from paper_1904_05717_gb300 import momms as M
    from paper_1904_05717_gb300 import synthetic as syn

    M.lib(build_if_missing=True)
    stream = torch.cuda.current_stream()
    mode = {"auto": M.MODE_AUTO, "native": M.MODE_NATIVE, "emulated": M.MODE_EMULATED}[args.mode]
    member = {"auto": M.MEMBER_AUTO, "C2": M.MEMBER_C2, "A2": M.MEMBER_A2, "B2": M.MEMBER_B2,
              "A1": M.MEMBER_A1}[args.member]
    h = M.Handle(mode=mode, member=member, slices=args.slices, scheme=SCHEMES[args.scheme])
    h.set_host_resident(1 if args.host_resident == "a" else 0)
    keep = []
    io = {}
    if args.shape == "host":
        m = n = args.size
        k = args.host_k or args.size
        hosts = [torch.from_numpy(np.ascontiguousarray(syn.matrix("uniform", r, c, syn.workload_seed(1, nm)).T)).pin_memory()
                 for r, c, nm in ((m, k, "A"), (k, n, "B"), (m, n, "C"))]
        keep.append(hosts)
        hA, hB, hC = (t.data_ptr() for t in hosts)
        flops = 2.0 * m * n * k
        workload = (f"FP64 GEMM C := A*B + C, m=n={m} k={k}, A, B, C in pinned host memory, uniform[-1,1] "
                    f"(seeded SplitMix64); out-of-core product, Resident {args.host_resident.upper()} at the HBM "
                    f"level, member {args.member} inside each block")

        def step():
            M.check(M.momms_gemm_host(h, m, n, k, 1.0, hA, m, hB, k, 1.0, hC, m, int(args.device_gb * 2 ** 30),
                                      args.block, stream), "momms_gemm_host")
            io.update(h.report())
    elif args.shape in ("trsm", "trmm"):
        m = n = args.size
        A_h = syn.matrix("uniform", m, m, syn.workload_seed(5, "A")) / np.sqrt(m)
        A_h[np.diag_indices(m)] = 1.0 + syn.unit_uniform(syn.workload_seed(5, "C"), m)
        A = M.DeviceMatrix.from_numpy(np.tril(A_h))
        B0 = M.DeviceMatrix.from_numpy(syn.matrix("uniform", m, n, syn.workload_seed(5, "B")))
        B = M.DeviceMatrix(m, n)
        flops = 1.0 * m * m * n
        fn = M.momms_trsm if args.shape == "trsm" else M.momms_trmm
        workload = (f"{'triangular solve B := A^-1 B' if args.shape == 'trsm' else 'triangular product B := A B'}, "
                    f"A {m}x{m} lower (off-diagonal uniform[-1,1]/sqrt(m), diagonal in [1,2]), B {m}x{n} "
                    f"uniform[-1,1] (seeded SplitMix64), restored from a device copy every step (counted); "
                    f"flops m^2 n")

        def step():
            B.storage.copy_(B0.storage)
            M.check(fn(h, M.LEFT, M.LOWER, M.OP_N, M.NON_UNIT, m, n, 1.0, A.ptr, A.ld, B.ptr, B.ld, stream),
                    args.shape)
    elif args.shape == "syrk":
        n = k = args.size
        A = M.DeviceMatrix.from_numpy(syn.matrix("uniform", n, k, syn.workload_seed(6, "A")))
        C = M.DeviceMatrix.from_numpy(syn.matrix("uniform", n, n, syn.workload_seed(6, "C")))
        flops = 1.0 * n * (n + 1) * k
        workload = (f"symmetric rank-k update C := A A^T + C on the lower triangle, n=k={n}, uniform[-1,1] "
                    f"(seeded SplitMix64); flops n (n + 1) k")

        def step():
            M.check(M.momms_syrk(h, M.LOWER, M.OP_N, n, k, 1.0, A.ptr, A.ld, 1.0, C.ptr, C.ld, stream), "syrk")
    elif args.shape == "backward":
        m, k, n = 4096, 2048, 4096
        A = M.DeviceMatrix.from_numpy(syn.matrix("normal", m, k, syn.workload_seed(2, "A")))
        B = M.DeviceMatrix.from_numpy(syn.matrix("normal", k, n, syn.workload_seed(2, "B")))
        G = M.DeviceMatrix.from_numpy(syn.matrix("normal", m, n, syn.workload_seed(2, "dC")))
        gA, gB = M.DeviceMatrix(m, k), M.DeviceMatrix(k, n)
        flops = 2 * 2.0 * m * n * k
        workload = ("backward of C = A B: dA = dC B^T (4096x2048) and dB = A^T dC (2048x4096), A 4096x2048, "
                    "B 2048x4096, dC 4096x4096, N(0,1) (seeded SplitMix64)")

        def step():
            M.check(M.momms_gemm_backward(h, m, n, k, A.ptr, A.ld, B.ptr, B.ld, G.ptr, G.ld, gA.ptr, gA.ld, gB.ptr,
                                          gB.ld, stream), "momms_gemm_backward")
    else:
        count = 2000
        sizes = syn.log_uniform_sizes(syn.workload_seed(4, "A"), count, 32, 2048)
        mats = []
        for i, (m_, n_, k_) in enumerate(sizes):
            m_, n_, k_ = int(m_), int(n_), int(k_)
            mats.append((M.DeviceMatrix.from_numpy(syn.matrix("uniform", m_, k_, 100000 + 3 * i)),
                         M.DeviceMatrix.from_numpy(syn.matrix("uniform", k_, n_, 100001 + 3 * i)),
                         M.DeviceMatrix.from_numpy(syn.matrix("uniform", m_, n_, 100002 + 3 * i))))
        keep.append(mats)
        ms_, ns_, ks_ = ([int(s_[j]) for s_ in sizes] for j in range(3))
        flops = sum(2.0 * a * b * c for a, b, c in zip(ms_, ns_, ks_))
        args_ = dict(m=ms_, n=ns_, k=ks_, alpha=[1.0] * count, A=[t[0].ptr for t in mats], lda=[t[0].ld for t in mats],
                     B=[t[1].ptr for t in mats], ldb=[t[1].ld for t in mats], beta=[1.0] * count,
                     C=[t[2].ptr for t in mats], ldc=[t[2].ld for t in mats])
        workload = ("batched C := A B + C, 2000 problems, m, n, k i.i.d. log-uniform in [32, 2048], "
                    "uniform[-1,1] (seeded SplitMix64)")

        def step():
            M.check(M.momms_gemm_batched(h, stream=stream, **args_), "momms_gemm_batched")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rep = h.report()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    if io:
        workload += (f"; block {io['ooc_block']}, {io['h2d_bytes']} B host->device and {io['d2h_bytes']} B "
                     f"device->host per step")
    line = {"metric": METRIC, "value": flops / (ms * 1e-3) / 1e12, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "mode": args.mode,
                       "path": "emulated" if rep["mode"] == M.MODE_EMULATED else "native",
                       "slices_last_call": int(rep["slices"]), "moduli_last_call": int(rep["moduli"])},
            "roofline": None, "e2e": None, "gpu_launches": int(rep["launches"]) * args.steps,
            "clocks": clk.summary(), "device_status": h.device_status(stream), "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    h.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.shape in ("backward", "batched", "host", "trsm", "trmm", "syrk"):
        return run_side_workload(args)
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_1904_05717_gb300 import momms as M
    from paper_1904_05717_gb300 import synthetic as syn

    M.lib(build_if_missing=True)
    m, n, k = shape_of(args)
    flops = 2.0 * m * n * k
    stream = torch.cuda.current_stream()
    mode = {"auto": M.MODE_AUTO, "native": M.MODE_NATIVE, "emulated": M.MODE_EMULATED}[args.mode]
    member = {"auto": M.MEMBER_AUTO, "C2": M.MEMBER_C2, "A2": M.MEMBER_A2, "B2": M.MEMBER_B2,
              "A1": M.MEMBER_A1}[args.member]

    # inputs generated on the host (seeded), copied once: device-resident for `value`
    A_h = syn.matrix("uniform", m, k, syn.workload_seed(1, "A"))
    B_h = syn.matrix("uniform", k, n, syn.workload_seed(1, "B"))
    C_h = syn.matrix("uniform", m, n, syn.workload_seed(1, "C"))
    dA = M.DeviceMatrix.from_numpy(A_h)
    dB = M.DeviceMatrix.from_numpy(B_h)
    dC = M.DeviceMatrix.from_numpy(C_h)
    dC0 = dC.storage.clone()

    h = M.Handle(mode=mode, member=member, slices=args.slices, scheme=SCHEMES[args.scheme])
    h.set_raster_group(args.group)
    h.set_max_ctas(args.ctas)
    h.set_cta_pairs({"auto": 0, "off": 1, "on": 2}[args.cta_pairs])
    h.set_tile_n(args.tile_n)
    h.set_plan_on_device(1 if args.plan == "device" else 0)

    def step():
        M.check(M.momms_gemm_ex(h, 0, 0, m, n, k, 1.0, dA.ptr, dA.ld, dB.ptr, dB.ld, 1.0, dC.ptr, dC.ld, stream),
                "momms_gemm_ex")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rep = h.report()
    launches_per_step = int(rep["launches"])

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # the dominant product launch of every timed step is bracketed by a CUDA event pair that the
    # library records on the launching stream (momms_set_kernel_timing)
    h.set_kernel_timing(args.steps)
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    value, ms = aggregate_throughput(flops, e0.elapsed_time(e1) / args.steps, world)
    k_total_ms, k_launches = h.kernel_timing()
    h.set_kernel_timing(0)
    clocks = clk.summary()
    status = h.device_status(stream)

    # ---- the dominant kernel: its launch time inside the timed steps (above), and alone (same digits or
    # residues, same launch configuration), per-launch CUDA events
    S, bb = int(rep["slices"]), int(rep["digit_bits"])
    n_mod, op_bits = int(rep["moduli"]), int(rep["operand_bits"])
    roof = None
    if rep["mode"] == M.MODE_EMULATED:
        k_pad = -(-k // 64) * 64
        e = torch.empty(m, dtype=torch.int32, device="cuda"); ef = torch.empty(m, dtype=torch.uint8, device="cuda")
        f = torch.empty(n, dtype=torch.int32, device="cuda"); ff = torch.empty(n, dtype=torch.uint8, device="cuda")
        M.check(M.momms_emu_scale(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr(), stream), "scale")
        M.check(M.momms_emu_scale(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr(), stream), "scale")
        planes = n_mod if n_mod else S
        Ad = torch.empty((planes, m, k_pad), dtype=torch.float16, device="cuda")
        Bd = torch.empty((planes, n, k_pad), dtype=torch.float16, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        if n_mod:
            # modular encoding: the residue planes, then one residue product per modulus
            M.check(M.momms_emu_residues(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr(), op_bits, k,
                                         Ad.data_ptr(), m, k_pad, stream), "residues")
            M.check(M.momms_emu_residues(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr(), op_bits, k,
                                         Bd.data_ptr(), n, k_pad, stream), "residues")
            nbytes = M.momms_emu_scratch_bytes()
            scratch = torch.empty(nbytes // 8, dtype=torch.float64, device="cuda")
            res = torch.empty(n_mod * m * n, dtype=torch.uint8, device="cuda")

            def product():
                M.check(M.momms_emu_residue_gemm(m, n, k, op_bits, Ad.data_ptr(), Bd.data_ptr(), m, n, k_pad,
                                                 int(rep["member"]), res.data_ptr(), scratch.data_ptr(), nbytes,
                                                 st.data_ptr(), stream), "residue gemm")
            products = n_mod
            kernel = ("momms::emu::residue_pair_kernel (tcgen05.mma.cta_group::2 kind::f16, 256 x 192 tiles on CTA "
                      "pairs; modular encoding: one residue product per modulus)" if rep["cta_pairs"] else
                      f"momms::emu::slice_gemm_kernel<{int(rep['tile_n'])}, 0, 1> (tcgen05 kind::f16; modular "
                      f"encoding: one residue product per modulus)")
            capture = NCU_RESIDUE_CAPTURE
        else:
            M.check(M.momms_emu_split(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr(), S, bb, Ad.data_ptr(),
                                      m, k_pad, stream), "split")
            M.check(M.momms_emu_split(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr(), S, bb, Bd.data_ptr(),
                                      n, k_pad, stream), "split")
            nbytes = M.momms_emu_scratch_bytes_for(m, n, k, S)
            scratch = torch.empty(nbytes // 8, dtype=torch.float64, device="cuda")
            Cs = M.DeviceMatrix(m, n)

            def product():
                M.check(M.momms_emu_slice_gemm(m, n, k, S, bb, Ad.data_ptr(), Bd.data_ptr(), m, n, k_pad,
                                               e.data_ptr(), ef.data_ptr(), f.data_ptr(), ff.data_ptr(), 1.0, 0.0,
                                               Cs.ptr, Cs.ld, int(rep["member"]), scratch.data_ptr(), nbytes,
                                               st.data_ptr(), stream), "slice gemm")
            products = S * (S + 1) // 2
            kernel = f"momms::emu::slice_gemm_kernel<{int(rep['tile_n'])}, 0|1, 0, 0> (tcgen05 kind::f16; main + tail launch)"
            capture = NCU_SLICE_CAPTURE
        evs = []
        reps = max(3, min(args.steps, 10))
        for i in range(reps + 1):
            a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            product()
            a1.record(stream)
            if i > 0:  # first launch is a warm-up
                evs.append((a0, a1))
        torch.cuda.synchronize()
        alone_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        # the launch time inside the timed steps is the figure; alone, for comparison
        slice_ms = k_total_ms / k_launches if k_launches else alone_ms
        tensor_flops = products * 2.0 * m * n * k  # algorithmic: every digit-pair / residue product
        achieved = tensor_flops / (slice_ms * 1e-3) / 1e12
        peaks, src = measured_peaks()
        # the steps' product launches run for well under a second at a time: the burst rate bounds them
        peak = float(peaks.get("bf16_tflops"))
        sustained = float(peaks.get("bf16_tflops_sustained", peak))
        traffic = None
        if capture is not None and args.shape == "square" and args.member in ("auto", "C2"):
            traffic = capture["dram_bytes"] * tensor_flops / capture["tensor_flops"]
        stale = capture is not None and not capture.get("current", True)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None if stale else traffic,
                "traffic_source": (capture or {}).get("source"),
                "kernel": kernel,
                "peak_source": f"{src} bf16_tflops (burst; fp16 rate = bf16 rate)",
                "frac_of_sustained": achieved / sustained,
                "algorithmic_flops_per_launch": tensor_flops, "launch_ms": slice_ms,
                "launch_ms_how": (f"CUDA events on the launching stream around the product launch of each of the "
                                  f"{k_launches} timed steps (mean)" if k_launches else
                                  "CUDA events around the product launched alone"),
                "launch_ms_alone": alone_ms}
        if stale:
            roof["traffic_last_capture"] = traffic
        # what the product's MMA instruction alone reaches (operands resident in shared memory, no
        # loads or drains): tcgen05 kind::f16 M 128 x N 192 on every SM (momms_probe_peak kind 2)
        try:
            roof["instruction_probe_tflops"] = M.momms_probe_peak(2, stream)
        except Exception:
            roof["instruction_probe_tflops"] = None
        del Ad, Bd, scratch

    # ---- native FP64 DMMA path on the same inputs (the other half of the metric)
    native = None
    if args.native_steps > 0:
        hn = M.Handle(mode=M.MODE_NATIVE, member=member)
        dC.storage.copy_(dC0)
        M.check(M.momms_gemm_ex(hn, 0, 0, m, n, k, 1.0, dA.ptr, dA.ld, dB.ptr, dB.ld, 1.0, dC.ptr, dC.ld, stream), "native")
        torch.cuda.synchronize()
        n0 = torch.cuda.Event(enable_timing=True); n1 = torch.cuda.Event(enable_timing=True)
        n0.record(stream)
        for _ in range(args.native_steps):
            M.check(M.momms_gemm_ex(hn, 0, 0, m, n, k, 1.0, dA.ptr, dA.ld, dB.ptr, dB.ld, 1.0, dC.ptr, dC.ld, stream),
                    "native")
        n1.record(stream)
        torch.cuda.synchronize()
        native_ms = n0.elapsed_time(n1) / args.native_steps
        native_tflops = flops / (native_ms * 1e-3) / 1e12
        dmma_peak = M.momms_probe_peak(0, stream)
        hn.close()
        native = {"value": native_tflops, "unit": UNIT, "ms_per_gemm": native_ms, "dmma_peak_probe_tflops": dmma_peak,
                  "frac_of_probe": native_tflops / dmma_peak if dmma_peak else None}

    # ---- end to end through the public API with host buffers (pinned), copies inside the timed region.
    # Every step copies its inputs A, B, C host->device and its result C device->host.  Two device
    # buffer sets and a copy stream let step i+1's copies run while step i computes.
    A_p = torch.from_numpy(np.ascontiguousarray(A_h.T)).pin_memory()
    B_p = torch.from_numpy(np.ascontiguousarray(B_h.T)).pin_memory()
    C_p = torch.from_numpy(np.ascontiguousarray(C_h.T)).pin_memory()
    C_out = torch.empty_like(C_p).pin_memory()
    h2d = (m * k + k * n + m * n) * 8
    d2h = m * n * 8
    sets = [(dA, dB, dC), (M.DeviceMatrix(m, k), M.DeviceMatrix(k, n), M.DeviceMatrix(m, n))]
    copy_s = torch.cuda.Stream()  # host -> device
    back_s = torch.cuda.Stream()  # device -> host (the other copy direction, its own engine)
    comp_s = stream
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]
    ev_read = [torch.cuda.Event(), torch.cuda.Event()]

    def h2d_into(i):
        A_, B_, C_ = sets[i % 2]
        with torch.cuda.stream(copy_s):
            if i >= 2:
                copy_s.wait_event(ev_read[i % 2])  # the set's previous result has been read back
            A_.storage.copy_(A_p, non_blocking=True)
            B_.storage.copy_(B_p, non_blocking=True)
            C_.storage.copy_(C_p, non_blocking=True)
            ev_in[i % 2].record(copy_s)

    def e2e_run(count):
        h2d_into(0)
        for i in range(count):
            if i + 1 < count:
                h2d_into(i + 1)
            A_, B_, C_ = sets[i % 2]
            comp_s.wait_event(ev_in[i % 2])
            M.check(M.momms_gemm_ex(h, 0, 0, m, n, k, 1.0, A_.ptr, A_.ld, B_.ptr, B_.ld, 1.0, C_.ptr, C_.ld,
                                    comp_s), "momms_gemm_ex")
            ev_done[i % 2].record(comp_s)
            with torch.cuda.stream(back_s):
                back_s.wait_event(ev_done[i % 2])
                C_out.copy_(C_.storage, non_blocking=True)
                ev_read[i % 2].record(back_s)
        torch.cuda.synchronize()

    e2e_run(2)
    esteps = max(3, min(args.steps, 20))
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_run(esteps)
    e2e_s = time.perf_counter() - t0
    e2e_value, e2e_ms = aggregate_throughput(flops, e2e_s * 1e3 / esteps, world)

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.shape == "square":
        sample = OracleSample(n)
        v, desc = sample.measure(args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": sample.cores, "kind": "oracle", "sample": desc}
        # the error of one step of the timed path against the oracle, on 16 rows and 16 columns of C
        # drawn at random (seeded) over the whole matrix
        dC.storage.copy_(dC0)
        step()
        torch.cuda.synchronize()
        C_gpu = dC.to_numpy()
        rng = np.random.default_rng(20191)
        rows = np.sort(rng.choice(m, size=min(16, m), replace=False))
        cols = np.sort(rng.choice(n, size=min(16, n), replace=False))
        ratio = max(oracle_error_ratio(A_h[rows, :], B_h, C_h[rows, :], C_gpu[rows, :], k),
                    oracle_error_ratio(A_h, B_h[:, cols], C_h[:, cols], C_gpu[:, cols], k))
        accuracy = {"max_error_over_bound": ratio, "rows_checked": [int(x) for x in rows],
                    "columns_checked": [int(x) for x in cols],
                    "bound": "4 k 2^-53 (|A||B| + |C0|)(1 + 4 k 2^-53) + 2^-1021, componentwise",
                    "slices": int(h.report()["slices"]) if h.report()["mode"] == M.MODE_EMULATED else 0,
                    "moduli": int(h.report()["moduli"]), "operand_bits": int(h.report()["operand_bits"])}

    if rank == 0:
        emulated = rep["mode"] == M.MODE_EMULATED
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64",
            "dtype_detail": (("FP64-accurate; emulated path, modular encoding: operands truncated to "
                              f"{op_bits}-bit integers, residues modulo {n_mod} coprime moduli <= 255 as fp16 on "
                              "tcgen05 kind::f16, exact FP32 accumulation drained to int32, Chinese remainder "
                              "reconstruction in integer arithmetic (approximate CRT), one FP64 rounding")
                             if (emulated and n_mod) else
                             (f"FP64-accurate; emulated path: {S} slices of {bb}-bit integer digits in fp16 on "
                              f"tcgen05 kind::f16, exact FP32 accumulation drained to int32, int64/FP64 recombination")
                             if emulated else "native FP64 DMMA"),
            "data": "synthetic",
            "config": {"workload": workload_name(args), "path": "emulated" if emulated else "native",
                       "slices": S, "digit_bits": bb, "moduli": n_mod, "operand_bits": op_bits,
                       "encoding": ("moduli" if n_mod else "slices") if emulated else None,
                       "member": M.MEMBER_NAMES.get(int(rep["member"]), "auto"),
                       "raster_group": int(rep["group"]), "ctas": int(rep["ctas"]),
                       "cta_pairs": int(rep["cta_pairs"]), "plan": args.plan,
                       "l2": "operands exceed L2 (126 MB) at the default size: no flush between steps",
                       "replicas": world},
            "roofline": roof,
            "native": native,
            "emulated_vs_native": (value / world / native["value"]) if (native and emulated) else None,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms, "steps": esteps,
                    "how": "host wall clock over all steps; pinned host buffers; the copies are torch "
                           "tensor copies (cudaMemcpyAsync) around the public call momms_gemm_ex on device "
                           "buffers: the inputs of step i+1 are copied in on one stream and the result of "
                           "step i-1 copied out on another while step i computes (two device buffer sets)"},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "device_status": status,
            "cpu_baseline": cpu,
            "accuracy": accuracy,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
