"""Bandwidth-ratio experiment: which family member wins as bandwidth per flop drops.

Sec. 5.2 (Fig. 6) lowers the main-memory bandwidth of one CPU and finds that the
member keeping more of the problem resident in the last-level cache pulls ahead of
Goto's algorithm, by 30-40 % at the lowest bandwidth, while at high bandwidth the
gap disappears.  On one GPU the memory system is fixed, so this sweep moves the
compute-to-bandwidth ratio in the two ways that remain:

* background traffic -- ``momms_stream_copy`` on H SMs of a second stream takes HBM
  bandwidth away from the product running on the other SMs (the counterpart of the
  slower memory setting);
* engine -- the native FP64 DMMA kernel (about 1 TFLOP/s) needs orders of magnitude
  fewer bytes per second than the emulated slice products (about 1.4 PFLOP/s of fp16
  tensor work), so only the latter can become bandwidth-bound.

At every point it times each member -- C2 (Resident C at the L2 level), A2, B2 and
A1 (the blocked, Goto-like order that does not design for L2) -- through the public
C ABI, beside the HBM bytes the I/O model predicts for that member's slice products.

    python -m paper_1904_05717_gb300.experiments [--size 8192] [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import math
import sys

from . import iomodel
from . import momms as M
from . import synthetic as syn

MEMBER_IDS = {"C2": M.MEMBER_C2, "A2": M.MEMBER_A2, "B2": M.MEMBER_B2, "A1": M.MEMBER_A1}


def _events_ms(torch, stream, fn, reps):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    return e0, e1


class Background:
    """HBM traffic on `sms` SMs of its own stream: a streaming copy between two buffers
    larger than L2, repeated long enough to outlast the timed product."""

    def __init__(self, torch, nbytes=1 << 31):
        self.torch = torch
        self.nbytes = nbytes
        self.src = torch.empty(nbytes // 8, dtype=torch.float64, device="cuda").uniform_()
        self.dst = torch.empty_like(self.src)
        self.stream = torch.cuda.Stream()
        self.pass_ms = {}

    def calibrate(self, sms):
        """Time of one copy pass on `sms` SMs alone, and its HBM rate (read + write)."""
        torch = self.torch
        if sms not in self.pass_ms:
            self.launch(sms, 1)
            torch.cuda.synchronize()
            e0, e1 = _events_ms(torch, self.stream, lambda: self.launch(sms, 1), 3)
            torch.cuda.synchronize()
            self.pass_ms[sms] = e0.elapsed_time(e1) / 3
        ms = self.pass_ms[sms]
        return ms, 2.0 * self.nbytes / (ms * 1e-3) / 1e9

    def launch(self, sms, repeats):
        M.check(M.momms_stream_copy(self.dst.data_ptr(), self.src.data_ptr(), self.nbytes, sms, repeats,
                                    self.stream), "momms_stream_copy")


def _operands(torch, m, n, k, seed):
    A = M.DeviceMatrix.from_numpy(syn.matrix("uniform", m, k, seed))
    B = M.DeviceMatrix.from_numpy(syn.matrix("uniform", k, n, seed + 1))
    C = M.DeviceMatrix.from_numpy(syn.matrix("uniform", m, n, seed + 2))
    return A, B, C


DEFAULT_POINTS = ((152, 0), (114, 38), (76, 0), (76, 38), (76, 76))


SCHEMES = {"auto": M.SCHEME_AUTO, "slices": M.SCHEME_SLICES, "moduli": M.SCHEME_MODULI}


def run(size=8192, members=("C2", "A2", "B2", "A1"), points=DEFAULT_POINTS, reps=3, native_size=4096, slices=6,
        engines=("emulated", "native"), check_results=False, scheme="auto"):
    """Times every (engine, point, member); a point is (product CTAs, background SMs).  The
    native kernel keeps its default grid (one CTA per tile) at every point.  Returns one dict
    per measurement.

    With `check_results` each product computed beside background traffic is compared bit
    for bit with the same product computed alone (concurrency must not change it)."""
    import torch

    M.lib()
    sms_total = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    for ctas, H in points:
        if ctas + H > sms_total:
            raise ValueError(f"point {(ctas, H)}: product CTAs plus background SMs exceed {sms_total} SMs")
    bg = Background(torch) if any(H for _, H in points) else None
    stream = torch.cuda.current_stream()
    rows = []
    for engine in engines:
        emulated = engine == "emulated"
        n = size if emulated else native_size
        A, B, C = _operands(torch, n, n, n, syn.workload_seed(1, "A"))
        seen = set()
        for ctas, H in points:
            key = (ctas if emulated else 0, H)
            if key in seen:
                continue  # the native grid ignores the product CTA count
            seen.add(key)
            for mem in members:
                h = M.Handle(mode=M.MODE_EMULATED if emulated else M.MODE_NATIVE, member=MEMBER_IDS[mem],
                             slices=slices if emulated else 0, scheme=SCHEMES[scheme])
                h.set_max_ctas(ctas if emulated else 0)

                def call():
                    M.check(M.momms_gemm_ex(h, 0, 0, n, n, n, 1.0, A.ptr, A.ld, B.ptr, B.ld, 0.0, C.ptr, C.ld,
                                            stream), "momms_gemm_ex")

                call()
                torch.cuda.synchronize()
                alone = C.storage.clone() if check_results else None
                e0, e1 = _events_ms(torch, stream, call, 1)
                torch.cuda.synchronize()
                alone_ms = e0.elapsed_time(e1)
                rep = h.report()
                point = {"engine": engine, "size": n, "member": mem, "background_sms": H,
                         "product_ctas": int(rep["ctas"]), "group": int(rep["group"]), "slices": int(rep["slices"]),
                         "moduli": int(rep["moduli"])}
                if H:
                    pass_ms, alone_gbs = bg.calibrate(H)
                    # enough passes to outlast the timed products even if they slow down 3x
                    repeats = max(1, math.ceil(3.0 * reps * alone_ms / pass_ms) + 1)
                    b0 = torch.cuda.Event(enable_timing=True)
                    b1 = torch.cuda.Event(enable_timing=True)
                    b0.record(bg.stream)
                    bg.launch(H, repeats)
                    b1.record(bg.stream)
                    point["background_alone_gbs"] = alone_gbs
                e0, e1 = _events_ms(torch, stream, call, reps)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                point["ms"] = ms
                point["tflops"] = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
                if H:
                    # the background started before the first product and ended after the last
                    point["background_covered"] = b0.elapsed_time(e0) >= 0.0 and e1.elapsed_time(b1) >= 0.0
                if emulated and rep["moduli"]:
                    # modular encoding: the residue product's operand planes and residue bytes (its
                    # units visit the rows of the A1 member in A2's order)
                    mod = iomodel.modular_dram_bytes(MEMBER_IDS["A2" if mem == "A1" else mem], n, n, n,
                                                     int(rep["moduli"]), ctas=int(rep["ctas"]), group=int(rep["group"]))
                elif emulated:
                    mod = iomodel.emulated_dram_bytes(MEMBER_IDS[mem], n, n, n, int(rep["slices"]),
                                                      ctas=int(rep["ctas"]), group=int(rep["group"]),
                                                      beta_nonzero=False)
                if emulated:
                    point["model_slice_dram_gb"] = mod["total"] / 1e9
                    point["model_gbs_at_measured_time"] = mod["total"] / (ms * 1e-3) / 1e9
                if check_results:
                    point["bitwise_equal_to_alone"] = bool(torch.equal(C.storage, alone))
                rows.append(point)
                h.close()
    return rows


def table(rows):
    """Markdown table: one line per measurement, with the time relative to C2 at the same point."""
    c2 = {(r["engine"], r["product_ctas"] if r["engine"] == "emulated" else 0, r["background_sms"]): r["ms"]
          for r in rows if r["member"] == "C2"}
    out = ["| engine | n | product CTAs | background SMs | member | group | ms | TFLOP/s | ms / C2 | "
           "model product HBM GB | model GB/s at that time | background alone GB/s |",
           "|---|---|---|---|---|---|---|---|---|---|---|---|"]
    for r in rows:
        b = c2.get((r["engine"], r["product_ctas"] if r["engine"] == "emulated" else 0, r["background_sms"]))
        out.append("| {engine} | {size} | {product_ctas} | {background_sms} | {member} | {group} | {ms:.2f} | {tf:.2f} | "
                   "{rel} | {gb} | {gbs} | {bgs} |".format(
                       tf=r["tflops"], rel=f"{r['ms'] / b:.3f}" if b else "-",
                       gb=f"{r['model_slice_dram_gb']:.1f}" if "model_slice_dram_gb" in r else "-",
                       gbs=f"{r['model_gbs_at_measured_time']:.0f}" if "model_gbs_at_measured_time" in r else "-",
                       bgs=f"{r['background_alone_gbs']:.0f}" if "background_alone_gbs" in r else "-", **r))
    return "\n".join(out)


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--size", type=int, default=8192)
    p.add_argument("--native-size", type=int, default=4096)
    p.add_argument("--points", default=",".join(f"{c}:{h}" for c, h in DEFAULT_POINTS),
                   help="comma-separated product_ctas:background_sms pairs")
    p.add_argument("--members", default="C2,A2,B2,A1")
    p.add_argument("--engines", default="emulated,native")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--scheme", default="auto", choices=sorted(SCHEMES))
    p.add_argument("--json", default=None)
    a = p.parse_args(argv)
    points = tuple(tuple(int(v) for v in pt.split(":")) for pt in a.points.split(","))
    rows = run(size=a.size, members=tuple(a.members.split(",")), points=points, reps=a.reps,
               native_size=a.native_size, engines=tuple(a.engines.split(",")), scheme=a.scheme)
    print(table(rows))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rows, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
