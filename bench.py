#!/usr/bin/env python
"""Benchmark of the even-odd preconditioned twisted-mass operator on one GB300.

Headline step: one application of the asymmetric even-even operator (eq. 2.2 LHS)
    M_asym = R_ee - kappa^2 H_eo R_oo^-1 H_oe
to a 32^3 x 64 non-degenerate doublet field (kappa = 0.1612, mu-bar = 0.135,
eps-bar = 0.15, antiperiodic time), FP32 storage and arithmetic, 12-real links.  The
step is the two fused launches tm_precond_op makes (tm_dslash with TM_EPI_TWINV, then
TM_EPI_TWXPAY_ASYM), issued through the C ABI with CUDA events between them on the
launching stream.  Flop convention: 1320 per hopping site and flavour; the twist R 48
and R^-1 72 per site and flavour (doublet: 192 and 240 per site), xpay 48 per flavour
-> 5808 flops per even site for the doublet (2808 one flavour).

Printed: one JSON line (rank 0).  Extra keys: per-precision / per-operator table,
CG time-to-solution, roofline of the dominant kernel, oracle CPU baseline, clocks.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_FULL = (32, 32, 32, 64)
KAPPA, MU_ND, EPS_ND, MU_DEG = 0.1612, 0.135, 0.15, 0.004
FLOPS_PER_SITE = {1: 2808, 2: 5808}          # M_asym per even site (flop convention above)
FLOPS_WILSON = 2 * 1320 + 48                 # M_asym at mu = eps = 0 (R = 1): two hops and the xpay
FLOPS_SYM = {1: 2832, 2: 5856}               # M_sym per even site
SPINOR_BYTES = {8: 192, 16: 192, 4: 96, 2: 52}  # per site and flavour; FP16 includes the 4-byte norm
REAL_BYTES = {8: 8, 16: 8, 4: 4, 2: 2}          # storage bytes per real (16 = DF64, a float pair)


def link_reals(prec, recon):
    return 12 if (prec == 16 and recon == 8) else recon  # DF64 keeps 12 reals for recon-8 handles


def asym_bytes(prec, nf, recon):
    """Algorithmic bytes per even site of M_asym: 16 links + 5 spinor passes (each launch reads 8 links
    and the input spinor and writes one; the second also reads x)."""
    return 16 * link_reals(prec, recon) * REAL_BYTES[prec] + 5 * SPINOR_BYTES[prec] * nf


def launch_bytes(prec, nf, recon):
    """(kernel A, kernel B) bytes per output site: A reads 8 links + 1 spinor, writes 1; B also reads x."""
    link = 8 * link_reals(prec, recon) * REAL_BYTES[prec]
    s = SPINOR_BYTES[prec] * nf
    return link + 2 * s, link + 3 * s


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during a timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def kernel_source_hash(clover=False):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1311_4462_gb300", "csrc")
    files = (["tm_core.cuh", "tm_clover.cuh", "tm_dslash.cuh", "tm_dslash_clov_f32.cu"] if clover else
             ["tm_core.cuh", "tm_dslash.cuh", "tm_dslash_f32.cu"])
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic(kernel_key):
    """Per-launch DRAM bytes of the dominant kernel from profiles/traffic.txt, if taken on this source."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(path):
            if line.startswith("#") or not line.strip():
                continue
            key, srchash, nbytes = line.split()[:3]
            if key == kernel_key and srchash == kernel_source_hash(clover=kernel_key.startswith("k_dslash_clov")):
                return float(nbytes)
    except OSError:
        pass
    return None


def aggregate_ranks(total_ms, units_local, world, device=None):
    """Whole-job throughput of independent replicas: the slowest rank's time bounds the job, and
    the work is every rank's units.  Returns (max_ms, units_per_second_total)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms), float(units_local)], dtype=torch.float64,
                         device=device if device is not None else "cpu")
        tmax, tsum = t.clone(), t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        total_ms, units = float(tmax[0].item()), float(tsum[1].item())
    else:
        units = float(units_local)
    return total_ms, units / (total_ms * 1e-3)


# ------------------------------------------------------------------------------------------- ours
def headline_config(args, nf, prec, recon, L, world):
    """The benchmark's workload description, shared by both arms."""
    flops_site = (CLOVER_FLOPS if args.csw else FLOPS_PER_SITE)[nf]
    return {"workload": ("M_asym (eq. 2.2 LHS), non-degenerate doublet %s, kappa=0.1612, mu=0.135, eps=0.15"
                         % "x".join(map(str, L)) if nf == 2 else
                         "M_asym (eq. 2.2 LHS), one flavour %s, kappa=0.1612, mu=0.004"
                         % "x".join(map(str, L))) + ", %s storage, recon-%d" % (args.prec.upper(), recon)
                        + (", clover c_sw=%g" % args.csw if args.csw else ""),
            "lattice": list(L), "flavours": nf, "storage": args.prec, "recon": recon,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2: links 403 MB, each spinor parity 201 MB, no flush",
            "flops_per_even_site": flops_site,
            "bytes_per_even_site": asym_bytes(prec, nf, recon) + (CLOVER_BYTES[prec] if args.csw else 0)}


FORMS = {0: "thread per site", 2: "register pipeline", 3: "register cap 128x4", 4: "register cap 64x8",
         5: "register cap 256x2", 6: "shared-memory staged pipeline (cp.async)",
         7: "shared-memory staged pipeline, 3 buffers", 8: "staged pipeline, flavour-paired hop",
         9: "staged pipeline, 3 buffers, flavour-paired hop"}


def launch_form(table, prec, csw=0.0):
    """The launch form the tune table selects for this precision's no-prologue hopping launches."""
    for e in table.split():
        f = e.split(":")
        if csw and f[0] == prec and f[1] == "c":
            if f[2] == "6":
                return "clover, shared-memory staged pipeline (3 blocks per SM)"
            return "clover, %s blocks per SM" % f[2]
        if not csw and f[0] == prec and f[1] == "0":
            return "%s (variant %s)" % (FORMS.get(int(f[2]), "?"), f[2])
    return "?"


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import inputs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    L = L_FULL
    t0 = time.time()
    U_np = inputs.gauge_field(L, 1002 + rank)
    psi_np = inputs.spinor_field(L, 2, 2002 + rank)
    gen_s = time.time() - t0
    U = torch.from_numpy(U_np).to(dev)
    prec, nf, recon = tmq.PRECS[args.prec], args.nf, args.recon
    if nf == 2:
        p_nd = tmq.Params(L, KAPPA, MU_ND, EPS_ND, flavor=tmq.TM_NDEG_DOUBLET, recon=recon)
    else:
        p_nd = tmq.Params(L, KAPPA, MU_DEG, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=recon)
    g = tmq.Gauge(p_nd, U)
    if args.csw:
        tmq.set_clover(g, args.csw)
    # the full run tunes its launch table; --quick (profiling) keeps the handle's default table so a
    # profiler's kernel filter sees only the benchmark's own launches
    tune_table = tmq.tune_export(g) if args.quick else tmq.autotune(g)
    psi = torch.from_numpy(psi_np if nf == 2 else psi_np[..., :1, :, :].copy()).to(dev)
    xe = tmq.pack(g, psi, 0, prec)
    tmp, out = tmq.Field(g, prec), tmq.Field(g, prec)
    stream = torch.cuda.current_stream()

    def step():
        tmq.dslash(g, tmp, xe, 1, tmq.TM_EPI_TWINV)
        tmq.dslash(g, out, tmp, 0, tmq.TM_EPI_TWXPAY_ASYM, xe)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clk = ClockSampler(dev.index)
    clk.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for k in range(K):
        evs[k][0].record(stream)
        tmq.dslash(g, tmp, xe, 1, tmq.TM_EPI_TWINV)
        evs[k][1].record(stream)
        tmq.dslash(g, out, tmp, 0, tmq.TM_EPI_TWXPAY_ASYM, xe)
        evs[k][2].record(stream)
    e_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    ta = [evs[k][0].elapsed_time(evs[k][1]) for k in range(K)]
    tb = [evs[k][1].elapsed_time(evs[k][2]) for k in range(K)]
    Vh = p_nd.Vh
    flops_site = CLOVER_FLOPS[nf] if args.csw else FLOPS_PER_SITE[nf]
    flops_step = flops_site * Vh
    total_ms, flops_per_s = aggregate_ranks(e_start.elapsed_time(e_end), flops_step * K, world, dev)
    ms_per_step = total_ms / K
    value = flops_per_s / 1e9
    la, lb = launch_bytes(prec, nf, recon)
    if args.csw:  # launch A reads the four clover blocks of L^-1, launch B the two of L
        la, lb = la + CLOVER_BYTES[prec] * 2 // 3, lb + CLOVER_BYTES[prec] // 3
    avg_launch_ms = (sum(ta) + sum(tb)) / (2 * K)
    steps_ms = sorted(a + b for a, b in zip(ta, tb))
    pct = lambda q: round(steps_ms[min(len(steps_ms) - 1, int(q * (len(steps_ms) - 1) + 0.5))], 5)
    achieved = ((la + lb) / 2 * Vh) / (avg_launch_ms * 1e-3) / 1e9
    peak, peak_src = load_peaks()
    traffic = read_traffic("k_dslash%s_%s_%s_r%d_%s" % ("_clov" if args.csw else "", args.prec,
                                                        "nd" if nf == 2 else "deg", recon, "x".join(map(str, L))))

    result = {
        "metric": "TM dslash GFLOPS & % HBM roofline per precision; CG time-to-1e-10 mixed vs FP64",
        "value": round(value, 1), "unit": "GFLOPS", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.prec, "data": "synthetic (seeded SU(3) links exp(0.3 i H), Gaussian spinors)",
        "config": headline_config(args, nf, prec, recon, L, world),
        "gpu_launches": 2 * K,
        "roofline": {"bound": "hbm", "kernel": "%s<%s, %s, recon-%d> (both launches of M_asym; launch form %s)"
                     % ("k_dslash_clov" if args.csw else "k_dslash", args.prec.upper(),
                        "doublet" if nf == 2 else "one flavour", recon, launch_form(tune_table, args.prec, args.csw)),
                     "achieved": round(achieved, 1), "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "bytes_per_launch_algorithmic": (la + lb) / 2 * Vh,
                     "launch_ms": {"twinv": round(statistics.mean(ta), 5), "twxpay": round(statistics.mean(tb), 5)}},
        "clocks": clocks,
        "step_ms_percentiles": {"p10": pct(0.1), "p50": pct(0.5), "p90": pct(0.9),
                                "source": "CUDA events around each step's two launches"},
        "launch_table": tune_table,
    }
    if rank == 0 and not args.quick and (args.prec, nf, recon, L, args.csw) != ("f32", 2, 12, (32, 32, 32, 64), 0.0):
        args.quick = True  # the extra sections describe the default workload only
    if rank == 0 and not args.quick:
        sections = [("e2e", lambda: e2e_ours(args, tmq, g, psi_np, dev, flops_step)),
                    ("per_precision", lambda: per_precision(tmq, U, psi, dev, args)),
                    ("l2_resident_16x16x16x32", lambda: l2_resident_section(tmq, dev, args)),
                    ("table1_analog", lambda: table1_section(tmq, U, psi, dev, args)),
                    ("cg", lambda: cg_section(tmq, g, U, psi, dev, args)),
                    ("multi_rhs", lambda: multi_rhs_section(tmq, U, dev, args)),
                    ("domain_decomposition", lambda: dd_section(tmq, U, psi, dev, args)),
                    ("batching", lambda: batching_section(tmq, U, dev, args)),
                    ("clover", lambda: clover_section(tmq, U, psi, dev, args)),
                    ("differentiation", lambda: force_section(tmq, dev, args)),
                    ("cpu_baseline", lambda: cpu_baseline(U_np, psi_np, args))]
        only = set(args.only.split(",")) if args.only else None
        for name, fn in sections:
            if only is None or name in only:
                result[name] = fn()
    result["input_generation_s"] = round(gen_s, 2)
    g.close()
    return result


def e2e_ours(args, tmq, g, psi_np, dev, flops_step):
    """The same step end to end through the public API with host buffers: each step copies a
    pinned host canonical complex64 field to the device, packs its even sites, applies M_asym,
    unpacks and copies the result field back to pinned host memory.  Steps are double-buffered
    on three streams (copy-in, compute, copy-out), so step k+1's host-to-device copy overlaps
    step k's compute and device-to-host copy; the time is the whole run over the steps.  The
    serial variant (one stream) and the variant that reads / writes the pinned host buffers in
    place from the pack kernels are reported beside it, and so is a client that keeps its host
    fields in the library's own layout (tm_field_upload / tm_field_download: the even sites' bytes,
    contiguous, so the copies run at the CPU-GPU link's rate); the fastest path is the line's e2e."""
    import numpy as np
    import torch

    host_in = torch.from_numpy(psi_np.astype(np.complex64)).pin_memory()
    host_out = [torch.zeros_like(host_in).pin_memory() for _ in range(2)]
    dev_in = [torch.empty(host_in.shape, dtype=torch.complex64, device=dev) for _ in range(2)]
    dev_out = [torch.zeros_like(dev_in[0]) for _ in range(2)]
    prec = tmq.TM_PREC_F32
    xe, tmp, out = tmq.Field(g, prec), tmq.Field(g, prec), tmq.Field(g, prec)
    cur = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_used = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    for e in ev_used + ev_out:
        e.record(cur)

    def run_overlapped(n):
        last = None
        for k in range(n):
            b = k % 2
            s_in.wait_event(ev_used[b])  # dev_in[b] no longer read by step k-2
            with torch.cuda.stream(s_in):
                dev_in[b].copy_(host_in, non_blocking=True)
            ev_in[b].record(s_in)
            cur.wait_event(ev_in[b])
            cur.wait_event(ev_out[b])    # dev_out[b] drained by step k-2's copy-out
            tmq.pack(g, dev_in[b], 0, prec, out=xe)
            tmq.precond_op(g, out, xe, tmp, tmq.TM_PC_ASYM, False)
            tmq.unpack(g, out, 0, canon=dev_out[b])
            ev_used[b].record(cur)
            s_out.wait_event(ev_used[b])
            with torch.cuda.stream(s_out):
                host_out[b].copy_(dev_out[b], non_blocking=True)
            ev_out[b].record(s_out)
            last = ev_out[b]
        cur.wait_event(last)

    def step_serial():
        dev_in[0].copy_(host_in, non_blocking=True)
        tmq.pack(g, dev_in[0], 0, prec, out=xe)
        tmq.precond_op(g, out, xe, tmp, tmq.TM_PC_ASYM, False)
        tmq.unpack(g, out, 0, canon=dev_out[0])
        host_out[0].copy_(dev_out[0], non_blocking=True)

    def step_in_place():
        tmq.pack(g, host_in, 0, prec, out=xe)
        tmq.precond_op(g, out, xe, tmp, tmq.TM_PC_ASYM, False)
        tmq.unpack(g, out, 0, canon=host_out[0])

    # in place on two streams: step k runs on stream k % 2 with its own fields, so the pack of one
    # step (reading host memory) overlaps the unpack of the other (writing host memory)
    streams = [cur, torch.cuda.Stream()]
    fields = [(xe, tmp, out)] + [tuple(tmq.Field(g, prec) for _ in range(3))]
    ev_done = [torch.cuda.Event() for _ in range(2)]

    def run_in_place_overlapped(n):
        ev_start = torch.cuda.Event()
        ev_start.record(cur)
        streams[1].wait_event(ev_start)  # the second stream starts inside the timed region
        for k in range(n):
            b = k % 2
            st = streams[b]
            fx, ft, fo = fields[b]
            with torch.cuda.stream(st):
                tmq.pack(g, host_in, 0, prec, out=fx, stream=st)
                tmq.precond_op(g, fo, fx, ft, tmq.TM_PC_ASYM, False, stream=st)
                tmq.unpack(g, fo, 0, canon=host_out[b], stream=st)
            ev_done[b].record(st)
        cur.wait_event(ev_done[(n - 1) % 2])
        cur.wait_event(ev_done[n % 2])

    # host fields in the library's own layout (FP32 even parity, tm_field_upload / download): the
    # same bytes as the canonical path's even sites, but contiguous, so they move at the copy rate
    hp_in, _ = tmq.host_buffers(g, prec)
    tmq.download(g, tmq.pack(g, dev_in[0].copy_(host_in), 0, prec), hp_in)
    hp_out = [tmq.host_buffers(g, prec)[0] for _ in range(2)]
    xin = [tmq.Field(g, prec) for _ in range(2)]
    xout = [tmq.Field(g, prec) for _ in range(2)]
    torch.cuda.synchronize()

    def run_packed_overlapped(n):
        last = None
        for k in range(n):
            b = k % 2
            s_in.wait_event(ev_used[b])  # xin[b] no longer read by step k-2
            tmq.upload(g, xin[b], hp_in, stream=s_in)
            ev_in[b].record(s_in)
            cur.wait_event(ev_in[b])
            cur.wait_event(ev_out[b])    # xout[b] drained by step k-2's copy-out
            tmq.precond_op(g, xout[b], xin[b], tmp, tmq.TM_PC_ASYM, False)
            ev_used[b].record(cur)
            s_out.wait_event(ev_used[b])
            tmq.download(g, xout[b], hp_out[b], stream=s_out)
            ev_out[b].record(s_out)
            last = ev_out[b]
        cur.wait_event(last)

    n = max(4, min(20, args.steps))

    def timed(fn, steps_fn=None):
        fn(3) if steps_fn is None else [steps_fn() for _ in range(3)]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        if steps_fn is None:
            fn(n)
        else:
            for _ in range(n):
                steps_fn()
        e1.record(cur)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    ms = timed(run_overlapped)
    ms_serial = timed(None, step_serial)
    ms_inplace = timed(None, step_in_place)
    ms_inplace2 = timed(run_in_place_overlapped)
    ms_packed = timed(run_packed_overlapped)
    full = host_in.numel() * 8
    gf = lambda t: round(flops_step / (t * 1e-3) / 1e9, 1)
    copies = {"value": gf(ms), "ms_per_step": round(ms, 4), "h2d_bytes_per_step": full, "d2h_bytes_per_step": full,
              "path": "pinned host complex64 canonical field -> cudaMemcpy -> tm_pack -> tm_precond_op -> tm_unpack "
                      "-> cudaMemcpy to pinned host; double-buffered over copy-in / compute / copy-out streams"}
    in_place = {"value": gf(ms_inplace2), "ms_per_step": round(ms_inplace2, 4), "h2d_bytes_per_step": full // 2,
                "d2h_bytes_per_step": full // 2,
                "path": "tm_pack reads the even sites of the pinned host complex64 canonical field in place over the "
                        "CPU-GPU link -> tm_precond_op -> tm_unpack writes them to pinned host memory in place; "
                        "consecutive steps on two streams"}
    packed = {"value": gf(ms_packed), "ms_per_step": round(ms_packed, 4), "h2d_bytes_per_step": hp_in.numel(),
              "d2h_bytes_per_step": hp_out[0].numel(),
              "path": "pinned host FP32 even-parity field in the library's layout -> tm_field_upload -> "
                      "tm_precond_op -> tm_field_download to pinned host; double-buffered over copy-in / compute / "
                      "copy-out streams"}
    best = min((copies, in_place, packed), key=lambda d: d["ms_per_step"])
    out_d = {"value": best["value"], "unit": "GFLOPS", "ms_per_step": best["ms_per_step"],
             "h2d_bytes_per_step": best["h2d_bytes_per_step"], "d2h_bytes_per_step": best["d2h_bytes_per_step"],
             "path": best["path"],
             "packed_host_fields_double_buffered": packed,
             "staged_copies_double_buffered": copies, "in_place_two_streams": in_place,
             "serial_copies": {"value": gf(ms_serial), "ms_per_step": round(ms_serial, 4)},
             "in_place_one_stream": {"value": gf(ms_inplace), "ms_per_step": round(ms_inplace, 4)}}
    return out_d


def time_op(fn, reps, flush=None):
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def per_precision(tmq, U, psi, dev, args):
    """M_asym, M_sym and adjoints for both doublets, all precisions, recon 12 (and 18/8 for FP32/FP16)."""
    import torch
    peak, _ = load_peaks()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2, zeroed between reps
    rows = []
    L = L_FULL
    for nf, mu, eps in [(2, MU_ND, EPS_ND), (1, MU_DEG, 0.0)]:
        for recon in (12, 18, 8):
            p = tmq.Params(L, KAPPA, mu, eps, flavor=(tmq.TM_NDEG_DOUBLET if nf == 2 else tmq.TM_TWIST_PLUS),
                           recon=recon)
            g = tmq.Gauge(p, U)
            tmq.autotune(g)
            src = psi if nf == 2 else psi[..., :1, :, :].contiguous()
            for prec in (tmq.TM_PREC_F32, tmq.TM_PREC_F16, tmq.TM_PREC_F64, tmq.TM_PREC_DF64):
                if recon == 8 and prec in (tmq.TM_PREC_F64, tmq.TM_PREC_DF64):
                    continue
                xe = tmq.pack(g, src, 0, prec)
                out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
                for pc in (0, 1):
                    for dag in (0, 1):
                        if recon != 12 and (pc or dag):
                            continue
                        if prec == tmq.TM_PREC_DF64 and (pc or dag):
                            continue
                        reps = 3 if prec in (8, 16) else 10
                        ms = time_op(lambda: tmq.precond_op(g, out, xe, tmp, pc, dag), reps, flush)
                        fl = (FLOPS_SYM if pc else FLOPS_PER_SITE)[nf] * p.Vh
                        by = asym_bytes(prec, nf, recon) * p.Vh
                        row = {"op": ("M_sym" if pc else "M_asym") + ("^dag" if dag else ""),
                               "flavours": nf, "prec": {8: "f64", 4: "f32", 2: "f16", 16: "df64"}[prec], "recon": recon,
                               "us": round(ms * 1e3, 1), "gflops": round(fl / (ms * 1e-3) / 1e9, 1),
                               "gbs": round(by / (ms * 1e-3) / 1e9, 1), "hbm_frac": round(by / (ms * 1e-3) / 1e9 / peak, 3)}
                        if prec in (8, 16):
                            row["fp64_alu_frac_of_nominal_1250"] = round(fl / (ms * 1e-3) / 1e9 / 1250.0, 3)
                        rows.append(row)
                del xe, out, tmp
            g.close()
    return rows


def l2_resident_section(tmq, dev, args):
    """M_asym of the 16^3x32 one-flavour lattice (kappa 0.1612, mu 0.004, recon 12) in FP64, FP32 and
    FP16.  Its links (25 MB in FP32) and spinors fit in the 129 MB L2, so the times are reported with
    that label and no HBM fraction; consecutive applications without a flush."""
    import torch
    from paper_1311_4462_gb300 import inputs
    L = (16, 16, 16, 32)
    p = tmq.Params(L, KAPPA, MU_DEG, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    g = tmq.Gauge(p, torch.from_numpy(inputs.gauge_field(L, 1001)).to(dev))
    tmq.autotune(g)
    src = torch.from_numpy(inputs.spinor_field(L, 1, 2001)).to(dev)
    rows = []
    for prec in (tmq.TM_PREC_F64, tmq.TM_PREC_F32, tmq.TM_PREC_F16):
        xe = tmq.pack(g, src, 0, prec)
        out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
        ms = time_op(lambda: tmq.precond_op(g, out, xe, tmp, 0, False), 50)
        by = asym_bytes(prec, 1, 12) * p.Vh
        rows.append({"op": "M_asym", "prec": {8: "f64", 4: "f32", 2: "f16"}[prec], "us": round(ms * 1e3, 2),
                     "gflops": round(FLOPS_PER_SITE[1] * p.Vh / (ms * 1e-3) / 1e9, 1),
                     "algorithmic_gbs": round(by / (ms * 1e-3) / 1e9, 1), "memory": "L2-resident"})
        del xe, out, tmp
    g.close()
    return {"lattice": list(L), "flavours": 1, "recon": 12, "rows": rows,
            "note": "working set inside L2 (no HBM roofline); median of 50 back-to-back applications"}


# Table 1 of the paper (single GTX Titan, 32^3x64, asymmetric operator, GFLOPS) for context
PAPER_TABLE1 = {("double", 12): (184, 190, 163), ("double", 8): (179, 183, 115), ("single", 12): (401, 415, 516),
                ("single", 8): (472, 487, 567), ("half", 12): (732, 759, 879), ("half", 8): (829, 858, 624)}


def table1_section(tmq, U, psi, dev, args):
    """Analog of the paper's Table 1 on GB300: M_asym GFLOPS for Wilson (mu = 0), degenerate and
    non-degenerate twisted mass, double / single / half storage, 12- and 8-real links, 32^3x64."""
    import torch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ops = {"wilson": (1, 0.0, 0.0), "deg_tm": (1, MU_DEG, 0.0), "nd_tm": (2, MU_ND, EPS_ND)}
    precs = {"double": tmq.TM_PREC_F64, "single": tmq.TM_PREC_F32, "half": tmq.TM_PREC_F16}
    rows = []
    for recon in (12, 8):
        handles = {}
        for name, (nf, mu, eps) in ops.items():
            p = tmq.Params(L_FULL, KAPPA, mu, eps, flavor=(tmq.TM_NDEG_DOUBLET if nf == 2 else tmq.TM_TWIST_PLUS),
                           recon=recon)
            handles[name] = (p, tmq.Gauge(p, U), nf)
            tmq.autotune(handles[name][1])
        for pname, prec in precs.items():
            row = {"prec": pname, "recon": recon}
            for name, (p, g, nf) in handles.items():
                src = psi if nf == 2 else psi[..., :1, :, :].contiguous()
                xe = tmq.pack(g, src, 0, prec)
                out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
                ms = time_op(lambda: tmq.precond_op(g, out, xe, tmp, 0, False), 3 if prec == 8 else 10, flush)
                # the Wilson operator counts no twist work (the kernel still multiplies by R = 1)
                fl = FLOPS_WILSON if name == "wilson" else FLOPS_PER_SITE[nf]
                row[name] = round(fl * p.Vh / (ms * 1e-3) / 1e9, 1)
                del xe, out, tmp
            row["paper_kepler_wilson_deg_nd"] = PAPER_TABLE1[(pname, recon)]
            row["flops_per_even_site"] = {"wilson": FLOPS_WILSON, "deg_tm": FLOPS_PER_SITE[1],
                                          "nd_tm": FLOPS_PER_SITE[2]}
            rows.append(row)
        for p, g, nf in handles.values():
            g.close()
    return rows


def cg_section(tmq, g, U, psi, dev, args):
    """Time to a 1e-10 FP64 true residual (normal equations) on the 32^3x64 doublet, asym and sym
    PC: plain FP64 CG vs reliable-update mixed CG with FP16 and FP32 sloppy storage; and the
    16^3x32 one-flavour system with FP64 CG plus odd-site reconstruction."""
    import torch
    from paper_1311_4462_gb300 import inputs

    def run(gg, bp, pc, reps, **kw):
        out = []
        for _ in range(reps):
            xe = tmq.Field(gg, tmq.TM_PREC_F64)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = tmq.solve(gg, xe, bp, pc=pc, tol=1e-10, maxiter=20000, check=False, **kw)
            e1.record()
            torch.cuda.synchronize()
            st["ms"] = e0.elapsed_time(e1)
            out.append(st)
        best = sorted(out, key=lambda d: d["ms"])[len(out) // 2]
        return {"ms": round(best["ms"], 2), "iterations": best["iterations"],
                "reliable_updates": best["reliable_updates"], "true_residual": best["true_residual"],
                "status": best["status"]}

    res = {"tolerance": 1e-10, "residual": "FP64 |bhat - A^dag A x|/|bhat|, A = M_pc, bhat = A^dag b'",
           "links": "recon 12 for FP32 / FP16 / DF64, 18 reals for FP64 (TM_GAUGE_F64_FULL_LINKS)"}
    # the solver's handle: FP64 links uncompressed (the FP64 operator is bound by the FP64 pipe)
    g = tmq.Gauge(g.params, U, f64_full_links=True)
    b = psi
    be, bo = tmq.pack(g, b, 0, tmq.TM_PREC_F64), tmq.pack(g, b, 1, tmq.TM_PREC_F64)
    nd = {}
    for pc, pname in ((0, "asym"), (1, "sym")):
        bp = tmq.Field(g, tmq.TM_PREC_F64)
        tmq.prepare_rhs(g, bp, be, bo, pc, False)
        run(g, bp, pc, 1, solver="mixed", sloppy_prec=tmq.TM_PREC_F16)  # warm-up
        nd[pname] = {
            "fp64_cg": run(g, bp, pc, 1, solver="cg"),
            "mixed_f16": run(g, bp, pc, 3, solver="mixed", sloppy_prec=tmq.TM_PREC_F16),
            "mixed_f32": run(g, bp, pc, 3, solver="mixed", sloppy_prec=tmq.TM_PREC_F32),
            "mixed_f32_df64_true_residual": run(g, bp, pc, 3, solver="mixed", sloppy_prec=tmq.TM_PREC_F32,
                                                true_prec=tmq.TM_PREC_DF64),
        }
        best = min(nd[pname]["mixed_f16"]["ms"], nd[pname]["mixed_f32"]["ms"],
                   nd[pname]["mixed_f32_df64_true_residual"]["ms"])
        nd[pname]["speedup_mixed_vs_fp64"] = round(nd[pname]["fp64_cg"]["ms"] / best, 2)
    res["doublet_32x32x32x64"] = nd
    del be, bo, bp
    g.close()
    # one flavour 16^3x32, kappa 0.1612, mu 0.004: FP64 CG + reconstruction, full-system residual
    L2 = (16, 16, 16, 32)
    p2 = tmq.Params(L2, KAPPA, MU_DEG, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    g2 = tmq.Gauge(p2, torch.from_numpy(inputs.gauge_field(L2, 1001)).to(dev))
    b2 = torch.from_numpy(inputs.spinor_field(L2, 1, 2001)).to(dev)
    be2, bo2 = tmq.pack(g2, b2, 0, tmq.TM_PREC_F64), tmq.pack(g2, b2, 1, tmq.TM_PREC_F64)
    bp2 = tmq.Field(g2, tmq.TM_PREC_F64)
    tmq.prepare_rhs(g2, bp2, be2, bo2, 0, False)
    st64 = run(g2, bp2, 0, 3, solver="cg")
    stmx = run(g2, bp2, 0, 3, solver="mixed", sloppy_prec=tmq.TM_PREC_F16)
    xe = tmq.Field(g2, tmq.TM_PREC_F64)
    tmq.solve(g2, xe, bp2, tol=1e-10)
    xo = tmq.Field(g2, tmq.TM_PREC_F64)
    tmq.reconstruct_odd(g2, xo, bo2, xe)
    re_, ro_ = tmq.Field(g2, tmq.TM_PREC_F64), tmq.Field(g2, tmq.TM_PREC_F64)
    tmq.mat(g2, re_, ro_, xe, xo)
    full = tmq.unpack(g2, re_, 0) + tmq.unpack(g2, ro_, 1)
    fres = float(torch.linalg.vector_norm(full - b2) / torch.linalg.vector_norm(b2))
    res["one_flavour_16x16x16x32"] = {"fp64_cg": st64, "mixed_f16": stmx, "full_system_residual": fres}
    g2.close()
    return res


# clover-twisted-mass (the paper's next step): flops and bytes per even site of M_asym, in the
# flop convention above (hermitian 6x6 block times a vector: 252 flops; L = two blocks per
# flavour plus the twist, L^-1 = four blocks per flavour plus the twist)
CLOVER_CSW = 1.6
CLOVER_FLOPS = {1: 2 * 1320 + (4 * 252 + 48) + (2 * 252 + 48) + 48,
                2: 4 * 1320 + (8 * 252 + 192) + (4 * 252 + 192) + 96}
CLOVER_BYTES = {8: 6 * 36 * 8, 4: 6 * 36 * 4, 2: 6 * (80 + 4)}  # 4 blocks (launch A) + 2 blocks (launch B)


def clover_section(tmq, U, psi, dev, args):
    """TM-clover M_asym / M_sym (c_sw = 1.6) at 32^3x64 for both doublets and all storage precisions,
    and time to 1e-10 of FP64 CG vs mixed FP32 CG for the non-degenerate doublet."""
    import torch
    peak, _ = load_peaks()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    rows = []
    cg = {}
    tables = {}
    for nf, mu, eps in [(1, MU_DEG, 0.0), (2, MU_ND, EPS_ND)]:
        p = tmq.Params(L_FULL, KAPPA, mu, eps, flavor=(tmq.TM_NDEG_DOUBLET if nf == 2 else tmq.TM_TWIST_PLUS),
                       recon=12)
        g = tmq.Gauge(p, U)
        tmq.set_clover(g, CLOVER_CSW)
        tables["flavours_%d" % nf] = tmq.autotune(g)
        src = psi if nf == 2 else psi[..., :1, :, :].contiguous()
        for prec in (tmq.TM_PREC_F32, tmq.TM_PREC_F16, tmq.TM_PREC_F64):
            xe = tmq.pack(g, src, 0, prec)
            out, tmp = tmq.Field(g, prec), tmq.Field(g, prec)
            for pc in (0, 1):
                reps = 3 if prec == 8 else 10
                ms = time_op(lambda: tmq.precond_op(g, out, xe, tmp, pc, False), reps, flush)
                fl = CLOVER_FLOPS[nf] * p.Vh
                by = (asym_bytes(prec, nf, 12) + CLOVER_BYTES[prec]) * p.Vh
                rows.append({"op": "M_sym" if pc else "M_asym", "flavours": nf,
                             "prec": {8: "f64", 4: "f32", 2: "f16"}[prec], "recon": 12, "us": round(ms * 1e3, 1),
                             "gflops": round(fl / (ms * 1e-3) / 1e9, 1), "gbs": round(by / (ms * 1e-3) / 1e9, 1),
                             "hbm_frac": round(by / (ms * 1e-3) / 1e9 / peak, 3)})
            del xe, out, tmp
        if nf == 2:
            be, bo = tmq.pack(g, psi, 0, tmq.TM_PREC_F64), tmq.pack(g, psi, 1, tmq.TM_PREC_F64)
            bp = tmq.Field(g, tmq.TM_PREC_F64)
            tmq.prepare_rhs(g, bp, be, bo, 0, False)

            def solve(**kw):
                xe = tmq.Field(g, tmq.TM_PREC_F64)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st = tmq.solve(g, xe, bp, tol=1e-10, maxiter=20000, check=False, **kw)
                e1.record()
                torch.cuda.synchronize()
                return {"ms": round(e0.elapsed_time(e1), 2), "iterations": st["iterations"],
                        "reliable_updates": st["reliable_updates"], "true_residual": st["true_residual"],
                        "status": st["status"]}

            solve(solver="mixed", sloppy_prec=tmq.TM_PREC_F32)  # warm-up
            cg = {"fp64_cg": solve(solver="cg"), "mixed_f32": solve(solver="mixed", sloppy_prec=tmq.TM_PREC_F32),
                  "mixed_f16": solve(solver="mixed", sloppy_prec=tmq.TM_PREC_F16)}
            cg["speedup_mixed_vs_fp64"] = round(cg["fp64_cg"]["ms"] / min(cg["mixed_f32"]["ms"], cg["mixed_f16"]["ms"]), 2)
        g.close()
    return {"csw": CLOVER_CSW, "lattice": list(L_FULL), "flops_per_even_site": CLOVER_FLOPS,
            "operators": rows, "cg_nd_asym_tol_1e-10": cg, "launch_tables": tables}


def force_section(tmq, dev, args):
    """The differentiation row at 24^3x48 one flavour (kappa 0.1612, mu 0.004): tm_force (the
    su(3)-projected link gradient, canonical output) in FP64 and FP32 with its algorithmic bytes
    and HBM fraction, and the pseudofermion action S = phi^dag (M^dag M)^-1 phi with its
    U-gradient through torch.autograd (two mixed-precision solves to 1e-10, then the force)."""
    import torch
    from paper_1311_4462_gb300 import autograd as tag
    from paper_1311_4462_gb300 import inputs
    peak, _ = load_peaks()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    L = (24, 24, 24, 48)
    p = tmq.Params(L, KAPPA, MU_DEG, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    U = torch.from_numpy(inputs.gauge_field(L, 1003)).to(dev)
    psi = torch.from_numpy(inputs.spinor_field(L, 1, 2003)).to(dev)
    gv = torch.from_numpy(inputs.spinor_field(L, 1, 2103)).to(dev)
    g = tmq.Gauge(p, U)
    V = 2 * p.Vh
    rows = []
    for prec in (tmq.TM_PREC_F64, tmq.TM_PREC_F32):
        w = REAL_BYTES[prec]
        pe, po = tmq.pack(g, psi, 0, prec), tmq.pack(g, psi, 1, prec)
        ge, go = tmq.pack(g, gv, 0, prec), tmq.pack(g, gv, 1, prec)
        out = torch.empty(p.gauge_shape, dtype=torch.complex128 if prec == 8 else torch.complex64, device=dev)
        ms = time_op(lambda: tmq.force(g, pe, po, ge, go, coef=1.0, project=True, out=out), 10, flush)
        # each input field read once, each link once (for the projection), each gradient written once
        by = 2 * V * 24 * w + 4 * V * 12 * w + 4 * V * 18 * w
        rows.append({"prec": {8: "f64", 4: "f32"}[prec], "us": round(ms * 1e3, 1),
                     "gbs": round(by / (ms * 1e-3) / 1e9, 1), "hbm_frac": round(by / (ms * 1e-3) / 1e9 / peak, 3),
                     "bytes_per_launch": by})
    g.close()
    phi = torch.from_numpy(inputs.spinor_field(L, 1, 2203)).to(dev)
    Ug = U.clone().requires_grad_(True)
    times = []
    for _ in range(2):  # the first run warms up
        Ug.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = tag.PseudofermionAction.apply(Ug, phi, p, 1e-10, "mixed")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        S.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        times.append((t1 - t0, t2 - t1))
    return {"lattice": list(L), "force": rows,
            "pseudofermion_action": {"forward_s": round(times[-1][0], 3), "backward_s": round(times[-1][1], 4),
                                     "solves": "two mixed FP32 CG solves to 1e-10 (M^dag z = phi, M X = z)",
                                     "S": float(S.detach())}}


def multi_rhs_section(tmq, U, dev, args):
    """The multi-RHS operator: M_asym on N = 16 right-hand sides (Z2 noise) in one launch per factor,
    32^3x64, one flavour (kappa 0.1612, mu 0.004) and the doublet, FP32 and FP16 storage, recon 12,
    autotuned launch shape; time per source against the single-RHS application.  Amortised bytes per
    even site and source: 16 links x L x w / N + 5 spinor passes x S x N_f (the links are read once
    per site for all N sources)."""
    import torch
    peak, _ = load_peaks()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    N = 16
    rows, tables = [], {}
    for nf, mu, eps in [(1, MU_DEG, 0.0), (2, MU_ND, EPS_ND)]:
        p = tmq.Params(L_FULL, KAPPA, mu, eps, flavor=(tmq.TM_NDEG_DOUBLET if nf == 2 else tmq.TM_TWIST_PLUS),
                       recon=12)
        g = tmq.Gauge(p, U)
        tables["flavours_%d" % nf] = tmq.autotune(g)
        for prec in (tmq.TM_PREC_F32, tmq.TM_PREC_F16):
            xe = tmq.noise_z2(g, tmq.Field(g, prec, N), 0, 5000)
            out, tmp = tmq.Field(g, prec, N), tmq.Field(g, prec, N)
            ms = time_op(lambda: tmq.precond_op(g, out, xe, tmp, 0, False), 5, flush)
            x1 = tmq.noise_z2(g, tmq.Field(g, prec), 0, 5000)
            o1, t1 = tmq.Field(g, prec), tmq.Field(g, prec)
            ms1 = time_op(lambda: tmq.precond_op(g, o1, x1, t1, 0, False), 10, flush)
            by = (16 * link_reals(prec, 12) * REAL_BYTES[prec] / N + 5 * SPINOR_BYTES[prec] * nf) * p.Vh
            gbs = by / (ms / N * 1e-3) / 1e9
            rows.append({"flavours": nf, "prec": {4: "f32", 2: "f16"}[prec], "nrhs": N,
                         "us_per_source": round(ms / N * 1e3, 1), "single_rhs_us": round(ms1 * 1e3, 1),
                         "amortised_bytes_per_source": by, "amortised_gbs": round(gbs, 1),
                         "hbm_frac": round(gbs / peak, 3),
                         "gflops_per_source": round(FLOPS_PER_SITE[nf] * p.Vh / (ms / N * 1e-3) / 1e9, 1)})
            del xe, out, tmp, x1, o1, t1
        g.close()
    return {"lattice": list(L_FULL), "operator": "M_asym (eq. 2.2 LHS), recon 12", "rows": rows,
            "launch_tables": tables}


def dd_section(tmq, U, psi, dev, args):
    """The domain-decomposed operator (sec. 2.1) emulated on one GPU: every time slab in this process,
    faces moved by device copies that overlap the interior launches.  M_asym of the 32^3x64 doublet
    (FP32, recon 12) cut into R = 1, 2, 4, 8 slabs, per application, against the undecomposed handle
    (one GPU runs all R slabs' launches one after another, so this is the decomposition's overhead,
    not a scaling measurement); and the analogue of Table 2: the decomposed double-single
    reliable-update CG with asymmetric and symmetric PC on the same system, R = 1 and 4."""
    import torch
    from paper_1311_4462_gb300 import dd, inputs
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    p = tmq.Params(L_FULL, KAPPA, MU_ND, EPS_ND, flavor=tmq.TM_NDEG_DOUBLET, recon=12)
    prec = tmq.TM_PREC_F32
    rows = []
    for R in (1, 2, 4, 8):
        if L_FULL[3] % R or (L_FULL[3] // R) % 2:
            continue
        slabs = dd.make_slabs(p, U, R)
        tr = dd.LocalTransport()
        ins = dd.pack_slabs(slabs, dd.split_field(slabs, psi), 0, prec)
        outs, tmps = [s.field(prec) for s in slabs], [s.field(prec) for s in slabs]
        ms = time_op(lambda: dd.precond_op(slabs, outs, ins, tmps, tr, 0, False), 10, flush)
        face = slabs[0].faces(prec).nbytes
        rows.append({"slabs": R, "us": round(ms * 1e3, 1), "face_bytes": face,
                     "faces_per_application": 4 * R, "gflops": round(FLOPS_PER_SITE[2] * p.Vh / (ms * 1e-3) / 1e9, 1)})
        for s_ in slabs:
            s_.close()
        del ins, outs, tmps
    # Table 2 analogue: the decomposed double-single reliable-update CG (the paper's multi-GPU solver),
    # asymmetric vs symmetric PC, on the 32^3x64 doublet, 1 and 4 slabs
    cg = []
    for R in (1, 4):
        slabs = dd.make_slabs(p, U, R)
        tr = dd.LocalTransport()
        parts = dd.split_field(slabs, psi)
        bes, bos = dd.pack_slabs(slabs, parts, 0), dd.pack_slabs(slabs, parts, 1)
        for pc in (0, 1):
            bps, xes = [s_.field() for s_ in slabs], [s_.field() for s_ in slabs]
            dd.prepare_rhs(slabs, bps, bes, bos, tr, pc)
            torch.cuda.synchronize()
            t0 = time.time()
            st = dd.cg(slabs, xes, bps, tr, pc=pc, tol=1e-10, sloppy_prec=tmq.TM_PREC_F32, delta=1e-5)
            torch.cuda.synchronize()
            cg.append({"slabs": R, "pc": "sym" if pc else "asym", "iterations": st["iterations"],
                       "reliable_updates": st["reliable_updates"], "true_residual": st["true_residual"],
                       "s": round(time.time() - t0, 3)})
        for s_ in slabs:
            s_.close()
    return {"operator": {"lattice": list(L_FULL), "workload": "M_asym, doublet, FP32, recon 12", "rows": rows},
            "cg_doublet_32x32x32x64_mixed_f32_tol_1e-10": cg,
            "note": "all slabs on one GPU: the time is the decomposition's overhead, not scaling"}


def batching_section(tmq, U, dev, args):
    """Loop estimator Tr[gamma5 M^-1] on the 32^3x64 one-flavour lattice (kappa 0.1612, mu 0.004):
    256 Z2 sources, 16 per batched mixed-precision CG to 1e-8 with source dropping and CUDA-graph
    replay; solves/s against one-at-a-time FP64 CG (timed on 4 sources), and the per-source error
    of the batched solutions against FP64 solves of the same sources."""
    import numpy as np
    import torch
    from paper_1311_4462_gb300 import loops

    p = tmq.Params(L_FULL, KAPPA, MU_DEG, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    g = tmq.Gauge(p, U)
    tmq.autotune(g)
    nsrc = 256 if L_FULL == (32, 32, 32, 64) else 32
    out = {"lattice": list(L_FULL), "sources": nsrc, "per_batch": 16, "tol": 1e-8,
           "true_residual_precision": "df64"}
    for name, sl in (("mixed_f32", tmq.TM_PREC_F32), ("mixed_f16", tmq.TM_PREC_F16)):
        # true residuals in DF64: for one flavour the double-float operator beats FP64 (3.8 vs 5.2 ms)
        res = loops.g5_trace(g, nsources=nsrc, batch=16, seed0=3000, tol=1e-8, solver="mixed", sloppy_prec=sl,
                             use_graph=True, return_solutions=(name == "mixed_f32"), true_prec=tmq.TM_PREC_DF64)
        out[name] = {"solves_per_s": round(res["solves_per_second"], 2), "seconds": round(res["solve_seconds"], 2),
                     "estimate_re": res["estimate"].real, "estimate_im": res["estimate"].imag,
                     "stderr": res["stderr"], "iterations_first_batch": res["iterations"][:16]}
        if name == "mixed_f32":
            sols = res["solutions"][0]
    # one-at-a-time FP64 CG on the first 4 sources: rate, and per-source error of the batched solutions
    errs, t64 = [], 0.0
    for k in range(4):
        ee, eo = tmq.Field(g, tmq.TM_PREC_F64), tmq.Field(g, tmq.TM_PREC_F64)
        tmq.noise_z2(g, ee, 0, 3000 + k)
        tmq.noise_z2(g, eo, 1, 3000 + k)
        bp, xe, xo = tmq.Field(g, 8), tmq.Field(g, 8), tmq.Field(g, 8)
        torch.cuda.synchronize()
        t0 = time.time()
        tmq.prepare_rhs(g, bp, ee, eo, 0, False)
        tmq.solve(g, xe, bp, tol=1e-8)
        tmq.reconstruct_odd(g, xo, eo, xe, False)
        torch.cuda.synchronize()
        t64 += time.time() - t0
        ref = torch.cat([tmq.unpack(g, xe, 0).reshape(-1), tmq.unpack(g, xo, 1).reshape(-1)])
        got = torch.cat([tmq.unpack(g, sols[0], 0)[k].reshape(-1), tmq.unpack(g, sols[1], 1)[k].reshape(-1)])
        errs.append(float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref)))
    out["fp64_one_at_a_time_solves_per_s"] = round(4 / t64, 3)
    out["speedup_batched_vs_fp64"] = round(out["mixed_f32"]["solves_per_s"] / (4 / t64), 2)
    out["per_source_rel_error_vs_fp64"] = errs
    g.close()
    return out


def cpu_baseline(U_np, psi_np, args):
    """The FP64 oracle as it stands (OpenMP over the host cores) on one full M_asym application."""
    import oracle
    po = oracle.Params(L_FULL, KAPPA, MU_ND, EPS_ND, flavor=2)
    x = oracle.project_parity(po, psi_np, 0)
    t0 = time.time()
    n = 0
    while True:
        oracle.apply_M_pc(po, U_np, x)
        n += 1
        if time.time() - t0 > 8.0 or n >= 3:
            break
    dt = (time.time() - t0) / n
    Vh = po.L[0] * po.L[1] * po.L[2] * po.L[3] // 2
    return {"value": round(FLOPS_PER_SITE[2] * Vh / dt / 1e9, 3), "unit": "GFLOPS", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{n} full M_asym application(s) of the 32^3x64 doublet, FP64, "
                                        f"{dt:.2f} s each"}


def solve_only(args):
    """One solve of the headline system (32^3x64 doublet, asymmetric PC, tol 1e-10), run twice (the
    first warms up): the command the solver's launch list is captured on."""
    import torch

    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import inputs
    p = tmq.Params(L_FULL, KAPPA, MU_ND, EPS_ND, flavor=tmq.TM_NDEG_DOUBLET, recon=args.recon)
    g = tmq.Gauge(p, torch.from_numpy(inputs.gauge_field(L_FULL, 1002)).cuda(), f64_full_links=True)
    b = torch.from_numpy(inputs.spinor_field(L_FULL, 2, 2002)).cuda()
    be, bo = tmq.pack(g, b, 0, tmq.TM_PREC_F64), tmq.pack(g, b, 1, tmq.TM_PREC_F64)
    bp = tmq.Field(g, tmq.TM_PREC_F64)
    tmq.prepare_rhs(g, bp, be, bo, 0, False)
    kw = {"cg": {"solver": "cg"}, "mixed_f32": {"solver": "mixed", "sloppy_prec": tmq.TM_PREC_F32},
          "mixed_f16": {"solver": "mixed", "sloppy_prec": tmq.TM_PREC_F16}}[args.solve]
    out = []
    for _ in range(2):
        xe = tmq.Field(g, tmq.TM_PREC_F64)
        torch.cuda.synchronize()
        t0 = time.time()
        st = tmq.solve(g, xe, bp, tol=1e-10, maxiter=20000, **kw)
        torch.cuda.synchronize()
        out.append({"s": round(time.time() - t0, 4), "iterations": st["iterations"],
                    "reliable_updates": st["reliable_updates"], "true_residual": st["true_residual"]})
    g.close()
    return {"solve": args.solve, "lattice": list(L_FULL), "runs": out}


def multi_only(args):
    """M_asym on 16 Z2 sources in one multi-RHS launch per factor (the handle's default multi-RHS
    form), at the headline lattice: the command the multi-RHS kernel's profile is captured on."""
    import torch

    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import inputs
    nf = args.nf
    p = tmq.Params(L_FULL, KAPPA, MU_ND if nf == 2 else MU_DEG, EPS_ND if nf == 2 else 0.0,
                   flavor=tmq.TM_NDEG_DOUBLET if nf == 2 else tmq.TM_TWIST_PLUS, recon=args.recon)
    prec = {"f32": tmq.TM_PREC_F32, "f16": tmq.TM_PREC_F16}[args.multi]
    g = tmq.Gauge(p, torch.from_numpy(inputs.gauge_field(L_FULL, 1002)).cuda(), precs=(prec,))
    N = 16
    xe = tmq.noise_z2(g, tmq.Field(g, prec, N), 0, 5000)
    out, tmp = tmq.Field(g, prec, N), tmq.Field(g, prec, N)
    for _ in range(args.warmup):
        tmq.precond_op(g, out, xe, tmp, 0, False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        tmq.precond_op(g, out, xe, tmp, 0, False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    table = tmq.tune_export(g)
    g.close()
    return {"multi": args.multi, "flavours": nf, "lattice": list(L_FULL), "nrhs": N, "us_per_source": round(ms / N * 1e3, 1),
            "launch_table": table}


def force_only(args):
    """tm_force (projected) at 24^3x48 one flavour in FP32 or FP64: the command the force kernel's
    profile is captured on; prints its time and algorithmic bandwidth."""
    import torch

    import paper_1311_4462_gb300 as tmq
    from paper_1311_4462_gb300 import inputs
    L = (24, 24, 24, 48)
    prec = {"f32": tmq.TM_PREC_F32, "f64": tmq.TM_PREC_F64}[args.force]
    p = tmq.Params(L, KAPPA, MU_DEG, 0.0, flavor=tmq.TM_TWIST_PLUS, recon=12)
    g = tmq.Gauge(p, torch.from_numpy(inputs.gauge_field(L, 1003)).cuda(), precs=(prec,))
    psi = torch.from_numpy(inputs.spinor_field(L, 1, 2003)).cuda()
    gv = torch.from_numpy(inputs.spinor_field(L, 1, 2103)).cuda()
    pe, po = tmq.pack(g, psi, 0, prec), tmq.pack(g, psi, 1, prec)
    ge, go = tmq.pack(g, gv, 0, prec), tmq.pack(g, gv, 1, prec)
    out = torch.empty(p.gauge_shape, dtype=torch.complex128 if prec == 8 else torch.complex64, device="cuda")
    for _ in range(args.warmup):
        tmq.force(g, pe, po, ge, go, coef=1.0, project=True, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        tmq.force(g, pe, po, ge, go, coef=1.0, project=True, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    V, w = 2 * p.Vh, REAL_BYTES[prec]
    by = 2 * V * 24 * w + 4 * V * 12 * w + 4 * V * 18 * w
    g.close()
    return {"force": args.force, "lattice": list(L), "us": round(ms * 1e3, 1), "gbs": round(by / (ms * 1e-3) / 1e9, 1)}


# -------------------------------------------------------------------------------------- reference
def run_reference(args):
    """The oracle (plain FP64 C, OpenMP) timed as the reference arm on a bounded sub-lattice sample."""
    import numpy as np

    import oracle
    from paper_1311_4462_gb300 import inputs

    oracle.build()
    K, W = args.steps, args.warmup
    # calibrate the oracle's time per site, then take the largest sample lattice (x = y = 32,
    # z and t shrunk, then all four halved) whose K + W applications fit in about a minute
    Lc = (32, 32, 32, 4)
    po = oracle.Params(Lc, KAPPA, MU_ND, EPS_ND, flavor=2)
    Uc = inputs.gauge_field(Lc, 1002)
    xc = oracle.project_parity(po, inputs.spinor_field(Lc, 2, 2002), 0)
    t0 = time.time()
    oracle.apply_M_pc(po, Uc, xc)
    per_site = (time.time() - t0) / (32 ** 3 * 4)
    target = 60.0 / max(K + W, 1) / per_site  # sites per step
    cands = [(32, 32, z, t) for t in (64, 32, 16, 8, 4, 2) for z in (32, 16, 8, 4, 2)]
    cands += [(16, 16, 2, 2), (8, 8, 2, 2), (4, 4, 2, 2), (2, 2, 2, 2)]
    L = next((c for c in sorted(cands, key=lambda c: -np.prod(c)) if np.prod(c) <= target), (2, 2, 2, 2))
    po = oracle.Params(L, KAPPA, MU_ND, EPS_ND, flavor=2)
    U = inputs.gauge_field(L, 1002)
    x = oracle.project_parity(po, inputs.spinor_field(L, 2, 2002), 0)
    for _ in range(W):
        oracle.apply_M_pc(po, U, x)
    t0 = time.time()
    for _ in range(K):
        oracle.apply_M_pc(po, U, x)
    dt = time.time() - t0
    Vh = int(np.prod(L)) // 2
    value = FLOPS_PER_SITE[2] * Vh * K / dt / 1e9
    sample = ("%s sub-lattice of the 32^3x64 doublet workload (same parameters), one FP64 M_asym application "
              "per step" % "x".join(map(str, L)))
    return {"metric": "TM dslash GFLOPS & % HBM roofline per precision; CG time-to-1e-10 mixed vs FP64",
            "impl": "reference", "value": round(value, 3), "unit": "GFLOPS", "n_gpus": args.gpus, "steps": K,
            "warmup": W, "ms_per_step": round(dt / K * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded SU(3) links exp(0.3 i H), Gaussian spinors)",
            "device": "host cores (the FP64 CPU oracle)",
            "config": headline_config(args, 2, 4, 12, L_FULL, 1),
            "cpu_baseline": {"value": round(value, 3), "unit": "GFLOPS", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "GFLOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="headline step only (no tables, e2e or baselines)")
    ap.add_argument("--csw", type=float, default=0.0, help="time the clover-twisted-mass operator with this c_sw")
    ap.add_argument("--lattice", default=None, help="override the lattice, e.g. 32,32,32,32 (profiling runs)")
    ap.add_argument("--prec", default="f32", choices=["f64", "f32", "f16"], help="headline storage (profiling runs)")
    ap.add_argument("--nf", type=int, default=2, choices=[1, 2], help="flavours of the headline step (profiling runs)")
    ap.add_argument("--recon", type=int, default=12, choices=[18, 12, 8], help="link storage (profiling runs)")
    ap.add_argument("--only", default=None, help="comma-separated extra sections to run (default: all)")
    ap.add_argument("--solve", default=None, choices=["cg", "mixed_f32", "mixed_f16"],
                    help="profiling run: only this solve (asymmetric PC, 1e-10) of the headline system, twice")
    ap.add_argument("--multi", default=None, choices=["f32", "f16"],
                    help="profiling run: only the 16-source multi-RHS M_asym (--nf flavours), --warmup + --steps times")
    ap.add_argument("--force", default=None, choices=["f32", "f64"],
                    help="profiling run: only tm_force at 24^3x48 (one flavour), --warmup + --steps launches")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.lattice:
        global L_FULL
        L_FULL = tuple(int(v) for v in args.lattice.split(","))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.solve or args.force or args.multi:
        if rank == 0:
            fn = solve_only if args.solve else (force_only if args.force else multi_only)
            print(json.dumps(fn(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
