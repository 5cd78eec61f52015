#!/usr/bin/env python3
"""Benchmark of the RLFC hot path on GB300.

One step = the whole hot path on one synthetic light field: decode every block
of every view (Algorithm 2 over the full light field) and render n new views
by quadrilinear interpolation with on-demand block decode (Section 3.6).
Default workload: 9 x 9 views of 512 x 512 RGB, 5 textured planes at
disparities -2..2, sigma 1 noise, 3-level tree (3, 3), 4 x 4 blocks,
residual threshold 4 (the middle of the 1 / 4 / 8 sweep), 1000 new 512 x 512
views at seeded random (u, v) with the focus on one of the planes.

value = output pixels per second of the step (the 21.2 Mpx decoded light
field plus 262 Mpx of rendered views) in Mpix/s; "parts" splits it into
decode-all Mpix/s and rendered 512 x 512 views/s.  The stream is encoded once
by the library's GPU encoder and stays resident; each timed step is bracketed
by CUDA events on the launching stream after a 256 MiB write that flushes L2.

--impl reference times the CPU oracle (the plain C restatement of the paper)
on the host cores on a bounded sample of the same workload, scaled to the
same unit.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lf_synth  # noqa: E402

METRIC = "decoded Mpix/s and % HBM roofline; 512×512 views/s; served p50/p99 view latency"
UNIT = "Mpix/s"


# dram__bytes_read.sum + dram__bytes_write.sum of one launch, from an ncu
# capture of the same kernel build on this workload (config, tau, views,
# kernel); a kernel missing here reports null
TRAFFIC_PER_LAUNCH = {
    # render_native_kernel, first timed step of `bench.py --steps 2 --warmup 1` (ncu one-pass
    # dram__bytes_read.sum 86.56 MB + dram__bytes_write.sum 3.09 GB)
    ("plain", 4, 1000, "render_native_kernel"): 86_560_000 + 3_090_000_000,
    # decode_all_kernel on the 17x17x1024^2 light field at tau 4 (ncu one-pass, third launch:
    # dram__bytes_read.sum 100.21 MB + dram__bytes_write.sum 853.10 MB; the rest of the
    # 909 MB of output is still in L2 when the kernel ends)
    ("batching", 4, 0, "decode_all_kernel"): 100_210_000 + 853_100_000,
}

# smsp__inst_executed.sum of one launch (warp instructions), from the same kind
# of one-pass ncu capture (`--metrics smsp__inst_executed.sum ... -s 3 -c 3`
# on `bench.py --steps 2 --warmup 1`); the kernels are integer and
# conversion work bound by instruction issue more than by DRAM
INSTR_PER_LAUNCH = {
    ("plain", 4, 1000, "render_native_kernel"): 1_072_146_688,
    ("batching", 4, 0, "decode_all_kernel"): 458_440_390,
}
# issue peak: 152 SMs x 4 schedulers x one warp instruction per cycle at the
# 2070 MHz maximum SM clock
ISSUE_PEAK = 152 * 4 * 2.070e9


NI_ = 48   # block statistics: the learned aid's network input width


def _bf16_sustained():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["bf16_tflops_sustained"])
    return 1700.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _workload(args):
    p = dict(lf_synth.PRESETS[args.config])
    n_views = args.n_views if args.n_views else p.get("n_render", 16)
    W, H = p.get("render_size", (p["W"], p["H"]))
    tau = args.tau if args.tau is not None else p["taus"][len(p["taus"]) // 2]
    return p, n_views, W, H, tau


def _config_json(p, n_views, out_w, out_h, tau, extra=None):
    c = {"workload": f"{args_config_name(p)}: {p['U']}x{p['V']} views of {p['W']}x{p['H']} RGB, "
                     f"{len(p['disparities'])} planes, sigma {p['sigma']}, {p['L']}-level tree {tuple(p['c'][1:])}, "
                     f"4x4 blocks, tau {tau}; full decode + {n_views} new {out_w}x{out_h} views",
         "U": p["U"], "V": p["V"], "W": p["W"], "H": p["H"], "levels": p["L"], "tau": tau,
         "n_render": n_views, "render_size": [out_w, out_h],
         "l2": "flushed by a 256 MiB write before every timed step"}
    if extra:
        c.update(extra)
    return c


def args_config_name(p):
    for k, v in lf_synth.PRESETS.items():
        if v["id"] == p["id"]:
            return k
    return "custom"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, uuid: str):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.uuid}", f"--query-gpu={','.join(self.FIELDS)}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) != len(self.FIELDS):
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for name, val in zip(names, f[3:]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _algorithmic_bytes(info, n_views_lf, n_render, out_w, out_h):
    nloc = info.nloc_x * info.nloc_y
    stream_read = info.record_bytes + 4 * (3 * nloc + 1) + info.top_bytes
    decode = stream_read + n_views_lf * info.W * info.H * 3
    render = stream_read + n_render * out_w * out_h * 12
    return decode, render, stream_read


def _needed_views(cams, U, V):
    """Grid views the renderer blends for these cameras: the 2 x 2 neighbours
    of each clamped camera position."""
    need = set()
    for u, v, _ in cams:
        cu, cv = min(max(float(u), 0.0), U - 1.0), min(max(float(v), 0.0), V - 1.0)
        i0 = min(int(cu), max(U - 2, 0))
        j0 = min(int(cv), max(V - 2, 0))
        for j in (j0, min(j0 + 1, V - 1)):
            for i in (i0, min(i0 + 1, U - 1)):
                need.add(j * U + i)
    return len(need)


def _kernel_bytes(info, stream_read, n_views_lf, n_needed, n_render, out_w, out_h):
    """Algorithmic bytes of one launch of each library kernel on this
    workload: what the step it implements must read and write at least."""
    px_view = info.W * info.H
    out_px = n_render * out_w * out_h
    return {
        # compressed stream read once, RGB8 written
        "decode_all_kernel": stream_read + 3 * px_view * n_views_lf,
        # the renderer's decode of the views it samples: the stream read (the
        # packed views it writes are the renderer's own intermediate)
        "decode_all_kernel<packed>": stream_read,
        # camera table read, one mask byte per view written
        "mark_needed_kernel": 12 * n_render + n_views_lf,
        # float RGB written (the decoded views it reads are the renderer's
        # own intermediate, not bytes the method must move)
        "render_native_kernel": 12 * out_px,
        "render_tiled_kernel": stream_read + 12 * out_px,
        "render_direct_kernel": stream_read + 12 * out_px,
    }


def max_over_ranks(vals, world, device):
    """Element-wise maximum of per-rank timings over all ranks (the slowest
    replica sets the job's time); identity on one rank."""
    if world <= 1:
        return list(vals)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_mpix_per_s(world, px_per_rank, ms):
    """Whole-job throughput: every replica processes px_per_rank pixels per
    step, the step lasting the slowest rank's ms."""
    return world * px_per_rank / (ms * 1e-3) / 1e6


DTYPE = "int decode + fp32 render"


def _median(xs):
    return float(np.median(np.asarray(xs, dtype=np.float64)))


def _timed_calls(torch, fn, reps, flush, warmup=3):
    """Per-call device times (ms) of `reps` calls of fn, each after a write
    that flushes L2, bracketed by CUDA events on the current stream."""
    cur = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    ms = []
    for k in range(reps):
        flush.fill_(k & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        fn()
        b.record(cur)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def _traced(rlfc, torch, fn, reps, flush):
    """Per-kernel launch counts and summed durations (the library's own CUDA
    events) over `reps` flushed calls of fn."""
    rlfc.trace_read(reset=True)
    rlfc.trace_enable(True)
    for k in range(reps):
        flush.fill_(k & 255)
        fn()
    torch.cuda.synchronize()
    tr = rlfc.trace_read(reset=True)
    rlfc.trace_enable(False)
    return tr


def _extra_parts(rlfc, torch, args, p, tau, st, out_lf, flush, peak, world):
    """Beside the step: the plain decode at the other thresholds of the sweep,
    the full decode of the 17 x 17 x 1024^2 light field (the bandwidth test of
    the decoder) and 10^6 random block requests on it, batched and as one warp
    per request.  Device times are medians over at least 20 flushed calls."""
    reps = max(args.steps, 20)
    U, V = p["U"], p["V"]
    out = {}
    px_lf = U * V * p["W"] * p["H"]
    if not args.no_sweep:
        d_lf = lf_synth.make_lightfield_torch(U, V, p["W"], p["H"], p["disparities"], p["sigma"], p["id"],
                                              p.get("contrast", False))
        for t in p.get("taus", [tau]):
            if t == tau:
                continue
            s_t = rlfc.Stream(rlfc.encode(d_lf, U, V, p["L"], p["c"], tau_p=t, tau_b=16 * t))
            b_t, _, _ = _algorithmic_bytes(s_t.info, U * V, 0, 0, 0)
            ms = max_over_ranks([_median(_timed_calls(torch, lambda: s_t.decode_all(out_lf), reps, flush))], world,
                                "cuda")[0]
            out[f"decode_all_tau{t}"] = {"ms": ms, "mpix_s": px_lf / (ms * 1e-3) / 1e6, "algorithmic_bytes": b_t,
                                         "gbs": b_t / (ms * 1e-3) / 1e9, "hbm_frac": b_t / (ms * 1e-3) / 1e9 / peak,
                                         "stream_bytes": int(s_t.info.stream_bytes)}
            s_t.close()
        del d_lf
    roof_dec = None
    if not args.no_batching:
        pb = lf_synth.PRESETS["batching"]
        t0 = time.time()
        d_b = lf_synth.preset_lightfield_torch("batching")
        torch.cuda.synchronize()
        t_synth = time.time() - t0
        tb = pb["taus"][0]
        s_b = rlfc.Stream(rlfc.encode(d_b, pb["U"], pb["V"], pb["L"], pb["c"], tau_p=tb, tau_b=16 * tb))
        del d_b
        ib = s_b.info
        nv = pb["U"] * pb["V"]
        px_b = nv * pb["W"] * pb["H"]
        lf_b = torch.empty((nv, pb["H"], pb["W"], 3), dtype=torch.uint8, device="cuda")
        ms_b = _timed_calls(torch, lambda: s_b.decode_all(lf_b), reps, flush)
        tr = _traced(rlfc, torch, lambda: s_b.decode_all(lf_b), reps, flush)
        alg_b, _, _ = _algorithmic_bytes(ib, nv, 0, 0, 0)
        med_b = max_over_ranks([_median(ms_b)], world, "cuda")[0]
        k_launch, k_tot = tr.get("decode_all_kernel", (1, med_b))
        k_ms = max_over_ranks([k_tot / max(k_launch, 1)], world, "cuda")[0]
        out["decode_all_17x17x1024"] = {
            "ms": med_b, "mpix_s": px_b / (med_b * 1e-3) / 1e6, "algorithmic_bytes": alg_b,
            "gbs": alg_b / (med_b * 1e-3) / 1e9, "hbm_frac": alg_b / (med_b * 1e-3) / 1e9 / peak,
            "kernel_ms": k_ms, "stream_bytes": int(ib.stream_bytes), "synth_s": t_synth,
            "workload": f"{pb['U']}x{pb['V']} views of {pb['W']}x{pb['H']}, 8 planes -3..3, contrast-modulated, "
                        f"3-level tree {tuple(pb['c'][1:])}, tau {tb}: every block of every view"}
        roof_dec = {"bound": "hbm", "kernel": "decode_all_kernel", "workload": "17x17x1024^2 full decode",
                    "achieved": alg_b / (k_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": alg_b / (k_ms * 1e-3) / 1e9 / peak, "bytes_per_launch": alg_b, "avg_launch_ms": k_ms,
                    "traffic": TRAFFIC_PER_LAUNCH.get(("batching", tb, 0, "decode_all_kernel")),
                    "peak_source": "measured hbm_gbs (burst copy)" if _peaks()[1] == "measured" else "fallback"}
        instr = INSTR_PER_LAUNCH.get(("batching", tb, 0, "decode_all_kernel"))
        if instr is not None:
            roof_dec["issue"] = {"achieved": instr / (k_ms * 1e-3), "peak": ISSUE_PEAK, "unit": "warp instructions/s",
                                 "frac": instr / (k_ms * 1e-3) / ISSUE_PEAK, "instructions_per_launch": instr}
        # 10^6 uniform random (view, location) requests
        n = pb["n_requests"]
        pv, pl = lf_synth.random_requests(n, nv, s_b.nloc, pb["id"])
        views = torch.from_numpy(pv.view(np.int32)).cuda()
        locs = torch.from_numpy(pl.view(np.int32)).cuda()
        ref_blocks = torch.empty((n, 4, 4, 3), dtype=torch.uint8, device="cuda")
        blocks = torch.empty((n, 4, 4, 3), dtype=torch.uint8, device="cuda")
        per_req = max_over_ranks([_median(_timed_calls(torch, lambda: s_b.decode_blocks(views, locs, ref_blocks),
                                                       reps, flush))], world, "cuda")[0]
        bt = rlfc.Batch(s_b, n)
        bt.config = dict(graph=0)
        chosen = dict(bt.autotune(views, locs, blocks))
        bt.config = dict(graph=1)
        chosen["graph"] = 1
        blocks.zero_()
        g_ms = max_over_ranks([_median(_timed_calls(torch, lambda: bt.decode(views, locs, blocks), reps, flush))],
                              world, "cuda")[0]
        same = bool(torch.equal(blocks, ref_blocks))
        out["batched_requests_1e6"] = {
            "ms": g_ms, "requests_per_s": n / (g_ms * 1e-3), "mpix_s": 16 * n / (g_ms * 1e-3) / 1e6,
            "config": chosen, "identical_to_per_request": same,
            "note": "persistent binned kernel, autotuned, replayed as a CUDA graph"}
        out["per_request_1e6"] = {"ms": per_req, "requests_per_s": n / (per_req * 1e-3),
                                  "mpix_s": 16 * n / (per_req * 1e-3) / 1e6, "note": "one warp per request"}
        out["batched_speedup_vs_per_request"] = per_req / g_ms
        bt.close()
        s_b.close()
        del lf_b, views, locs, blocks, ref_blocks
    return out, roof_dec


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1805_06019_gb300 import rlfc

    p, n_render, out_w, out_h, tau = _workload(args)
    U, V = p["U"], p["V"]
    d_lf = lf_synth.make_lightfield_torch(U, V, p["W"], p["H"], p["disparities"], p["sigma"], p["id"],
                                          p.get("contrast", False))
    data = rlfc.encode(d_lf, U, V, p["L"], p["c"], tau_p=tau, tau_b=16 * tau)
    lf = d_lf.cpu().numpy() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    del d_lf
    st = rlfc.Stream(data)
    cams = lf_synth.random_views(n_render, U, V, p["id"], d_choices=p["disparities"])
    uv = torch.from_numpy(cams[:, :2].copy()).cuda()
    disp = torch.from_numpy(cams[:, 2].copy()).cuda()
    out_lf = torch.empty((U * V, p["H"], p["W"], 3), dtype=torch.uint8, device="cuda")
    out_views = torch.empty((n_render, out_h, out_w, 3), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    cur = torch.cuda.current_stream()

    def step():
        st.decode_all(out_lf)
        st.render(uv, disp, out_w, out_h, out_views)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    clocks = ClockSampler(str(torch.cuda.get_device_properties(local).uuid))
    if not str(clocks.uuid).startswith("GPU-"):
        clocks.uuid = "GPU-" + str(clocks.uuid)
    clocks.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    rlfc.trace_read(reset=True)
    rlfc.trace_enable(True)
    for k in range(args.steps):
        flush.fill_(k & 255)
        a, b, c = evs[k]
        a.record(cur)
        st.decode_all(out_lf)
        b.record(cur)
        st.render(uv, disp, out_w, out_h, out_views)
        c.record(cur)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    trace = rlfc.trace_read(reset=True)
    rlfc.trace_enable(False)
    t_dec = [a.elapsed_time(b) for a, b, _ in evs]
    t_ren = [b.elapsed_time(c) for _, b, c in evs]
    t_step = [a.elapsed_time(c) for a, _, c in evs]
    # the same calls back to back without the flush: warm-L2 figures beside
    # the flushed ones (the compressed stream stays in L2 between calls)
    wev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        a, b, c = wev[k]
        a.record(cur)
        st.decode_all(out_lf)
        b.record(cur)
        st.render(uv, disp, out_w, out_h, out_views)
        c.record(cur)
    torch.cuda.synchronize()
    dec_warm, ren_warm = max_over_ranks([_median([a.elapsed_time(b) for a, b, _ in wev]),
                                         _median([b.elapsed_time(c) for _, b, c in wev])], world, "cuda")
    step_ms, dec_ms, ren_ms, step_mean = max_over_ranks(
        [_median(t_step), _median(t_dec), _median(t_ren), float(np.mean(t_step))], world, "cuda")

    info = st.info
    px_lf = U * V * p["W"] * p["H"]
    px_render = n_render * out_w * out_h
    value = job_mpix_per_s(world, px_lf + px_render, step_ms)
    peak, peak_src = _peaks()
    b_dec, b_ren, stream_read = _algorithmic_bytes(info, U * V, n_render, out_w, out_h)
    dec_gbs = b_dec / (dec_ms * 1e-3) / 1e9
    ren_gbs = b_ren / (ren_ms * 1e-3) / 1e9
    parts = {
        "decode_all": {"ms": dec_ms, "mpix_s": px_lf / (dec_ms * 1e-3) / 1e6, "algorithmic_bytes": b_dec,
                       "gbs": dec_gbs, "hbm_frac": dec_gbs / peak, "ms_warm": dec_warm,
                       "note": f"the step's light field at tau {tau}; the stream stays in L2 across calls"},
        "render": {"ms": ren_ms, "ms_warm": ren_warm, "views_per_s": n_render / (ren_ms * 1e-3),
                   "mpix_s": px_render / (ren_ms * 1e-3) / 1e6,
                   "algorithmic_bytes": b_ren, "gbs": ren_gbs, "hbm_frac": ren_gbs / peak},
    }
    # per-kernel durations from the library's own CUDA events (on the
    # launching stream, inside the timed region); the roofline is that of the
    # kernel with the most device time
    n_needed = _needed_views(cams, U, V)
    kbytes = _kernel_bytes(info, stream_read, U * V, n_needed, n_render, out_w, out_h)
    kernels = {}
    for name, (launches, tot) in trace.items():
        avg = tot / max(launches, 1)
        gbs = kbytes.get(name, 0) / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
        kernels[name] = {"launches": launches, "avg_ms": avg, "share": tot / max(sum(t for _, t in trace.values()), 1e-9),
                         "algorithmic_bytes": kbytes.get(name), "gbs": gbs, "hbm_frac": gbs / peak}
        instr = INSTR_PER_LAUNCH.get((args.config, tau, n_render, name))
        if instr is not None and avg > 0:
            kernels[name]["issue_frac"] = instr / (avg * 1e-3) / ISSUE_PEAK
    top = max(kernels, key=lambda k: kernels[k]["avg_ms"] * kernels[k]["launches"])
    roof = {"bound": "hbm", "kernel": top, "achieved": kernels[top]["gbs"], "peak": peak, "unit": "GB/s",
            "frac": kernels[top]["gbs"] / peak, "peak_source": f"{peak_src} hbm_gbs (burst copy)",
            "traffic": TRAFFIC_PER_LAUNCH.get((args.config, tau, n_render, top)),
            "bytes_per_launch": kernels[top]["algorithmic_bytes"], "avg_launch_ms": kernels[top]["avg_ms"]}
    instr_top = INSTR_PER_LAUNCH.get((args.config, tau, n_render, top))
    if instr_top is not None:
        # the same kernel against the instruction-issue ceiling
        ach = instr_top / (kernels[top]["avg_ms"] * 1e-3)
        roof["issue"] = {"achieved": ach, "peak": ISSUE_PEAK, "unit": "warp instructions/s", "frac": ach / ISSUE_PEAK,
                         "instructions_per_launch": instr_top,
                         "peak_source": "derived: 152 SMs x 4 schedulers x 1 warp instruction/cycle x 2070 MHz"}
    gpu_launches = sum(l for l, _ in trace.values())

    # end to end through the C ABI: per-step camera upload from pinned host
    # memory, decode + render, and download of every output to pinned memory.
    # Outputs are double-buffered so that step k's downloads (on a copy
    # stream) overlap step k + 1's decode and render; every step's copies lie
    # inside the timed region.
    def end_to_end(u8: bool):
        h_uv = torch.from_numpy(cams[:, :2].copy()).pin_memory()
        h_disp = torch.from_numpy(cams[:, 2].copy()).pin_memory()
        vdt = torch.uint8 if u8 else torch.float32
        d_uv = [uv, torch.empty_like(uv)]
        d_disp = [disp, torch.empty_like(disp)]
        d_lf = [out_lf, torch.empty_like(out_lf)]
        d_views = [torch.empty(out_views.shape, dtype=vdt, device="cuda") for _ in range(2)]
        h_lf = [torch.empty(out_lf.shape, dtype=torch.uint8).pin_memory() for _ in range(2)]
        h_views = [torch.empty(out_views.shape, dtype=vdt).pin_memory() for _ in range(2)]
        copy_st = torch.cuda.Stream()
        e_steps = max(args.steps, 5)
        done = [None, None]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for k in range(e_steps):
            b = k & 1
            if done[b] is not None:
                cur.wait_event(done[b])          # buffer b's previous download finished
            d_uv[b].copy_(h_uv, non_blocking=True)
            d_disp[b].copy_(h_disp, non_blocking=True)
            st.decode_all(d_lf[b])
            st.render(d_uv[b], d_disp[b], out_w, out_h, d_views[b])
            ready = torch.cuda.Event()
            ready.record(cur)
            copy_st.wait_event(ready)
            with torch.cuda.stream(copy_st):
                h_lf[b].copy_(d_lf[b], non_blocking=True)
                h_views[b].copy_(d_views[b], non_blocking=True)
            done[b] = torch.cuda.Event()
            done[b].record(copy_st)
        cur.wait_stream(copy_st)
        e1.record(cur)
        torch.cuda.synchronize()
        e_ms = max_over_ranks([e0.elapsed_time(e1) / e_steps], world, "cuda")[0]
        return {"value": job_mpix_per_s(world, px_lf + px_render, e_ms), "unit": UNIT, "ms_per_step": e_ms,
                "h2d_bytes_per_step": int(h_uv.numel() * 4 + h_disp.numel() * 4),
                "d2h_bytes_per_step": int(h_lf[0].numel() + h_views[0].numel() * h_views[0].element_size()),
                "steps": e_steps,
                "note": "downloads of step k overlap step k+1 on a copy stream; the device-to-host link "
                        "bounds it"}

    e2e = e2e_u8 = None
    if not args.no_e2e:
        e2e = end_to_end(False)
        e2e_u8 = end_to_end(True)
        e2e_u8["note"] = "the same step with 8-bit views (rlfc_render_views_u8), " + e2e_u8["note"]
    # the render call with 8-bit output, device-timed like the step
    views8 = torch.empty(out_views.shape, dtype=torch.uint8, device="cuda")
    r8_ms = max_over_ranks([_median(_timed_calls(torch, lambda: st.render(uv, disp, out_w, out_h, views8),
                                                 max(args.steps, 20), flush))], world, "cuda")[0]
    del views8
    parts["render_u8"] = {"ms": r8_ms, "views_per_s": n_render / (r8_ms * 1e-3),
                          "mpix_s": px_render / (r8_ms * 1e-3) / 1e6,
                          "note": "rlfc_render_views_u8: the same views as 8-bit RGB (3 B/px written)"}
    extra, roof_dec = _extra_parts(rlfc, torch, args, p, tau, st, out_lf, flush, peak, world)
    parts.update(extra)
    if not args.no_learned and world == 1:
        lr_ = learned_result(args, tau=lf_synth.PRESETS["learned"]["taus"][0])
        parts["learned_aid"] = {k: lr_[k] for k in ("agreement_heldout", "majority_class_share", "plain", "search",
                                                    "aided", "aided_vs_plain", "train_s", "decision_ns_per_block",
                                                    "network_on_tensor_cores")}
        parts["learned_aid"]["workload"] = lr_["config"]["workload"]
    if not args.no_serving and world == 1:
        parts["serving_vs_per_request"] = serving_compare(rlfc, torch, [float(r) for r in args.compare_rates.split(",")],
                                                          args.compare_seconds)

    cpu = None
    if lf is not None:
        cpu = cpu_baseline(p, lf, tau, n_render, out_w, out_h, cams, sample_views=args.cpu_sample_views)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
                "config": _config_json(p, n_render, out_w, out_h, tau, {"parallelism": f"replicas{world}"}),
                "timing": {"ms_per_step_median": step_ms, "ms_per_step_mean": step_mean,
                           "steps_timed": args.steps, "l2": "flushed by a 256 MiB write before every timed step"},
                "parts": parts, "kernels": kernels, "roofline": roof, "roofline_decode": roof_dec,
                "cpu_baseline": cpu, "e2e": e2e, "e2e_u8": e2e_u8,
                "gpu_launches": gpu_launches, "clocks": clk, "stream_bytes": int(info.stream_bytes)}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def _oracle_stream(p, lf, tau):
    import oracle
    return oracle.Stream(oracle.encode(lf, p["U"], p["V"], B=4, L=p["L"], c=p["c"], tau_p=tau, tau_b=16 * tau))


def _oracle_sample(p, st, n_render, out_w, out_h, cams, sample_views, threads=1):
    """Oracle time for decode-all plus `sample_views` renders on `threads`
    host threads (the oracle's decode splits views over threads; renders run
    one per thread, the C calls releasing the interpreter lock), scaled to the
    workload's n_render renders."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    dec = st.decode_all(nthreads=threads)
    t_dec = time.perf_counter() - t0
    k = min(sample_views, n_render)

    def one(r):
        oracle.render_view(dec, p["U"], p["V"], float(cams[r, 0]), float(cams[r, 1]), float(cams[r, 2]),
                           out_w, out_h)

    t0 = time.perf_counter()
    if threads == 1:
        for r in range(k):
            one(r)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(one, range(k)))
    t_ren = time.perf_counter() - t0
    step_s = t_dec + t_ren * n_render / k
    px = p["U"] * p["V"] * p["W"] * p["H"] + n_render * out_w * out_h
    return px / step_s / 1e6, step_s, t_dec + t_ren, k


def cpu_baseline(p, lf, tau, n_render, out_w, out_h, cams, sample_views=50):
    """The oracle on every host core (the whole workload: decode-all and every
    render), and on one core (a sample, scaled)."""
    ost = _oracle_stream(p, lf, tau)
    ncpu = os.cpu_count() or 1
    value, step_s, spent, k = _oracle_sample(p, ost, n_render, out_w, out_h, cams, n_render, threads=ncpu)
    v1, step1, spent1, k1 = _oracle_sample(p, ost, n_render, out_w, out_h, cams, sample_views)
    return {"value": value, "unit": UNIT, "cores": ncpu, "kind": "oracle",
            "sample": f"oracle decode of all {p['U'] * p['V']} views plus all {k} renders "
                      f"({spent:.1f} s on {ncpu} threads)",
            "step_s": step_s, "host_cpus": ncpu,
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "step_s": step1,
                              "sample": f"oracle decode of all {p['U'] * p['V']} views plus {k1} of the "
                                        f"{n_render} renders ({spent1:.1f} s, 1 thread), render time "
                                        f"scaled to {n_render} views"}}


def run_reference(args):
    """The oracle (the plain C restatement of the paper) as the reference arm:
    every step is the whole workload on the host cores, the decode of every
    view and all renders, nothing extrapolated."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    p, n_render, out_w, out_h, tau = _workload(args)
    lf = lf_synth.preset_lightfield(args_config_name(p))
    cams = lf_synth.random_views(n_render, p["U"], p["V"], p["id"], d_choices=p["disparities"])
    ncpu = os.cpu_count() or 1
    ost = _oracle_stream(p, lf, tau)
    for _ in range(args.warmup):
        _oracle_sample(p, ost, n_render, out_w, out_h, cams, n_render, threads=ncpu)
    steps = [_oracle_sample(p, ost, n_render, out_w, out_h, cams, n_render, threads=ncpu)
             for _ in range(args.steps)]
    step_s = _median([s[1] for s in steps])
    px = p["U"] * p["V"] * p["W"] * p["H"] + n_render * out_w * out_h
    value = px / step_s / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
            "config": _config_json(p, n_render, out_w, out_h, tau, {"parallelism": f"replicas{world}"}),
            "timing": {"ms_per_step_median": step_s * 1e3, "ms_per_step_mean": float(np.mean([s[1] for s in steps])) * 1e3,
                       "steps_timed": args.steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": ncpu,
                             "sample": f"per step: oracle decode of all {p['U'] * p['V']} views plus all {n_render} "
                                       f"renders ({ncpu} threads), median over {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _stream_location_words(data: bytes):
    """Words of the three channel records of every block location, from the
    stream's offset table (format v1 header: 16 little-endian uint32)."""
    h = np.frombuffer(data[:64], dtype="<u4")
    U, V, W, H, B = (int(x) for x in h[2:7])
    nloc = ((W + B - 1) // B) * ((H + B - 1) // B)
    off = np.frombuffer(data, dtype="<u4", count=3 * nloc + 1, offset=int(h[12]))
    return (off[3::3] - off[0:-1:3]).astype(np.int64), nloc


def run_batching(args):
    """10^6 uniform random (view, location) block requests per launch on the
    17 x 17 x 1024^2 light field: the persistent binned kernel (autotuned,
    eager and replayed as a CUDA graph) against one warp per request, plus a
    full decode of the same light field."""
    import torch
    from paper_1805_06019_gb300 import rlfc

    torch.cuda.set_device(0)
    p = dict(lf_synth.PRESETS["batching"])
    tau = args.tau if args.tau is not None else p["taus"][0]
    n = args.n_requests or p["n_requests"]
    U, V = p["U"], p["V"]
    t0 = time.time()
    if args.view_size and args.view_size != p["W"]:
        # the same scene and tree at a smaller view size (profiling case)
        p["W"] = p["H"] = args.view_size
        lf = lf_synth.make_lightfield(U, V, p["W"], p["H"], p["disparities"], p["sigma"], p["id"], True)
    else:
        lf = lf_synth.preset_lightfield("batching")
    t_synth = time.time() - t0
    d_lf = torch.from_numpy(lf).cuda()
    data = rlfc.encode(d_lf, U, V, p["L"], p["c"], tau_p=tau, tau_b=16 * tau)
    del d_lf
    st = rlfc.Stream(data)
    info = st.info
    pv, pl = lf_synth.random_requests(n, U * V, st.nloc, p["id"])
    views = torch.from_numpy(pv.view(np.int32)).cuda()
    locs = torch.from_numpy(pl.view(np.int32)).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    cur = torch.cuda.current_stream()
    out_ref = torch.empty((n, 4, 4, 3), dtype=torch.uint8, device="cuda")
    out = torch.empty((n, 4, 4, 3), dtype=torch.uint8, device="cuda")

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(cur)
            fn()
            b.record(cur)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms)), float(np.mean(ms))

    per_req_ms, _ = timed(lambda: st.decode_blocks(views, locs, out_ref), args.steps, args.warmup)
    b = rlfc.Batch(st, n)
    b.config = dict(graph=0)
    chosen = b.autotune(views, locs, out)
    eager_ms, _ = timed(lambda: b.decode(views, locs, out), args.steps, args.warmup)
    identical_eager = bool(torch.equal(out, out_ref))
    # per-kernel split of the eager path
    rlfc.trace_read(reset=True)
    rlfc.trace_enable(True)
    eager_trace_steps = args.steps
    for _ in range(eager_trace_steps):
        flush.fill_(1)
        b.decode(views, locs, out)
    torch.cuda.synchronize()
    trace = rlfc.trace_read(reset=True)
    rlfc.trace_enable(False)
    b.config = dict(graph=1)
    out.zero_()
    graph_ms, _ = timed(lambda: b.decode(views, locs, out), args.steps, args.warmup)
    identical_graph = bool(torch.equal(out, out_ref))

    # full decode of the light field, the bandwidth-bound form of the decoder
    lf_out = torch.empty((U * V, p["H"], p["W"], 3), dtype=torch.uint8, device="cuda")
    dec_ms, _ = timed(lambda: st.decode_all(lf_out), args.steps, args.warmup)

    peak, peak_src = _peaks()
    loc_words, nloc = _stream_location_words(data)
    hit = np.unique(pl)
    rec_bytes_hit = int(4 * loc_words[hit].sum())
    # records of the locations hit, their offsets and top-RKV blocks, the
    # requests read, 48 B written per request
    alg_batch = rec_bytes_hit + 12 * len(hit) + 96 * info.n_top * len(hit) + 8 * n + 48 * n
    stream_read = info.record_bytes + 4 * (3 * nloc + 1) + info.top_bytes
    alg_dec = stream_read + U * V * p["W"] * p["H"] * 3
    kern = {}
    for name, (launches, tot) in trace.items():
        kern[name] = {"launches": launches, "avg_ms": tot / max(launches, 1)}
    dk = kern.get("decode_binned_kernel", {"avg_ms": eager_ms})
    kbytes_binned = rec_bytes_hit + 12 * len(hit) + 96 * info.n_top * len(hit) + 4 * n + 8 * n + 48 * n
    dk_gbs = kbytes_binned / (dk["avg_ms"] * 1e-3) / 1e9

    # end to end: requests uploaded from pinned memory, blocks downloaded
    h_v = torch.from_numpy(pv.view(np.int32)).pin_memory()
    h_l = torch.from_numpy(pl.view(np.int32)).pin_memory()
    h_out = torch.empty(out.shape, dtype=torch.uint8).pin_memory()
    e_steps = min(args.steps, 5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for _ in range(e_steps):
        views.copy_(h_v, non_blocking=True)
        locs.copy_(h_l, non_blocking=True)
        b.decode(views, locs, out)
        h_out.copy_(out, non_blocking=True)
    e1.record(cur)
    torch.cuda.synchronize()
    e_ms = e0.elapsed_time(e1) / e_steps

    # CPU oracle on a bounded sample of the requests
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ost = oracle.Stream(oracle.encode(lf, U, V, B=4, L=p["L"], c=p["c"], tau_p=tau, tau_b=16 * tau))
        t_enc = time.perf_counter() - t0
        k = min(n, args.cpu_sample_requests)
        t0 = time.perf_counter()
        for r in range(k):
            ost.decode_block(int(pv[r]), int(pl[r]))
        t_cpu = time.perf_counter() - t0
        cpu = {"value": 16 * k / t_cpu / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle DecompressLFIBlock for the first {k} of the {n} requests "
                         f"({t_cpu:.1f} s, 1 thread, one call each; stream written by the oracle "
                         f"encoder in {t_enc:.0f} s)", "host_cpus": os.cpu_count()}

    px = 16 * n
    line = {"metric": METRIC, "value": px / (graph_ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": graph_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int decode", "data": "synthetic",
            "config": {"workload": f"batching: {U}x{V} views of {p['W']}x{p['H']} RGB, 8 planes -3..3, "
                                   f"contrast-modulated, 3-level tree {tuple(p['c'][1:])}, 4x4 blocks, tau {tau}; "
                                   f"{n} uniform random (view, location) requests per launch",
                       "U": U, "V": V, "W": p["W"], "H": p["H"], "levels": p["L"], "tau": tau,
                       "n_requests": n, "stream_bytes": int(info.stream_bytes),
                       "locations_hit": int(len(hit)), "nloc": int(nloc),
                       "l2": "flushed by a 256 MiB write before every timed launch",
                       "synth_s": t_synth},
            "batched_graph": {"ms": graph_ms, "requests_per_s": n / (graph_ms * 1e-3),
                              "config": chosen, "identical_to_per_request": identical_graph},
            "batched_eager": {"ms": eager_ms, "requests_per_s": n / (eager_ms * 1e-3),
                              "identical_to_per_request": identical_eager},
            "per_request": {"ms": per_req_ms, "requests_per_s": n / (per_req_ms * 1e-3)},
            "speedup_vs_per_request": per_req_ms / graph_ms,
            "kernels": kern,
            "roofline": {"bound": "hbm", "kernel": "decode_binned_kernel", "achieved": dk_gbs, "peak": peak,
                         "unit": "GB/s", "frac": dk_gbs / peak, "peak_source": f"{peak_src} hbm_gbs (burst copy)",
                         "traffic": TRAFFIC_PER_LAUNCH.get(("batching", tau, n, "decode_binned_kernel")),
                         "bytes_per_launch": kbytes_binned, "avg_launch_ms": dk["avg_ms"]},
            "algorithmic_bytes_per_call": alg_batch,
            "decode_all": {"ms": dec_ms, "mpix_s": U * V * p["W"] * p["H"] / (dec_ms * 1e-3) / 1e6,
                           "algorithmic_bytes": alg_dec, "gbs": alg_dec / (dec_ms * 1e-3) / 1e9,
                           "hbm_frac": alg_dec / (dec_ms * 1e-3) / 1e9 / peak},
            "e2e": {"value": px / (e_ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": e_ms,
                    "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 48 * n, "steps": e_steps},
            "cpu_baseline": cpu,
            "gpu_launches": sum(v["launches"] for v in kern.values())}
    print(json.dumps(line))


def _serve_trace(rlfc, srv, ids, grids, pool, rate, n, preset_id, u8):
    """Submit n requests arriving as a seeded Poisson process at `rate` to
    srv (light field uniform over `ids`, camera and focus plane uniform), each
    into a free pinned destination of `pool` (reused once its request has
    completed), and wait for every completion.  Latency is submit -> view in
    pinned host memory."""
    arr = lf_synth.poisson_arrivals(rate, n, preset_id=preset_id)
    lf_i, fu, fv, fd = lf_synth.serving_requests(n, len(ids), preset_id=preset_id)
    free = {k: list(range(len(v))) for k, v in pool.items()}
    owner = {}
    comps, waited = [], 0
    base = rlfc.Server.now() + 0.05
    for i in range(n):
        U, V, W, H, disp = grids[lf_i[i]]
        while not free[(W, H)]:
            waited += 1
            for c in srv.poll():
                comps.append(c)
                free[owner[c["ticket"]][0]].append(owner[c["ticket"]][1])
        slot = free[(W, H)].pop()
        while rlfc.Server.now() < base + arr[i]:
            pass
        t = srv.submit(ids[lf_i[i]], fu[i] * (U - 1), fv[i] * (V - 1),
                       disp[min(int(fd[i] * len(disp)), len(disp) - 1)], pool[(W, H)][slot])
        owner[t] = ((W, H), slot)
        if i % 16 == 0:
            for c in srv.poll():
                comps.append(c)
                free[owner[c["ticket"]][0]].append(owner[c["ticket"]][1])
    comps += srv.poll(wait=True)
    lat = np.array([c["t_done"] - c["t_submit"] for c in comps]) * 1e3
    span = max(c["t_done"] for c in comps) - min(c["t_submit"] for c in comps)
    px = sum(grids[c["lf"]][2] * grids[c["lf"]][3] for c in comps)
    return {"format": "u8" if u8 else "f32", "rate_req_s": rate, "requests": n,
            "ok": int(sum(c["status"] == 0 for c in comps)),
            "views_per_s": len(comps) / span, "mpix_s": px / span / 1e6,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_batch": float(np.mean([c["batch"] for c in comps])),
            "client_waits_for_buffers": waited}


def serving_compare(rlfc, torch, rates, seconds, pool_size=256):
    """The served form against the plain per-request launch on the same GPU:
    the three 5 x 5 x 256^2 serving light fields (tau 2 / 4 / 8) resident, the
    same seeded Poisson trace of 8-bit 256^2 view requests at each rate, through
    the server configured two ways: one render call per request on one stream
    (calls queue in the stream), and continuous batching (up to 64 views per
    call, four streams, one call in flight per stream)."""
    streams, grids = [], []
    for name, tau in lf_synth.SERVING_FLEET:
        if name != "serving_small":
            continue
        p = lf_synth.PRESETS[name]
        d_lf = lf_synth.preset_lightfield_torch(name)
        streams.append(rlfc.Stream(rlfc.encode(d_lf, p["U"], p["V"], p["L"], p["c"], tau_p=tau, tau_b=16 * tau)))
        grids.append((p["U"], p["V"], p["W"], p["H"], p["disparities"]))
        del d_lf
    W, H = grids[0][2], grids[0][3]
    pool = {(W, H): [torch.empty((H, W, 3), dtype=torch.uint8).pin_memory() for _ in range(pool_size)]}
    forms = {"per_request": dict(n_streams=1, max_batch=1, max_inflight=64),
             "served": dict(n_streams=4, max_batch=64, max_inflight=1)}
    out = {}
    for form, cfg in forms.items():
        srv = rlfc.Server(memory_budget=1 << 30, **cfg)
        ids = [srv.add(st) for st in streams]
        # a short warm-up trace, then the measured rates
        _serve_trace(rlfc, srv, ids, grids, pool, 2000.0, 200, 40, True)
        out[form] = {"config": cfg, "rates": [_serve_trace(rlfc, srv, ids, grids, pool, r, max(int(r * seconds), 200),
                                                           41 + ri, True) for ri, r in enumerate(rates)]}
        srv.close()
    for st in streams:
        st.close()
    sat = {f: max(x["views_per_s"] for x in v["rates"]) for f, v in out.items()}
    out["max_views_per_s"] = sat
    out["served_over_per_request_at_saturation"] = sat["served"] / sat["per_request"]
    out["workload"] = ("3 resident 5x5x256^2 light fields (tau 2/4/8), 8-bit 256^2 view requests, the same seeded "
                       f"Poisson trace per rate ({seconds} s each); latency = submit to view in pinned host memory")
    return out


def run_serving(args):
    """Eight resident light fields (three 5x5x256^2, three 9x9x512^2, two
    17x17x1024^2), view requests at their native sizes arriving as a Poisson
    process at several rates, served with continuous batching; latency is
    submit -> view copied to pinned host memory.  Each output format (float
    RGB, 8-bit RGB) runs the same rates."""
    import torch
    from paper_1805_06019_gb300 import rlfc

    torch.cuda.set_device(0)
    streams, grids = [], []
    t0 = time.time()
    for name, tau in lf_synth.SERVING_FLEET:
        p = lf_synth.PRESETS[name]
        lf = lf_synth.preset_lightfield(name)
        d_lf = torch.from_numpy(lf).cuda()
        data = rlfc.encode(d_lf, p["U"], p["V"], p["L"], p["c"], tau_p=tau, tau_b=16 * tau)
        del d_lf, lf
        streams.append(rlfc.Stream(data))
        grids.append((p["U"], p["V"], p["W"], p["H"], p["disparities"]))
    t_setup = time.time() - t0
    resident = sum(int(s.info.device_bytes) for s in streams)
    budget = args.serve_budget << 20
    srv = rlfc.Server(n_streams=args.serve_streams, max_batch=args.serve_max_batch, memory_budget=budget,
                      max_inflight=args.serve_inflight)
    ids = [srv.add(s) for s in streams]
    rates = [float(r) for r in args.serve_rates.split(",")]
    formats = args.serve_formats.split(",")
    results = []
    pools = {}
    for fmt, ri, rate in [(f, ri, r) for f in formats for ri, r in enumerate(rates)]:
        # pinned destinations per format, reused once their request has completed
        if fmt not in pools:
            pools.clear()
            pools[fmt] = {}
            for U, V, W, H, _ in grids:
                if (W, H) not in pools[fmt]:
                    pools[fmt][(W, H)] = [torch.empty((H, W, 3), dtype=torch.uint8 if fmt == "u8" else torch.float32)
                                          .pin_memory() for _ in range(args.serve_pool)]
        pool = pools[fmt]
        n = max(int(rate * args.serve_seconds), 50)
        results.append(_serve_trace(rlfc, srv, ids, grids, pool, rate, n, 4 + ri, fmt == "u8"))
    srv.close()
    top = [r for r in results if r["format"] == formats[0]][-1]
    line = {"metric": METRIC, "value": top["mpix_s"], "unit": UNIT, "n_gpus": 1, "steps": len(rates), "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving: 8 resident light fields (3x 5x5x256^2 tau 2/4/8, 3x 9x9x512^2 "
                                   "tau 2/4/8, 2x 17x17x1024^2 tau 4/8), native-size view requests, "
                                   "Poisson arrivals; latency = submit to view in pinned host memory",
                       "formats": formats, "value_format": formats[0], "rates": rates, "seconds_per_rate": args.serve_seconds,
                       "n_streams": args.serve_streams, "max_batch": args.serve_max_batch,
                       "max_inflight": args.serve_inflight,
                       "memory_budget_mib": args.serve_budget, "resident_device_bytes": resident,
                       "setup_s": t_setup},
            "serving": results}
    print(json.dumps(line))


def run_learned(args):
    print(json.dumps(learned_result(args)))


def learned_result(args, tau=None):
    """The learned encoder aid on the 15 x 15 x 625 x 434 light field
    (lenslet-like disparities within +-1, sigma 2, 3-level (3, 5) tree):
    level-0 blocks labelled by the exhaustive (shift, mode) search, the
    network trained on the GPU, mode agreement on held-out blocks, and bpp /
    PSNR of the plain, searched and aided encodes."""
    import torch
    from paper_1805_06019_gb300 import learned, rlfc

    torch.cuda.set_device(0)
    p = lf_synth.PRESETS["learned"]
    U, V, W, H, L, c = p["U"], p["V"], p["W"], p["H"], p["L"], p["c"]
    if tau is None:
        tau = args.tau if args.tau is not None else p["taus"][0]
    lam = args.lam_q8
    d = lf_synth.preset_lightfield_torch("learned")
    lf = d.cpu().numpy()
    px = U * V * W * H
    cur = torch.cuda.current_stream()

    def ev_time(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        r = fn()
        b.record(cur)
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    plain = rlfc.encode(d, U, V, L, c, tau_p=tau, tau_b=16 * tau)
    searched, resid, label, index, n = learned.leaf_dataset(d, U, V, L, c, tau, 16 * tau, 0, tau, lam)
    x, y = learned.features(resid, label, index, n)
    g = torch.Generator(device="cpu")
    g.manual_seed(0)
    perm = torch.randperm(n, generator=g).cuda()
    n_train = int(0.9 * n)
    tr, te = perm[:n_train], perm[n_train:]
    # an untimed epoch of a throwaway network loads the kernels first
    xt, yt = x[tr], y[tr]
    learned.Aid(seed=1).train(xt[:65536], yt[:65536], epochs=1, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    aid = learned.Aid(seed=0)
    t0 = time.time()
    hist = aid.train(xt, yt, epochs=args.epochs, batch=4096, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    # multiply-adds of one sample's step: forward 48x64 + 64x64 + 64x112, the
    # weight gradients the same, the deltas 112x64 + 64x64 (each counted
    # once, not once per BF16 part of a split operand)
    flop_sample = 2 * (3 * (NI_ * 64 + 64 * 64 + 64 * 112) - NI_ * 64)
    train_tflops = flop_sample * n_train * args.epochs / train_s / 1e12
    pred_te = aid.predict(x[te])
    agree = float((pred_te == y[te]).float().mean().item())
    classes = torch.bincount(y[tr].long(), minlength=256)
    majority = float(classes.max().item()) / n_train
    pred_all = aid.predict(x)
    agree_all = float((pred_all == y).float().mean().item())
    aided = learned.encode_aided(d, U, V, L, c, tau, 16 * tau, aid, x, index, resid.shape[0], 0, tau, lam)
    # per-block decision time: exhaustive search vs statistics + network
    blocks = resid.index_select(0, index.long())
    for _ in range(3):
        learned.search(blocks, 0, tau, lam)
        xs, _ = learned.features(blocks, None, None, n)
        aid.predict(xs)
    _, t_search = ev_time(lambda: learned.search(blocks, 0, tau, lam))
    _, t_feat = ev_time(lambda: learned.features(blocks, None, None, n))
    _, t_pred = ev_time(lambda: aid.predict(xs))

    def quality(data):
        dec = rlfc.Stream(data).decode_all().cpu().numpy()
        return {"bytes": len(data), "bpp": 8.0 * len(data) / px, "psnr_db": learned.psnr_ycocg(lf, dec)}

    q_plain, q_search, q_aided = quality(plain), quality(searched), quality(aided)
    hist_labels = torch.bincount(y.long(), minlength=256).cpu().numpy()
    shift_share = [float(hist_labels[(s_ << 5):(s_ << 5) + 28].sum()) / n for s_ in range(4)]
    line = {"metric": METRIC, "value": agree, "unit": "mode agreement (held-out blocks)", "n_gpus": 1,
            "steps": args.epochs, "warmup": 0, "ms_per_step": train_s * 1e3 / max(args.epochs, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)",
            "data": "synthetic",
            "config": {"workload": f"learned encoder aid: {U}x{V} views of {W}x{H} RGB, disparities within "
                                   f"+-1, sigma 2, 3-level tree {tuple(c[1:])}, tau {tau}; level-0 blocks kept "
                                   f"by the energy test labelled by the exhaustive (shift, mode) search "
                                   f"(tau_err {tau}, lambda {lam}/256); 90/10 split",
                       "labelled_blocks": n, "train_blocks": n_train, "epochs": args.epochs, "batch": 4096},
            "train_loss_per_epoch": hist, "train_s": train_s,
            "agreement_heldout": agree, "agreement_all": agree_all, "majority_class_share": majority,
            "label_shift_share": shift_share,
            "plain": q_plain, "search": q_search, "aided": q_aided,
            "aided_vs_plain": {"bpp_change": q_aided["bpp"] - q_plain["bpp"],
                               "psnr_change_db": q_aided["psnr_db"] - q_plain["psnr_db"]},
            "aided_vs_search": {"bpp_change": q_aided["bpp"] - q_search["bpp"],
                                "psnr_change_db": q_aided["psnr_db"] - q_search["psnr_db"]},
            "decision_ns_per_block": {"search": t_search * 1e6 / n, "statistics": t_feat * 1e6 / n,
                                      "network": t_pred * 1e6 / n},
            "network_on_tensor_cores": {
                "train_tflops": train_tflops, "train_frac_of_bf16_sustained": train_tflops / _bf16_sustained(),
                "predict_tflops": 2 * (NI_ * 64 + 64 * 64 + 64 * 112) / (t_pred * 1e-3 / n) / 1e12,
                "note": "mma.sync m16n8k16 BF16 with FP32 accumulation; FP32 activations and deltas as BF16 "
                        "high + residual parts; the layers are 48-112 wide, so the kernels are bound by "
                        "fragment loads and synchronisation, not by the tensor pipe"}}
    return line


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="plain", choices=["plain", "tiny"])
    ap.add_argument("--tau", type=int, default=None)
    ap.add_argument("--n-views", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the other thresholds' decode parts")
    ap.add_argument("--no-batching", action="store_true",
                    help="skip the 17x17x1024^2 full-decode and 10^6-request parts")
    ap.add_argument("--no-serving", action="store_true", help="skip the served vs per-request part")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned encoder aid part")
    ap.add_argument("--compare-rates", default="5000,10000,20000,40000,80000")
    ap.add_argument("--compare-seconds", type=float, default=1.0)
    ap.add_argument("--cpu-sample-views", type=int, default=400)
    ap.add_argument("--workload", choices=["step", "batching", "serving", "learned"], default="step",
                    help="step: decode-all + render (default); batching: random block requests; "
                         "serving: Poisson view requests on resident light fields")
    ap.add_argument("--serve-rates", default="500,1000,2000,5000")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-max-batch", type=int, default=64)
    ap.add_argument("--serve-budget", type=int, default=2048, help="MiB of outputs in flight")
    ap.add_argument("--serve-inflight", type=int, default=1, help="render calls queued per stream")
    ap.add_argument("--serve-pool", type=int, default=48, help="pinned destinations per view size")
    ap.add_argument("--serve-formats", default="f32,u8", help="output formats served, in order (f32, u8)")
    ap.add_argument("--n-requests", type=int, default=None)
    ap.add_argument("--view-size", type=int, default=None, help="batching: view side (default 1024)")
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--lam-q8", type=int, default=256, help="distortion weight of the mode search, /256")
    ap.add_argument("--cpu-sample-requests", type=int, default=200000)
    args = ap.parse_args()
    if args.workload == "batching" and args.impl == "ours":
        run_batching(args)
    elif args.workload == "serving" and args.impl == "ours":
        run_serving(args)
    elif args.workload == "learned" and args.impl == "ours":
        run_learned(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
