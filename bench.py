"""Benchmark of the AD-LBR hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timed unit ("step"): one coherence-enhancing-diffusion step on a 4096 x 4096
FP32 synthetic fingerprint-like image (sigma = 1, rho = 4, alpha = 1e-4 so
kappa <= 100, C = 1e-5, dt = 0.02): the tensor stage D(J_rho(grad u_sigma)),
the AD-LBR stencils of D (re-built every step), and one explicit step
u <- u - dt A u.  Inputs are resident in HBM; the working set (about 1 GB)
is larger than L2, so no flush is needed between steps.

Under torchrun every rank advances its own image (independent units, no
collective on the data path: weak scaling); the reported time is the max over
ranks and ``value`` is the points of all ranks per second.

``--impl reference`` times the FP64 CPU oracle (the only reference this
method has: the paper ships no code) on a bounded crop of the same workload.
"""
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

METRIC = "AD-LBR apply Gpts/s (% HBM roofline); implicit step ms, NN-PCG vs CG @1e-6"
UNIT = "Gpts/s"
N_SIDE = 4096
CED = dict(sigma=1.0, rho=4.0, alpha=1e-4, C=1e-5, dt=0.02)
SEED = 1
# Algorithmic FP32 operations per point of the fused tensor stage (an FMA
# counts once): sigma blurs 2 x 7, gradient and products 7, rho blurs
# 2 x 3 x 25, eigen epilogue 20.  It is held against the FP32 issue peak:
# SMs x 128 FP32 lanes x the maximum SM clock (fp32_peak_tops).
ALU_OPS_PER_POINT = 2 * 7 + 7 + 2 * 3 * 25 + 20


def fp32_peak_tops():
    """(peak in T operations/s, how it was derived): the device's SM count,
    128 FP32 lanes per SM, the maximum SM clock of MEASURED_PEAKS.json (else
    the device's own)."""
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    mhz, src = None, "device"
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            mhz = json.load(f).get("sm_max_mhz")
        src = "MEASURED_PEAKS.json sm_max_mhz"
    if not mhz:
        mhz = getattr(props, "clock_rate", 2070000) / 1000.0
    return sms * 128 * mhz * 1e6 / 1e12, "derived: %d SMs x 128 FP32 lanes x %.0f MHz (%s)" % (sms, mhz, src)
# DRAM bytes (read + write) of one launch at 4096^2, from an ncu capture of the
# current kernels (dram__bytes_read.sum + dram__bytes_write.sum, one launch each,
# second warm-up step of this benchmark's CED step)
TRAFFIC_4096 = {"ced_fused_kernel": 67.203e6 + 140.874e6, "build2d_kernel": 201.391e6 + 225.406e6,
                # operator + finalize
                "explicit_step": 402.739e6 + 48.194e6 + 134.228e6 + 19.020e6,
                # fused build and operator + finalize (the memset's 67 MB write is
                # not a kernel and is not counted)
                "build_step": 471.089e6 + 294.640e6 + 134.228e6 + 19.020e6}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-implicit", action="store_true", help="skip the implicit-step measurement")
    p.add_argument("--no-3d", action="store_true", help="skip the 3D measurement and precision study")
    p.add_argument("--no-batch", action="store_true", help="skip the batched-step measurement")
    p.add_argument("--no-ced3d", action="store_true", help="skip the 3D CED measurement")
    p.add_argument("--no-eed3d", action="store_true", help="skip the 3D edge-enhancing measurement")
    p.add_argument("--no-spectral", action="store_true", help="skip the periodic spectral study")
    p.add_argument("--no-ann", action="store_true", help="skip the A-NN comparison scheme")
    p.add_argument("--precision-steps", type=int, default=100)
    p.add_argument("--config", type=int, choices=[1, 2, 3, 4, 5], default=2,
                   help="workload: 2 (default) is the headline CED step and its full line; 1, 3, 4 and 5 "
                        "run only that workload's measurement (64^2 FP64 steps, the 256^3 precision "
                        "study, the 2048^2 implicit step, the serving batch) and print it as one line")
    p.add_argument("--cpu-configs", action="store_true",
                   help="only time the oracle on samples of the other workloads (64^2 FP64 build and steps, "
                        "3D steps, CG iterations, batch items), one thread and every host core")
    p.add_argument("--profile-cg", action="store_true",
                   help="only run three plain-CG implicit solves at 2048^2 (for ncu launch lists)")
    p.add_argument("--profile-unet", action="store_true",
                   help="only run four tensor-core U-Net forwards at 512^2 (for ncu launch lists)")
    p.add_argument("--profile-gather", action="store_true",
                   help="only run three gather-form applications of the operator on 2048^2 CED stencils "
                        "(for ncu)")
    p.add_argument("--profile-fcg", action="store_true",
                   help="only run two 40-iteration flexible-CG solves with the U-Net preconditioner "
                        "at 2048^2 (for ncu launch lists)")
    return p.parse_args()


# ----------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_uuid=None):
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "50"]
        if dev_uuid:
            cmd += ["-i", dev_uuid]
        self.lines = []
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        rows = [l for (t, l) in self.lines if t0 - 0.05 <= t <= t1 + 0.05] or [l for _, l in self.lines]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in rows:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[3 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def init_dist(backend="nccl"):
    """(world size, rank, local rank) from the torchrun environment; joins the
    process group when there is more than one rank."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x):
    """Max of a host scalar over ranks (the slowest rank's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank):
    """Each rank advances its own image (independent units, weak scaling)."""
    return SEED + rank


def job_value(ws, points_per_rank, ms_max):
    """Whole-job throughput: the points of all ranks over the slowest rank's time."""
    return ws * points_per_rank / (ms_max * 1e-3) / 1e9


def time_ms(fn, reps, stream):
    """Mean device time of fn() over reps calls (CUDA events on `stream`)."""
    import torch
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


# ----------------------------------------------------------------- sub-measurements
def bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def unet_forward_measurement(params, H, W, reps=20):
    """The preconditioner's network (25 -> 16/32/64 channels, batch 1, H x W)
    on the tensor cores and on the FP32 SIMT kernels: CUDA-event times over
    `reps` forwards, and the tensor-core forward's dense FLOPs (2 per
    multiply-add of every convolution) against the measured BF16 peak."""
    import torch
    from paper_1301_3925_gb300 import adlbr as ab
    from paper_1301_3925_gb300 import nn
    net = ab.adlbr_unet_create(nn.NF, 16, 32, 64, 1, H, W)
    try:
        x = torch.randn(nn.NF * H * W, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
        y = torch.empty(H * W, device="cuda")
        res = {}
        for name, tc in (("fp32_ms", False), ("tc_ms", True)):
            ab.adlbr_unet_set_tensor_cores(net, tc)
            for _ in range(3):
                ab.adlbr_unet_forward(net, params, x, y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                ab.adlbr_unet_forward(net, params, x, y)
            e1.record()
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1) / reps
    finally:
        ab.adlbr_unet_destroy(net)
    # per layer: (co, ci, k) at full, half, quarter resolution
    scale = [1, 1, 4, 4, 16, 16, 4, 4, 1, 1, 1]
    flops = sum(2.0 * co * ci * k * k * H * W / sc
                for (co, ci, k), sc in zip(nn.layer_shapes(nn.NF, 16, 32, 64), scale))
    pk, src = bf16_peak()
    tf = flops / (res["tc_ms"] * 1e-3) / 1e12
    res.update({"grid": [H, W], "gflop": flops / 1e9, "tc_tflops": tf, "bf16_peak_tflops": pk,
                "peak_source": src, "frac_bf16_peak": tf / pk,
                "note": "latency-bound: per-row copy / MMA / epilogue chains over short strips"})
    return res


def implicit_measurement(peak):
    """Implicit step (I + dt A) x = u_n on 2048^2, smooth random orientation,
    kappa in [1, 50], dt = 200 / max A_zz, tolerance 1e-6: plain CG, flexible
    CG with the Jacobi part of the preconditioner alone, and flexible CG with
    the trained U-Net preconditioner (trained here on three other right-hand
    sides of the same operator; training time reported separately)."""
    import torch
    import synth
    from paper_1301_3925_gb300 import adlbr as ab
    from paper_1301_3925_gb300 import nn
    n = 2048
    D = torch.from_numpy(synth.smooth_field2d(n, n, 3, 1.0, 50.0, 16).reshape(3, -1)
                         .astype(np.float32)).cuda()
    g = ab.grid((n, n))
    h = ab.adlbr_build_stencils(g, D, ab.F32, ab.F32)
    try:
        dt = 200.0 / ab.adlbr_stencils_max_diag(h)
        b = torch.from_numpy(synth.u_uniform((n, n), 3).astype(np.float32).ravel()).cuda()
        x = torch.empty_like(b)
        out = {"grid": [n, n], "dt": dt, "rtol": 1e-6, "rhs": "U[0,1] seed 3",
               "field": "smooth orientation, kappa in [1, 50], 16x16 lattice, seed 3"}

        def solve(precond=0, desc=None):
            x.copy_(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, rel = ab.adlbr_step_implicit(h, b, x, dt, 1e-6, 4000, precond=precond, nn=desc)
            torch.cuda.synchronize()
            fb = ab.adlbr_last_fallback() if precond else 0
            return it, rel, (time.perf_counter() - t0) * 1e3, fb

        solve()
        cg = [solve() for _ in range(3)]
        out["cg"] = {"iters": cg[-1][0], "relres": cg[-1][1], "ms": float(np.median([c[2] for c in cg]))}
        solve(2)
        jp = [solve(2) for _ in range(3)]
        out["jacobi_pcg"] = {"iters": jp[-1][0], "relres": jp[-1][1], "ms": float(np.median([c[2] for c in jp]))}
        t0 = time.perf_counter()
        rhs = [torch.from_numpy(synth.u_uniform((n, n), 100 + k).astype(np.float32).ravel()).cuda()
               for k in range(3)]
        params, log = nn.fit(h, rhs, dt, rounds=3, steps=(1500, 700, 700), crop=48)
        torch.cuda.synchronize()
        out["train_s"] = time.perf_counter() - t0
        out["train_loss"] = [r["loss"][-1][1] for r in log]
        jac = params.clone()
        jac[-17:] = 0.0
        for name, th in (("jacobi_fcg", jac), ("nn_fcg", params)):
            pc = nn.Preconditioner(th, n, n)
            try:
                solve(1, pc.desc)
                r = [solve(1, pc.desc) for _ in range(3)]
            finally:
                pc.close()
            out[name] = {"iters": r[-1][0], "relres": r[-1][1], "ms": float(np.median([c[2] for c in r])),
                         "fell_back_to_cg": bool(r[-1][3])}
        out["nn_vs_cg_wallclock"] = out["cg"]["ms"] / out["nn_fcg"]["ms"]
        out["jacobi_pcg_vs_cg_wallclock"] = out["cg"]["ms"] / out["jacobi_pcg"]["ms"]
        out["unet_forward"] = unet_forward_measurement(params, n // nn.RF, n // nn.RF)
        return out
    finally:
        ab.adlbr_stencils_destroy(h)


def profile_cg():
    """Three plain-CG solves of the 2048^2 implicit step (profiling entry)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1301_3925_gb300 import adlbr as ab
    n = 2048
    D = torch.from_numpy(synth.smooth_field2d(n, n, 3, 1.0, 50.0, 16).reshape(3, -1)
                         .astype(np.float32)).cuda()
    g = ab.grid((n, n))
    h = ab.adlbr_build_stencils(g, D, ab.F32, ab.F32)
    dt = 200.0 / ab.adlbr_stencils_max_diag(h)
    b = torch.from_numpy(synth.u_uniform((n, n), 3).astype(np.float32).ravel()).cuda()
    x = torch.empty_like(b)
    for _ in range(3):
        x.copy_(b)
        it, rel = ab.adlbr_step_implicit(h, b, x, dt, 1e-6, 4000)
    torch.cuda.synchronize()
    ab.adlbr_stencils_destroy(h)
    print(json.dumps({"profile_cg": {"iters": it, "relres": rel}}))
    return 0


def profile_fcg():
    """Two flexible-CG solves of the 2048^2 implicit step with the tensor-core
    U-Net preconditioner, stopped after 40 iterations (profiling entry).  The
    network is untrained (He-normal weights, output layer scaled by 1e-3):
    an iteration runs the same kernels as with trained weights."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1301_3925_gb300 import adlbr as ab
    from paper_1301_3925_gb300 import nn
    n = 2048
    D = torch.from_numpy(synth.smooth_field2d(n, n, 3, 1.0, 50.0, 16).reshape(3, -1)
                         .astype(np.float32)).cuda()
    g = ab.grid((n, n))
    h = ab.adlbr_build_stencils(g, D, ab.F32, ab.F32)
    dt = 200.0 / ab.adlbr_stencils_max_diag(h)
    b = torch.from_numpy(synth.u_uniform((n, n), 3).astype(np.float32).ravel()).cuda()
    x = torch.empty_like(b)
    shapes = nn.layer_shapes(nn.NF, 16, 32, 64)
    th = nn.init_params(sum(co * ci * k * k + co for co, ci, k in shapes), shapes, 1)
    th[-17:] *= 1e-3   # output layer (16 weights + bias)
    pc = nn.Preconditioner(torch.from_numpy(th).cuda(), n, n)
    out = []
    try:
        for _ in range(2):
            x.copy_(b)
            try:
                out.append(ab.adlbr_step_implicit(h, b, x, dt, 1e-6, 40, precond=1, nn=pc.desc))
            except ab.AdlbrError as e:   # E_NOT_CONVERGED after 40 iterations
                out.append(str(e).split(":")[0])
        torch.cuda.synchronize()
    finally:
        pc.close()
        ab.adlbr_stencils_destroy(h)
    print(json.dumps({"profile_fcg": {"solves": [str(o) for o in out]}}))
    return 0


def profile_gather():
    """Three applications of the operator in its gather form on the CED
    stencils of a 2048^2 crop of the fingerprint image (F16 weights, FP32 u);
    the first builds the table (profiling entry)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_1301_3925_gb300 import adlbr as ab
    n = 2048
    g = ab.grid((n, n))
    u = torch.from_numpy(synth.fingerprint(N_SIDE, SEED)[:n, :n].astype(np.float32).ravel()).cuda()
    scratch = torch.empty(ab.adlbr_ced_scratch_bytes(g), dtype=torch.uint8, device="cuda")
    h = ab.adlbr_ced_stencils(None, g, u, scratch, *(CED[k] for k in ("sigma", "rho", "alpha", "C")), ab.F16)
    Au = torch.empty_like(u)
    try:
        ab.adlbr_stencils_set_operator(h, ab.OP_GATHER)
        for _ in range(3):
            ab.adlbr_apply(h, u, Au, ab.F32)
        torch.cuda.synchronize()
    finally:
        ab.adlbr_stencils_destroy(h)
    print(json.dumps({"profile_gather": {"Au_abs_max": float(Au.abs().max())}}))
    return 0


def batch_measurement(peak, steps=20):
    """Serving-style batch: 64 images (sides U{256..2048}) and 8 volumes
    (sides U{64..192}), each with its own seeded field (kappa_i ~ U[5, 100]:
    smooth 2D orientation field / 3D needle field), F16 weights, FP32 u,
    dt_i = 1 / max A_zz.  `steps` batched steps (one graph launch each,
    autotuned tile shapes) against the same steps issued item by item."""
    import torch
    import synth
    from paper_1301_3925_gb300 import adlbr as ab
    items = synth.batch_items()
    st = torch.cuda.current_stream()
    hs, us, dts = [], [], []
    pts2, pts3 = 0, 0
    try:
        for k, it in enumerate(items):
            shape = it["shape"]
            if it["dim"] == 2:
                D = synth.smooth_field2d_torch(*shape, it["seed"], 1.0, it["kappa"], 16).reshape(3, -1)
                pts2 += shape[0] * shape[1]
            else:
                D = torch.from_numpy(synth.needle_field3d(shape[0], it["seed"], kappa=it["kappa"],
                                                          dtype=np.float32).reshape(6, -1)).cuda()
                pts3 += shape[0] ** 3
            h = ab.adlbr_build_stencils(ab.grid(shape), D, ab.F32, ab.F16)
            hs.append(h)
            del D
            dts.append(1.0 / ab.adlbr_stencils_max_diag(h))
            us.append(torch.rand(int(np.prod(shape)), device="cuda",
                                 generator=torch.Generator(device="cuda").manual_seed(it["seed"])))
        t0 = time.perf_counter()
        b = ab.adlbr_batch_create(hs, us, dts, autotune=True)
        tune_s = time.perf_counter() - t0
        try:
            shape, tuned_ms, points, ntiles = ab.adlbr_batch_config(b)
            ab.adlbr_batch_step(b, 2)
            ms = time_ms(lambda: ab.adlbr_batch_step(b, steps), 1, st) / steps
        finally:
            ab.adlbr_batch_destroy(b)
        scratch = [torch.empty(ab.adlbr_step_scratch_bytes(h, ab.F32), dtype=torch.uint8, device="cuda")
                   for h in hs]

        def looped():
            for _ in range(steps):
                for h, u, d, sc in zip(hs, us, dts, scratch):
                    ab.adlbr_step_explicit(h, u, sc, ab.F32, d, 1)

        ms_loop = time_ms(looped, 1, st) / steps
        algo = 24 * pts2 + 36 * pts3
        gbs = algo / (ms * 1e-3) / 1e9
        return {"items": {"images": sum(1 for i in items if i["dim"] == 2),
                          "volumes": sum(1 for i in items if i["dim"] == 3)},
                "points": points, "steps": steps, "tiles": ntiles,
                "shape": {"tile2d": list(shape[:2]), "block3d": list(shape[2:])},
                "create_s": tune_s, "tuned_accumulate_ms": tuned_ms,
                "ms_per_step": ms, "gpts": points / (ms * 1e-3) / 1e9, "gbs": gbs,
                "frac_hbm": gbs / peak, "bytes_per_point": {"2d": 24, "3d": 36},
                "looped_ms_per_step": ms_loop, "speedup_vs_looped": ms_loop / ms,
                "kernel_launches_per_step": {"batched": 3, "looped": 2 * len(hs)}}
    finally:
        for h in hs:
            ab.adlbr_stencils_destroy(h)


def spectral_measurement(n=128, k=7):
    """The periodic spectral study (Fig. Eigen): the k smallest eigenvalues of
    the scheme for D = [[19/2, 6], [6, 4]] on an n x n periodic grid by LOBPCG
    on the FP64 operator (preconditioned by the library's CG), scaled by n^2
    (h = 1/n) and set beside 4 pi^2 <m, D m>, the continuous eigenvalues."""
    import time
    import torch
    from paper_1301_3925_gb300 import adlbr as ab
    from paper_1301_3925_gb300 import spectral
    D = np.array([[9.5, 6.0], [6.0, 4.0]])
    planes = torch.tensor([D[0, 0], D[0, 1], D[1, 1]], dtype=torch.float64, device="cuda")
    # warm-up on a 16^2 grid: the first use of the library's FP64 kernels and
    # of the block algebra (cuBLAS handles, host eigensolver) is paid here,
    # not in the timed study (it made the timed figure swing by seconds)
    hw = ab.adlbr_build_stencils(ab.grid((16, 16), ab.PERIODIC), planes[:, None].expand(3, 256).contiguous(),
                                 ab.F64, ab.F64)
    try:
        spectral.lobpcg_smallest(hw, 256, k, tol=1e-8)
    finally:
        ab.adlbr_stencils_destroy(hw)
    Dd = planes[:, None].expand(3, n * n).contiguous()
    h = ab.adlbr_build_stencils(ab.grid((n, n), ab.PERIODIC), Dd, ab.F64, ab.F64)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        theta, _, its = spectral.lobpcg_smallest(h, n * n, k, tol=1e-10)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
    finally:
        ab.adlbr_stencils_destroy(h)
    r = np.arange(-8, 9)
    mx, my = np.meshgrid(r, r, indexing="ij")
    cont = np.sort(4 * np.pi ** 2 * (D[0, 0] * mx ** 2 + 2 * D[0, 1] * mx * my + D[1, 1] * my ** 2).ravel())[:k]
    scaled = theta * n * n
    return {"grid": [n, n], "D": D.tolist(), "k": k, "lobpcg_iters": its, "ms": ms,
            "n2_lambda": [float(v) for v in scaled], "continuous": [float(v) for v in cont],
            "max_rel_dev": float(np.abs(scaled - cont)[1:].max() / cont[1:].max())}


def ann_measurement(peak):
    """The A-NN comparison scheme (Sec. 4.1, Remark rem:WG) beside AD-LBR on
    the GPU: Fig. Radius (largest stencil radius over 3600 orientations at
    kappa = 10, both schemes built by the library), and build and operator
    times on a 2048^2 smooth field (kappa <= 10, F16 weights, FP32 u)."""
    import torch
    import synth
    from paper_1301_3925_gb300 import adlbr as ab
    out = {}
    th = np.linspace(0, np.pi, 3600, endpoint=False)
    D = torch.from_numpy(synth.D_from_angle(th, 10.0).reshape(3, -1)).cuda()
    g = ab.grid((1, th.size))
    for name, sch in (("adlbr", ab.SCHEME_ADLBR), ("ann", ab.SCHEME_ANN)):
        h = ab.adlbr_build_stencils_scheme(g, D, ab.F64, ab.F64, sch)
        try:
            offs = torch.zeros((th.size, 3, 2), dtype=torch.int16, device="cuda")
            w = torch.zeros((th.size, 3), dtype=torch.float64, device="cuda")
            ab.adlbr_stencils_export(h, offs, w)
            out["fig_radius_max_" + name] = float(offs.double().pow(2).sum(-1).sqrt().max())
        finally:
            ab.adlbr_stencils_destroy(h)
    n = 2048
    Ds = torch.from_numpy(synth.smooth_field2d(n, n, 3, 1.0, 10.0, 16).reshape(3, -1).astype(np.float32)).cuda()
    gg = ab.grid((n, n))
    u = torch.rand(n * n, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    Au = torch.empty_like(u)
    st = torch.cuda.current_stream()
    for name, sch in (("adlbr", ab.SCHEME_ADLBR), ("ann", ab.SCHEME_ANN)):
        h = ab.adlbr_build_stencils_scheme(gg, Ds, ab.F32, ab.F16, sch)
        try:
            ab.adlbr_stencils_check(h)
            bms = time_ms(lambda: ab.adlbr_build_stencils_scheme(gg, Ds, ab.F32, ab.F16, sch, out=h), 10, st)
            ams = time_ms(lambda: ab.adlbr_apply(h, u, Au, ab.F32), 20, st)
            offs = torch.zeros((n * n, 3, 2), dtype=torch.int16, device="cuda")
            w = torch.zeros((n * n, 3), dtype=torch.float32, device="cuda")
            ab.adlbr_stencils_export(h, offs, w)
            r = offs.double().pow(2).sum(-1).sqrt().max(-1).values
            out[name + "_2048"] = {"build_ms": bms, "apply_ms": ams, "apply_gpts": n * n / (ams * 1e-3) / 1e9,
                                   "radius_mean": float(r.mean()), "radius_max": float(r.max())}
            del offs, w
        finally:
            ab.adlbr_stencils_destroy(h)
    out["field_2048"] = "smooth orientation, kappa in [1, 10], 16x16 lattice, seed 3"
    return out


def eed3d_measurement(steps=10, precond=2, C=7.7e-6):
    """The 3D edge-enhancing experiment (Sec. 5, 3D MRI data) on a synthetic
    stand-in of the scan's shape: 100 x 256 x 256 voxels (z, y, x) of nested
    ellipsoidal shells and inner balls plus N(0, 0.15^2) noise (seed 1);
    sigma 0.5, rho 4 as in the paper, C = 7.7e-6 (so that the largest
    anisotropy ratio is about the paper's 11.2 on this volume); `steps` steps
    of dt = 1e-4 with h = 1/256 (6.55 in grid units, so implicit steps):
    tensor, stencils (F32 weights), CG to 1e-6."""
    import torch
    import synth
    from paper_1301_3925_gb300 import adlbr as ab
    shape = (100, 256, 256)
    N = int(np.prod(shape))
    dt = 1e-4 * 256 * 256
    u0, noisy = synth.shells3d(shape, 1)
    g = ab.grid(shape)
    u = torch.from_numpy(noisy.astype(np.float32).ravel()).cuda()
    x = torch.empty_like(u)
    D = torch.empty(6 * N, dtype=torch.float32, device="cuda")
    scratch = torch.empty(ab.adlbr_ced_scratch_bytes(g), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    h = None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t_tensor, t_build, t_solve, iters = [], [], [], []
    kappa = None
    try:
        for k in range(steps):
            ev[0].record(st)
            ab.adlbr_eed_tensor(g, u, D, 0.5, 4.0, C, scratch)
            ev[1].record(st)
            h = ab.adlbr_build_stencils(g, D, ab.F32, ab.F32, out=h)
            ev[2].record(st)
            x.copy_(u)
            it, _ = ab.adlbr_step_implicit(h, u, x, dt, 1e-6, 4000, precond=precond)
            u.copy_(x)
            ev[3].record(st)
            torch.cuda.synchronize()
            ab.adlbr_stencils_check(h)
            t_tensor.append(ev[0].elapsed_time(ev[1]))
            t_build.append(ev[1].elapsed_time(ev[2]))
            t_solve.append(ev[2].elapsed_time(ev[3]))
            iters.append(it)
            if k == 0:
                # anisotropy ratio of the first tensor on 400,000 sampled voxels
                idx = np.random.default_rng(0).choice(N, 400_000, replace=False)
                d = D.view(6, N)[:, torch.from_numpy(idx).cuda()].double().cpu().numpy()
                M = np.stack([np.stack([d[0], d[3], d[4]], -1), np.stack([d[3], d[1], d[5]], -1),
                              np.stack([d[4], d[5], d[2]], -1)], -2)
                ev3 = np.linalg.eigvalsh(M)
                kappa = float(np.sqrt(ev3[:, 2] / ev3[:, 0]).max())
    finally:
        if h:
            ab.adlbr_stencils_destroy(h)
    ug = u.double().cpu().numpy().reshape(shape)
    rms = lambda a: float(np.sqrt(np.mean(a ** 2)))
    ms = float(np.mean(t_tensor) + np.mean(t_build) + np.mean(t_solve))
    return {"grid": list(shape), "steps": steps, "C": C, "dt_grid_units": dt, "precond": precond,
            "max_kappa_sampled": kappa, "paper_max_kappa": 11.2,
            "ms_per_step": ms, "tensor_ms": float(np.mean(t_tensor)), "stencils_ms": float(np.mean(t_build)),
            "implicit_ms": float(np.mean(t_solve)), "cg_iters_mean": float(np.mean(iters)),
            "gpts_per_step": N / (ms * 1e-3) / 1e9,
            "rms_to_clean": {"noisy": rms(noisy - u0), "result": rms(ug - u0)},
            "input": "synthetic stand-in for the 256 x 256 x 100 MRI scan (not available)"}


def ced3d_measurement(steps=20, precond=2):
    """The 3D coherence-enhancing experiment: 100^3 radial image cos(2 (r/R)^3)
    plus Gaussian noise of variance 0.5 (seed 8), sigma 0.5, rho 4, alpha 1e-2,
    C 1e-5, `steps` steps of dt = 1e-3 on [0,1]^3 (dt = 10 in grid units, so
    implicit steps): tensor, stencils (F32 weights), CG to 1e-6 (precond 0:
    plain; 2: preconditioned by the diagonal)."""
    import torch
    import synth
    from paper_1301_3925_gb300 import adlbr as ab
    n = 100
    dt = 1e-3 * n * n
    u0, noisy = synth.radial3d(n, 8)
    g = ab.grid((n, n, n))
    u = torch.from_numpy(noisy.astype(np.float32).ravel()).cuda()
    x = torch.empty_like(u)
    scratch = torch.empty(ab.adlbr_ced_scratch_bytes(g), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    h = None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_tensor, t_solve, iters = [], [], []
    try:
        for _ in range(steps):
            ev[0].record(st)
            h = ab.adlbr_ced_stencils(h, g, u, scratch, 0.5, 4.0, 1e-2, 1e-5, ab.F32)
            ev[1].record(st)
            x.copy_(u)
            it, _ = ab.adlbr_step_implicit(h, u, x, dt, 1e-6, 4000, precond=precond)
            u.copy_(x)
            ev[2].record(st)
            torch.cuda.synchronize()
            t_tensor.append(ev[0].elapsed_time(ev[1]))
            t_solve.append(ev[1].elapsed_time(ev[2]))
            iters.append(it)
    finally:
        if h:
            ab.adlbr_stencils_destroy(h)
    ug = u.double().cpu().numpy().reshape(n, n, n)
    rms = lambda a: float(np.sqrt(np.mean(a ** 2)))
    ms = float(np.mean(t_tensor) + np.mean(t_solve))
    return {"grid": [n, n, n], "steps": steps, "dt_grid_units": dt, "precond": precond,
            "ms_per_step": ms, "tensor_and_stencils_ms": float(np.mean(t_tensor)),
            "implicit_ms": float(np.mean(t_solve)), "cg_iters_mean": float(np.mean(iters)),
            "gpts_per_step": n ** 3 / (ms * 1e-3) / 1e9,
            "rms_to_clean": {"noisy": rms(noisy - u0), "result": rms(ug - u0)}}


def volume_measurement(peak, steps):
    """3D 256^3 needle field (eigenvalues 1, 1/400, 1/400, smooth random
    orientation on a 16^3 lattice, seed 2): stencil build, operator and
    explicit-step throughput, and the precision study: `steps` explicit steps
    at dt = 1 / max A_zz with u in FP64, FP32, FP16 and BF16 (FP16 weights for
    the FP32 / FP16 / BF16 runs, FP64 weights for the FP64 run), errors
    relative to the FP64 run, and the error of one step."""
    import torch
    import synth
    from paper_1301_3925_gb300 import adlbr as ab
    n = 256
    N = n ** 3
    D = torch.from_numpy(synth.needle_field3d(n, 2, dtype=np.float32).reshape(6, -1)).cuda()
    g = ab.grid((n, n, n))
    st = torch.cuda.current_stream()
    out = {"grid": [n, n, n], "field": "needle, kappa 20, 16^3 lattice, seed 2"}
    h16 = ab.adlbr_build_stencils(g, D, ab.F32, ab.F16)
    h64 = ab.adlbr_build_stencils(g, D, ab.F32, ab.F64)
    try:
        ms = time_ms(lambda: ab.adlbr_build_stencils(g, D, ab.F32, ab.F16, out=h16), 5, st)
        out["build_ms"] = ms
        out["build_gpts"] = N / (ms * 1e-3) / 1e9
        u0 = synth.u_uniform((n, n, n), 2).ravel()
        u32 = torch.from_numpy(u0.astype(np.float32)).cuda()
        Au = torch.empty_like(u32)
        ms = time_ms(lambda: ab.adlbr_apply(h16, u32, Au, ab.F32), 10, st)
        # u in (4), offsets (12), weights (6 x f16 + scale lane = 16), Au out (4)
        gbs = 36 * N / (ms * 1e-3) / 1e9
        out["apply"] = {"ms": ms, "gpts": N / (ms * 1e-3) / 1e9, "gbs": gbs, "frac_hbm": gbs / peak,
                        "bytes_per_point": 36}
        dt = 1.0 / ab.adlbr_stencils_max_diag(h64)
        out["dt"] = dt
        runs = {}
        cases = (("f64", h64, torch.float64, ab.F64), ("f32", h16, torch.float32, ab.F32),
                 ("f16", h16, torch.float16, ab.F16), ("bf16", h16, torch.bfloat16, ab.BF16))
        u64 = torch.from_numpy(u0).cuda()
        sc64 = torch.empty(ab.adlbr_step_scratch_bytes(h64, ab.F64), dtype=torch.uint8, device="cuda")
        for name, h, dtype, code in cases:
            u = u64.to(dtype, copy=True)
            scratch = torch.empty(ab.adlbr_step_scratch_bytes(h, code), dtype=torch.uint8, device="cuda")
            # one step from the same (rounded) u^n against the FP64 step of it
            u1, r1 = u.clone(), u.to(torch.float64, copy=True)
            ab.adlbr_step_explicit(h, u1, scratch, code, dt, 1)
            ab.adlbr_step_explicit(h64, r1, sc64, ab.F64, dt, 1)
            torch.cuda.synchronize()
            step_err = (u1.double() - r1).abs().max().item() / r1.abs().max().item()
            ab.adlbr_step_explicit(h, u1, scratch, code, dt, 2)   # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ab.adlbr_step_explicit(h, u, scratch, code, dt, steps)
            torch.cuda.synchronize()
            runs[name] = (u.double(), (time.perf_counter() - t0) * 1e3 / steps, step_err)
        ref = runs["f64"][0]
        scale = ref.abs().max().item()
        out["precision"] = {"steps": steps, "weights": "F16 (F64 for the f64 run)",
                            "error": "relative L-inf against the FP64 run; per step: one step from the same "
                                     "rounded u^n against the FP64 step of it"}
        for name, (u, ms, e1) in runs.items():
            out["precision"][name] = {"ms_per_step": ms, "rel_linf_vs_f64": (u - ref).abs().max().item() / scale,
                                      "per_step_rel_linf": e1}
        return out
    finally:
        ab.adlbr_stencils_destroy(h16)
        ab.adlbr_stencils_destroy(h64)


# ----------------------------------------------------------------- CPU oracle
def oracle_ced_steps(u, nsteps):
    """The FP64 oracle's CED loop (tensor, stencils, explicit step)."""
    import oracle
    from oracle import ced
    n = u.shape
    for _ in range(nsteps):
        D = ced.ced_tensor(u, CED["sigma"], CED["rho"], CED["alpha"], CED["C"])
        offs, w, st, _ = oracle.build2d(*D)
        u = oracle.step_explicit(n, oracle.NEUMANN, offs, w, u, CED["dt"], 1)
    return u


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), and nproc."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part", "hardware")):
                        name = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return name or "unknown", os.cpu_count() or 1


def _oracle_worker(args):
    """One all-core leg process: CED steps of the oracle on its own crop for
    about `budget_s` seconds; returns (points processed, seconds)."""
    k, side, budget_s = args
    import synth
    r0 = (k * side) % (N_SIDE - side)
    img = synth.fingerprint(N_SIDE, SEED)[r0:r0 + side, :side].copy()
    oracle_ced_steps(img[:64, :64].copy(), 1)
    t0 = time.perf_counter()
    steps, u = 0, img
    while time.perf_counter() - t0 < budget_s:
        u = oracle_ced_steps(u, 1)
        steps += 1
    return steps * side * side, time.perf_counter() - t0


CPU_CONFIG_UNITS = {1: "runs/s (build + 10 explicit steps, 64^2 FP64 spiral)",
                    3: "Gpts/s (3D explicit steps, 64^3 crop of the needle field)",
                    4: "G point-iterations/s (plain CG on a 512^2 kappa <= 50 field, dt = 200 / max A_zz)",
                    5: "Gpts/s (explicit steps on a 256^2 image and a 64^3 volume of the batch's kind)"}


def _cfg_runner(cfg, k):
    """The oracle's work unit for workload `cfg` in process k: returns a
    function that runs it once and gives the units it processed."""
    import oracle
    import synth
    if cfg == 1:
        D = synth.spiral_field(64, 10.0).reshape(3, -1)
        u0 = synth.u_uniform((64, 64), k)

        def run():
            offs, w, st, _ = oracle.build2d(*D)
            dt = oracle.dt_limit((64, 64), oracle.NEUMANN, offs, w)
            oracle.step_explicit((64, 64), oracle.NEUMANN, offs, w, u0, dt, 10)
            return 1
        return run
    if cfg == 3:
        n = 64
        offs, w, st, _ = oracle.build3d(synth.needle_field3d(n, 2 + k, kappa=20.0).reshape(6, -1))
        dt = oracle.dt_limit((n, n, n), oracle.NEUMANN, offs, w)
        state = {"u": synth.u_uniform((n, n, n), k)}

        def run():
            state["u"] = oracle.step_explicit((n, n, n), oracle.NEUMANN, offs, w, state["u"], dt, 1)
            return n ** 3
        return run
    if cfg == 4:
        n = 512
        offs, w, st, _ = oracle.build2d(*synth.smooth_field2d(n, n, 3 + k, 1.0, 50.0, 16).reshape(3, -1))
        dt = 200.0 / oracle.diag((n, n), oracle.NEUMANN, offs, w).max()
        b = synth.u_uniform((n, n), 3 + k)

        def run():
            _, it, _ = oracle.cg((n, n), oracle.NEUMANN, offs, w, b, b, dt, 1e-6, 20)
            return n * n * it
        return run
    # cfg == 5
    D2 = synth.smooth_field2d(256, 256, 100 + k, 1.0, 50.0, 16).reshape(3, -1)
    o2, w2, _, _ = oracle.build2d(*D2)
    d2 = oracle.dt_limit((256, 256), oracle.NEUMANN, o2, w2)
    o3, w3, _, _ = oracle.build3d(synth.needle_field3d(64, 200 + k, kappa=20.0).reshape(6, -1))
    d3 = oracle.dt_limit((64, 64, 64), oracle.NEUMANN, o3, w3)
    st = {"a": synth.u_uniform((256, 256), k), "b": synth.u_uniform((64, 64, 64), k)}

    def run():
        st["a"] = oracle.step_explicit((256, 256), oracle.NEUMANN, o2, w2, st["a"], d2, 1)
        st["b"] = oracle.step_explicit((64, 64, 64), oracle.NEUMANN, o3, w3, st["b"], d3, 1)
        return 256 * 256 + 64 ** 3
    return run


def _cfg_worker(args):
    """Runs workload `cfg`'s oracle unit for about `budget_s` seconds after one
    untimed run; returns (units, seconds)."""
    cfg, k, budget_s = args
    run = _cfg_runner(cfg, k)
    run()
    t0 = time.perf_counter()
    units = 0
    while time.perf_counter() - t0 < budget_s:
        units += run()
    return units, time.perf_counter() - t0


def one_thread_env():
    """Pins the numerical libraries of processes spawned from here on to one
    thread each (numpy's BLAS would otherwise start a thread per core in
    every process of an all-core leg)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def cpu_configs(budget_s=4.0):
    """The oracle on samples of the other workloads, one thread (one spawned
    process) and then every host core (one spawned process per core, each on
    its own sample), every process with single-threaded numerical libraries."""
    import multiprocessing as mp
    model, ncpu = cpu_model()
    one_thread_env()
    ctx = mp.get_context("spawn")
    out = {}
    for cfg in (1, 3, 4, 5):
        with ctx.Pool(1) as pool:
            u1, t1 = pool.map(_cfg_worker, [(cfg, 0, budget_s)])[0]
        with ctx.Pool(ncpu) as pool:
            res = pool.map(_cfg_worker, [(cfg, k, budget_s) for k in range(ncpu)])
        allv = sum(r[0] for r in res) / max(r[1] for r in res)
        scale = 1.0 if cfg == 1 else 1e-9
        out[str(cfg)] = {"unit": CPU_CONFIG_UNITS[cfg], "single_thread": u1 / t1 * scale,
                         "all_core": allv * scale, "cores": ncpu}
    print(json.dumps({"cpu_configs": out, "cpu_model": model, "nproc": ncpu, "kind": "oracle",
                      "budget_s_per_leg": budget_s}))
    return 0


def small_measurement():
    """The 64^2 FP64 spiral workload on the GPU: stencil build (FP64 D and
    weights), the explicit limit dt = 1 / max A_zz (read back to the host) and
    10 explicit steps, per run."""
    import torch
    import synth
    from paper_1301_3925_gb300 import adlbr as ab
    n = 64
    D = torch.from_numpy(synth.spiral_field(n, 10.0).reshape(3, -1)).cuda()
    u0 = torch.from_numpy(synth.u_uniform((n, n), 0).ravel()).cuda()
    u = u0.clone()
    g = ab.grid((n, n))
    h = ab.adlbr_build_stencils(g, D, ab.F64, ab.F64)
    scratch = torch.empty(ab.adlbr_step_scratch_bytes(h, ab.F64), dtype=torch.uint8, device="cuda")
    try:
        def run():
            ab.adlbr_build_stencils(g, D, ab.F64, ab.F64, out=h)
            dt = 1.0 / ab.adlbr_stencils_max_diag(h)
            u.copy_(u0)
            ab.adlbr_step_explicit(h, u, scratch, ab.F64, dt, 10)
        for _ in range(5):
            run()
        torch.cuda.synchronize()
        reps = 200
        t0 = time.perf_counter()
        for _ in range(reps):
            run()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / reps
    finally:
        ab.adlbr_stencils_destroy(h)
    return {"grid": [n, n], "ms_per_run": ms, "runs_per_s": 1e3 / ms,
            "run": "build (FP64) + max A_zz to the host + 10 explicit steps, wall clock per run"}


def cpu_baseline(budget_s=12.0, side=1024, all_side=512, all_budget_s=10.0):
    """Times the oracle as it stands on crops of the workload: one thread on a
    side^2 crop, then every host core at once, each core a separate process
    (spawned: the parent has used the GPU) advancing its own all_side^2 crop.
    Returns the all-core throughput in Gpts/s, the cores used and a dict of
    details."""
    import multiprocessing as mp
    import synth
    img = synth.fingerprint(N_SIDE, SEED)[:side, :side].copy()
    oracle_ced_steps(img[:64, :64].copy(), 1)       # build + warm the oracle
    t0 = time.perf_counter()
    steps = 0
    u = img
    while True:
        u = oracle_ced_steps(u, 1)
        steps += 1
        if time.perf_counter() - t0 > budget_s or steps >= 20:
            break
    dt = time.perf_counter() - t0
    one = steps * side * side / dt / 1e9
    model, ncpu = cpu_model()
    one_thread_env()
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(ncpu) as pool:
        res = pool.map(_oracle_worker, [(k, all_side, all_budget_s) for k in range(ncpu)])
    wall = time.perf_counter() - t0
    pts = sum(r[0] for r in res)
    span = max(r[1] for r in res)
    allc = pts / span / 1e9
    sample = ("all-core leg: %d processes (one per host core, spawned), each advancing its own %dx%d crop "
              "of the 4096^2 image by CED steps (tensor + stencils + explicit step) of the FP64 oracle for "
              "about %.0f s (%.1f s wall with start-up); single-thread leg: %d steps on the top-left %dx%d "
              "crop, %.1f s" % (ncpu, all_side, all_side, all_budget_s, wall, steps, side, side, dt))
    return allc, ncpu, {"sample": sample, "single_thread_value": one, "single_thread_cores": 1,
                        "cpu_model": model, "nproc": ncpu}


def _ref_worker(k, crop, warmup, steps, barrier, out):
    """One process of the reference arm: `warmup` untimed CED steps of the
    oracle on its copy of the crop, then (after every process has reached the
    barrier) `steps` timed ones; puts (k, seconds) on `out`."""
    oracle_ced_steps(crop[:64, :64].copy(), 1)
    u = crop
    for _ in range(warmup):
        u = oracle_ced_steps(u, 1)
    barrier.wait(timeout=900)
    t0 = time.perf_counter()
    for _ in range(steps):
        u = oracle_ced_steps(u, 1)
    out.put((k, time.perf_counter() - t0))


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on every host core.
    One process per core (spawned), each advancing its own copy of the top-left
    512^2 crop of the 4096^2 workload; a step is one CED step on every core at
    once, timed from a common barrier to the slowest process."""
    import multiprocessing as mp
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import synth
    side = 512
    crop = synth.fingerprint(N_SIDE, SEED)[:side, :side].copy()
    model, ncpu = cpu_model()
    one_thread_env()
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(ncpu), ctx.Queue()
    procs = [ctx.Process(target=_ref_worker, args=(k, crop, args.warmup, args.steps, barrier, out))
             for k in range(ncpu)]
    for p in procs:
        p.start()
    import queue
    spans = []
    while len(spans) < ncpu:
        try:
            spans.append(out.get(timeout=5)[1])
        except queue.Empty:
            if any(p.exitcode not in (None, 0) for p in procs):
                for p in procs:
                    if p.is_alive():
                        p.terminate()
                raise RuntimeError("a reference-arm process failed")
    for p in procs:
        p.join(timeout=60)
    el = max(spans)
    value = ncpu * args.steps * side * side / el / 1e9
    sample = ("each step: one CED step of the FP64 oracle (numpy tensor stage, C stencils and operator) "
              "on every host core at once, %d processes (spawned, one thread each), each on its own copy "
              "of the top-left %dx%d crop of the 4096^2 workload; CPU %s" % (ncpu, side, side, model))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncpu, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict():
    return {"workload": "ced2d_4096_fp32", "grid": [N_SIDE, N_SIDE], "sigma": CED["sigma"],
            "rho": CED["rho"], "alpha": CED["alpha"], "C": CED["C"], "dt": CED["dt"],
            "kappa_max": 100, "u": "f32", "D": "f32", "weights": "f16", "offsets": "int16",
            "boundary": "neumann", "l2": "working set ~1 GB > L2 (no flush needed)",
            "image": "sum of 8 random sinusoids, period U[6,12] px, + N(0, 0.2^2), seed 1"}


# ----------------------------------------------------------------- GPU arm
def profile_unet():
    """Four forwards of the 2048^2 preconditioner's network (25 -> 16/32/64
    channels at 512^2, batch 1) on the tensor cores (profiling entry)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1301_3925_gb300 import adlbr as ab
    from paper_1301_3925_gb300 import nn
    H = W = 512
    net = ab.adlbr_unet_create(nn.NF, 16, 32, 64, 1, H, W)
    try:
        P = ab.adlbr_unet_num_params(net)
        th = torch.from_numpy(nn.init_params(P, nn.layer_shapes(nn.NF, 16, 32, 64), 1)).float().cuda()
        x = torch.randn(nn.NF * H * W, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
        y = torch.empty(H * W, device="cuda")
        ab.adlbr_unet_set_tensor_cores(net, True)
        for _ in range(4):
            ab.adlbr_unet_forward(net, th, x, y)
        torch.cuda.synchronize()
    finally:
        ab.adlbr_unet_destroy(net)
    print(json.dumps({"profile_unet": {"y_abs_max": float(y.abs().max())}}))
    return 0


CONFIG_WORKLOADS = {
    1: "64x64 FP64 spiral field (kappa 10): stencil build and 10 explicit steps at the stability limit",
    3: "256^3 needle field (eigenvalues 1, 1/20^2, 1/20^2): build, operator, 100-step precision study "
       "(FP32, FP16, BF16 u against FP64)",
    4: "2048^2 implicit step (I + dt A) u = u_n, dt = 200 x the explicit limit, kappa <= 50: CG, "
       "Jacobi-PCG, U-Net-preconditioned flexible CG to 1e-6",
    5: "serving batch: 64 images 256^2-2048^2 and 8 volumes 64^3-192^3, one graph launch per step"}


def run_config(args):
    """One workload other than the headline, on one GPU: its measurement as
    one JSON line (the entry of the full line that covers it)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    peak, peak_src = measured_peaks()
    if args.config == 1:
        res = small_measurement()
        value, unit, hib = res["runs_per_s"], "runs/s", True
    elif args.config == 3:
        res = volume_measurement(peak, args.precision_steps)
        value, unit, hib = 256 ** 3 / (res["precision"]["f32"]["ms_per_step"] * 1e-3) / 1e9, "Gpts/s", True
    elif args.config == 4:
        res = implicit_measurement(peak)
        value, unit, hib = res["cg"]["ms"], "ms", False
    else:
        res = batch_measurement(peak)
        value, unit, hib = res["gpts"], "Gpts/s", True
    print(json.dumps({"config_id": args.config, "workload": CONFIG_WORKLOADS[args.config], "value": value,
                      "unit": unit, "higher_is_better": hib, "n_gpus": 1, "dtype": "see result",
                      "data": "synthetic", "peak_hbm_gbs": peak, "peak_source": peak_src, "result": res}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.cpu_configs:
        import __graft_entry__
        __graft_entry__.build()
        return cpu_configs()
    import torch
    if args.profile_cg:
        return profile_cg()
    if args.profile_unet:
        return profile_unet()
    if args.profile_fcg:
        return profile_fcg()
    if args.profile_gather:
        return profile_gather()
    if args.config != 2:
        return run_config(args)

    ws, rank, local = init_dist()
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    barrier(ws)
    import synth
    from paper_1301_3925_gb300 import adlbr as ab

    n = N_SIDE
    N = n * n
    g = ab.grid((n, n))
    img = synth.fingerprint(n, rank_seed(rank)).astype(np.float32)
    u0 = torch.from_numpy(img.ravel()).cuda()
    u = u0.clone()
    scratch = torch.empty(ab.adlbr_ced_scratch_bytes(g), dtype=torch.uint8, device="cuda")
    Dbuf = scratch[6 * N * 4: 9 * N * 4].view(torch.float32)
    acc = scratch[9 * N * 4: 10 * N * 4].view(torch.float32)
    stream = torch.cuda.current_stream()
    h = None
    S = (CED["sigma"], CED["rho"], CED["alpha"], CED["C"])

    def step():
        # the tensor stage, then the stencil build and the explicit step in
        # one call (one fused kernel for this workload), each timed on its own
        nonlocal h
        ab.adlbr_ced_tensor(g, u, Dbuf, *S, scratch)
        h = ab.adlbr_build_step_explicit(g, Dbuf, ab.F32, ab.F16, h, u, acc, CED["dt"])

    for _ in range(max(args.warmup, 3)):
        step()
    ab.adlbr_stencils_check(h)
    torch.cuda.synchronize()

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.time()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(K):
        e = ev[k]
        e[0].record(stream)
        ab.adlbr_ced_tensor(g, u, Dbuf, *S, scratch)
        e[1].record(stream)
        h = ab.adlbr_build_step_explicit(g, Dbuf, ab.F32, ab.F16, h, u, acc, CED["dt"])
        e[2].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    t1 = time.time()
    clocks = sampler.stop(t0, t1)
    ab.adlbr_stencils_check(h)
    total_ms = start.elapsed_time(end)
    total_ms = allmax(ws, total_ms)
    st_tensor = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    st_bstep = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    ms_step = total_ms / K

    # the same step as three calls (tensor, build, explicit step with the
    # stand-alone operator), each timed: the stages before the fusion
    ev2 = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(10)]
    u_side = u.clone()
    for e in ev2:
        e[0].record(stream)
        ab.adlbr_ced_tensor(g, u_side, Dbuf, *S, scratch)
        e[1].record(stream)
        h = ab.adlbr_build_stencils(g, Dbuf, ab.F32, ab.F16, out=h)
        e[2].record(stream)
        ab.adlbr_step_explicit(h, u_side, acc, ab.F32, CED["dt"], 1)
        e[3].record(stream)
    torch.cuda.synchronize()
    del u_side
    st_build = float(np.mean([e[1].elapsed_time(e[2]) for e in ev2[2:]]))
    st_step = float(np.mean([e[2].elapsed_time(e[3]) for e in ev2[2:]]))
    value = job_value(ws, N, ms_step)

    # roofline of the dominant kernel; the others beside it
    peak, peak_src = measured_peaks()

    def roof_of(name, ms):
        if name == "ced_fused_kernel":
            # issue-bound FP32 arithmetic: algorithmic FP32 operations per point
            # (an FMA counts once) against the FP32 issue rate of the GPU
            a = ALU_OPS_PER_POINT * N / (ms * 1e-3) / 1e12
            pk, pk_src = fp32_peak_tops()
            return {"kernel": name, "bound": "alu", "achieved": a, "peak": pk, "unit": "Tops/s",
                    "frac": a / pk, "traffic": TRAFFIC_4096.get(name), "peak_source": pk_src,
                    "ops_per_point": ALU_OPS_PER_POINT, "units_per_launch": N}
        # build_step: D in 12 + stencils out 16 + u in 4 + u out 4
        bpp = {"build_step": 12 + 16 + 4 + 4, "build2d_kernel": 12 + 8 + 8, "explicit_step": 4 + 16 + 4}[name]
        a = bpp * N / (ms * 1e-3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
                "traffic": TRAFFIC_4096.get(name), "peak_source": peak_src, "bytes_per_point": bpp,
                "units_per_launch": N}

    stage_ms = {"ced_fused_kernel": st_tensor, "build_step": st_bstep}
    dom = max(stage_ms, key=stage_ms.get)
    roof = roof_of(dom, stage_ms[dom])
    roof["others"] = [roof_of(k, v) for k, v in stage_ms.items() if k != dom]
    if dom == "build_step" or "build_step" in stage_ms:
        for r in [roof] + roof["others"]:
            if r["kernel"] == "build_step":
                r["kernels"] = "memset + build_accumulate2d_tma (stencil build fused into the operator) + finalize"
    unfused = {"build2d_kernel": roof_of("build2d_kernel", st_build), "explicit_step": roof_of("explicit_step", st_step),
               "build_ms": st_build, "explicit_step_ms": st_step,
               "note": "the same step as separate calls (build, then the stand-alone operator), 8 steps "
                       "after 2 untimed, for comparison"}
    step_gbs = 24 * N / (st_step * 1e-3) / 1e9

    # the operator alone on the step's stencils (adlbr_apply: zero Au, accumulate)
    Au = torch.empty_like(u)
    apply_ms = time_ms(lambda: ab.adlbr_apply(h, u, Au, ab.F32), 20, stream)
    apply_gbs = 24 * N / (apply_ms * 1e-3) / 1e9
    apply_sub = {"ms": apply_ms, "gpts": N / (apply_ms * 1e-3) / 1e9, "gbs": apply_gbs,
                 "frac_hbm": apply_gbs / peak, "bytes_per_point": 24,
                 "stencils": "CED kappa <= 100 (4096^2 fingerprint)", "form": "scatter (the default)"}
    # the same applications in the gather form (its table built first, not timed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ab.adlbr_stencils_set_operator(h, ab.OP_GATHER)
    ab.adlbr_apply(h, u, Au, ab.F32)
    torch.cuda.synchronize()
    table_ms = (time.perf_counter() - t0) * 1e3
    g_ms = time_ms(lambda: ab.adlbr_apply(h, u, Au, ab.F32), 20, stream)
    ab.adlbr_stencils_set_operator(h, ab.OP_AUTO)
    apply_sub["gather_form"] = {"ms": g_ms, "gpts": N / (g_ms * 1e-3) / 1e9,
                                "frac_hbm_24B": 24 * N / (g_ms * 1e-3) / 1e9 / peak,
                                "first_call_with_table_build_ms": table_ms,
                                "note": "deterministic gather form, measured beside the scatter; slower, "
                                        "so not the default"}

    # End to end through the C ABI with host buffers: every step copies its
    # input image from pinned host memory and reads its result back.  As a
    # serving loop would, the copies of one request overlap the compute of
    # its neighbours: a host-to-device stream, the compute stream and a
    # device-to-host stream, three device buffers in rotation.
    e2e = None
    if not args.no_e2e:
        Ke = max(6, min(K, 50))
        host = torch.from_numpy(img.ravel()).pin_memory()
        outs = [torch.empty_like(host).pin_memory() for _ in range(3)]
        bufs = [torch.empty_like(u) for _ in range(3)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

        def step_on(buf):
            nonlocal h
            ab.adlbr_ced_tensor(g, buf, Dbuf, *S, scratch)
            h = ab.adlbr_build_step_explicit(g, Dbuf, ab.F32, ab.F16, h, buf, acc, CED["dt"])

        def run(n):
            done_out = [None] * 3
            for k in range(n):
                j = k % 3
                with torch.cuda.stream(s_in):
                    if done_out[j] is not None:
                        s_in.wait_event(done_out[j])   # the buffer's previous result is read out
                    bufs[j].copy_(host, non_blocking=True)
                    ev_in = torch.cuda.Event()
                    ev_in.record(s_in)
                stream.wait_event(ev_in)
                step_on(bufs[j])
                ev_c = torch.cuda.Event()
                ev_c.record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_c)
                    outs[j].copy_(bufs[j], non_blocking=True)
                    done_out[j] = torch.cuda.Event()
                    done_out[j].record(s_out)

        run(3)
        torch.cuda.synchronize()
        barrier(ws)
        t_e0 = time.perf_counter()
        run(Ke)
        torch.cuda.synchronize()
        e2e_ms = allmax(ws, (time.perf_counter() - t_e0) * 1e3) / Ke
        assert torch.equal(outs[(Ke - 1) % 3], bufs[(Ke - 1) % 3].cpu())
        e2e = {"value": job_value(ws, N, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 4 * N,
               "pipeline": "H2D / compute / D2H on three streams, three device buffers"}

    implicit = None if args.no_implicit or rank != 0 else implicit_measurement(peak)
    volume = None if args.no_3d or rank != 0 else volume_measurement(peak, args.precision_steps)
    batch = None if args.no_batch or rank != 0 else batch_measurement(peak)
    eed3d = None
    if not args.no_eed3d and rank == 0:
        eed3d = eed3d_measurement()
    ced3d = None
    if not args.no_ced3d and rank == 0:
        ced3d = ced3d_measurement(precond=2)
        plain = ced3d_measurement(precond=0)
        ced3d["plain_cg"] = {k: plain[k] for k in ("ms_per_step", "implicit_ms", "cg_iters_mean", "rms_to_clean")}
    spectral_study = None if args.no_spectral or rank != 0 else spectral_measurement()
    ann_study = None if args.no_ann or rank != 0 else ann_measurement(peak)
    small = small_measurement() if rank == 0 else None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, cores, det = cpu_baseline()
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": det["sample"],
               "single_thread_value": det["single_thread_value"], "cpu_model": det["cpu_model"],
               "nproc": det["nproc"]}

    if rank == 0:
        line = {"metric": METRIC, "value": value,
                "value_is": "one CED step of the hot path (tensor stage, stencil build, explicit step with "
                            "the operator; the build runs inside the operator's kernel, each point starting from its previous stencil, certified exactly) on the 4096^2 image, "
                            "points per second; the operator alone is apply_gpts / apply_frac_hbm",
                "apply_gpts": apply_sub["gpts"], "apply_frac_hbm": apply_sub["frac_hbm"],
                "unit": UNIT, "n_gpus": ws, "steps": K,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks,
                # per step: the fused tensor kernel, the stencil build fused into
                # the operator, and the finalize kernel
                "gpu_launches": K * 3,
                "stages_ms": {"tensor": st_tensor, "build_step": st_bstep},
                "unfused": unfused,
                "explicit_step": {"gpts": N / (st_step * 1e-3) / 1e9, "gbs": step_gbs,
                                  "frac_hbm": step_gbs / peak, "bytes_per_point": 24,
                                  "note": "the stand-alone explicit step (memset, operator, finalize) "
                                          "on the step's stencils"},
                "apply": apply_sub, "implicit": implicit, "volume3d": volume, "batch": batch,
                "ced3d": ced3d, "eed3d": eed3d, "spectral": spectral_study, "ann": ann_study, "small_64_fp64": small}
        print(json.dumps(line))
    ab.adlbr_stencils_destroy(h)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
