"""Benchmark of the pseudo-spectral NS + Cahn-Hilliard channel time step.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Prints ONE JSON line (rank 0).  A step is one full time step (Sec. 2.2 steps i)-v)) of one
channel: six kernels - z right-hand sides (Chebyshev DCTs, assembly, AB2), tau solves, z update
+ backward DCTs, y backward pass, fused x-line kernel (transforms + products), y forward pass
(eight with --cheb tc: the Chebyshev transforms then run as two tensor-core launches).
Default workload: the 512 x 256 x 257 channel in mixed precision (Re_tau = 300, 64 drops; float32
x/y transforms and products, float64 along z), the other precisions and Chebyshev methods of the
same grid beside it (variants, with the float64 step's own roofline).  Points = nx ny nz
(unpadded); the metric is Mpoints * steps / s of the whole job.

* value: device time of K steps on the handle's stream (CUDA events, barrier + synchronize on
  both sides, max over ranks); the per-step working set (~8 GB at 512 x 256 x 257, ~0.8 GB at
  128^3) is larger than L2.
* e2e: the user path through the C ABI with host buffers: upload of u, v, w, phi from pinned host
  memory, K steps, download of u, v, w, phi, timed on the host clock after a synchronize.
* roofline: the dominant kernel of the step, its algorithmic FLOPs (or bytes) per launch over
  its CUDA-event launch time, against the float64 ALU peak (no float64 figure is in the
  measured-peaks file: 152 SMs x 2.07 GHz x 4 flop/clk/SM = 1.26 TFLOP/s nominal) or the
  measured HBM copy bandwidth.
* cpu_baseline: the CPU oracle on a bounded sample of the same workload (rank 0, N = 1), credited
  with the fraction of a step it covered; --impl reference runs the same sampled oracle step as
  its steps.
* N > 1: N independent replicas, one per rank ("replicas only": the single-grid step does not
  shard without all-to-all transposes); value = all ranks' points * steps / max time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time steps/s & Mpoints·step/s per grid; % HBM roofline; mixed vs FP64"
UNIT = "Mpoints*step/s"
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12   # 2 DFMA per clock per SM (recipe: 1.25 TF/s)
# double-float x/y kernels run float64-equivalent arithmetic on the float32 pipe (128 lanes per SM
# per clock): 11 float32 instructions per double-float addition, 7 per multiplication, 18 per
# fused multiply-add (2 flops); with the float64 instruction mix of the transforms (10.2 M adds,
# 5.4 M FMAs, 2.4 M multiplications per 128^3 zrhs) that is 9.67 instructions per flop
DF_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 9.67 / 1e12


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, MB) of kernels of the
# current build from one ncu capture each (128 x 128 x 129 workloads, steady-state launches);
# absent entries report null.  Re-capture when a kernel changes.
TRAFFIC_MB = {
    ("channel_128x128x129", 0, "xline"): 152.8 + 185.4,
    ("channel_128x128x129", 0, "ybwd"): 84.6 + 135.3,
    ("channel_128x128x129", 2, "xline"): 153.2 + 193.1,
    ("channel_128x128x129", 2, "ybwd"): 84.7 + 134.8,
    # coefficient-space z kernels of the tensor-core method (the same kernels at any precision)
    ("channel_128x128x129", 0, "zsolve"): 93.5 + 8.9,
    ("channel_128x128x129", 1, "zsolve"): 93.5 + 8.9,
    ("channel_128x128x129", 2, "zsolve"): 93.5 + 8.9,
    # 512 x 256 x 257 (full-size captures of the default bench command, its Chebyshev method
    # trial included, and of the FP64 step on the same grid)
    ("channel_512x256x257_mixed", 1, "zsolve"): 4747.8 + 3621.8,
    ("channel_512x256x257_mixed", 1, "zbwd"): 1343.6 + 1427.6,
    ("channel_512x256x257_mixed", 0, "zsolve"): 4753.3 + 3623.4,
    ("channel_512x256x257_mixed", 0, "zbwd"): 1343.7 + 2096.8,
    ("channel_512x256x257_mixed", 0, "xline"): 2434.1 + 3591.5,
    ("channel_512x256x257_mixed", 0, "ybwd"): 1610.9 + 2393.1,
    # current step kernels (full-size captures of the default bench command's kernels with
    # --cheb tc, and of the 128^3 mixed tensor-core and float64 FFT-method steps)
    ("channel_512x256x257_mixed", 1, "cheb_fwd"): 964.4 + 2390.7,
    ("channel_512x256x257_mixed", 1, "cheb_bwd"): 1368.9 + 1220.4,
    ("channel_512x256x257_mixed", 1, "zrhs_coef"): 3331.3 + 2004.2,
    ("channel_512x256x257_mixed", 1, "zbwd_coef"): 1342.3 + 2287.4,
    ("channel_512x256x257_mixed", 1, "xline"): 1783.4 + 2107.7,
    ("channel_512x256x257_mixed", 1, "yfwd"): 1819.3 + 906.6,
    ("channel_512x256x257_mixed", 1, "ybwd"): 805.6 + 1174.0,
    ("channel_128x128x129", 1, "cheb_fwd"): 60.6 + 63.3,
    ("channel_128x128x129", 1, "cheb_bwd"): 85.3 + 8.3,
    ("channel_128x128x129", 1, "zrhs_coef"): 218.3 + 80.1,
    ("channel_128x128x129", 0, "zbwd_coef"): 83.9 + 88.1,
    ("channel_128x128x129", 1, "zbwd_coef"): 83.9 + 88.1,
    ("channel_128x128x129", 2, "zbwd_coef"): 83.9 + 88.1,
    ("channel_128x128x129", 1, "yfwd"): 114.2 + 32.6,
    ("channel_128x128x129", 1, "ybwd"): 42.0 + 27.9,
    ("channel_128x128x129", 0, "zrhs"): 218.3 + 73.3,
    ("channel_128x128x129", 0, "yfwd"): 228.3 + 85.9,
    ("channel_128x128x129", 0, "zbwd"): 84.0 + 82.6,
    ("channel_128x128x129_adjoint", 0, "adj_xline"): 380.7 + 130.9,
    ("channel_128x128x129_adjoint", 0, "adj_zsolve"): 102.4 + 28.2,
    ("channel_128x128x129_adjoint", 0, "adj_zrhs"): 135.1 + 223.7,
}


def traffic_bytes(workload, prec, kernel, cheb="fft"):
    """ncu DRAM bytes of one launch; the z kernels of the tensor-core method (coefficient-space
    variants) have their own entries, "zrhs_coef" and "zbwd_coef"; the tensor-core transforms'
    entries are per precision."""
    if cheb == "tc" and kernel in ("zrhs", "zbwd"):
        kernel += "_coef"
    v = TRAFFIC_MB.get((workload, prec, kernel))
    return None if v is None else v * 1e6


# the float64 FMA rate measured on this device by the library's probe (ch_fp64_fma_rate), filled
# in by main() before the rooflines are formed
MEASURED_FMA = {}


def tensor_peak():
    """Measured bf16 dense tensor peak (burst: the kernel is timed inside a short step)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured bf16 dense (cuBLAS burst)"
    return 1900.0, "fallback bf16 dense"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6785.9), "measured"
    return 6800.0, "fallback"


# ---- algorithmic work per launch --------------------------------------------------------------
def fft_flops(n):
    """5 n log2 n: the conventional flop count of a complex FFT of length n."""
    return 5.0 * n * math.log2(n)


def kernel_work(w, prec, cheb="fft"):
    """Algorithmic flops (an FMA counts 2) and bytes per launch of the step kernels (the six of
    the FFT method and the two tensor-core Chebyshev transforms).  cheb = "tc": zrhs and zbwd are
    the coefficient-space variants (no DCTs; float64 coefficients in and out)."""
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    Mx, Px, Py, N = nx // 2, 3 * nx // 2, 3 * ny // 2, nz - 1
    b = 8 if prec == 1 else 16
    S = Mx * ny * nz           # spectral points per field
    Y = Mx * Py * nz           # y-padded points per field
    lines = Mx * ny
    # complex DCT-I of a line: 5 N log2 N (an N-point complex FFT per complex line, the count of
    # the scope table; the paper's 2N-point even extension would be twice that); a derivative =
    # 4 flops per coefficient
    dct = fft_flops(N)
    # zrhs: the 7 combined non-linear lines in, 7 DCTs, 7 derivatives, assembly, AB2 and the
    # right-hand sides (56 flops per coefficient)
    zrhs_fl = lines * (7 * dct + 7 * 4 * nz + 56 * nz)
    zrhs_by = S * (b * 7 + 16 * 3 + 16 * 3 + 16 * 3 + 16 * 3)   # NL, state, hist in/out, R out
    zsolve_fl = lines * nz * (5 * 30 + 8)                       # 5 sweeps + influence correction
    zsolve_by = S * 16 * 3 * 2
    zbwd_fl = lines * (5 * dct + 2 * 4 * nz + 40 * nz)
    zbwd_by = S * (16 * 3 + 16 * 2 + 16 * 3 + b * 5)             # R, state in, state out, 5 out
    yb_fl = 6 * Mx * nz * fft_flops(Py)
    yb_by = (5 * S + 6 * Y) * b
    x_fl = Py * nz * (16 * 0.5 * fft_flops(Px) + 45 * Px)       # packed real FFTs + products
    x_by = 15 * Y * b
    # forward y pass: 9 product fields in, the 7 combined lines out (42 flops per spectral point
    # for the i kx, i ky combinations)
    yf_fl = 9 * Mx * nz * fft_flops(Py) + 42 * S
    yf_by = (9 * Y + 7 * S) * b
    # Chebyshev transforms on the tensor cores (CH_CHEB_TC): tensor-pipe flops issued (36 digit
    # products of 2 M Nout K each, M = real rows, Nout and K padded as the kernel pads them) and
    # the bytes of the fields read and written once
    Kp, NT, nNt = tc_tiles(nz)
    rows = 2 * lines
    tcf_fl = 36 * 2.0 * (7 * rows) * (NT * nNt) * Kp
    tcf_by = 7 * S * (b + 16)
    tcb_fl = 36 * 2.0 * (5 * rows) * (NT * nNt) * Kp
    tcb_by = 5 * S * (16 + b)
    if cheb == "tc":
        zrhs_fl = lines * (7 * 4 * nz + 56 * nz)
        zrhs_by = S * (16 * 7 + 16 * 3 + 16 * 3 + 16 * 3 + 16 * 3)
        zbwd_fl = lines * (2 * 4 * nz + 40 * nz)
        zbwd_by = S * (16 * 3 + 16 * 2 + 16 * 3 + 16 * 5)
    return {"zrhs": (zrhs_fl, zrhs_by), "zsolve": (zsolve_fl, zsolve_by),
            "zbwd": (zbwd_fl, zbwd_by), "ybwd": (yb_fl, yb_by), "xline": (x_fl, x_by),
            "yfwd": (yf_fl, yf_by), "cheb_fwd": (tcf_fl, tcf_by), "cheb_bwd": (tcb_fl, tcb_by)}


def tc_tiles(nz):
    """K padding, output slice width and slice count of the tensor-core Chebyshev kernel (the
    library's rule: the slices cover the outputs n < N = nz - 1, 48 wide unless 64-wide ones pad
    20 % less; the last output is summed exactly outside the MMAs)."""
    N = nz - 1
    Kp = (nz + 15) // 16 * 16
    c48, c64 = (N + 47) // 48 * 48, (N + 63) // 64 * 64
    NT = 48 if 5 * c48 <= 4 * c64 else 64
    return Kp, NT, (N + NT - 1) // NT


def cufft_transforms_ms(w, prec, reps=5, warmup=2, dev="cuda"):
    """Timed comparison only: the transforms of one step done with cuFFT through torch.fft, as a
    library user would write them (zero padding / truncation by copies, layouts as stored):
    12 Chebyshev DCT-I (5 backward + 7 forward, each a 2N-point FFT of the even extension),
    6 y inverse FFTs and 9 y forward FFTs of length Py, 7 x c2r and 9 x r2c of length Px.
    The products, assembly and solves are not included.  Returns (z ms, x-y ms) per step."""
    import torch
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    Mx, Px, Py, N = nx // 2, 3 * nx // 2, 3 * ny // 2, nz - 1
    h = ny // 2
    cd = torch.complex64 if prec == 1 else torch.complex128
    rd = torch.float32 if prec == 1 else torch.float64
    spec = torch.randn(12, Mx, ny, nz, dtype=torch.complex128, device=dev)
    ymod = torch.randn(6, Mx, ny, nz, dtype=cd, device=dev)
    prod = torch.randn(9, Px, Py, nz, dtype=rd, device=dev)

    def zpart():
        ext = torch.cat([spec, spec.flip(-1)[..., 1:-1]], dim=-1)      # even extension, 2N
        return torch.fft.fft(ext, dim=-1)

    def xypart():
        pad = torch.zeros(6, Mx, Py, nz, dtype=cd, device=dev)
        pad[:, :, :h] = ymod[:, :, :h]
        pad[:, :, Py - h + 1:] = ymod[:, :, h + 1:]
        yb = torch.fft.ifft(pad, dim=2)
        xin = torch.cat([yb, yb[3:4]], dim=0)                          # 7 fields (phi_x from phi)
        phys = torch.fft.irfft(xin, n=Px, dim=1)                       # (7, Px, Py, nz)
        xf = torch.fft.rfft(prod, dim=1)[:, :Mx]                       # (9, Mx, Py, nz)
        yf = torch.fft.fft(xf, dim=2)
        out = torch.cat([yf[:, :, :h], yf[:, :, Py - h:]], dim=2)
        return phys, out

    res = []
    for fn in (zpart, xypart):
        for _ in range(warmup):
            fn()
        if dev == "cpu":                 # shape check of the comparison (no timing meaning)
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            res.append((time.perf_counter() - t0) * 1e3 / reps)
            continue
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        res.append(a.elapsed_time(b) / reps)
    del spec, ymod, prod
    if dev != "cpu":
        torch.cuda.empty_cache()
    return res[0], res[1]


PREC_NAMES = {0: "fp64", 1: "mixed", 2: "dfloat"}
DTYPES = {0: "f64", 1: "f32 transforms/products + f64 solves",
          2: "double-float (float pair, ~48-bit) transforms/products + f64 solves"}


def precision_accuracy(binding, w, fields, steps, device, prec=1):
    """Step of precision `prec` against the FP64 step from the same fields after `steps` steps:
    per-field max relative difference (max |a - b| / max |b|; velocity_scale: the largest of
    the velocity components' max |a - b| over max |u|), phi mass drift of each path relative to
    the initial mass, and relative differences of the mass, kinetic energy, int |grad phi|^2 and
    free energy."""
    import torch
    kw = dict(re_tau=w["re_tau"], we=w["we"], ch=w["ch"], pe=w["pe"], dt=w["dt"])
    out = {}
    res = {}
    for pr in (0, prec):
        g = binding.Grid(w["nx"], w["ny"], w["nz"], precision=pr, device=device, **kw)
        g.set_fields(*[torch.from_numpy(f) for f in fields])
        m0 = g.diagnostics()["mass"]
        g.step(steps)
        d = g.diagnostics()
        res[pr] = ([f.cpu() for f in g.get_fields()], d, m0)
        g.close()
        torch.cuda.empty_cache()
    (f64, d64, m64), (f32, d32, m32) = res[0], res[prec]
    out["rel_err"] = {n: float((a - b).abs().max() / b.abs().max())
                      for n, a, b in zip(("u", "v", "w", "phi"), f32, f64)}
    umax = float(f64[0].abs().max())
    out["rel_err"]["velocity_scale"] = max(float((a - b).abs().max()) / umax
                                           for a, b in zip(f32[:3], f64[:3]))
    out["mass_drift_fp64"] = (d64["mass"] - m64) / abs(m64)
    out["mass_drift_" + PREC_NAMES[prec]] = (d32["mass"] - m32) / abs(m32)
    for k in ("mass", "kinetic", "grad2", "free_energy"):
        out[k + "_rel_diff"] = (d32[k] - d64[k]) / abs(d64[k])
    out["steps"] = steps
    return out


def dct_gemm_ms(w, reps=5, warmup=2, dev="cuda"):
    """Timed comparison only: the seven forward Chebyshev transforms of one step as one dense
    float64 matrix product (cuBLAS through torch.matmul): the (N+1) x (N+1) DCT-I matrix times
    the real and imaginary parts of 7 x Mx x Ny lines.  Returns (ms, TFLOP/s)."""
    import torch
    nz = w["nz"]
    ncols = 7 * (w["nx"] // 2) * w["ny"] * 2
    C = torch.randn(nz, nz, dtype=torch.float64, device=dev)
    X = torch.randn(nz, ncols, dtype=torch.float64, device=dev)
    for _ in range(warmup):
        torch.matmul(C, X)
    if dev == "cpu":
        t0 = time.perf_counter()
        for _ in range(reps):
            torch.matmul(C, X)
        ms = (time.perf_counter() - t0) * 1e3 / reps
    else:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            torch.matmul(C, X)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
    del C, X
    return ms, 2.0 * nz * nz * ncols / (ms * 1e-3) / 1e12


def adjoint_work(w):
    """Algorithmic flops and bytes per launch of the reverse step's kernels (FP64)."""
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    Mx, Px, Py, N = nx // 2, 3 * nx // 2, 3 * ny // 2, nz - 1
    S, Y, lines = Mx * ny * nz, Mx * Py * nz, Mx * ny
    dct = fft_flops(N)
    f = kernel_work(w, 0)
    return {
        "zbwd": (lines * (5 * dct + 2 * 4 * nz + 40 * nz), S * 16 * (3 + 5)),
        "ybwd": f["ybwd"],
        "adj_zsolve": (lines * nz * (5 * 30 + 12), S * 16 * 3 * 3),
        "adj_zrhs": (lines * (7 * dct + 7 * 4 * nz + 150 * nz), S * 16 * (3 + 3 + 3 + 3 + 3 + 9)),
        "adj_ybwd": (9 * Mx * nz * fft_flops(Py), 9 * (S + Y) * 16),
        "adj_xline": (Py * nz * (23 * 0.5 * fft_flops(Px) + 60 * Px), (6 + 9 + 6) * Y * 16),
        "adj_yfwd": (6 * Mx * nz * fft_flops(Py), 6 * (S + Y) * 16),
        "fold_dy": (8 * S, 4 * S * 16),
        "adj_zbwd": (lines * (5 * dct + 2 * 4 * nz + 30 * nz), S * 16 * (5 + 3 + 3)),
    }


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device):
    """Largest x over the ranks of the default process group (x itself when world == 1)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(points, steps, world, seconds):
    """Whole-job Mpoints*step/s of `world` independent replicas, each advancing `points` for
    `steps` steps, timed by the slowest rank (`seconds`)."""
    return world * points * steps / seconds / 1e6


def oracle_channel(w):
    from oracle.channel import Channel, Params
    from paper_2406_01322_gb300 import inputs
    p = Params(nx=w["nx"], ny=w["ny"], nz=w["nz"], re_tau=w["re_tau"], we=w["we"], ch=w["ch"],
               pe=w["pe"], dt=w["dt"])
    c = Channel(p)
    c.set_fields(*inputs.initial_fields(**w))
    return c


ORACLE_SAMPLE = dict(nplanes=1, nlines=16)


def oracle_sampled_step(c, rng, nplanes=1, nlines=16):
    """One oracle step on a bounded sample of the workload, timed as it runs.

    * non-linear terms: the oracle's own nonlinear_spectral on a copy of the channel whose
      Chebyshev matrices keep `nplanes` random z-planes (rows of the backward matrix, columns of
      the forward one): the velocity recovery runs on every line, the x-y transforms and products
      on those planes only;
    * assembly and right-hand sides (the oracle's assemble and rhs) on one random wavenumber row
      (all kx of one ky);
    * implicit solves (solve_lines) of `nlines` random lines of that row.
    Returns (seconds, fraction): the sample's wall time and the smallest fraction of the full
    step's work any part covered (planes / Nz, lines / all lines), which is what the sample is
    credited with (an under-estimate of the work done)."""
    import copy
    import numpy as np
    Nz, Ny, Mx = c.p.nz, c.p.ny, c.Mx
    planes = np.sort(rng.choice(Nz, size=min(nplanes, Nz), replace=False))
    j = int(rng.integers(1, Ny // 2))
    ms = np.sort(rng.choice(np.arange(1, Mx), size=min(nlines, Mx - 1), replace=False))
    t0 = time.perf_counter()
    s = copy.copy(c)
    s.Bm = c.Bm[planes]
    s.Fm = c.Fm[:, planes]
    nl = s.nonlinear_spectral()
    r = copy.copy(c)                     # the wavenumber row j as a one-row channel
    r.iky = c.iky[:, [j], :]
    r.k2 = c.k2[[j], :]
    r.omega, r.w, r.phi = (a[:, [j], :] for a in (c.omega, c.w, c.phi))
    h = r.assemble([a[:, [j], :] for a in nl])
    H = h if c.hist is None else tuple(1.5 * a - 0.5 * b[:, [j], :] for a, b in zip(h, c.hist))
    rr = r.rhs(H)
    r.solve_lines([(0, int(m)) for m in ms], *rr)
    t1 = time.perf_counter()
    frac = min(len(planes) / Nz, len(ms) / len(c.all_lines()))
    return t1 - t0, frac


def sample_note(w, nplanes, nlines):
    return (f"per step: the oracle's non-linear terms on {nplanes} of {w['nz']} z-planes "
            f"(velocity recovery on every line), assembly and right-hand sides of one "
            f"wavenumber row, implicit solves of {nlines} of its lines; credited with the "
            f"smallest fraction of the full step any part covered; numpy FP64 oracle, BLAS "
            f"threads = host cores, FFTs single-threaded")


def oracle_baseline(w, nsteps=2):
    """cpu_baseline: the oracle on `nsteps` sampled steps of the workload (oracle_sampled_step).
    Returns (Mpoints*step/s credited, seconds per sampled step, extrapolated seconds per full
    step)."""
    import numpy as np
    c = oracle_channel(w)
    rng = np.random.default_rng(0)
    pts = w["nx"] * w["ny"] * w["nz"]
    tot, work = 0.0, 0.0
    for _ in range(nsteps):
        sec, frac = oracle_sampled_step(c, rng, **ORACLE_SAMPLE)
        tot += sec
        work += frac * pts
    return work / tot / 1e6, tot / nsteps, tot / (work / pts)


def run_reference(args, w, config):
    """The CPU oracle (the reference arm) on the machine's host cores: each step (warm-up and timed)
    is one sampled oracle step (oracle_sampled_step), so the whole run stays within minutes.
    ms_per_step is the sampled step's measured time; value is the work credited to the samples
    over that time; the extrapolated time of a full oracle step is a separate, labelled field."""
    import numpy as np
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count()
    c = oracle_channel(w)
    rng = np.random.default_rng(0)
    for _ in range(args.warmup):
        oracle_sampled_step(c, rng, **ORACLE_SAMPLE)
    tot, fracs = 0.0, 0.0
    for _ in range(args.steps):
        sec, frac = oracle_sampled_step(c, rng, **ORACLE_SAMPLE)
        tot += sec
        fracs += frac
    pts = w["nx"] * w["ny"] * w["nz"]
    val = fracs * pts / tot / 1e6
    t_step = tot / max(1, args.steps)
    out = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference", "config": config,
           "extrapolated_full_oracle_step_s": tot / fracs,
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample_note(w, **ORACLE_SAMPLE)},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_ensemble(args):
    """32 uneven channels (mixed precision; --precision 0 or 2 for FP64 or double-float x/y)
    advanced by grouped persistent launches, after the
    autotuner; the same members stepped one by one with their own graphs are timed beside it.
    With --cheb tc every member's z transforms run on the tensor cores (two launches per member
    per step beside the six grouped ones)."""
    import torch
    from paper_2406_01322_gb300 import binding, build, inputs
    build.build_library()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    prec = 1 if args.precision is None else args.precision
    ms = [dict(m, precision=prec) for m in inputs.ensemble_members()]
    ens = binding.Ensemble(ms, precision=prec, device=f"cuda:{local}")
    # auto: the tensor-core method, which steps this ensemble faster (35.5 against 43.8 ms per
    # mixed step after autotuning)
    tc = args.cheb in ("tc", "auto")
    if tc:
        ens.set_chebyshev(binding.CHEB_TC)
    for i, (g, m) in enumerate(zip(ens.grids, ms)):
        g.set_fields(*[torch.from_numpy(a) for a in inputs.initial_fields(**m)])
    ens.step(1)
    tuning = ens.autotune(reps=2)
    ens.step(args.warmup)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        tot_ms, kms = ens.step_timed(args.steps)
    torch.cuda.synchronize()
    # the same members, one ch_step per member per step (graph replays, no grouping)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        for g in ens.grids:
            g.step(1)
    t1.record()
    torch.cuda.synchronize()
    seq_ms = t0.elapsed_time(t1)
    pts = sum(m["nx"] * m["ny"] * m["nz"] for m in ms)
    # e2e: every member's fields from pinned host memory, K grouped steps, fields back to pinned
    # host memory, on the host clock
    host = [[torch.from_numpy(a).pin_memory() for a in inputs.initial_fields(**m)] for m in ms]
    outs = [[torch.empty_like(h).pin_memory() for h in hs] for hs in host]
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    for g, hs in zip(ens.grids, host):
        g.set_fields_host(*hs)
    ens.step(args.steps)
    for g, os_ in zip(ens.grids, outs):
        g.get_fields_host(os_)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t_e
    nbytes = sum(4 * m["nx"] * m["ny"] * m["nz"] * 8 for m in ms)
    names = list(binding.Ensemble.STAGES)
    out = {"metric": METRIC, "value": pts * args.steps / (tot_ms * 1e-3) / 1e6, "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None,
           "dtype": {0: "f64", 1: "f32 x/y transforms and products, f64 z transforms and solves",
                     2: "double-float x/y transforms and products, f64 z transforms and solves"}[prec]
                    + (" (z transforms as exact-split bf16 tensor-core products)" if tc else ""),
           "data": "synthetic",
           "config": {"workload": "ensemble_32_uneven", "members": len(ms),
                      "points": pts, "precision": PREC_NAMES[prec],
                      "chebyshev": "tc" if tc else "fft"},
           "sequential_members_ms_per_step": seq_ms / args.steps,
           "e2e": {"value": pts * args.steps / e2e_s / 1e6, "unit": UNIT,
                   "h2d_bytes_per_step": nbytes / args.steps,
                   "d2h_bytes_per_step": nbytes / args.steps,
                   "note": "set_fields_host of every member + K grouped steps + get_fields_host"},
           "stage_ms_per_step": {n: kms[i] / args.steps for i, n in enumerate(names)},
           "tuning": tuning, "gpu_launches": (6 + (2 * len(ms) if tc else 0)) * args.steps,
           "clocks": clk.summary()}
    ens.close()
    print(json.dumps(out))


def run_adjoint(args):
    """Gradient of J = 1/2 int |u|^2 + int |grad phi|^2 after the workload's steps with respect to
    the initial fields: forward run with checkpoints every 10 steps, then segment recomputation
    and the reverse sweep (torch.autograd through the library's adjoint kernels).  A bench step
    is one gradient; value = points x differentiated steps x gradients / device time."""
    import torch
    from paper_2406_01322_gb300 import binding, build, inputs
    build.build_library()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    w = dict(inputs.WORKLOADS[args.workload])
    nsteps = w["steps"]
    fields = inputs.initial_fields(**dict(w, seed=w["seed"] + rank))
    kw = dict(re_tau=w["re_tau"], we=w["we"], ch=w["ch"], pe=w["pe"], dt=w["dt"])
    g = binding.Grid(w["nx"], w["ny"], w["nz"], precision=0, device=f"cuda:{local}", **kw)
    dev = [torch.from_numpy(f).cuda() for f in fields]

    def gradient(ts):
        ts = [t.detach().requires_grad_(True) for t in ts]
        J = binding.objective_after(g, *ts, nsteps, checkpoint_every=10)
        J.backward()
        return J, [t.grad for t in ts]

    for _ in range(args.warmup):
        gradient(dev)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record()
        for _ in range(args.steps):
            gradient(dev)
        e1.record()
        torch.cuda.synchronize()
    tot_ms = e0.elapsed_time(e1)
    pts = w["nx"] * w["ny"] * w["nz"]
    value = pts * nsteps * args.steps / (tot_ms * 1e-3) / 1e6
    # forward-only reference on the same grid: nsteps plain steps
    g.set_fields(*dev)
    e0.record()
    g.step(nsteps)
    e1.record()
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    # e2e: pinned host fields in, gradients out to pinned host memory, per gradient
    host = [torch.from_numpy(f).pin_memory() for f in fields]
    outs = [torch.empty_like(h).pin_memory() for h in host]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ts = [h.to("cuda", non_blocking=True) for h in host]
        _, gr = gradient(ts)
        for o, a in zip(outs, gr):
            o.copy_(a, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # per-kernel times of one instrumented reverse sweep (states recomputed and saved first)
    g.set_fields(*dev)
    states = []
    for _ in range(nsteps):
        states.append(g.get_state())
        g.step(1)
    g.adjoint_begin()
    kms = [0.0] * len(binding.Grid.ADJ_KERNELS)
    for st in reversed(states):
        for i, v in enumerate(g.adjoint_step_timed(st)):
            kms[i] += v
    g.adjoint_end()
    names = list(binding.Grid.ADJ_KERNELS)
    work = adjoint_work(w)
    k = max(range(len(names)), key=lambda i: kms[i])
    per_launch_ms = kms[k] / nsteps
    fl, by = work[names[k]]
    ach = fl / (per_launch_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS,
            "traffic": traffic_bytes(args.workload, 0, names[k]), "kernel": names[k],
            "peak_kind": "float64 FMA pipe: 152 SMs x 2.07 GHz x 4 flop/clk (nominal)",
            "kernel_share": {n: kms[i] / sum(kms) for i, n in enumerate(names)},
            "kernel_ms_per_reverse_step": {n: kms[i] / nsteps for i, n in enumerate(names)},
            "note": "kernel times from an instrumented step-by-step reverse sweep, which "
                    "recomputes each state's fields (zbwd, ybwd); the timed gradients reverse "
                    "whole segments that keep them"}
    nbytes = 4 * pts * 8
    # launches of this library per gradient: set_fields 10 (4 x r2c, y pass, projection, four
    # for the products), 6 per forward step, objective 2, restore of the final state 4,
    # adjoint seed 2, per segment a restore (4) and 6 per recomputed step, 7 per reverse step
    # (the segment keeps the y-padded fields), gradient 6 (projection transpose, y pass, 4 c2r)
    nseg = -(-nsteps // 10)
    launches = 10 + 6 * nsteps + 2 + 4 + 2 + 4 * nseg + 6 * (nsteps - nseg) + 7 * nsteps + 6
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "grid": [w["nx"], w["ny"], w["nz"]],
                      "differentiated_steps": nsteps, "checkpoint_every": 10,
                      "precision": "fp64", "l2": "working set larger than L2 (no flush)",
                      "step": "one gradient: forward with checkpoints, recomputation, reverse"},
           "forward_only_ms": fwd_ms, "gradient_over_forward": (tot_ms / args.steps) / fwd_ms,
           "e2e": {"value": pts * nsteps * args.steps / e2e_s / 1e6, "unit": UNIT,
                   "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
           "gpu_launches": launches * args.steps, "roofline": roof, "clocks": clk.summary()}
    g.close()
    print(json.dumps(out))


def roofline_of(workload, w, prec, cheb, kms, steps, ms_step, names):
    """Roofline of the dominant kernel of a timed run (kms: summed ms per kernel over `steps`
    steps, in the order of `names`), the per-kernel times and shares, and the step-level HBM
    fraction (the step's algorithmic bytes over its time, against the measured copy peak)."""
    work = kernel_work(w, prec, cheb)
    # the FFT method launches no tensor-core transforms: their timed entries are empty gaps
    active = [i for i, n in enumerate(names) if cheb == "tc" or not n.startswith("cheb")]
    if cheb != "tc":
        work = {n: v for n, v in work.items() if not n.startswith("cheb")}
    k = max(active, key=lambda i: kms[i])
    name = names[k]
    per_launch_ms = kms[k] / steps
    fl, by = work[name]
    hbm, hbm_kind = peaks()
    traffic = traffic_bytes(workload, prec, name, cheb)
    # float64 kernels (all of precision 0, the z kernels of every precision) are ALU-bound and
    # measured against the float64 peak, the double-float x/y kernels (float64-accurate work on
    # the float32 pipe) against the double-float rate of the float32 pipe, float32 kernels
    # against HBM
    fp64_like = (prec != 1) or name.startswith("z")
    if prec == 2 and not name.startswith("z") and not name.startswith("cheb"):
        ach = fl / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": DF_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / DF_PEAK_TFLOPS, "traffic": traffic, "kernel": name,
                "peak_kind": "double-float on the float32 pipe: 152 SMs x 128 lanes x 2.07 GHz / "
                             "9.67 float32 instructions per float64-equivalent flop (nominal)"}
    elif name.startswith("cheb"):
        tpk, tpk_kind = tensor_peak()
        ach = fl / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": tpk, "unit": "TFLOP/s",
                "frac": ach / tpk, "traffic": traffic, "kernel": name, "peak_kind": tpk_kind}
    elif fp64_like:
        ach = fl / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": name,
                "peak_kind": "float64 FMA pipe: 152 SMs x 2.07 GHz x 4 flop/clk (nominal)"}
    else:
        ach = by / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": traffic, "kernel": name, "peak_kind": f"{hbm_kind} copy bandwidth"}
    roof["algorithmic_per_launch"] = {"flops": fl, "bytes": by}
    if roof["bound"] == "alu" and roof["peak"] == FP64_PEAK_TFLOPS and MEASURED_FMA.get("tflops"):
        roof["fp64_fma_measured_tflops"] = MEASURED_FMA["tflops"]
        roof["frac_of_measured_fma_rate"] = roof["achieved"] / MEASURED_FMA["tflops"]
    ksum = sum(kms[i] for i in active)
    roof["kernel_share"] = {names[i]: kms[i] / ksum for i in active}
    roof["kernel_ms_per_step"] = {names[i]: kms[i] / steps for i in active}
    step_bytes = sum(v[1] for v in work.values())
    roof["step_algorithmic_bytes"] = step_bytes
    roof["hbm_frac_step"] = (step_bytes / (ms_step * 1e-3) / 1e9) / hbm
    return roof


def precision_variants(binding, w, workload, fields, kw, steps, device, main):
    """The same workload in the other precision modes and Chebyshev methods than the headline
    run `main` = (precision, method): device time per step over `steps` steps (after 3 warm-up
    steps) and the max relative field difference from the float64 FFT path after 3 + `steps`
    steps from the same fields.  The float64 FFT step (the comparison base) also reports its
    per-kernel times, its dominant kernel's roofline and its step-level HBM fraction."""
    import torch
    out, final = {}, {}
    pts = w["nx"] * w["ny"] * w["nz"]
    names = list(binding.Grid.KERNELS)
    combos = [(0, 0, 0), (2, 0, 0), (1, 0, 0), (0, 1, 0), (2, 1, 0), (1, 1, 0)]
    combos += [(0, 0, 1), (main[0], 0, 1)] if main[0] != 0 else [(0, 0, 1)]
    for pr, cheb, prune in combos:
        g = binding.Grid(w["nx"], w["ny"], w["nz"], precision=pr, device=device, **kw)
        g.set_chebyshev(cheb)
        g.set_fft_pruning(prune)
        g.set_fields(*[torch.from_numpy(f) for f in fields])
        g.step(3)
        tot, kms = g.step_timed(steps)
        final[(pr, cheb, prune)] = [f.cpu() for f in g.get_fields()]
        g.close()
        torch.cuda.empty_cache()
        if (pr, cheb, prune) == main:
            continue
        name = PREC_NAMES[pr] + ("_tc" if cheb else "") + ("_pruned" if prune else "")
        dt = DTYPES[pr] + (" (Chebyshev transforms: exact-split bf16 tensor-core products, "
                           "float64-accurate)" if cheb else "") + (
            " (pruned x/y transforms of the 3/2-rule padding)" if prune else "")
        v = {"ms_per_step": tot / steps, "dtype": dt,
             "value": pts * steps / (tot * 1e-3) / 1e6,
             "max_rel_field_diff_vs_fp64": None if (pr, cheb, prune) == (0, 0, 0) else max(
                 float((a - b).abs().max() / b.abs().max())
                 for a, b in zip(final[(pr, cheb, prune)], final[(0, 0, 0)]))}
        if (pr, cheb, prune) == (0, 0, 0):
            v["roofline"] = roofline_of(workload, w, 0, "fft", kms, steps, tot / steps, names)
        out[name] = v
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 100; adjoint workload: gradients, default 5)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="channel_512x256x257_mixed")
    ap.add_argument("--precision", type=int, default=None,
                    help="0 fp64, 1 mixed (fp32 x/y), 2 double-float x/y")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the comparison against the FP64 path (precision 1 and 2)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the other precisions and Chebyshev methods of the same workload")
    ap.add_argument("--cheb", default="auto", choices=["auto", "fft", "tc"],
                    help="Chebyshev transforms of the step: N-point DCT-I in float64 (fft), "
                         "the exact-split matrix product on the tensor cores (tc), or whichever "
                         "of the two steps faster on this grid (auto: timed before the run)")
    ap.add_argument("--prune", type=int, default=0, choices=[0, 1],
                    help="pruned x/y transforms of the 3/2-rule padding (ch_set_fft_pruning)")
    ap.add_argument("--grid", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"),
                    help="run the workload's physics on another grid (smaller cases of the same "
                         "kernels for profiling); the workload name then carries the grid")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 5 if args.workload == "channel_128x128x129_adjoint" else 100

    from paper_2406_01322_gb300 import inputs
    if args.workload == "ensemble_32_uneven":
        run_ensemble(args)
        return
    if args.workload == "channel_128x128x129_adjoint" and args.impl == "native":
        run_adjoint(args)
        return
    w = dict(inputs.WORKLOADS[args.workload])
    if args.grid is not None:
        w.update(nx=args.grid[0], ny=args.grid[1], nz=args.grid[2])
        args.workload = f"{args.workload}@{args.grid[0]}x{args.grid[1]}x{args.grid[2]}"
    prec = w["precision"] if args.precision is None else args.precision
    _, world0, _ = dist_env()
    config = {"workload": args.workload, "grid": [w["nx"], w["ny"], w["nz"]],
              "precision": PREC_NAMES[prec], "chebyshev": args.cheb,
              "pruned_xy_transforms": bool(args.prune),
              "parallelism": "replicas" if world0 > 1 else "single",
              "l2": "step working set larger than L2 (no flush)"}
    if args.impl == "reference":
        run_reference(args, w, config)
        return

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2406_01322_gb300 import build
    if rank == 0:
        build.build_library()
    if world > 1:
        dist.barrier()
    from paper_2406_01322_gb300 import binding
    MEASURED_FMA["tflops"] = binding.fp64_fma_rate()

    fields = inputs.initial_fields(**dict(w, seed=w["seed"] + rank))
    kw = dict(re_tau=w["re_tau"], we=w["we"], ch=w["ch"], pe=w["pe"], dt=w["dt"])
    g = binding.Grid(w["nx"], w["ny"], w["nz"], precision=prec, device=f"cuda:{local}", **kw)
    g.set_fft_pruning(args.prune)
    cheb_trial = {}
    if args.cheb == "auto":
        # the Chebyshev method is part of the kernel choice, not of the workload: time both on
        # this grid (a few steps each, untimed in the result) and run the faster
        for name, m in (("fft", binding.CHEB_FFT), ("tc", binding.CHEB_TC)):
            g.set_chebyshev(m)
            g.set_fields(*[torch.from_numpy(f) for f in fields])
            g.step(2)
            t, _ = g.step_timed(3)
            cheb_trial[name] = t / 3
        pick = 1.0 if cheb_trial["tc"] < cheb_trial["fft"] else 0.0
        cheb = "tc" if max_over_ranks(pick, world, "cuda") > 0.5 else "fft"
    else:
        cheb = args.cheb
    g.set_chebyshev(binding.CHEB_TC if cheb == "tc" else binding.CHEB_FFT)
    g.set_fields(*[torch.from_numpy(f) for f in fields])
    g.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-timed region
    barrier()
    with ClockSampler(local) as clk:
        tot_ms, kms = g.step_timed(args.steps)
    barrier()
    tot_ms = max_over_ranks(tot_ms, world, "cuda")
    pts = w["nx"] * w["ny"] * w["nz"]
    value = replica_throughput(pts, args.steps, world, tot_ms * 1e-3)
    ms_step = tot_ms / args.steps

    # ---- e2e through the C ABI with host buffers
    host = [torch.from_numpy(f).pin_memory() for f in fields]
    outs = [torch.empty_like(h).pin_memory() for h in host]
    barrier()
    t0 = time.perf_counter()
    g.set_fields_host(*host)
    g.step(args.steps)
    g.get_fields_host(outs)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_val = replica_throughput(pts, args.steps, world, e2e_s)
    nbytes = 4 * pts * 8

    # ---- roofline of the dominant kernel
    names = list(binding.Grid.KERNELS)
    roof = roofline_of(args.workload, w, prec, cheb, kms, args.steps, ms_step, names)

    if rank != 0:
        g.close()
        if world > 1:
            dist.destroy_process_group()
        return
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "steps_per_s": 1e3 / ms_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": DTYPES[prec],
           "data": "synthetic",
           "config": config,
           "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": nbytes / args.steps,
                   "d2h_bytes_per_step": nbytes / args.steps,
                   "note": "set_fields_host + K steps + get_fields_host per job, bytes / K"},
           "gpu_launches": g.launches_per_step() * args.steps,
           "chebyshev_method": cheb,
           "roofline": roof,
           "clocks": clk.summary()}
    if cheb_trial:
        out["chebyshev_trial_ms_per_step"] = cheb_trial
    g.close()
    torch.cuda.empty_cache()
    dev = f"cuda:{local}"
    if world == 1 and not args.no_variants:
        out["variants"] = precision_variants(binding, w, args.workload, fields, kw, args.steps,
                                             dev, (prec, 1 if cheb == "tc" else 0,
                                                   args.prune))
    if world == 1 and prec != 0 and not args.no_accuracy:
        acc = precision_accuracy(binding, w, fields, w["steps"], dev, prec)
        if prec == 1:
            from paper_2406_01322_gb300.bounds import MIXED_BOUNDS
            acc["bounds"] = MIXED_BOUNDS
            acc["bounds_met"] = all(
                [acc["rel_err"][n] <= MIXED_BOUNDS[n] for n in acc["rel_err"]]
                + [abs(acc[k + "_rel_diff"]) <= MIXED_BOUNDS[k]
                   for k in ("mass", "kinetic", "grad2", "free_energy")])
        out[PREC_NAMES[prec] + "_vs_fp64"] = acc
    if world == 1:
        zc, xyc = cufft_transforms_ms(w, prec)
        ours_xy = sum(roof["kernel_ms_per_step"][n] for n in ("ybwd", "xline", "yfwd"))
        gm, gtf = dct_gemm_ms(w)
        kms_step = roof["kernel_ms_per_step"]
        zrhs_ms = kms_step["zrhs"] + (kms_step.get("cheb_fwd", 0.0) if cheb == "tc" else 0.0)
        out["dct_as_gemm_comparison"] = {
            "fp64_gemm_ms_for_7_forward_dcts": gm, "fp64_gemm_tflops": gtf,
            "ours_zrhs_ms": zrhs_ms,
            "note": "the 7 forward DCTs of one step as one cuBLAS float64 GEMM, against our whole "
                    "forward z stage: zrhs (7 DCTs + derivatives + assembly), or with the "
                    "tensor-core method its forward transform of the seven combined lines "
                    "plus the coefficient-space zrhs"}
        out["cufft_comparison"] = {
            "cufft_z_dct_ms_per_step": zc, "cufft_xy_ms_per_step": xyc,
            "cufft_transforms_ms_per_step": zc + xyc,
            "ours_step_ms": ms_step, "ours_ybwd_xline_yfwd_ms": ours_xy,
            "note": "cuFFT (torch.fft) timed on the transforms of one step only (no products, "
                    "assembly or solves); ours_ybwd_xline_yfwd_ms also includes the products"}
    if world == 1 and not args.no_cpu_baseline:
        val, t_sample, t_full = oracle_baseline(w, nsteps=2)
        out["cpu_baseline"] = {"value": val, "unit": UNIT, "cores": os.cpu_count(),
                               "kind": "oracle", "sample": sample_note(w, **ORACLE_SAMPLE),
                               "seconds_per_sampled_step": t_sample,
                               "extrapolated_full_oracle_step_s": t_full}
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
