#!/usr/bin/env python3
"""Benchmark of the electron scattering self-energy (Eq. 3) on GB300.

One step = one sse_sigma_fwd call: Sigma^< and Sigma^> for every atom,
energy and kz of the workload (default: the Si-FinFET-shaped problem,
NA=1024, NB=4, Norb=10, NE=512, Nkz=Nqz=7, Nw=32), inputs resident in HBM.
Default mode: FP64 through the convolution theorem (fp64_fft); the other
modes (direct FP64, BF16X3, TF32, FP32 transforms, FP32 transforms with the
block products on the tensor cores (f16x3_fft), and the transform modes
with anti-Hermitian inputs) are timed on the same inputs in the "compare"
object, with their error against this run's result; Pi (Eq. 4), the adjoint
and the gradient in G follow in "pi" and "adjoint". Prints one JSON line
(rank 0).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload finfet|large|...]
                  [--mode fp64_fft|fp32_fft|f16x3_fft|fp64|tf32|bf16x3] [--antihermitian]

Metric: useful TFLOP/s of the paper-equivalent (regrouped, Sec. 5.1) flop
count, plus (E,kz) points/s. Multi-GPU (torchrun): the one workload split
into atom tiles (parallel.sigma_atom_sharded: a halo exchange of the
neighbours' G blocks over NCCL, then the library on each rank's atoms),
value = the workload's useful flops / the max over ranks of the step time
("strong"); the line reports the halo bytes against the paper's model.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import threading
import time

import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1912_10024_gb300 import binding as B  # noqa: E402
from paper_1912_10024_gb300.inputs import WORKLOADS, make_inputs, make_upstream  # noqa: E402

SCALE = 1.0 / (2.0 * math.pi)
# FP64 pipe of GB300: 152 SMs x 2 FP64 FMA/clock x 2 flop x 2070 MHz (unit count and maximum SM clock; a DFMA
# throughput probe measured 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# FP32 pipe: 152 SMs x 128 FP32 FMA/clock x 2 flop x 2070 MHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def n_valid(NE: int, Nw: int):
    """Number of in-range (w, sigma) terms for each energy."""
    return [sum(1 for w in range(Nw) if E - (w + 1) >= 0) + sum(1 for w in range(Nw) if E + (w + 1) < NE)
            for E in range(NE)]


def useful_flops(d, atoms=None, energies=None) -> float:
    """Paper-equivalent flops (Sec. 5.1 model after regrouping, exact in-range count):
    per (a, s, t, k, E): 24 Norb^3 per in-range (q, w, sigma) term + 24 Norb^3 final multiply."""
    nv = n_valid(d.NE, d.Nw)
    Es = range(d.NE) if energies is None else energies
    nA = d.NA if atoms is None else atoms
    per = sum(24 * d.Norb ** 3 * (d.Nqz * nv[E] + 1) for E in Es)
    return 2.0 * nA * d.NB * d.Nkz * per


def fp64_kernel_flops(d) -> float:
    """Real FP64 flops the FP64 kernel's algorithm performs (no zero taps counted):
    per (a, s, t, k, E): 9 Norb^2 complex MACs per in-range term at 3 FMA (6 flop) each,
    plus 12 Norb^3 complex MACs (8 flop) of block products."""
    nv = n_valid(d.NE, d.Nw)
    per = sum(54 * d.Norb ** 2 * d.Nqz * nv[E] + 96 * d.Norb ** 3 for E in range(d.NE))
    return 2.0 * d.NA * d.NB * d.Nkz * per


def fft_length(NE: int, Nw: int) -> int:
    """FFT length along E of the fp64_fft mode: the smallest 2^a 3^b >= NE + Nw."""
    L = NE + Nw
    while True:
        m = L
        for p in (2, 3):
            while m % p == 0:
                m //= p
        if m == 1:
            return L
        L += 1


def freq_count(d, half: bool) -> int:
    """Frequencies the product kernels evaluate: Nkz * L, or one of each (f, -f) pair with
    SSE_FLAG_ANTIHERMITIAN (the library's frequency map)."""
    L = fft_length(d.NE, d.Nw)
    if not half:
        return d.Nkz * L
    return d.Nkz * ((L - 1) // 2) + (d.Nkz // 2 + 1) * (2 if L % 2 == 0 else 1)


def spectral_prod_flops(d, half: bool = False) -> float:
    """FP64 flops one spec_prod_kernel launch (one type) executes: per (atom, slot, frequency) and block
    element, the weight block W_i (9 complex MACs at 4 FMA) and two block products (3 Norb complex
    MACs each at 3 FMA, Gauss form); 2 flops per FMA."""
    nel = d.Norb * d.Norb
    return 2.0 * d.NA * d.NB * freq_count(d, half) * nel * (36 + 18 * d.Norb)


def spectral_prod32_flops(d, half: bool = False) -> float:
    """FP32 flops one spec_prod32_kernel launch (one type) executes: per (atom, slot, frequency) and element of
    the block padded to an even order Np, P_j = G^ dH_j^H and sum_i dH_i U_i (3 Norb complex MACs each at
    4 FMA) and U_i = sum_j K_ij P_j (9 complex MACs at 4 FMA); 2 flops per FMA."""
    Np = d.Norb + (d.Norb & 1)
    return 2.0 * d.NA * d.NB * freq_count(d, half) * Np * Np * (36 + 24 * d.Norb)


def tc_shape(norb: int):
    """Tile shape of spec_prod_tc_kernel (mode F16X3_FFT): frequencies per 128-row tile and the padded GEMM sizes
    (fp16 elements): GEMM1 K1 x N1, GEMM2 K2 x N2 (N per part: the dH operand's hi or lo)."""
    r16 = lambda x: -(-x // 16) * 16  # noqa: E731
    return {"FT": 4 * (32 // norb), "K1": r16(2 * norb), "N1": r16(6 * norb), "K2": 8 * (-(-norb // 2) * 2),
            "N2": r16(2 * norb)}


def tc_tensor_flops(d, half: bool = False) -> float:
    """Tensor-pipe flops one spec_prod_tc_kernel launch (one type) issues (padding included): per 128-row tile of
    frequencies and bond, GEMM1 as hi x [B_hi | B_lo] (N = 2 N1) + lo x B_hi (N = N1) over K1, GEMM2 likewise with
    N2 over K2; 2 flops per multiply-add."""
    t = tc_shape(d.Norb)
    tiles = -(-freq_count(d, half) // t["FT"])
    per = 2.0 * 128 * (3 * t["N1"] * t["K1"] + 3 * t["N2"] * t["K2"])
    return per * tiles * d.NB * d.NA


def tc_useful_flops(d, half: bool = False) -> float:
    """The part of tc_tensor_flops that the split-precision products need, padding excluded: per (atom, bond,
    frequency) the two real-embedded GEMMs (Norb rows; K = 2 Norb, N = 6 Norb, then K = 6 Norb, N = 2 Norb), three
    FP16 products each; 2 flops per multiply-add."""
    n = d.Norb
    return 2.0 * 3 * n * (2 * n * 6 * n + 6 * n * 2 * n) * freq_count(d, half) * d.NB * d.NA


def spectral_pi_flops(d, half: bool = False) -> float:
    """FP64 flops one spec_pi_kernel launch (both types) executes: per (type, atom, slot, frequency) and block
    element, the half products dH_i^H G^ and dH_j G^ (3 Norb complex MACs each at 3 FMA) and the 9 trace
    terms (2 FMA each); 2 flops per FMA."""
    nel = d.Norb * d.Norb
    return 2.0 * 2 * d.NA * d.NB * freq_count(d, half) * nel * (18 * d.Norb + 18)


def spectral_adj_flops(d) -> float:
    """FP64 flops one spec_adj_kernel launch (one type) executes: per (atom, slot, frequency) and block
    element, 12 block products (3 Norb complex MACs each at 3 FMA), the coupling-gradient weights
    (6 complex MACs at 4 FMA per direction) and the weight-gradient traces (9 Norb^2 complex MACs at 4 FMA
    per frequency); 2 flops per FMA."""
    L = fft_length(d.NE, d.Nw)
    nel = d.Norb * d.Norb
    return 2.0 * d.NA * d.NB * d.Nkz * L * nel * (36 * d.Norb + 108)


def mixed_tensor_flops(d, mode: str) -> float:
    """Tensor-pipe flops one sse_sigma_fwd launch issues in a mixed mode (padding included):
    per (atom, slot, type, kz, 128-row tile) and in-range (q, w, sigma) tap, kpad/kstep MMAs of
    128 x npad x kstep (the tile layout of the tcgen05 kernel)."""
    TE = 128 // d.Norb
    kstep = 16 if mode == "bf16x3" else 8
    kraw = 6 * d.Norb if mode == "bf16x3" else 2 * d.Norb
    kpad = -(-kraw // kstep) * kstep
    npad = -(-6 * d.Norb // 16) * 16
    taps = 0
    for E0 in range(0, d.NE, TE):
        taps += max(0, min(d.Nw, E0 + TE - 1)) + max(0, min(d.Nw, d.NE - 1 - E0))
    return 2.0 * 128 * npad * kpad * taps * d.Nqz * d.NB * d.Nkz * 2 * d.NA


def mixed_useful_flops(d, mode: str) -> float:
    """The part of mixed_tensor_flops that the method needs, padding excluded: per in-range tap the tile's energy rows
    (Norb each, the last tile ragged), K = 6 Norb (BF16X3: G_hi, G_lo, G_hi against W_hi, W_hi, W_lo) or 2 Norb
    (TF32) and N = 6 Norb."""
    TE = 128 // d.Norb
    kraw = 6 * d.Norb if mode == "bf16x3" else 2 * d.Norb
    rows_taps = 0
    for E0 in range(0, d.NE, TE):
        taps = max(0, min(d.Nw, E0 + TE - 1)) + max(0, min(d.Nw, d.NE - 1 - E0))
        rows_taps += min(TE, d.NE - E0) * d.Norb * taps
    return 2.0 * rows_taps * 6 * d.Norb * kraw * d.Nqz * d.NB * d.Nkz * 2 * d.NA


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per unit from one ncu capture at the adjoint workload,
# with the sha256 prefix of the captured kernel's own source text: the figure is dropped (None) once that kernel
# has changed.
NCU_TRAFFIC = {
    "spec_prod_kernel": (4815.4, "a19635f8b1e45065", "atom-frequency of one type"),
    "spec_pi_kernel": (5033.6, "9a225dfc2cb7d028", "type-atom-frequency"),
    "spec_adj_kernel": (13897.1, "3cadf5d36e3c5bb6", "atom-frequency of one type"),
    "spec_prod32_kernel": (1923.2, "f34fb6e78487019a", "atom-frequency of one type"),
    "spec_adj32_kernel": (7533.4, "8e9f1b2f0231170c", "atom-frequency of one type"),
    "spec_pi32_kernel": (2121.4, "3f8eabc933beac4b", "type-atom-frequency"),
    "spec_gradg32_kernel": (1863.7, "aa646c7c1d04f57d", "atom-frequency of one type"),
    "spec_prod_tc_kernel": (1865.6, "b6487e717de45e49", "atom-frequency of one type"),
}


def kernel_source_sha(kernel: str) -> str:
    """sha256 prefix of a kernel's source text in the library's sources: from the line that opens its definition
    (`__global__ ... <kernel>(`) to the first closing brace in column 0."""
    import glob
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1912_10024_gb300", "csrc")
    for path in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))):
        with open(path) as f:
            src = f.read()
        m = re.search(r"__global__[^;{]*?\b" + re.escape(kernel) + r"\(", src)
        if m is not None:
            end = src.find("\n}\n", m.end())
            return hashlib.sha256(src[m.start():end + 3].encode()).hexdigest()[:16]
    return ""


def ncu_traffic(kernel: str, units: float):
    """Per-launch DRAM traffic scaled from the ncu capture by the units one launch processes, or None
    when the kernel's source changed since the capture."""
    if kernel not in NCU_TRAFFIC:
        return None
    per, sha, _ = NCU_TRAFFIC[kernel]
    if kernel_source_sha(kernel) != sha:
        return None
    return per * units


def gpu_local_cpus(dev):
    """Host CPUs on the GPU's own NUMA node (sysfs local_cpulist of its PCI device), intersected with the CPUs this
    process may use; None when the system does not say."""
    try:
        pr = torch.cuda.get_device_properties(dev)
        path = "/sys/bus/pci/devices/%04x:%02x:%02x.0/local_cpulist" % (pr.pci_domain_id, pr.pci_bus_id,
                                                                        pr.pci_device_id)
        with open(path) as f:
            text = f.read().strip()
        cpus = set()
        for part in text.split(","):
            if "-" in part:
                lo, hi = part.split("-")
                cpus.update(range(int(lo), int(hi) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        return cpus or None
    except (AttributeError, OSError, ValueError):
        return None


FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def load_peaks(path=None):
    """Measured copy bandwidth and bf16 GEMM rates of this GPU model; the earlier GB300 measurement for any figure
    the file lacks (or for all of them, without a readable file), with the source saying which."""
    try:
        with open(path or os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            measured = json.load(f)
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"
    peaks = dict(FALLBACK_PEAKS)
    usable = {k: float(v) for k, v in measured.items() if k in FALLBACK_PEAKS and isinstance(v, (int, float)) and v > 0}
    peaks.update(usable)
    return peaks, "measured" if len(usable) == len(FALLBACK_PEAKS) else "measured, partly fallback"


def smi_gpu_id(local: int) -> str:
    """The GPU behind torch's device ``local`` as nvidia-smi names it: with CUDA_VISIBLE_DEVICES set, its entry number
    ``local`` (an index or a UUID; nvidia-smi counts every GPU of the machine), else ``local`` itself."""
    ids = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    return ids[local] if local < len(ids) else str(local)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: str):
        self.gpu, self.proc, self.lines = gpu, None, []

    def __enter__(self):
        if shutil.which("nvidia-smi"):
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "gpu": self.gpu}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "gpu": self.gpu}


def cpu_baseline(d, seconds: float, inp=None, seed: int = 0):
    """The FP64 oracle as it stands, on this host's cores, over a bounded sample:
    atom 0 and a growing block of energies around the middle, all kz, both types."""
    import oracle
    from oracle.subproblem import oracle_blocks
    if inp is None:
        # only atom 0's neighbourhood is copied to the host by oracle_blocks
        inp = make_inputs(d, seed=seed, device="cuda" if torch.cuda.is_available() else "cpu")
    threads = oracle.default_threads()
    nE, spent, flops, a = 1, 0.0, 0.0, 0
    E0 = d.NE // 2
    while spent < seconds and nE <= d.NE:
        lo = max(0, min(E0, d.NE - nE))
        t0 = time.perf_counter()
        oracle_blocks(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, a, lo, lo + nE,
                      nthreads=threads)
        dt = time.perf_counter() - t0
        spent += dt
        flops += useful_flops(d, atoms=1, energies=range(lo, lo + nE))
        last = (nE, dt)
        nE *= 2
    return {"value": flops / spent / 1e12, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"atom 0, energies around NE/2 in blocks of 1,2,...,{last[0]} ({spent:.1f} s total), "
                      f"all kz, Sigma^< and Sigma^>; FP64 C loops (pthreads)"}


def bench_config(args, d, world=1):
    """The workload description shared by both arms (the same keys and values for the same arguments)."""
    g_bytes = 2 * d.Nkz * d.NE * d.NA * d.Norb * d.Norb * 16
    return {"workload": args.workload, **d.__dict__, "mode": args.mode,
            "antihermitian_inputs_flag": bool(getattr(args, "antihermitian", False)),
            "l2": "inputs larger than L2 (G^<,G^> %.1f GB)" % (g_bytes / 1e9),
            "parallelism": "1 rank" if world == 1 else
                           f"atom tiles over {world} ranks (parallel.sigma_atom_sharded): one halo exchange of G "
                           f"over NCCL per step, then the library on the owned atoms"}


def run_reference(args, d, rank, world):
    if rank != 0:
        return 0
    inp = make_inputs(d, seed=0, device="cuda" if torch.cuda.is_available() else "cpu")
    cb = cpu_baseline(d, args.cpu_seconds, inp)
    steps = []
    for _ in range(args.warmup + args.steps):
        steps.append(cpu_baseline(d, args.cpu_seconds / 4, inp))
    vals = [s["value"] for s in steps[args.warmup:]]
    v = statistics.median(vals)
    out = {"impl": "reference", "metric": "SSE useful TFLOP/s (Eq. 3, paper-equivalent flops)", "value": v,
           "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(args, d, world),
           "cpu_baseline": {**cb, "value": v},
           "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_sharded(args, d, rank, world, local, dev):
    """N > 1: one global problem (the workload) split into atom tiles over the ranks (Sec. 4.2's communication-avoiding
    tiling). A step is parallel.sigma_atom_sharded on every rank: the halo exchange of the neighbours' G blocks over
    NCCL (one packed message per peer and direction), the rank-local problem, and the library call on the owned atoms.
    Strong scaling: value = the whole problem's useful flops / the max over ranks of the step time."""
    import torch.distributed as dist
    from paper_1912_10024_gb300 import parallel as P
    full = make_inputs(d, seed=0, device=dev)  # the same seeded problem on every rank; each keeps its tile
    a0, a1 = P.atom_range(d.NA, world, rank)
    nbr = full.nbr.cpu()
    G_own = (full.G_less[:, :, a0:a1].contiguous(), full.G_greater[:, :, a0:a1].contiguous())
    D_own = (full.D_less[:, :, a0:a1].contiguous(), full.D_greater[:, :, a0:a1].contiguous())
    dH_own = full.dH[a0:a1].contiguous()
    del full
    torch.cuda.empty_cache()
    flags = {"antihermitian": bool(args.antihermitian)}

    def step(profile=False):
        return P.sigma_atom_sharded(nbr, dH_own, D_own, G_own, d.NA, SCALE, mode=args.mode, profile=profile, **flags)

    S = None
    for _ in range(args.warmup):
        S = step()
    del S
    torch.cuda.synchronize(dev)
    dist.barrier()
    torch.cuda.synchronize(dev)
    B.sse_profile_read()  # drop anything recorded before the timed region
    stream = torch.cuda.current_stream(dev)
    with ClockSampler(smi_gpu_id(local)) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            S = step(profile=True)  # CUDA events around each library kernel, on this stream
        t1.record(stream)
        torch.cuda.synchronize(dev)
    dist.barrier()
    launches = sum(n for _name, _ms, n in B.sse_profile_read())
    t = torch.tensor([t0.elapsed_time(t1)], device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_per_step = float(t.item()) / args.steps
    # end to end through the same public calls: each step uploads the rank's G tiles from page-locked host memory,
    # runs the sharded call, and downloads its Sigma tiles
    e2e = None
    if not args.no_e2e:
        hG = [g.cpu().pin_memory() for g in G_own]
        hS = [torch.empty(g.shape, dtype=g.dtype).pin_memory() for g in G_own]
        dG = [torch.empty_like(g) for g in G_own]

        def e2e_step():
            for dst, src in zip(dG, hG):
                dst.copy_(src, non_blocking=True)
            Sd = P.sigma_atom_sharded(nbr, dH_own, D_own, dG, d.NA, SCALE, mode=args.mode, **flags)
            for dst, src in zip(hS, Sd):
                dst.copy_(src, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize(dev)
        dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        dist.barrier()
        te = torch.tensor([e0.elapsed_time(e1)], device=dev)
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
        bts = torch.tensor([float(sum(x.numel() * x.element_size() for x in hG))], device=dev, dtype=torch.float64)
        dist.all_reduce(bts, op=dist.ReduceOp.SUM)
        e_ms = float(te.item()) / args.steps
        e2e = {"value": useful_flops(d) / (e_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": e_ms,
               "h2d_bytes_per_step": float(bts.item()), "d2h_bytes_per_step": float(bts.item()),
               "how": "every rank: its G tiles uploaded from page-locked host memory, parallel.sigma_atom_sharded, "
                      "its Sigma tiles downloaded; bytes summed over the ranks"}
        del hG, hS, dG
    # halo bytes received per step (both types), against the paper's model with c = NB extra atoms per process
    halo = len(P.halo_atoms(nbr, a0, a1))
    blk = d.Nkz * d.NE * d.Norb * d.Norb * 16
    hb = torch.tensor([2.0 * halo * blk], device=dev, dtype=torch.float64)
    dist.all_reduce(hb, op=dist.ReduceOp.MAX)
    hsum = torch.tensor([2.0 * halo * blk], device=dev, dtype=torch.float64)
    dist.all_reduce(hsum, op=dist.ReduceOp.SUM)
    uf = useful_flops(d)
    if rank == 0:
        out = {"metric": "SSE useful TFLOP/s (Eq. 3, paper-equivalent flops)",
               "value": uf / (ms_per_step * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong",
               "vs_baseline": None,
               "dtype": {"fp64": "f64", "fp64_fft": "f64", "fp32_fft": "f32", "tf32": "tf32+f64",
                         "bf16x3": "bf16x3+f64", "f16x3_fft": "f32+f16x3"}[args.mode],
               "data": "synthetic (seeded; Si-FinFET-shaped)",
               "config": bench_config(args, d, world),
               "pts_per_s": d.NE * d.Nkz / (ms_per_step * 1e-3),
               "exchange": {"halo_bytes_received_max_rank": float(hb.item()),
                            "halo_bytes_received_all_ranks": float(hsum.item()),
                            "paper_model_bytes_per_rank": 2.0 * d.NB * blk,
                            "paper_model": "the G part of Sec. 4.2's all-to-all volume beyond the owned atoms: "
                                           "2 types x 16 B x Nkz x NE x c x Norb^2 with c = NB (T_E = 1)"},
               "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches}
        print(json.dumps(out))
    dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="finfet", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="fp64_fft", choices=sorted(B.MODES))
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other modes on the same inputs")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--antihermitian", action="store_true",
                    help="pass SSE_FLAG_ANTIHERMITIAN (the synthetic G and D blocks are exactly anti-Hermitian)")
    ap.add_argument("--no-pi", action="store_true", help="skip timing the phonon self-energy (Eq. 4)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip timing the FP64 adjoint")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    d = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, d, rank, world)

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        return run_sharded(args, d, rank, world, local, dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    inp = make_inputs(d, seed=rank, device=dev)
    mode = B.MODES[args.mode]
    run_flags = B.SSE_FLAG_ANTIHERMITIAN if args.antihermitian else 0
    dims = B.dims_of(inp.G_less, inp.D_less, inp.dH)
    ws = B.workspace(dims, mode, 0, dev)
    Sl = torch.empty_like(inp.G_less)
    Sg = torch.empty_like(inp.G_greater)
    stream = torch.cuda.current_stream(dev)

    def step(flags=0):
        rc = B.sse_sigma_fwd(dims, inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                             mode, flags | run_flags, Sl, Sg, ws, ws.numel(), stream)
        if rc != 0:
            raise B.SseError(rc, "sse_sigma_fwd")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    B.sse_profile_read()  # drop anything recorded before the timed region
    with ClockSampler(smi_gpu_id(local)) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            step(B.SSE_FLAG_PROFILE)  # CUDA events around each kernel, on this stream
        t1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    total_ms = t0.elapsed_time(t1)
    kernels = {name: (ms, n) for name, ms, n in B.sse_profile_read()}
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    uf = useful_flops(d)
    value = world * uf * args.steps / (total_ms * 1e-3) / 1e12
    pts = world * d.NE * d.Nkz * args.steps / (total_ms * 1e-3)

    # ---- end to end through the public API with host buffers ----
    # sse_sigma_fwd_host: pinned host inputs in, Sigma out; the uploads and downloads run on a second
    # stream and overlap the compute of the other type (transform modes)
    e2e = None
    if not args.no_e2e:
        # page-locked buffers allocated (first touch) from the CPUs of the GPU's own NUMA node where known, as a
        # NUMA-aware caller would; the binding is reported
        local = gpu_local_cpus(dev)
        saved = os.sched_getaffinity(0)
        if local:
            os.sched_setaffinity(0, local)
        host = {n: getattr(inp, n).cpu().pin_memory() for n in ("nbr", "dH", "D_less", "D_greater", "G_less",
                                                                  "G_greater")}
        hSl = torch.empty(Sl.shape, dtype=Sl.dtype).pin_memory()
        hSg = torch.empty(Sg.shape, dtype=Sg.dtype).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = 2 * Sl.numel() * Sl.element_size()
        nbuf = B.sse_sigma_fwd_host_bytes(dims, mode, run_flags)
        dbuf = torch.empty(nbuf, dtype=torch.uint8, device=dev)
        cp = torch.cuda.Stream(device=dev)

        def hstep():
            rc = B.sse_sigma_fwd_host(dims, host["nbr"], host["dH"], host["D_less"], host["D_greater"],
                                      host["G_less"], host["G_greater"], SCALE, mode, run_flags, hSl, hSg, dbuf,
                                      nbuf, stream, cp)
            if rc != 0:
                raise B.SseError(rc, "sse_sigma_fwd_host")

        hstep()  # warm-up
        torch.cuda.synchronize(dev)
        # the host link as seen from these buffers: one plain copy of G^< each way
        l0, l1, l2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        gdev = dbuf[:host["G_less"].numel() * host["G_less"].element_size()].view(torch.complex128).view(
            host["G_less"].shape)
        l0.record(stream)
        gdev.copy_(host["G_less"], non_blocking=True)
        l1.record(stream)
        hSl.copy_(gdev, non_blocking=True)
        l2.record(stream)
        torch.cuda.synchronize(dev)
        gbytes = host["G_less"].numel() * host["G_less"].element_size()
        link = {"h2d_gbs": gbytes / (l0.elapsed_time(l1) * 1e-3) / 1e9,
                "d2h_gbs": gbytes / (l1.elapsed_time(l2) * 1e-3) / 1e9}
        del gdev
        barrier()
        nsteps = max(args.steps, 3)  # host copies vary more than kernels: time at least three steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nsteps):
            hstep()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        e2e_ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([e2e_ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_ms = float(t.item())
        same = bool(torch.equal(hSl, Sl.cpu()) and torch.equal(hSg, Sg.cpu()))
        e2e = {"value": world * uf * nsteps / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / nsteps,
               "steps": nsteps, "api": "sse_sigma_fwd_host (pinned host buffers, copies on a second stream)",
               "same_bytes_as_device_call": same, "host_link": link,
               "host_cpus": ("GPU-local NUMA node, %d CPUs" % len(local)) if local else "unbound"}
        del host, hSl, hSg, dbuf
        os.sched_setaffinity(0, saved)

    # ---- the other modes on the same inputs (the metric's FP64-versus-mixed comparison) ----
    compare = None
    if not args.no_compare and rank == 0:
        compare = {}
        ref = (Sl.clone(), Sg.clone())
        bounds = {"fp64": 1e-12, "fp64_fft": 1e-12, "bf16x3": 2e-5, "tf32": 2e-3, "fp64_fft_antihermitian": 1e-12,
                  "fp32_fft": 2e-6, "fp32_fft_antihermitian": 2e-6, "f16x3_fft": 2e-6, "f16x3_fft_antihermitian": 2e-6}
        variants = [("fp64", 0), ("bf16x3", 0), ("tf32", 0), ("fp64_fft", 0),
                    ("fp64_fft_antihermitian", B.SSE_FLAG_ANTIHERMITIAN), ("fp32_fft", 0),
                    ("fp32_fft_antihermitian", B.SSE_FLAG_ANTIHERMITIAN), ("f16x3_fft", 0),
                    ("f16x3_fft_antihermitian", B.SSE_FLAG_ANTIHERMITIAN)]
        for mname, mflags in variants:
            if mname == args.mode and mflags == run_flags:
                continue
            m = B.MODES[mname.replace("_antihermitian", "")]
            wsm = B.workspace(dims, m, 0, dev)
            Ml, Mg = torch.empty_like(Sl), torch.empty_like(Sg)

            def mstep():
                rc = B.sse_sigma_fwd(dims, inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater,
                                     SCALE, m, mflags, Ml, Mg, wsm, wsm.numel(), stream)
                if rc != 0:
                    raise B.SseError(rc, "sse_sigma_fwd")

            mw = 1 if mname == "fp64" else max(3, args.warmup)  # the direct FP64 kernel runs about a minute
            for _ in range(mw):
                mstep()
            torch.cuda.synchronize(dev)
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            for _ in range(args.steps):
                mstep()
            m1.record(stream)
            torch.cuda.synchronize(dev)
            mms = m0.elapsed_time(m1) / args.steps
            err = max(float((Ml - ref[0]).abs().max() / ref[0].abs().max()),
                      float((Mg - ref[1]).abs().max() / ref[1].abs().max()))
            compare[mname] = {"value": uf / (mms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": mms,
                              "warmup": mw, "speedup_of_this_run": mms / ms_per_step,
                              "max_normwise_diff_vs_this_run": err, "stated_bound_vs_oracle": bounds[mname]}
            del wsm, Ml, Mg
        del ref
        torch.cuda.empty_cache()

    # the forward's workspace and outputs are not needed past this point (room for Pi and the adjoint)
    del ws
    Sl = Sg = None
    torch.cuda.empty_cache()

    # ---- the phonon self-energy Pi of Eq. (4) on the same inputs ----
    pi_line = None
    if not args.no_pi and rank == 0:
        pd = B.sse_dims(d.NA, d.NB, d.Norb, d.NE, d.Nkz, d.Nqz, d.Nw, 0, d.NA)
        wsp = torch.empty(B.sse_pi_workspace_bytes(pd, B.SSE_MODE_FP64, 0), dtype=torch.uint8, device=dev)
        shape = (d.Nqz, d.Nw, d.NA, d.NB + 1, 3, 3)
        Pout = (torch.empty(shape, dtype=torch.complex128, device=dev),
                torch.empty(shape, dtype=torch.complex128, device=dev))

        def pstep(flags=0):
            B.pi(inp.G_less, inp.G_greater, inp.dH, inp.nbr, d.Nqz, d.Nw, scale=SCALE, out=Pout, ws=wsp,
                 stream=stream, profile=bool(flags), antihermitian=args.antihermitian)

        for _ in range(max(3, args.warmup)):
            pstep()
        torch.cuda.synchronize(dev)
        B.sse_profile_read()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            pstep(1)
        p1.record(stream)
        torch.cuda.synchronize(dev)
        pms = p0.elapsed_time(p1) / args.steps
        pk = {name: (ms, n) for name, ms, n in B.sse_profile_read()}
        ks = pk["spec_pi_kernel"][0] * 1e-3 / pk["spec_pi_kernel"][1]
        ach = spectral_pi_flops(d, args.antihermitian) / ks / 1e12
        pi_line = {"op": "Pi^<, Pi^> of Eq. 4 (sse_pi_fwd, FP64 via the convolution theorem)",
                   "ms_per_step": pms, "warmup": max(3, args.warmup),
                   "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                "frac": ach / FP64_PEAK_TFLOPS, "kernel": "spec_pi_kernel", "launch_ms": ks * 1e3,
                                "traffic": ncu_traffic("spec_pi_kernel", 2 * d.NA * freq_count(d, args.antihermitian)),
                                "kernels": {k: {"ms_per_step": v[0] / args.steps,
                                                "launches_per_step": v[1] / args.steps} for k, v in pk.items()}}}
        # the same Pi with FP32 transforms and products (mode FP32_FFT), compared with the FP64 result
        ref_p = tuple(x.clone() for x in Pout)
        del wsp
        torch.cuda.empty_cache()
        m32 = B.MODES["fp32_fft"]
        wsp = torch.empty(B.sse_pi_workspace_bytes(pd, m32, 0), dtype=torch.uint8, device=dev)

        def pstep32():
            B.pi(inp.G_less, inp.G_greater, inp.dH, inp.nbr, d.Nqz, d.Nw, scale=SCALE, out=Pout, ws=wsp,
                 stream=stream, antihermitian=args.antihermitian, mode="fp32_fft")

        for _ in range(max(3, args.warmup)):
            pstep32()
        torch.cuda.synchronize(dev)
        p0.record(stream)
        for _ in range(args.steps):
            pstep32()
        p1.record(stream)
        torch.cuda.synchronize(dev)
        pi_line["fp32_fft"] = {"ms_per_step": p0.elapsed_time(p1) / args.steps,
                               "normwise_diff_vs_fp64": max(float((x - y).abs().max() / y.abs().max())
                                                            for x, y in zip(Pout, ref_p)),
                               "stated_bound": 2e-6}
        del wsp, Pout, ref_p
        torch.cuda.empty_cache()

    # ---- the FP64 adjoint (transform-based) on the same inputs ----
    adj_line = None
    if not args.no_adjoint and rank == 0:
        W, V = make_upstream(d, seed=1000 + rank, device=dev)
        mfft = B.MODES["fp64_fft"]
        wsa = B.workspace(dims, mfft, 0, dev)
        gout = (torch.empty_like(inp.dH), torch.empty_like(inp.D_less), torch.empty_like(inp.D_greater))

        def astep(flags=0):
            rc = B.sse_sigma_bwd(dims, inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                                 mfft, flags, W, V, gout[0], gout[1], gout[2], wsa, wsa.numel(), stream)
            if rc != 0:
                raise B.SseError(rc, "sse_sigma_bwd")

        for _ in range(max(3, args.warmup)):
            astep()
        torch.cuda.synchronize(dev)
        B.sse_profile_read()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            astep(B.SSE_FLAG_PROFILE)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        ams = a0.elapsed_time(a1) / args.steps
        ak = {name: (ms, n) for name, ms, n in B.sse_profile_read()}
        ks = ak["spec_adj_kernel"][0] * 1e-3 / ak["spec_adj_kernel"][1]
        ach = spectral_adj_flops(d) / ks / 1e12
        adj_line = {"op": "adjoint of Eq. 3 (sse_sigma_bwd, FP64 via the transforms): grad dH, D^<, D^>",
                    "ms_per_step": ams, "warmup": max(3, args.warmup),
                    "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                 "frac": ach / FP64_PEAK_TFLOPS, "kernel": "spec_adj_kernel",
                                 "launch_ms": ks * 1e3,
                                 "traffic": ncu_traffic("spec_adj_kernel", d.NA * d.Nkz * fft_length(d.NE, d.Nw)),
                                 "kernels": {k: {"ms_per_step": v[0] / args.steps,
                                                 "launches_per_step": v[1] / args.steps} for k, v in ak.items()}}}
        # the same adjoint with FP32 transforms and products (mode FP32_FFT)
        ref_g = tuple(x.clone() for x in gout)
        m32 = B.MODES["fp32_fft"]
        del wsa
        torch.cuda.empty_cache()
        wsa = B.workspace(dims, m32, 0, dev)

        def astep32():
            rc = B.sse_sigma_bwd(dims, inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                                 m32, 0, W, V, gout[0], gout[1], gout[2], wsa, wsa.numel(), stream)
            if rc != 0:
                raise B.SseError(rc, "sse_sigma_bwd")

        for _ in range(max(3, args.warmup)):
            astep32()
        torch.cuda.synchronize(dev)
        a0.record(stream)
        for _ in range(args.steps):
            astep32()
        a1.record(stream)
        torch.cuda.synchronize(dev)
        adj_line["fp32_fft"] = {"ms_per_step": a0.elapsed_time(a1) / args.steps,
                                "normwise_diff_vs_fp64": dict(zip(("g_dH", "g_D_less", "g_D_greater"),
                                                                  (float((x - y).abs().max() / y.abs().max())
                                                                   for x, y in zip(gout, ref_g)))),
                                "stated_bound": 1e-5}
        del ref_g
        # gradient w.r.t. G^<, G^> (sse_sigma_bwd_g), same upstream, FP64 and FP32 transforms; a mode whose
        # workspace does not fit next to the inputs and outputs is reported as skipped
        del wsa
        torch.cuda.empty_cache()
        gG = (torch.empty_like(inp.G_less), torch.empty_like(inp.G_greater))
        adj_line["grad_G"] = {}
        sample = None
        for gname, gm in (("fp64_fft", mfft), ("fp32_fft", m32)):
            need = B.sse_sigma_bwd_g_workspace_bytes(dims, gm, 0)
            free = torch.cuda.mem_get_info(dev)[0]
            if need + (2 << 30) > free:
                adj_line["grad_G"][gname] = {"skipped": f"workspace {need / 1e9:.1f} GB > free {free / 1e9:.1f} GB"}
                continue
            wsg = torch.empty(need, dtype=torch.uint8, device=dev)

            def gstep(flags=0):
                rc = B.sse_sigma_bwd_g(dims, inp.nbr, inp.dH, inp.D_less, inp.D_greater, SCALE, gm, flags, W, V,
                                       gG[0], gG[1], wsg, wsg.numel(), stream)
                if rc != 0:
                    raise B.SseError(rc, "sse_sigma_bwd_g")

            for _ in range(max(3, args.warmup)):
                gstep()
            torch.cuda.synchronize(dev)
            B.sse_profile_read()
            a0.record(stream)
            for _ in range(args.steps):
                gstep(B.SSE_FLAG_PROFILE)
            a1.record(stream)
            torch.cuda.synchronize(dev)
            gk = {name: (ms, n) for name, ms, n in B.sse_profile_read()}
            entry = {"op": f"gradient w.r.t. G^<, G^> (sse_sigma_bwd_g, mode {gname.upper()})",
                     "ms_per_step": a0.elapsed_time(a1) / args.steps,
                     "kernels": {k: {"ms_per_step": v[0] / args.steps,
                                     "launches_per_step": v[1] / args.steps} for k, v in gk.items()}}
            # every 7th energy of every atom: a strided sample of both outputs
            cur = (gG[0][:, ::7].clone(), gG[1][:, ::7].clone())
            if sample is None:
                sample = cur
            else:
                entry["normwise_diff_vs_fp64_sampled"] = max(float((x - y).abs().max() / y.abs().max())
                                                             for x, y in zip(cur, sample))
                entry["stated_bound"] = 1e-5
            del cur
            adj_line["grad_G"][gname] = entry
            del wsg
            torch.cuda.empty_cache()
        del W, V, gout, gG, sample
        torch.cuda.empty_cache()

    out = None
    if rank == 0:
        def kernel_s(name):
            ms, n = kernels[name]
            return ms * 1e-3 / n, n

        if args.mode == "fp64":
            ks, n = kernel_s("sigma_fp64_fwd_kernel")
            achieved = fp64_kernel_flops(d) / (n / args.steps) / ks / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "sigma_fp64_fwd_kernel",
                    "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2070 MHz (DFMA probe: 1.25)"}
        elif args.mode == "fp32_fft":
            ks, n = kernel_s("spec_prod32_kernel")
            achieved = spectral_prod32_flops(d, args.antihermitian) / ks / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_PEAK_TFLOPS,
                    "traffic": ncu_traffic("spec_prod32_kernel", d.NA * freq_count(d, args.antihermitian)),
                    "kernel": "spec_prod32_kernel",
                    "peak_source": "derived: 152 SM x 128 FFMA/clk x 2 flop x 2070 MHz (FFMA probe: 73)"}
        elif args.mode == "f16x3_fft":
            peaks, src = load_peaks()
            ks, n = kernel_s("spec_prod_tc_kernel")
            key = "bf16_tflops_sustained" if ks > 1.0 else "bf16_tflops"
            achieved = tc_tensor_flops(d, args.antihermitian) / ks / 1e12
            useful = tc_useful_flops(d, args.antihermitian) / ks / 1e12
            roof = {"bound": "tensor", "achieved": achieved, "peak": peaks[key], "unit": "TFLOP/s",
                    "frac": achieved / peaks[key], "useful_achieved": useful, "useful_frac": useful / peaks[key],
                    "traffic": ncu_traffic("spec_prod_tc_kernel", d.NA * freq_count(d, args.antihermitian)),
                    "kernel": "spec_prod_tc_kernel",
                    "peak_source": f"{src} {key} (kind::f16 with fp16 operands runs at the bf16 rate)",
                    "achieved_counts": "tensor work issued, padded tiles included; useful_*: the products "
                                       "the method needs"}
        elif args.mode == "fp64_fft":
            ks, n = kernel_s("spec_prod_kernel")
            achieved = spectral_prod_flops(d, args.antihermitian) / ks / 1e12
            units = d.NA * freq_count(d, args.antihermitian)
            roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": ncu_traffic("spec_prod_kernel", units),
                    "traffic_source": "ncu capture at the adjoint workload, bytes per atom-frequency x units",
                    "kernel": "spec_prod_kernel",
                    "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2070 MHz (DFMA probe: 1.25)"}
        else:
            peaks, src = load_peaks()
            ks, n = kernel_s("sigma_mixed_kernel")
            key = "bf16_tflops_sustained" if ks > 1.0 else "bf16_tflops"
            peak = peaks[key] * (1.0 if args.mode == "bf16x3" else 1.1 / 2.25)
            achieved = mixed_tensor_flops(d, args.mode) / (n / args.steps) / ks / 1e12
            useful = mixed_useful_flops(d, args.mode) / (n / args.steps) / ks / 1e12
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "useful_achieved": useful, "useful_frac": useful / peak,
                    "achieved_counts": "tensor work issued, padded tiles included; useful_*: the products "
                                       "the method needs",
                    "traffic": None, "kernel": "sigma_mixed_kernel",
                    "peak_source": f"{src} {key}" + ("" if args.mode == "bf16x3"
                                                     else " x 1.1/2.25 (tf32/bf16 nominal)")}
        roof["launch_ms"] = ks * 1e3
        roof["kernel_share_of_step"] = kernels[roof["kernel"]][0] / total_ms
        roof["kernels"] = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                           for k, v in kernels.items()}
        out = {"metric": "SSE useful TFLOP/s (Eq. 3, paper-equivalent flops)", "value": value, "unit": "TFLOP/s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": {"fp64": "f64", "fp64_fft": "f64", "fp32_fft": "f32", "tf32": "tf32+f64",
                         "bf16x3": "bf16x3+f64", "f16x3_fft": "f32+f16x3"}[args.mode],
               "data": "synthetic (seeded; Si-FinFET-shaped)",
               "config": bench_config(args, d, world),
               "pts_per_s": pts, "roofline": roof, "clocks": clk.summary(), "e2e": e2e,
               "gpu_launches": sum(v[1] for v in kernels.values())}
        if compare:
            out["compare"] = compare
        if pi_line:
            out["pi"] = pi_line
        if adj_line:
            out["adjoint"] = adj_line
        if world == 1 and not args.no_cpu:
            Sl = Sg = None
            torch.cuda.empty_cache()
            out["cpu_baseline"] = cpu_baseline(d, args.cpu_seconds, inp)
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
