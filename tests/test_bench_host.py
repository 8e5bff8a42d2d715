"""Host-side checks of bench.py (no GPU): the flop counts and frequency counts it reports are recomputed by
brute-force enumeration, the kernel-source hashes resolve, and the reference arm (the FP64 oracle timed on the
host cores) prints one JSON line with the contract's keys."""
import argparse
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1912_10024_gb300.inputs import TINY, Dims  # noqa: E402


@pytest.mark.parametrize("d", [TINY, Dims(NA=3, NB=2, Norb=3, NE=9, Nkz=2, Nqz=2, Nw=4)])
def test_useful_flops_is_the_term_count(d):
    """Per (type, atom, slot, kz, E): 24 Norb^3 per in-range (q, w, sigma) term of Eq. (3) plus 24 Norb^3 for the
    final multiply; the terms are enumerated one by one."""
    total = 0
    for _t in range(2):
        for _a in range(d.NA):
            for _s in range(d.NB):
                for _k in range(d.Nkz):
                    for E in range(d.NE):
                        terms = sum(1 for _q in range(d.Nqz) for w in range(d.Nw) for sigma in (1, -1)
                                    if 0 <= E - sigma * (w + 1) < d.NE)
                        total += 24 * d.Norb ** 3 * (terms + 1)
    assert bench.useful_flops(d) == total


@pytest.mark.parametrize("norb", [1, 3, 4, 7, 10])
def test_tensor_core_tile_counts(norb):
    """spec_prod_tc_kernel's issued and useful tensor work, enumerated per 128-row tile of frequencies and bond: FP16
    MMAs of K = 16 over the padded K, N and all 128 rows, against the unpadded real GEMMs of the used rows."""
    d = Dims(NA=3, NB=2, Norb=norb, NE=40, Nkz=3, Nqz=2, Nw=11)
    t = bench.tc_shape(norb)
    nfreq = bench.freq_count(d, False)
    issued = useful = 0
    for f0 in range(0, nfreq, t["FT"]):
        rows = min(t["FT"], nfreq - f0) * norb
        for _s in range(d.NB):
            for _a in range(d.NA):
                issued += 3 * (2 * 128 * t["N1"] * t["K1"] + 2 * 128 * t["N2"] * t["K2"])
                useful += 3 * (2 * rows * (6 * norb) * (2 * norb) + 2 * rows * (2 * norb) * (6 * norb))
    assert bench.tc_tensor_flops(d) == issued
    assert bench.tc_useful_flops(d) == useful
    assert t["K1"] >= 2 * norb and t["N1"] >= 6 * norb and t["K2"] >= 6 * norb and t["N2"] >= 2 * norb


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_mixed_useful_work_is_within_the_issued_work(mode):
    """Useful rows x K x N per in-range tap never exceeds the padded 128 x npad x kpad, and equals it where the
    padding vanishes (Norb = 8: 16 energies fill 128 rows, 6 Norb = 48 fills N and K)."""
    for d in (Dims(NA=2, NB=2, Norb=10, NE=50, Nkz=2, Nqz=2, Nw=7), Dims(NA=2, NB=1, Norb=8, NE=32, Nkz=1, Nqz=1, Nw=3)):
        u, p = bench.mixed_useful_flops(d, mode), bench.mixed_tensor_flops(d, mode)
        assert 0 < u <= p
    d = Dims(NA=2, NB=1, Norb=8, NE=32, Nkz=1, Nqz=1, Nw=3)
    if mode == "bf16x3":
        assert bench.mixed_useful_flops(d, mode) == bench.mixed_tensor_flops(d, mode)


def test_fft_length_is_the_smallest_2a3b():
    smooth = sorted(2 ** a * 3 ** b for a in range(14) for b in range(9))
    for NE in (1, 7, 32, 61, 256, 512, 1000, 1024):
        for Nw in (1, 4, 16, 32, 64):
            want = next(x for x in smooth if x >= NE + Nw)
            assert bench.fft_length(NE, Nw) == want


@pytest.mark.parametrize("Nkz", [1, 2, 3, 4, 7, 9])
@pytest.mark.parametrize("NE,Nw", [(32, 4), (61, 5), (70, 5), (512, 32)])
def test_half_spectrum_count_is_one_per_pair(Nkz, NE, Nw):
    """With anti-Hermitian inputs one frequency of each (f, -f) pair is evaluated: the count equals the number of
    orbits of f -> -f on the (kz, E) frequency grid."""
    d = Dims(NA=1, NB=1, Norb=1, NE=NE, Nkz=Nkz, Nqz=1, Nw=Nw)
    L = bench.fft_length(NE, Nw)
    seen, orbits = set(), 0
    for kap in range(Nkz):
        for eps in range(L):
            if (kap, eps) in seen:
                continue
            orbits += 1
            seen.add((kap, eps))
            seen.add(((Nkz - kap) % Nkz, (L - eps) % L))
    assert bench.freq_count(d, True) == orbits
    assert bench.freq_count(d, False) == Nkz * L


def test_kernel_sources_resolve():
    for k in list(bench.NCU_TRAFFIC) + ["spec_prod_kernel", "fft_e_kernel", "fft_e4_kernel", "fft_e4p_kernel",
                                        "dft_kz_kernel", "spec_gradg_kernel"]:
        assert len(bench.kernel_source_sha(k)) == 16, k
    assert bench.kernel_source_sha("no_such_kernel") == ""
    assert bench.ncu_traffic("no_such_kernel", 1.0) is None


def test_reference_arm_prints_the_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--steps", "1", "--warmup", "1", "--cpu-seconds", "1"],
                       capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
                "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["value"] > 0 and out["higher_is_better"] is True
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
    assert out["config"]["workload"] == "tiny"
    # the GPU arm's config for the same arguments: same keys, same values
    args = argparse.Namespace(workload="tiny", mode=out["config"]["mode"], antihermitian=False)
    assert out["config"] == bench.bench_config(args, TINY, 1)


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun (N > 1) rank 0 alone times the oracle and prints; the other ranks exit 0 and print nothing."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_peaks_fall_back_per_figure(tmp_path):
    """The roofline denominators: the measured file's figures where present, the earlier GB300 measurement where a
    figure (or the whole file) is missing, and the source says which."""
    full = tmp_path / "full.json"
    full.write_text(json.dumps({"hbm_gbs": 6793.4, "bf16_tflops": 1897.2, "bf16_tflops_sustained": 1714.1,
                                "gpu_name": "x"}))
    peaks, src = bench.load_peaks(str(full))
    assert src == "measured" and peaks["hbm_gbs"] == 6793.4 and peaks["bf16_tflops_sustained"] == 1714.1
    part = tmp_path / "part.json"
    part.write_text(json.dumps({"hbm_gbs": 7000.0, "bf16_tflops": "n/a"}))
    peaks, src = bench.load_peaks(str(part))
    assert src == "measured, partly fallback" and peaks["hbm_gbs"] == 7000.0
    assert peaks["bf16_tflops"] == bench.FALLBACK_PEAKS["bf16_tflops"]
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert bench.load_peaks(str(bad)) == (bench.FALLBACK_PEAKS, "fallback")
    assert bench.load_peaks(str(tmp_path / "missing.json"))[1] == "fallback"


def test_clock_samples_come_from_the_gpu_torch_uses(monkeypatch):
    """nvidia-smi numbers every GPU of the machine; torch numbers the visible ones: the sampler maps one to the
    other through CUDA_VISIBLE_DEVICES (indices or UUIDs)."""
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,2")
    assert bench.smi_gpu_id(0) == "5" and bench.smi_gpu_id(1) == "2"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-1234abcd")
    assert bench.smi_gpu_id(0) == "GPU-1234abcd"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.smi_gpu_id(3) == "3"
    clk = bench.ClockSampler("7")
    clk.lines = ["1965, 2070, 900.1, Not Active, Not Active, Not Active, Active", "garbage"]
    out = clk.summary()
    assert out == {"sm_mhz": 1965.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 1, "gpu": "7"}
