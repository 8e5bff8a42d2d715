"""The compile-time cosines and sines of the register-codelet transforms and of the kz DFT (cx_cis in
csrc/sse_fft32.cuh: an exact reduction of 2 pi k / n to a quadrant, then Taylor series) against the C library's
long-double cos and sin, on the host: every k of every n up to 72 (the codelet and kz grid sizes), negative k and
k >= n included, once evaluated at run time and once forced to compile time. No GPU is used."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include "sse_spectral.cuh"

int main() {
    long double worst = 0.0L;
    for (long n = 1; n <= 72; ++n)
        for (long k = -n; k < 2 * n; ++k) {
            const sse::CxCis w = sse::cx_cis(k, n);
            const long double a = 2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)n;
            const long double ec = fabsl((long double)w.c - cosl(a)), es = fabsl((long double)w.s - sinl(a));
            if (ec > worst) worst = ec;
            if (es > worst) worst = es;
        }
    constexpr sse::CxCis w17 = sse::cx_cis(1, 7);   // evaluated by the compiler
    constexpr sse::CxCis w524 = sse::cx_cis(5, 24);
    const long double a17 = 2.0L * 3.14159265358979323846264338327950288L / 7.0L;
    const long double a524 = 2.0L * 3.14159265358979323846264338327950288L * 5.0L / 24.0L;
    long double cw = fabsl((long double)w17.c - cosl(a17));
    if (fabsl((long double)w17.s - sinl(a17)) > cw) cw = fabsl((long double)w17.s - sinl(a17));
    if (fabsl((long double)w524.c - cosl(a524)) > cw) cw = fabsl((long double)w524.c - cosl(a524));
    if (fabsl((long double)w524.s - sinl(a524)) > cw) cw = fabsl((long double)w524.s - sinl(a524));
    printf("%.6Le %.6Le\n", worst, cw);
    return 0;
}
"""


def test_compile_time_twiddles_match_the_c_library(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "twiddles.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "twiddles"
    cmd = [nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_1912_10024_gb300", "csrc"), str(src), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    worst, at_compile_time = (float(x) for x in out.stdout.split())
    assert worst < 1e-15, worst  # a few roundings of doubles below 1 (measured 3.6e-16), nothing more
    assert at_compile_time < 1e-15, at_compile_time
