"""The boundary from plain C: include/sse.h compiles as strict C99 and as C++17, and a C program that links libsse
(no PyTorch, no Python) sees every declared entry point and gets workspace sizes and status strings. Nothing here
touches a GPU: the calls made are the host-only queries."""
import os
import shutil
import subprocess

import pytest

from paper_1912_10024_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <stdio.h>
#include "sse.h"

int main(void) {
    /* every entry point, taken by address: a missing or mistyped export fails to link */
    const void* entry[] = {
        (const void*)&sse_workspace_bytes, (const void*)&sse_sigma_fwd, (const void*)&sse_sigma_fwd_host_bytes,
        (const void*)&sse_sigma_fwd_host, (const void*)&sse_sigma_bwd, (const void*)&sse_sigma_bwd_g_workspace_bytes,
        (const void*)&sse_sigma_bwd_g, (const void*)&sse_pi_workspace_bytes, (const void*)&sse_pi_fwd,
        (const void*)&sse_dcomb_fwd, (const void*)&sse_dcomb_bwd, (const void*)&sse_sigma_bwd_static,
        (const void*)&sse_profile_read, (const void*)&sse_strerror};
    sse_dims d = {16, 4, 4, 32, 3, 3, 4, 0, 16};
    sse_dims bad = d;
    unsigned i;
    bad.Nw = bad.NE; /* Nw < NE is required */
    for (i = 0; i < sizeof entry / sizeof entry[0]; ++i)
        if (!entry[i]) return 1;
    printf("%zu %zu %zu %zu\n", sse_workspace_bytes(&d, SSE_MODE_FP64_FFT, SSE_FLAG_SYMMETRIZE),
           sse_pi_workspace_bytes(&d, SSE_MODE_FP32_FFT, 0), sse_workspace_bytes(&bad, SSE_MODE_FP64, 0),
           (size_t)SSE_STATIC_SCRATCH_BYTES);
    printf("%s|%s\n", sse_strerror(SSE_ERR_UNSUPPORTED), sse_strerror(42));
    printf("%d\n", sse_profile_read(NULL, 0));
    return 0;
}
"""


def _compiler(name):
    c = shutil.which(name)
    if not c:
        pytest.skip(f"{name} not available")
    return c


@pytest.mark.parametrize("std", ["-std=c99", "-std=c11"])
def test_header_is_strict_c(tmp_path, std):
    src = tmp_path / "h.c"
    src.write_text('#include "sse.h"\nint sse_header_probe(void) { return (int)sizeof(sse_dims); }\n')
    subprocess.run([_compiler("gcc"), std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", INCLUDE, "-c",
                    str(src), "-o", str(tmp_path / "h.o")], check=True, capture_output=True, text=True)


def test_header_is_cxx(tmp_path):
    src = tmp_path / "h.cpp"
    src.write_text('#include "sse.h"\nint sse_header_probe() { return (int)sizeof(sse_dims); }\n')
    subprocess.run([_compiler("g++"), "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", INCLUDE, "-c",
                    str(src), "-o", str(tmp_path / "h.o")], check=True, capture_output=True, text=True)


def test_plain_c_program_links_and_queries(tmp_path):
    lib = B.library_path()
    B.load()  # builds the library if needed
    src = tmp_path / "prog.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "prog"
    libdir = os.path.dirname(lib)
    r = subprocess.run([_compiler("gcc"), "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", INCLUDE, str(src),
                        "-o", str(exe), "-L", libdir, "-lsse", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60, env=dict(os.environ,
                                                                                          CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr
    sizes, strings, prof = out.stdout.strip().splitlines()
    ws, wpi, wbad, static = (int(x) for x in sizes.split())
    d = B.sse_dims(16, 4, 4, 32, 3, 3, 4, 0, 16)
    assert ws == B.sse_workspace_bytes(d, B.SSE_MODE_FP64_FFT, B.SSE_FLAG_SYMMETRIZE) > 0
    assert wpi == B.sse_pi_workspace_bytes(d, B.SSE_MODE_FP32_FFT, 0) > 0
    assert wbad == 0 and static == B.SSE_STATIC_SCRATCH_BYTES
    assert strings == f"{B.sse_strerror(2)}|unknown status"
    assert prof == "0"
