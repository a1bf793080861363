"""Host-side check of the chunked sweep schedule (CPU only, no GPU call).

The tiled kernels map CTA u of a chunked launch to a tile column and a range of planes
with chunk_unit(); the last chunk of every column may be cut into split_last() pieces.
Every (column, plane) must be updated by exactly one CTA and every CTA must get at least
one plane, for any depth, chunk length and requested cut.  The functions are host-callable,
so a small host program built with nvcc walks all launches of a grid of cases.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2407_19868_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "pm_sweep_tiled.cuh"
using namespace pmgb;
int main() {
    long long cases = 0;
    for (int nz = 1; nz <= 70; ++nz)
        for (int zc = 1; zc <= nz + 3; ++zc)
            for (int split = 0; split <= 9; ++split)
                for (long long C : {1LL, 3LL, 7LL}) {
                    const int z = zc < nz ? zc : nz;  // the launch clamps the chunk to nz
                    const int K = (nz + z - 1) / z, S = split_last(nz, z, split);
                    if (S < 1) { printf("bad split %d %d %d\n", nz, zc, split); return 1; }
                    const long long grid = C * (K - 1 + S);
                    std::vector<int> hit((size_t)(C * nz), 0);
                    for (long long u = 0; u < grid; ++u) {
                        long long col; int m0, m1;
                        chunk_unit(u, C, nz, z, S, col, m0, m1);
                        if (col < 0 || col >= C || m0 < 0 || m1 > nz || m0 >= m1) {
                            printf("bad unit nz=%d zc=%d split=%d C=%lld u=%lld: col %lld [%d,%d)\n",
                                   nz, zc, split, C, u, col, m0, m1);
                            return 1;
                        }
                        for (int m = m0; m < m1; ++m) hit[(size_t)(col * nz + m)]++;
                    }
                    for (size_t i = 0; i < hit.size(); ++i)
                        if (hit[i] != 1) {
                            printf("plane covered %d times nz=%d zc=%d split=%d C=%lld\n", hit[i], nz, zc, split, C);
                            return 1;
                        }
                    // the requested cut is honoured whenever the last chunk is long enough
                    const int len = nz - (K - 1) * z;
                    if (split >= 1 && split <= len && (split - 1) * ((len + split - 1) / split) < len && S != split) {
                        printf("cut not honoured nz=%d zc=%d split=%d -> %d\n", nz, zc, split, S);
                        return 1;
                    }
                    ++cases;
                }
    printf("ok %lld\n", cases);
    return 0;
}
"""


def test_chunked_units_cover_every_plane_once(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "schedule.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "schedule"
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert out.stdout.startswith("ok")
