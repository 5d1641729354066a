"""Shared-memory layouts of the step kernels (csrc/rlbm_args.h), checked on the
host: a small C++ program includes the header, prints the layouts of the
tilings the kernels run, and the invariants are asserted here.

* Tile-staged kernel (PairTmaSmem): the TMA stage, the pair table and the
  mbarrier do not overlap and keep their alignment; where the angular sums and
  the per-site results alias the dead stage they fit inside it, else they
  follow the table; the benchmark's tiling (N = 2, K = 48, 16-bit, nine warps)
  takes the aliased layout and fits four CTAs per SM (228 KB, 1 KB reserved
  per CTA).
* The double-float per-site part: tile_smem_bytes_dd counts the angular sums,
  the per-site rows and the frame and partial sums of the direction split;
  pair_smem_total adds the split's rows exactly when pair_split holds
  (a thread for every (sample direction, site) item).
"""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2011_06856_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "rlbm_args.h"
using namespace rlbmk;
int main() {
    std::printf("[");
    bool first = true;
    const int cases[][5] = {  // N, K, storage bytes, two_d, G
        {2, 48, 2, 1, 9}, {2, 48, 4, 1, 9}, {3, 64, 4, 1, 8}, {3, 64, 2, 0, 8},
        {2, 16, 2, 0, 3}, {2, 16, 4, 1, 3}, {3, 12, 4, 1, 4}, {3, 32, 2, 1, 4}};
    for (const auto &c : cases) {
        const int N = c[0], K = c[1], es = c[2], G = c[4];
        const bool two_d = c[3] != 0;
        const int npop = (N + 1) * K;
        const PairTmaSmem L(N, G, npop, es, two_d);
        const size_t BW = size_t(kPairSites) + 2 * size_t(16 / es);
        std::printf("%s{\"N\":%d,\"K\":%d,\"es\":%d,\"two_d\":%d,\"G\":%d,\"stage_bytes\":%zu,"
                    "\"tab\":%zu,\"red\":%zu,\"sres\":%zu,\"bar\":%zu,\"total\":%zu,\"alias\":%d,"
                    "\"red_bytes\":%zu,\"sres_bytes\":%zu,\"npop\":%d,"
                    "\"dd\":%zu,\"split\":%d,\"split_rows\":%d,\"pair_bytes\":%zu,\"pair_total\":%zu}",
                    first ? "" : ",", N, K, es, two_d ? 1 : 0, G,
                    size_t(two_d ? 2 : 1) * size_t(npop) * BW * size_t(es), L.tab, L.red, L.sres, L.bar,
                    L.total, L.alias ? 1 : 0, size_t(5) * G * kPairSites * 4,
                    size_t(pair_site_rows(N)) * kPairSites * 4, npop, tile_smem_bytes_dd(N, G),
                    pair_split(N, G) ? 1 : 0, split_rows(N), pair_smem_bytes(N, G, false, es, two_d),
                    pair_smem_total(N, G, false, es, two_d));
        first = false;
    }
    std::printf("]\n");
    return 0;
}
"""


def cuda_include():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda.h")):
            return os.path.join(cand, "include")
    return None


@pytest.fixture(scope="module")
def layouts(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = cuda_include()
    if not cxx or not inc:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    d = tmp_path_factory.mktemp("layout")
    src, exe = d / "layout.cpp", d / "layout"
    src.write_text(PROGRAM)
    res = subprocess.run([cxx, "-std=c++17", "-O1", "-I", inc, "-I", CSRC, str(src), "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return json.loads(out)


def test_tile_staged_layout_regions_do_not_overlap(layouts):
    for c in layouts:
        assert c["tab"] % 128 == 0 and c["tab"] >= c["stage_bytes"], c
        tab_end = c["tab"] + c["npop"] * 3 * 16
        assert c["bar"] % 16 == 0 and c["bar"] >= tab_end, c
        if c["alias"]:
            # the sums and the per-site results sit inside the (dead) stage
            assert c["red"] == 0 and c["sres"] == c["red_bytes"], c
            assert c["red_bytes"] + c["sres_bytes"] <= c["stage_bytes"], c
        else:
            assert c["red"] >= tab_end and c["sres"] == c["red"] + c["red_bytes"], c
            assert c["bar"] >= c["sres"] + c["sres_bytes"], c
        assert c["total"] == c["bar"] + 16 + 1024, c  # + the 1 KB alignment slack of the base


def test_benchmark_tiling_fits_four_ctas_per_sm(layouts):
    c = next(c for c in layouts if (c["N"], c["K"], c["es"], c["two_d"], c["G"]) == (2, 48, 2, 1, 9))
    assert c["alias"]
    assert 4 * (c["total"] + 1024) <= 228 * 1024, c["total"]
    # without the aliasing the same tiling needs the sums and results on top: three CTAs
    assert 4 * (c["total"] + c["red_bytes"] + c["sres_bytes"] + 1024) > 228 * 1024


def test_double_float_split_layouts(layouts):
    for c in layouts:
        N, G = c["N"], c["G"]
        W = (N + 1) ** 2
        assert c["split_rows"] == 6 + 2 * (N + 1) + (N + 1) * 2 * W
        # per-tile kernel: sums [5][G][32], rows [2 W + 3][32], frame + partial sums, FP32
        assert c["dd"] == 4 * 32 * (5 * G + 2 * W + 3 + c["split_rows"])
        # pair kernels: the split's rows are added exactly when every item has a thread
        assert c["split"] == (G * 32 >= (N + 1) * 64)
        extra = c["pair_total"] - c["pair_bytes"]
        if c["es"] == 4 and c["split"]:
            assert extra == c["split_rows"] * 64 * 4, c
        else:
            assert extra == 0, c
