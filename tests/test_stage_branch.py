"""The stage body's switch node (no GPU needed): the branch index that the head
kernel sets (stage_branch in internal.h) and the branch bodies that the host
captures must correspond one to one.  A host program compiled from the same
header checks, for every handle configuration (with or without complement and
scoring kernels), that the combinations with work fill [0, stage_branches)
exactly once and that a stage without work selects no branch."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2109_04626_gb300", "csrc")

PROGRAM = r"""
#include "internal.h"
#include <cstdio>
#include <vector>
int main()
{
    using namespace fpc;
    int bad = 0;
    for (int hc = 0; hc < 2; ++hc)
        for (int hs = 0; hs < 2; ++hs) {
            const int nb = stage_branches(hc, hs);
            std::vector<int> hit(nb, 0);
            for (int sco = 0; sco <= hs; ++sco)
                for (int cmp = 0; cmp <= hc; ++cmp)
                    for (int kind = 0; kind <= STAGE_KIND_NONE; ++kind) {
                        if (kind == STAGE_KIND_NONE && (!cmp || sco)) continue;
                        const int i = stage_branch(kind, cmp, sco, hc, hs);
                        if (i < 0 || i >= nb) ++bad;
                        else ++hit[i];
                    }
            for (int i = 0; i < nb; ++i) bad += hit[i] != 1;
            bad += stage_branch(STAGE_KIND_NONE, 0, 0, hc, hs) != nb;
            bad += stage_branch(STAGE_KIND_NONE, 0, 1, hc, hs) != nb;
            // flags a handle cannot use fold onto the combination without them
            bad += stage_branch(2, 1, 1, hc, hs) != stage_branch(2, hc, hs, hc, hs);
            bad += stage_branch(STAGE_KIND_DIRECT, 1, 1, hc, hs) != stage_branch(STAGE_KIND_DIRECT, hc, hs, hc, hs);
            printf("%d %d %d\n", hc, hs, nb);
        }
    printf("bad %d\n", bad);
    return bad != 0;
}
"""


def test_stage_branch_map_is_one_to_one(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "branch.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "branch"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout
    lines = out.stdout.split("\n")
    # LANE_RANGES small-stage ranges + warp-per-test (+ none with the complement):
    # 7, 7 + 7 with scoring, 7 + 8 with the complement, 7 + 8 + 7 + 7 with both
    counts = {tuple(map(int, ln.split()[:2])): int(ln.split()[2]) for ln in lines if ln and ln[0].isdigit()}
    assert counts == {(0, 0): 7, (0, 1): 14, (1, 0): 15, (1, 1): 29}
    assert "bad 0" in out.stdout
