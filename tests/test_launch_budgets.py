"""Launch budgets of the persistent passes, on the CPU.

The persistent row and column passes size their blocks and shared memory from
constexpr formulas shared by host and device (kernels_persist.cuh): tile
columns, threads per block, staging and exchange areas, and whether the
column plan's twiddle table is copied into shared memory.  A launch whose
shared memory exceeds a block's limit falls back to the plain pass, so a
formula that grows past the limit would silently lose the persistent pass.
A small host program compiled against the header evaluates every size from 8
to 4096 points in both precisions and prints the plan; the test checks that
every persistent column pass fits (at most 512 threads, shared memory within
the limit), which column plans keep their twiddles in shared memory, and
which row passes fit.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2010_15069_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

CHECK = r"""
#include <cstdio>
#include <utility>
#include "kernels_persist.cuh"
using namespace spgpe;

template <class T, int LOGN> void col_plan() {
  constexpr int es = sizeof(cx<T>), N = 1 << LOGN, LOGE = col_loge_for(LOGN, es);
  constexpr int C = colp_cols_c<T>(LOGN, LOGE);
  const size_t tw = colp_tw_bytes<T>(LOGN, C, Plan<LOGN, LOGE>::entries());
  const size_t smem = kPipe * colp_buf_bytes(N, C, es) + (size_t)N * es + tw + kPipe * sizeof(uint64_t);
  printf("col %d %d %d %zu %zu\n", es, N, C * (N >> LOGE), tw, smem);
}
template <class T, int LOGN> void row_plan() {
  constexpr int es = sizeof(cx<T>), N = 1 << LOGN, LOGE = row_loge_for(LOGN, es), E = 1 << LOGE;
  printf("row %d %d %d %zu\n", es, N, rowu_block(N, E), rowu_smem(N, E, es, Plan<LOGN, LOGE>::entries()));
}
template <class T, int... L> void all(std::integer_sequence<int, L...>) {
  ((col_plan<T, L + 3>(), row_plan<T, L + 3>()), ...);
}
int main() {
  all<float>(std::make_integer_sequence<int, 10>{});
  all<double>(std::make_integer_sequence<int, 10>{});
  printf("colw %zu\nlimit %zu\n", colw_smem(), kMaxSmemPerBlock);
  return 0;
}
"""


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("budgets")
    src, exe = d / "check.cu", d / "check"
    src.write_text(CHECK)
    r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC, "-I", INCLUDE,
                        str(src), "-o", str(exe)], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout[-3000:]
    cols, rows, lim, colw = {}, {}, None, None
    for ln in r.stdout.splitlines():
        f = ln.split()
        if f[0] == "col":
            cols[(int(f[1]), int(f[2]))] = dict(threads=int(f[3]), tw=int(f[4]), smem=int(f[5]))
        elif f[0] == "row":
            rows[(int(f[1]), int(f[2]))] = dict(threads=int(f[3]), smem=int(f[4]))
        elif f[0] == "colw":
            colw = int(f[1])
        elif f[0] == "limit":
            lim = int(f[1])
    return cols, rows, colw, lim


def test_every_persistent_column_pass_fits_a_block(plans):
    cols, _, colw, lim = plans
    assert len(cols) == 20
    for (es, n), p in cols.items():
        assert p["threads"] <= 512, (es, n, p)
        assert p["smem"] <= lim, (es, n, p)
    assert colw <= lim


def test_column_plans_keep_their_twiddles_in_shared_memory_where_they_fit(plans):
    cols, _, _, lim = plans
    for es in (8, 16):
        # columns of 512 to 2048 rows keep the table (8, 16 and 32.5 KB) beside their tiles
        for n in (512, 1024, 2048):
            assert cols[(es, n)]["tw"] > 0, (es, n)
        # the 4096-row table (65 KB) would not fit beside the tiles and the K table
        assert cols[(es, 4096)]["tw"] == 0
        assert cols[(es, 4096)]["smem"] + 4080 * 16 > lim
    assert cols[(8, 2048)]["tw"] == 2032 * 16


def test_persistent_row_passes_fit_except_the_double_precision_4096_rows(plans):
    _, rows, _, lim = plans
    assert len(rows) == 20
    for (es, n), p in rows.items():
        if (es, n) == (16, 4096):
            assert p["smem"] > lim  # the launcher runs the plain row pass there
        else:
            assert p["smem"] <= lim, (es, n, p)
            assert p["threads"] <= 512, (es, n, p)
