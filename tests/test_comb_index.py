"""The reconfiguration's index arithmetic, checked on the CPU from the kernel
source itself: comb_blocks, comb_slots and comb_order_pos are cut out of
lrdmc_kernels.cu, compiled into a host harness with g++, and run for every
population size up to 5000 and for sampled sizes up to LRDMC_MAX_WALKERS.
For each size the grid stays within kMaxCombBlocks blocks and the shared
memory within kCombSmemMax, and the order positions that the blocks write
are a bijection of the slots onto 0..W-1 (no slot lost, none written
twice)."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1909_01589_gb300", "csrc")


def _function(src, signature):
    """The text of the function whose definition starts with `signature`,
    through its matching closing brace."""
    i = src.index(signature)
    j = src.index("{", i)
    depth = 0
    for k in range(j, len(src)):
        depth += src[k] == "{"
        depth -= src[k] == "}"
        if depth == 0:
            return src[i:k + 1]
    raise ValueError(signature)


def _constant(text, name):
    return int(eval(re.search(rf"constexpr int {name} = ([^;]+);", text).group(1)))


HARNESS = r"""
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>
#define __device__
#define __forceinline__ inline
constexpr int kCombThreads = %(threads)d;
constexpr int kMaxCombBlocks = %(blocks)d;
constexpr int kCombSmemMax = %(smem)d;
constexpr int kReconfigSmemW = %(smem_w)d;
%(functions)s
static int check(int W)
{
  const int G = comb_blocks(W);
  if (G < 1 || G > kMaxCombBlocks) return 1;
  const int R = comb_slots(W, G);
  if (R != (W + G - 1) / G) return 2;
  const long smem = (W <= kReconfigSmemW ? 8L * W : 0L) + 4L * R;
  if (smem > kCombSmemMax) return 3;
  const int Gn = (W + R - 1) / R, Rl = W - (Gn - 1) * R;
  std::vector<char> seen(W, 0);
  for (int g = 0; g < G; ++g) {
    const int b0 = std::min(W, g * R), b1 = std::min(W, b0 + R);
    for (int r = 0; r < b1 - b0; ++r) {
      const int pos = comb_order_pos(g, r, Gn, Rl);
      if (pos < 0 || pos >= W || seen[pos]) return 4;
      seen[pos] = 1;
    }
  }
  for (int i = 0; i < W; ++i)
    if (!seen[i]) return 5;
  return 0;
}
int main(int argc, char** argv)
{
  for (int a = 1; a < argc; ++a) {
    const int W = atoi(argv[a]);
    const int rc = check(W);
    if (rc) { printf("W=%%d failed (%%d)\n", W, rc); return 1; }
  }
  printf("ok %%d sizes\n", argc - 1);
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("needs g++")
    src = open(os.path.join(CSRC, "lrdmc_kernels.cu")).read()
    internal = open(os.path.join(CSRC, "lrdmc_internal.h")).read()
    functions = "\n".join([
        _function(src, "__device__ __forceinline__ int comb_slots(int W, int G)"),
        _function(src, "__device__ __forceinline__ int comb_order_pos(int g, int r, int Gn, int Rl)"),
        _function(src, "int comb_blocks(int W)\n"),
    ])
    code = HARNESS % dict(threads=_constant(internal, "kCombThreads"), blocks=_constant(internal, "kMaxCombBlocks"),
                          smem=_constant(internal, "kCombSmemMax"), smem_w=_constant(internal, "kReconfigSmemW"),
                          functions=functions)
    d = tmp_path_factory.mktemp("comb")
    cpp, exe = str(d / "comb.cpp"), str(d / "comb")
    open(cpp, "w").write(code)
    r = subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Werror", cpp, "-o", exe], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _run(exe, sizes):
    r = subprocess.run([exe, *map(str, sizes)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr


def test_every_small_population(harness):
    _run(harness, range(1, 5001))


def test_sampled_large_populations(harness):
    header = open(os.path.join(ROOT, "include", "lrdmc.h")).read()
    w_max = int(re.search(r"#define LRDMC_MAX_WALKERS (\d+)", header).group(1))
    rng = np.random.default_rng(5)
    sizes = set(rng.integers(5001, w_max + 1, 300).tolist())
    for p in range(12, 23):  # powers of two and their neighbours, up to 2^22
        sizes |= {2 ** p - 1, 2 ** p, 2 ** p + 1}
    sizes |= {16383, 16384, 16385, 32768, 32767, w_max - 1, w_max}
    _run(harness, sorted(s for s in sizes if 1 <= s <= w_max))
