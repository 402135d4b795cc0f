"""Index arithmetic of the kernels, checked on the CPU from the kernel source as it stands.

Symmetric storage.
``sym_tile_ij`` maps a packed tile number t to its block pair (I, J), I <= J, in the
row-by-row packing of an nb x nb upper triangle; the lane loop uses it for every tile it
reads.  The test takes the function's text from the kernel source as it stands, compiles it
with g++ (the CUDA qualifiers defined away), and checks every t of every nb the symmetric
storage accepts (nb (nb + 1) / 2 < 2^15, so nb <= 255) against the enumeration of the
packing.  The device may contract b2 * b2 - 8 t into one fused multiply-add, so a second
build spells that contraction out; the function's correction loops must make both exact.

Tensor-core layout.  ``qbf_index`` places the BF16 matrix in 128 x 64 tiles; it must be a
bijection onto [0, ld^2) in which tile (M tile, k-block) is one contiguous run of 8192
elements at position M tile * (ld / 64) + k-block, so that one TMA box of the
(ld^2 / 64) x 64 view is one contiguous 16 KB copy.  The split-K kernel's shared memory
(``tc_smem_bytes``, ``tc_pick_stages`` and the epilogue-slot constants, compiled from the
source) must hold its TMA ring and, after the main loop, the accumulators and the slots.
"""
import pathlib
import re
import subprocess

import numpy as np
import pytest

SRC = pathlib.Path(__file__).resolve().parent.parent / "paper_2408_04875_gb300" / "csrc" / "gemv_rows.cuh"

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <algorithm>
using std::max;
using std::min;
#define __device__
#define __forceinline__ inline
%s
int main()
{
    long bad = 0, checked = 0;
    for (int nb = 1; nb <= 255; ++nb) {
        int t = 0;
        for (int i = 0; i < nb; ++i)
            for (int j = i; j < nb; ++j, ++t) {
                int I = -1, J = -1;
                sym_tile_ij(t, nb, I, J);
                ++checked;
                if (I != i || J != j) {
                    if (bad < 5) std::printf("nb=%%d t=%%d -> (%%d,%%d), want (%%d,%%d)\n", nb, t, I, J, i, j);
                    ++bad;
                }
            }
    }
    std::printf("checked %%ld bad %%ld\n", checked, bad);
    return bad != 0;
}
"""


def _function_text() -> str:
    text = SRC.read_text()
    m = re.search(r"__device__ __forceinline__ void sym_tile_ij\(.*?\n}\n", text, re.S)
    assert m, "sym_tile_ij not found in the kernel source"
    return m.group(0)


@pytest.mark.parametrize("fused", [False, True], ids=["plain", "fma"])
def test_sym_tile_ij_matches_the_packing(tmp_path, fused):
    fn = _function_text()
    if fused:
        expr = "b2 * b2 - 8.f * (float)t"
        assert fn.count(expr) == 1
        fn = fn.replace(expr, "std::fma(b2, b2, -8.f * (float)t)")
    src = tmp_path / "tile_ij.cpp"
    src.write_text(HARNESS % fn)
    exe = tmp_path / "tile_ij"
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-o", str(exe), str(src)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout
    assert "checked 2796160 bad 0" in r.stdout, r.stdout


def test_engine_limits_symmetric_storage_to_the_checked_range():
    """The engine turns symmetric storage off once nb (nb + 1) / 2 reaches 2^15 (the ring
    entry's block field), so nb = 1 .. 255 above covers every instance that uses it."""
    engine = (SRC.parent / "engine.cu").read_text()
    assert "if (nb * (nb + 1) / 2 >= 0x8000) sym_ = false;" in engine
    assert 255 * 256 // 2 < 0x8000 <= 256 * 257 // 2


def _qbf_index_py():
    """qbf_index's body, taken from the source and evaluated with numpy integer arrays."""
    text = (SRC.parent / "ubqp_engine.cuh").read_text()
    m = re.search(r"size_t qbf_index\(size_t i, size_t j, size_t ld\)\s*\{\s*return (.*?);\s*\}", text, re.S)
    assert m, "qbf_index not found"
    expr = m.group(1)
    return lambda i, j, ld: eval(expr, {}, {"i": i, "j": j, "ld": ld})


@pytest.mark.parametrize("ld", [128, 256, 640, 2560])
def test_qbf_index_is_a_tiled_bijection(ld):
    f = _qbf_index_py()
    i, j = np.meshgrid(np.arange(ld, dtype=np.uint64), np.arange(ld, dtype=np.uint64), indexing="ij")
    idx = f(i, j, np.uint64(ld))
    assert np.array_equal(np.sort(idx.ravel()), np.arange(ld * ld, dtype=np.uint64))
    for M in range(ld // 128):
        for K in range(ld // 64):
            tile = idx[M * 128:(M + 1) * 128, K * 64:(K + 1) * 64]
            base = (M * (ld // 64) + K) * 8192
            # rows of 64 entries, one after the other, from the tile's base
            assert np.array_equal(tile, base + np.arange(8192, dtype=np.uint64).reshape(128, 64))


TC_HARNESS = r"""
#include <algorithm>
#include <cstddef>
#include <cstdio>
%s
int main()
{
    for (int two = 0; two < 2; ++two)
        for (int bn = 16; bn <= 128; bn += 16) {
            const int stages = tc_pick_stages(bn, two != 0);
            const size_t total = tc_smem_bytes(bn, two != 0, stages);
            const size_t stage = 128 * 128 + (size_t)bn * 128 * (two ? 2 : 1);
            std::printf("%%d %%d %%d %%zu %%zu %%zu %%d %%d\n", two, bn, stages, total, stage, kEpiSlotBytes,
                        kEpiSlot, kEpiDepth);
        }
    return 0;
}
"""


def _tc_source_parts() -> str:
    tc = (SRC.parent / "tc_gemm.cu").read_text()
    hdr = (SRC.parent / "ubqp_tc.cuh").read_text()
    parts = []
    for text, pat in ((hdr, r"constexpr int kTcMaxStages = .*?;"),
                      (tc, r"constexpr int kTcThreads = .*?;"),
                      (tc, r"constexpr int kEpiDepth = .*?;"),
                      (tc, r"constexpr int kEpiSlot = .*?;"),
                      (tc, r"constexpr size_t kEpiSlotBytes = .*?;"),
                      (tc, r"size_t tc_smem_bytes\(int bn, bool two, int stages\)\n\{.*?\n\}\n"),
                      (tc, r"int tc_pick_stages\(int bn, bool two\)\n\{.*?\n\}\n")):
        m = re.search(pat, text, re.S)
        assert m, pat
        parts.append(m.group(0))
    return "\n".join(parts)


def test_tc_shared_memory_holds_the_ring_and_the_epilogue_slots(tmp_path):
    """The split-K kernel's dynamic shared memory (tc_smem_bytes for the stage count
    tc_pick_stages gives) must hold, after the 1 KB alignment slack, the TMA ring of `stages`
    k-blocks and, once the ring is free, the accumulators (128 x bn FP32) followed by every
    warp's epilogue slots; the slots' offsets are 16-byte aligned (cp.async), and the total
    leaves room for the kernel's static shared memory (9 KB) under the 227 KB per CTA.  Every
    tile width the engine forms (multiples of 16 up to 128), one and two BF16 terms."""
    src = tmp_path / "tc_smem.cpp"
    src.write_text(TC_HARNESS % _tc_source_parts())
    exe = tmp_path / "tc_smem"
    subprocess.run(["g++", "-std=c++17", "-O1", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True, timeout=60).stdout.split("\n")
    rows = [list(map(int, ln.split())) for ln in out if ln.strip()]
    assert len(rows) == 16
    for two, bn, stages, total, stage, slot_bytes, slot, depth in rows:
        ring = total - 1024
        assert 2 <= stages <= 4
        assert ring >= stages * stage, (two, bn)
        assert ring >= 128 * bn * 4 + slot_bytes, (two, bn)
        assert (128 * bn * 4) % 16 == 0 and (slot * 4) % 16 == 0 and (depth * slot * 4) % 16 == 0
        assert slot >= 7 * 128                      # seven operand vectors of 128 rows
        assert total + 9 * 1024 <= 227 * 1024, (two, bn, total)
