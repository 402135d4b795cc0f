"""The compensated FP32 summation of the kernels, checked on the CPU from the kernel source.

``two_sum``, ``csum_add`` and ``csum_merge`` carry every compensated sum of the FP32 path
(the row dots, the symmetric tiles' column merge and block sums, the BB dot products).
Their text is taken from the kernel header as it stands and compiled with g++, with the
round-to-nearest intrinsics mapped to plain IEEE single-precision adds and subtracts (the
intrinsics exist to stop the device compiler from contracting into FMAs, so the host build
uses -ffp-contract=off).  Checked against exact sums in long double:
- TwoSum is error-free: s + e equals a + b exactly, over random pairs of wide exponent range;
- the compensated accumulation of long sequences with cancellation stays within
  2 eps |S| + 4 n eps^2 sum |v| of the exact sum S (eps = 2^-24), a bound that a plain
  FP32 sum of the same data breaks in most trials;
- merging two partial accumulators gives the same bound as one accumulation.
"""
import pathlib
import re
import subprocess

import pytest

HDR = pathlib.Path(__file__).resolve().parent.parent / "paper_2408_04875_gb300" / "csrc" / "ubqp_internal.cuh"

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>
struct float2 { float x, y; };
static inline float2 make_float2(float x, float y) { float2 r; r.x = x; r.y = y; return r; }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
#define __device__
#define __forceinline__ inline
%s
int main()
{
    std::mt19937_64 rng(12345);
    std::uniform_real_distribution<double> mant(-1.0, 1.0);
    std::uniform_int_distribution<int> ex(-30, 30);
    long bad_two_sum = 0;
    for (int t = 0; t < 2000000; ++t) {
        float a = (float)std::ldexp(mant(rng), ex(rng)), b = (float)std::ldexp(mant(rng), ex(rng));
        float s, e;
        two_sum(a, b, s, e);
        if ((long double)s + (long double)e != (long double)a + (long double)b) ++bad_two_sum;
    }
    const double eps = std::ldexp(1.0, -24);
    long bad_acc = 0, bad_merge = 0, bad_plain = 0;
    for (int trial = 0; trial < 200; ++trial) {
        const int n = 1000 + 500 * trial;
        float2 acc = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
        float plain = 0.f;
        long double exact = 0.0L, absum = 0.0L;
        for (int i = 0; i < n; ++i) {
            // values of mixed magnitude and sign: large terms that cancel plus small ones
            float v = (float)std::ldexp(mant(rng), (i %% 7 == 0) ? 20 : ex(rng) / 3);
            csum_add(acc, v);
            csum_add(i < n / 2 ? lo : hi, v);
            plain += v;
            exact += v;
            absum += std::fabs((long double)v);
        }
        const long double bound = 2 * eps * std::fabs(exact) + 4.0L * n * eps * eps * absum;
        if (std::fabs((long double)acc.x + acc.y - exact) > bound) ++bad_acc;
        float2 m = csum_merge(lo, hi);
        if (std::fabs((long double)m.x + m.y - exact) > bound) ++bad_merge;
        if (std::fabs((long double)plain - exact) > bound) ++bad_plain;
    }
    std::printf("two_sum %%ld acc %%ld merge %%ld plain %%ld of 200\n", bad_two_sum, bad_acc, bad_merge, bad_plain);
    return (bad_two_sum || bad_acc || bad_merge) ? 1 : 0;
}
"""


def _helpers() -> str:
    text = HDR.read_text()
    out = []
    for name in ("two_sum", "csum_add", "csum_merge"):
        m = re.search(r"__device__ __forceinline__ [a-z0-9_]+ " + name + r"\(.*?\n}\n", text, re.S)
        assert m, f"{name} not found in the kernel header"
        out.append(m.group(0))
    return "\n".join(out)


def test_two_sum_is_error_free_and_compensated_sums_meet_their_bound(tmp_path):
    src = tmp_path / "csum.cpp"
    src.write_text(HARNESS % _helpers())
    exe = tmp_path / "csum"
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-o", str(exe), str(src)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout
    m = re.search(r"plain (\d+) of 200", r.stdout)
    assert m and int(m.group(1)) >= 150, r.stdout        # a plain FP32 sum of the same data fails the bound
