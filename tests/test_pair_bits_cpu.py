"""The level conversions' integer arithmetic (split_pair, join_pair and the
helpers of the kernel header), compiled for the host with stand-ins for the
CUDA intrinsics, bit for bit against the host CPU's IEEE-754 conversions and
float64 addition (round to nearest even): random encodings (every class:
zeros, subnormals, normals, infinities, NaNs), values over the float32 range
and below it down to float64 subnormals, values a few units of the last
float64 place from a float32, exact float32 ties, and arbitrary float32 pairs
for the join.  The GPU's own conversions are compared in test_gpu_pairs."""
import shutil
import subprocess
from pathlib import Path

import pytest

HEADER = Path(__file__).resolve().parents[1] / "paper_1308_3214_gb300" / "csrc" / "molt_kernels.cuh"

SHIMS = r"""
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <random>
#include <cmath>
static inline int __double2hiint(double v) { uint64_t b; memcpy(&b, &v, 8); return (int)(b >> 32); }
static inline int __double2loint(double v) { uint64_t b; memcpy(&b, &v, 8); return (int)(uint32_t)b; }
static inline float __uint_as_float(unsigned u) { float f; memcpy(&f, &u, 4); return f; }
static inline unsigned __float_as_uint(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
static inline double __longlong_as_double(long long u) { double f; memcpy(&f, &u, 8); return f; }
static inline long long __double_as_longlong(double d) { long long u; memcpy(&u, &d, 8); return u; }
static inline float __double2float_rn(double v) { return (float)v; }
static inline int __clz(int x) { return x == 0 ? 32 : __builtin_clz((unsigned)x); }
static inline int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }
"""

MAIN = r"""
static bool same32(float a, float b) { return __float_as_uint(a) == __float_as_uint(b) || (std::isnan(a) && std::isnan(b)); }
static bool same64(double a, double b)
{
    return __double_as_longlong(a) == __double_as_longlong(b) || (std::isnan(a) && std::isnan(b));
}
int main()
{
    std::mt19937_64 g(20240611);
    long bad = 0, n = 0;
    auto chk = [&](double v) {
        float h, l;
        split_pair(v, h, l);
        const float rh = (float)v;
        ++n;
        if (!same32(h, rh)) { if (bad++ < 5) printf("high %a: %a %a\n", v, h, rh); return; }
        if (std::isfinite(v) && std::isfinite(rh)) {
            const float rl = (float)(v - (double)rh);
            if (!same32(l, rl)) { if (bad++ < 5) printf("low %a: %a %a\n", v, l, rl); return; }
        }
        const double j = join_pair(h, l), rj = (double)h + (double)l;
        if (!same64(j, rj)) { if (bad++ < 5) printf("join %a: %a %a -> %a %a\n", v, h, l, j, rj); }
    };
    const long M = 1000000;
    std::uniform_real_distribution<double> U(-2, 2);
    std::uniform_int_distribution<int> E(-160, 140), E2(-1080, -100), K(-1000, 1000);
    for (long i = 0; i < 4 * M; ++i) { uint64_t b = g(); double v; memcpy(&v, &b, 8); chk(v); }
    for (long i = 0; i < 4 * M; ++i) chk(std::ldexp(U(g), E(g)));
    for (long i = 0; i < 2 * M; ++i) chk(std::ldexp(U(g), E2(g)));
    for (long i = 0; i < M; ++i) {
        const float h = (float)std::ldexp(U(g), E(g));
        int e;
        std::frexp((double)h, &e);
        const double v = (double)h + std::ldexp((double)K(g), e - 53);
        chk(v); chk(-v);
        chk((double)h + std::ldexp(1.0, e - 25)); chk((double)h - std::ldexp(1.0, e - 25));
        chk(std::nextafter((double)h, 1.0)); chk(std::nextafter((double)h, -1.0));
    }
    long pbad = 0;
    for (long i = 0; i < 4 * M; ++i) {
        const uint64_t b = g();
        const unsigned hb = (unsigned)b, lb = (unsigned)(b >> 32);
        float h, l;
        memcpy(&h, &hb, 4); memcpy(&l, &lb, 4);
        if (!same64(join_pair(h, l), (double)h + (double)l)) { if (pbad++ < 5) printf("pair %a %a\n", h, l); }
        const float h2 = (float)std::ldexp(U(g), E(g)), l2 = (float)std::ldexp(U(g), E(g) - (int)(g() % 64));
        if (!same64(join_pair(h2, l2), (double)h2 + (double)l2)) { if (pbad++ < 5) printf("pair %a %a\n", h2, l2); }
    }
    printf("checked %ld values, %ld mismatches; %ld pair mismatches\n", n, bad, pbad);
    return (bad || pbad) ? 1 : 0;
}
"""


def conversion_source() -> str:
    text = HEADER.read_text()
    a = text.index("// --- level conversions (begin) ---")
    b = text.index("// --- level conversions (end) ---")
    return text[a:b].replace("__device__ __forceinline__", "static inline")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_pair_conversion_bits_on_host(tmp_path):
    src = tmp_path / "pairs.cpp"
    src.write_text(SHIMS + conversion_source() + MAIN)
    exe = tmp_path / "pairs"
    # no contraction: the host reference is plain IEEE arithmetic
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe), str(src)], check=True)
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, run.stdout + run.stderr
