"""The double-single split taken from the bits of a double (csrc/split.cuh)
against the plain conversions hi = RN_float(r), lo = RN_float(r - hi), bit for
bit, on the GPU: random doubles over the whole fast-path exponent range and
both fallbacks, round-to-even ties of either parity, roundings that carry into
the exponent, signed zeros, subnormals, infinities and NaN.  The widening of
a float to double from its bits against the conversion instruction, on every
one of the 2^32 float bit patterns."""
import os
import re
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1003_3896_gb300", "csrc")

SRC = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>
#include "split.cuh"

__global__ void check(const double *r, int n, unsigned long long *bad, int *first)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float hi, lo;
    nb::split_ds(r[t], hi, lo);
    const float h0 = __double2float_rn(r[t]);
    const float l0 = __double2float_rn(r[t] - (double)h0);
    const bool same_h = __float_as_int(hi) == __float_as_int(h0) || (h0 != h0 && hi != hi);
    const bool same_l = __float_as_int(lo) == __float_as_int(l0) || (l0 != l0 && lo != lo);
    if (!(same_h && same_l)) {
        atomicAdd(bad, 1ull);
        atomicMin(first, t);
    }
}

__global__ void check_widen(unsigned long long *bad, unsigned int *first)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < (1ull << 32);
         u += stride) {
        const float f = __uint_as_float((unsigned int)u);
        const double a = nb::widen(f), b = (double)f;
        const bool same = __double_as_longlong(a) == __double_as_longlong(b) || (a != a && b != b);
        if (!same) {
            atomicAdd(bad, 1ull);
            atomicMin(first, (unsigned int)u);
        }
    }
}

static double from_bits(uint64_t b) { double d; std::memcpy(&d, &b, 8); return d; }

int main()
{
    std::vector<double> v;
    uint64_t s = 0x9E3779B97F4A7C15ull;
    auto next = [&]() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; };
    // random mantissas over exponents 900 .. 1150 (fast path is 953 .. 1123)
    for (int e = 900; e <= 1150; ++e)
        for (int k = 0; k < 4000; ++k) {
            const uint64_t m = next() & 0xFFFFFFFFFFFFFull;
            const uint64_t sign = (next() & 1) << 63;
            v.push_back(from_bits(sign | ((uint64_t)e << 52) | m));
        }
    // ties (low 29 bits exactly half) with odd and even kept bit, carries
    for (int e : {953, 1000, 1023, 1050, 1123}) {
        for (int k = 0; k < 2000; ++k) {
            uint64_t m = next() & 0xFFFFFFFFFFFFFull;
            m = (m & ~0x1FFFFFFFull) | 0x10000000ull;
            v.push_back(from_bits(((uint64_t)e << 52) | m));
            v.push_back(from_bits((1ull << 63) | ((uint64_t)e << 52) | m));
        }
        v.push_back(from_bits(((uint64_t)e << 52) | 0xFFFFFFFFFFFFFull));
        v.push_back(from_bits(((uint64_t)e << 52) | 0xFFFFFF0000000ull | 0x10000000ull));
        v.push_back(from_bits(((uint64_t)e << 52) | 0xFFFFFFE000000ull | 0x10000000ull));
        v.push_back(from_bits((1ull << 63) | ((uint64_t)e << 52) | 0xFFFFFFFFFFFFFull));
    }
    // zeros, subnormals, tiny, huge, infinities, NaN
    for (uint64_t b : {0ull, 1ull << 63, 1ull, 0x000FFFFFFFFFFFFFull, 0x0010000000000000ull,
                       0x7FEFFFFFFFFFFFFFull, 0x7FF0000000000000ull, 0xFFF0000000000000ull,
                       0x7FF8000000000000ull})
        v.push_back(from_bits(b));
    const int n = (int)v.size();
    double *d_r = nullptr;
    unsigned long long *d_bad = nullptr;
    int *d_first = nullptr;
    if (cudaMalloc(&d_r, sizeof(double) * n) || cudaMalloc(&d_bad, 8) || cudaMalloc(&d_first, 4))
        return 2;
    const int big = n;
    cudaMemcpy(d_r, v.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
    cudaMemset(d_bad, 0, 8);
    cudaMemcpy(d_first, &big, 4, cudaMemcpyHostToDevice);
    check<<<(n + 255) / 256, 256>>>(d_r, n, d_bad, d_first);
    unsigned long long bad = 0;
    int first = 0;
    if (cudaMemcpy(&bad, d_bad, 8, cudaMemcpyDeviceToHost) ||
        cudaMemcpy(&first, d_first, 4, cudaMemcpyDeviceToHost))
        return 3;
    std::printf("checked %d mismatches %llu first %d\n", n, bad, first);
    if (bad) {
        uint64_t b;
        std::memcpy(&b, &v[first], 8);
        std::printf("first mismatch bits %016llx\n", (unsigned long long)b);
    }
    unsigned long long wbad = 0;
    unsigned int wfirst = 0xFFFFFFFFu;
    cudaMemset(d_bad, 0, 8);
    unsigned int *d_wfirst = nullptr;
    if (cudaMalloc(&d_wfirst, 4)) return 2;
    cudaMemcpy(d_wfirst, &wfirst, 4, cudaMemcpyHostToDevice);
    check_widen<<<152 * 16, 256>>>(d_bad, d_wfirst);
    if (cudaMemcpy(&wbad, d_bad, 8, cudaMemcpyDeviceToHost) ||
        cudaMemcpy(&wfirst, d_wfirst, 4, cudaMemcpyDeviceToHost))
        return 3;
    std::printf("widen checked 4294967296 mismatches %llu first %08x\n", wbad, wfirst);
    return (bad || wbad) ? 1 : 0;
}
"""


def test_split_matches_plain_conversions(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "split_check.cu"
    src.write_text(SRC)
    exe = tmp_path / "split_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert re.search(r"^checked \d+ mismatches 0 first", r.stdout, re.M), r.stdout
    assert "widen checked 4294967296 mismatches 0 first" in r.stdout, r.stdout


RSQ_SRC = r"""
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>
#include "split.cuh"

__global__ void powers(const double *r, int n, double *p1, double *p3)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    p1[t] = nb::rsqrt_pow<true>(r[t]);
    p3[t] = nb::rsqrt_pow<false>(r[t]);
}

int main()
{
    std::vector<double> v;
    uint64_t s = 0x2545F4914F6CDD1Dull;
    auto next = [&]() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; };
    for (int k = 0; k < 400000; ++k) {   // log-uniform over [1e-30, 1e30]
        const double u = (double)(next() >> 11) / 9007199254740992.0;
        v.push_back(std::pow(10.0, -30.0 + 60.0 * u));
    }
    // both ends of the float-estimate path and beyond it (library fallback)
    for (double e : {-125.0, -124.0, 125.0, 126.0, 127.0, -126.0, -127.0, 200.0, -200.0})
        for (int k = -3; k <= 3; ++k) v.push_back(std::ldexp(1.0 + k * 1e-3, (int)e));
    const int n = (int)v.size();
    double *d_r, *d_1, *d_3;
    if (cudaMalloc(&d_r, 8 * n) || cudaMalloc(&d_1, 8 * n) || cudaMalloc(&d_3, 8 * n)) return 2;
    cudaMemcpy(d_r, v.data(), 8 * n, cudaMemcpyHostToDevice);
    powers<<<(n + 255) / 256, 256>>>(d_r, n, d_1, d_3);
    std::vector<double> p1(n), p3(n);
    if (cudaMemcpy(p1.data(), d_1, 8 * n, cudaMemcpyDeviceToHost) ||
        cudaMemcpy(p3.data(), d_3, 8 * n, cudaMemcpyDeviceToHost))
        return 3;
    double worst1 = 0, worst3 = 0;
    for (int k = 0; k < n; ++k) {
        const long double R = v[k], e1 = 1.0L / std::sqrt(R), e3 = e1 * e1 * e1;
        const double u1 = (double)std::fabs((p1[k] - e1) / e1) / 0x1p-53;
        const double u3 = (double)std::fabs((p3[k] - e3) / e3) / 0x1p-53;
        if (u1 > worst1) worst1 = u1;
        if (u3 > worst3) worst3 = u3;
    }
    std::printf("rsqrt powers checked %d worst ulp R^-1/2 %.3f R^-3/2 %.3f\n", n, worst1, worst3);
    return 0;
}
"""


def test_rsqrt_powers_against_long_double(tmp_path):
    """The FP64 pair kernel's and the field's R^(-1/2) and R^(-3/2) (float
    estimate, series refinement in double): within 2.5 and 4.5 units of 2^-53
    of a long-double evaluation (quad precision on the GPU host's Arm
    toolchain) over 60 decades, the float-range edges and the library
    fallback beyond them (a CPU emulation of the refinement gave 1.5 and 3.3;
    a wrong series coefficient gives thousands)."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "rsq_check.cu"
    src.write_text(RSQ_SRC)
    exe = tmp_path / "rsq_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    m = re.search(r"worst ulp R\^-1/2 ([0-9.]+) R\^-3/2 ([0-9.]+)", r.stdout)
    assert m, r.stdout
    assert float(m.group(1)) <= 2.5 and float(m.group(2)) <= 4.5, r.stdout
