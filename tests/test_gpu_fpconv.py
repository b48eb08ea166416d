"""The integer-pipe helpers of paper_1603_04039_gb300/csrc/fpconv.cuh against
the FP64 forms they replace, bit for bit:
  * double <-> float conversions against the hardware conversions: random
    encodings over the whole exponent range, every rounding case of the 29
    dropped fraction bits (below, at and above one half, with an even and an
    odd kept fraction), carries into the exponent, overflow to infinity,
    results in the subnormal range, signed zeros, infinities and NaNs;
  * floor-and-clamp of the Morton-key quantisation against
    (uint32_t)fmin(fmax(floor(t), 0), maxv): integers, values just below and
    above them, negatives, -0, huge values, infinities, NaNs;
  * the domain test against lo <= p && p <= hi.
A small CUDA program including the header is built with nvcc and run."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <vector>
#include "fpconv.cuh"

__global__ void conv(const double *d, float *df, float *dh, const float *f, double *fd, double *fh, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    df[i] = apc::f64_to_f32_int(d[i]);
    dh[i] = __double2float_rn(d[i]);
    fd[i] = apc::f32_to_f64_int(f[i]);
    fh[i] = (double)f[i];
}

__global__ void quant(const double *t, uint32_t maxv, uint32_t *qi, uint32_t *qh, const double *lo,
                      const double *hi, int *ri, int *rh, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    qi[i] = apc::f64_floor_clamp_u32(t[i], maxv);
    qh[i] = (uint32_t)fmin(fmax(floor(t[i]), 0.0), (double)maxv);
    ri[i] = apc::f64_in_range(t[i], lo[i], hi[i]) ? 1 : 0;
    rh[i] = (t[i] >= lo[i] && t[i] <= hi[i]) ? 1 : 0;
}

static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t next() {   // SplitMix64
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double dbits(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static float fbits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }

int main() {
    std::vector<double> d;
    std::vector<float> f;
    // random encodings: all exponents, and exponents near the float range
    for (int i = 0; i < 2000000; ++i) d.push_back(dbits(next()));
    for (int i = 0; i < 2000000; ++i) {
        uint64_t b = next();
        uint64_t e = 1023 - 160 + (b >> 55) % 330;   // binary32 range and a margin on both sides
        d.push_back(dbits((b & 0x800FFFFFFFFFFFFFull) | (e << 52)));
    }
    // the dropped 29 bits at, just below and just above one half; kept fraction even and odd
    const uint64_t drops[] = {0x10000000ull, 0x0FFFFFFFull, 0x10000001ull, 0ull, 1ull, 0x1FFFFFFFull};
    for (int e = 1023 - 126; e <= 1023 + 127; ++e)
        for (uint64_t keep : {0ull, 1ull, 2ull, 0x7FFFFEull, 0x7FFFFFull, 0x2AAAAAull})
            for (uint64_t r : drops)
                for (uint64_t sg : {0ull, 1ull})
                    d.push_back(dbits((sg << 63) | ((uint64_t)e << 52) | (keep << 29) | r));
    // around the subnormal and overflow edges, zeros, infinities, NaNs, double subnormals
    for (int e = 1023 - 160; e <= 1023 - 120; ++e)
        for (int k = 0; k < 64; ++k) d.push_back(dbits(((uint64_t)e << 52) | (next() >> 12)));
    for (int e = 1023 + 126; e <= 1023 + 130; ++e)
        for (int k = 0; k < 64; ++k) d.push_back(dbits(((uint64_t)e << 52) | (next() >> 12)));
    const uint64_t special[] = {0ull, 0x8000000000000000ull, 0x7FF0000000000000ull, 0xFFF0000000000000ull,
                                0x7FF8000000000000ull, 1ull, 0x000FFFFFFFFFFFFFull, 0x47EFFFFFE0000000ull,
                                0x47EFFFFFF0000000ull, 0x47EFFFFFEFFFFFFFull, 0x36A0000000000000ull,
                                0x3690000000000000ull, 0x3810000000000000ull, 0x380FFFFFF0000000ull};
    for (uint64_t b : special) d.push_back(dbits(b));
    for (size_t i = 0; i < d.size(); ++i) f.push_back(fbits((uint32_t)next()));
    const uint32_t fspecial[] = {0u, 0x80000000u, 1u, 0x007FFFFFu, 0x00800000u, 0x7F7FFFFFu, 0x7F800000u,
                                 0xFF800000u, 0x7FC00000u, 0x3F800000u};
    for (int i = 0; i < 10; ++i) f[i] = fbits(fspecial[i]);
    const int n = (int)d.size();
    double *gd, *gfd, *gfh; float *gdf, *gdh, *gf;
    cudaMalloc(&gd, n * 8); cudaMalloc(&gfd, n * 8); cudaMalloc(&gfh, n * 8);
    cudaMalloc(&gdf, n * 4); cudaMalloc(&gdh, n * 4); cudaMalloc(&gf, n * 4);
    cudaMemcpy(gd, d.data(), n * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(gf, f.data(), n * 4, cudaMemcpyHostToDevice);
    conv<<<(n + 255) / 256, 256>>>(gd, gdf, gdh, gf, gfd, gfh, n);
    if (cudaDeviceSynchronize() != cudaSuccess) { printf("cuda error\n"); return 2; }
    std::vector<uint32_t> df(n), dh(n);
    std::vector<uint64_t> fd(n), fh(n);
    cudaMemcpy(df.data(), gdf, n * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(dh.data(), gdh, n * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(fd.data(), gfd, n * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(fh.data(), gfh, n * 8, cudaMemcpyDeviceToHost);
    long bad_d = 0, bad_f = 0, int_path = 0;
    for (int i = 0; i < n; ++i) {
        bool nan_a = (df[i] & 0x7FFFFFFFu) > 0x7F800000u, nan_b = (dh[i] & 0x7FFFFFFFu) > 0x7F800000u;
        if (!(nan_a && nan_b) && df[i] != dh[i]) ++bad_d;
        bool fn_a = (fd[i] & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull;
        bool fn_b = (fh[i] & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull;
        if (!(fn_a && fn_b) && fd[i] != fh[i]) ++bad_f;
        uint64_t b; memcpy(&b, &d[i], 8);
        int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
        if (e > 0 && e < 255) ++int_path;
    }
    // quantisation: t around every integer up to 2^22, random magnitudes, specials
    std::vector<double> t, lo, hi;
    for (int k = -4; k < (1 << 22) + 4; k += 97)
        for (double off : {-0.5, -1e-9, 0.0, 1e-9, 0.5}) t.push_back(k + off);
    for (int i = 0; i < 1000000; ++i) t.push_back(dbits(next()));
    for (int i = 0; i < 1000000; ++i) {
        uint64_t b = next();
        t.push_back(dbits((b & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(1023 - 30 + (b >> 58) % 60) << 52)));
    }
    for (uint64_t b : special) t.push_back(dbits(b));
    t.push_back(-0.0); t.push_back(2097151.0); t.push_back(2097152.0); t.push_back(nextafter(2097152.0, 0.0));
    for (size_t i = 0; i < t.size(); ++i) {
        // bounds: random finite pairs, a third of them around t itself
        double a = dbits(next() & 0xBFFFFFFFFFFFFFFFull), b = dbits(next() & 0xBFFFFFFFFFFFFFFFull);
        if (i % 3 == 0 && t[i] == t[i]) { a = t[i]; b = nextafter(t[i], 1e300); }
        if (i % 3 == 1 && t[i] == t[i]) { a = nextafter(t[i], -1e300); b = t[i]; }
        if (!(fabs(a) < 1e300)) a = -1.0;
        if (!(fabs(b) < 1e300)) b = 1.0;
        lo.push_back(a < b ? a : b); hi.push_back(a < b ? b : a);
    }
    const int nt = (int)t.size();
    double *gt, *glo, *ghi; uint32_t *gqi, *gqh; int *gri, *grh;
    cudaMalloc(&gt, nt * 8); cudaMalloc(&glo, nt * 8); cudaMalloc(&ghi, nt * 8);
    cudaMalloc(&gqi, nt * 4); cudaMalloc(&gqh, nt * 4); cudaMalloc(&gri, nt * 4); cudaMalloc(&grh, nt * 4);
    cudaMemcpy(gt, t.data(), nt * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(glo, lo.data(), nt * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(ghi, hi.data(), nt * 8, cudaMemcpyHostToDevice);
    long bad_q = 0, bad_r = 0, in_range = 0;
    for (uint32_t maxv : {2097151u, 1023u, 0x7FFFFFFFu}) {
        quant<<<(nt + 255) / 256, 256>>>(gt, maxv, gqi, gqh, glo, ghi, gri, grh, nt);
        if (cudaDeviceSynchronize() != cudaSuccess) { printf("cuda error\n"); return 2; }
        std::vector<uint32_t> qi(nt), qh(nt);
        std::vector<int> ri(nt), rh(nt);
        cudaMemcpy(qi.data(), gqi, nt * 4, cudaMemcpyDeviceToHost);
        cudaMemcpy(qh.data(), gqh, nt * 4, cudaMemcpyDeviceToHost);
        cudaMemcpy(ri.data(), gri, nt * 4, cudaMemcpyDeviceToHost);
        cudaMemcpy(rh.data(), grh, nt * 4, cudaMemcpyDeviceToHost);
        for (int i = 0; i < nt; ++i) {
            bad_q += qi[i] != qh[i];
            bad_r += ri[i] != rh[i];
            in_range += rh[i];
        }
    }
    printf("n %d int_path %ld bad_d2f %ld bad_f2d %ld nq %d bad_quant %ld bad_range %ld in_range %ld\n", n,
           int_path, bad_d, bad_f, nt, bad_q, bad_r, in_range);
    return 0;
}
"""


def test_integer_conversions_match_hardware(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "fpconv_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "fpconv_check"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_1603_04039_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout
    fields = dict(zip(out.split()[0::2], map(int, out.split()[1::2])))
    assert fields["int_path"] > 1_500_000, fields          # most inputs exercise the integer path
    assert fields["bad_d2f"] == 0 and fields["bad_f2d"] == 0, fields
    assert fields["bad_quant"] == 0 and fields["bad_range"] == 0, fields
    # both outcomes of the range test occur (three bounds runs over nq values)
    assert fields["nq"] < fields["in_range"] < 3 * fields["nq"], fields
