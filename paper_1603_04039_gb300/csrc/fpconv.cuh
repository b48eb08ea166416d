// fpconv.cuh -- binary64 <-> binary32 conversions, and the floor, clamp and
// range test of the Morton-key quantisation, on the integer pipe.
//
// GB300 runs FP64 arithmetic, and the conversions between double and float,
// on a pipe 58x narrower than FP32 (1.19 TFLOP/s measured).  A particle pass
// that converts seven values per particle spends most of its time there.
// These conversions work directly on the IEEE 754-2008 encodings -- binary64:
// sign, 11 exponent bits (bias 1023), 52 fraction bits; binary32: sign, 8
// exponent bits (bias 127), 23 fraction bits -- with integer instructions
// only, every case included (zeros, subnormal results and inputs, overflow to
// infinity, infinities, NaNs), and round to nearest, ties to even, the
// standard's default rounding; the floor-and-clamp and the range test read
// the same encodings.  Nothing here may reach the FP64 pipe: a
// hardware conversion kept for a rare case would be evaluated for every
// value once the compiler turns the branch into a select.  Checked bit for
// bit against the hardware conversions and the FP64 floor / fmin / fmax /
// comparison forms by tests/test_gpu_fpconv.py (NaNs compare as NaNs).
#pragma once

#include <cstdint>

namespace apc {

// double -> float, round to nearest even
__device__ __forceinline__ float f64_to_f32_int(double d) {
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int E = (int)((b >> 52) & 0x7FFu);
    const uint64_t frac = b & 0xFFFFFFFFFFFFFull;
    if (E == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (frac ? 0x400000u : 0u));   // inf, NaN
    const int e = E - 1023 + 127;
    if (e >= 255) return __uint_as_float(sign | 0x7F800000u);                               // overflow
    // significand with its leading bit, and the number of its low bits to drop:
    // 29 for a normal result, 29 + (1 - e) for a subnormal one
    const uint64_t sig = (E ? (1ull << 52) : 0ull) | frac;
    const int drop = e > 0 ? 29 : 29 + 1 - e;
    if (drop >= 64) return __uint_as_float(sign);                                            // below half the least subnormal
    const uint64_t keep = sig >> drop, rest = sig & ((1ull << drop) - 1ull), half = 1ull << (drop - 1);
    const uint32_t up = (rest > half || (rest == half && (keep & 1ull))) ? 1u : 0u;
    // a normal result adds its exponent field to the 24-bit significand (whose
    // leading bit then lands in the exponent field: one less exponent to add);
    // a carry out of the fraction moves into the exponent, to infinity at the
    // top, and a subnormal that rounds up to 2^-126 becomes the least normal
    const uint32_t r = e > 0 ? (((uint32_t)(e - 1) << 23) + (uint32_t)keep + up) : ((uint32_t)keep + up);
    return __uint_as_float(sign | r);
}

// float -> double (exact)
__device__ __forceinline__ double f32_to_f64_int(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    uint32_t hi, lo;
    if (e == 255) {                 // inf, NaN (payload kept)
        hi = sign | 0x7FF00000u | (m >> 3);
        lo = m << 29;
    } else if (e != 0) {            // normal
        hi = sign | ((e + 1023u - 127u) << 20) | (m >> 3);
        lo = m << 29;
    } else if (m == 0) {            // zero
        hi = sign;
        lo = 0u;
    } else {                        // subnormal float: m 2^-149, leading bit t
        const int t = 31 - __clz((int)m);
        const uint64_t fr = ((uint64_t)m << (52 - t)) & 0xFFFFFFFFFFFFFull;
        hi = sign | ((uint32_t)(t - 149 + 1023) << 20) | (uint32_t)(fr >> 32);
        lo = (uint32_t)fr;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// min(max(floor(t), 0), maxv) as an unsigned integer, for maxv < 2^31; NaN
// gives 0 (as fmin(fmax(NaN, 0), maxv) does)
__device__ __forceinline__ uint32_t f64_floor_clamp_u32(double t, uint32_t maxv) {
    const uint64_t b = (uint64_t)__double_as_longlong(t);
    const int E = (int)((b >> 52) & 0x7FFu);
    if ((b >> 63) || E < 1023) return 0u;                 // negative, -0, below 1
    if (E == 0x7FF) return (b & 0xFFFFFFFFFFFFFull) ? 0u : maxv;   // NaN, +inf
    const int ex = E - 1023;                               // t in [2^ex, 2^(ex+1))
    if (ex >= 31) return maxv;
    const uint64_t ip = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> (52 - ex);
    return ip > maxv ? maxv : (uint32_t)ip;
}

// lo <= p <= hi for finite lo, hi (false for NaN p), compared on the IEEE
// encodings mapped to integers of the same order
__device__ __forceinline__ int64_t f64_order_key(double v) {
    const int64_t b = __double_as_longlong(v);
    return b >= 0 ? b : (int64_t)(0x8000000000000000ull - (uint64_t)b);   // -0 maps to 0 like +0
}
__device__ __forceinline__ bool f64_in_range(double p, double lo, double hi) {
    const uint64_t b = (uint64_t)__double_as_longlong(p);
    if (((b >> 52) & 0x7FFu) == 0x7FFu && (b & 0xFFFFFFFFFFFFFull)) return false;   // NaN
    const int64_t k = f64_order_key(p);
    return k >= f64_order_key(lo) && k <= f64_order_key(hi);
}

}  // namespace apc
