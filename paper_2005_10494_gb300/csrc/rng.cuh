// Counter-based normals for the sampling kernels.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (hi0, lo0) = M0 * x0,  (hi1, lo1) = M1 * x2,
//   x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0),  k <- k + (W0, W1).
// Counter (call_lo, call_hi, key_lo, key_hi), Philox key (seed_lo, seed_hi).
// Word x -> u = (2 floor(x / 2^9) + 1) 2^-24 in (0, 1); Box-Muller on words
// (0,1) and (2,3): z = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1).
#pragma once

#include <cstdint>

#include "mcd_internal.cuh"

namespace mcd {

// Round keys rk0[r] = seed_lo + r W0, rk1[r] = seed_hi + r W1 are computed on
// the host and read from the kernel parameters (constant bank).

__device__ __forceinline__ void mulhilo(uint32_t m, uint32_t x, uint32_t& hi, uint32_t& lo) {
    const uint64_t p = static_cast<uint64_t>(m) * static_cast<uint64_t>(x);
    hi = static_cast<uint32_t>(p >> 32);
    lo = static_cast<uint32_t>(p);
}

// Rounds 2..10 of Philox on (x0, x1, x2, x3).
__device__ __forceinline__ uint4 philox_rounds_2_10(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3,
                                                    const uint32_t* __restrict__ rk0,
                                                    const uint32_t* __restrict__ rk1) {
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo(kPhiloxM0, x0, hi0, lo0);
        mulhilo(kPhiloxM1, x2, hi1, lo1);
        const uint32_t n0 = hi1 ^ x1 ^ rk0[r];
        const uint32_t n2 = hi0 ^ x3 ^ rk1[r];
        x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
    }
    return make_uint4(x0, x1, x2, x3);
}

// Full Philox4x32-10 on an arbitrary counter.
__device__ __forceinline__ uint4 philox_full(uint64_t call, uint64_t key, const uint32_t* rk0,
                                             const uint32_t* rk1) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo(kPhiloxM0, static_cast<uint32_t>(call), hi0, lo0);
    mulhilo(kPhiloxM1, static_cast<uint32_t>(key), hi1, lo1);
    const uint32_t x0 = hi1 ^ static_cast<uint32_t>(call >> 32) ^ rk0[0];
    const uint32_t x2 = hi0 ^ static_cast<uint32_t>(key >> 32) ^ rk1[0];
    return philox_rounds_2_10(x0, lo1, x2, lo0, rk0, rk1);
}

// Per-tile constants of the first round when the high word of the call index
// is fixed over the tile: round 1 maps (c_lo, c_hi, key_lo, key_hi) to
// (hi(M1 key_lo) ^ c_hi ^ k0, lo(M1 key_lo), hi(M0 c_lo) ^ key_hi ^ k1, lo(M0 c_lo)).
struct Round1 {
    uint32_t x0;      // hi(M1 key_lo) ^ c_hi ^ k0
    uint32_t x1;      // lo(M1 key_lo)
    uint32_t kx;      // key_hi ^ k1
};

__device__ __forceinline__ Round1 round1_consts(uint32_t call_hi, uint64_t key, const uint32_t* rk0,
                                                const uint32_t* rk1) {
    uint32_t hi1, lo1;
    mulhilo(kPhiloxM1, static_cast<uint32_t>(key), hi1, lo1);
    Round1 r;
    r.x0 = hi1 ^ call_hi ^ rk0[0];
    r.x1 = lo1;
    r.kx = static_cast<uint32_t>(key >> 32) ^ rk1[0];
    return r;
}

__device__ __forceinline__ uint4 philox_fast(uint32_t call_lo, const Round1& r1, const uint32_t* rk0,
                                             const uint32_t* rk1) {
    uint32_t hi0, lo0;
    mulhilo(kPhiloxM0, call_lo, hi0, lo0);
    return philox_rounds_2_10(r1.x0, r1.x1, hi0 ^ r1.kx, lo0, rk0, rk1);
}

// ---- FP32 Box-Muller ------------------------------------------------------
// 1.m in [1, 2) from the 23 high bits of x (x >> 9 has no bit in common with
// the exponent field, so the sum is the bitwise or; one shift-add).
__device__ __forceinline__ float one_point_m(uint32_t x) {
    return __uint_as_float((x >> 9) + 0x3f800000u);
}

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sin_approx(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float cos_approx(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two normals from words (w0, w1).  u0 = 1.m0 - (1 - 2^-24) and
// 2v = 2 (1 - u0) = fma(-2, u0, 2) are exact.  r^2 = -2 ln u0 comes from the
// hardware log2, whose absolute error (about 2.2e-7 in r^2) grows into a
// radius error of 1.1e-7 / r for small r; for 2v < 2^-10 the first term of
// -2 ln(1 - v) = 2v + v^2 + ... is used instead (error v^2 < 2.4e-7 there).
// The switch point balances the two, so the radius error stays below 4e-6.  The angle is 2 pi u1 - pi = 2 pi (1.m1) - (3 pi - 2 pi 2^-24)
// in (-pi, pi), where the approximate sine and cosine are most accurate, and
// (cos, sin)(2 pi u1) = -(cos, sin)(angle).
__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float& z0, float& z1) {
    const float u0 = one_point_m(w0) - 0x1.fffffep-1f;             // exact
    const float two_v = fmaf(-2.0f, u0, 2.0f);                       // exact
    const float lg = -1.38629436112f * lg2_approx(u0);
    const float r = sqrt_approx(two_v < 0x1p-10f ? two_v : lg);     // sqrt(-2 ln u0)
    const float ang = fmaf(6.28318530718f, one_point_m(w1), -9.42477758f);
    const float nr = -r;
    z0 = nr * cos_approx(ang);
    z1 = nr * sin_approx(ang);
}

// ---- FP64 Box-Muller ------------------------------------------------------
__device__ __forceinline__ double uniform64(uint32_t x) {
    return (2.0 * static_cast<double>(x >> 9) + 1.0) * 0x1p-24;
}

// Not inlined: the FP64 path is a precision reference, and one out-of-line
// copy keeps the many unrolled instantiations small.
static __device__ __noinline__ void box_muller(uint32_t w0, uint32_t w1, double& z0, double& z1) {
    const double u0 = uniform64(w0);
    const double u1 = uniform64(w1);
    const double r = sqrt(-2.0 * log(u0));
    double s, c;
    sincospi(2.0 * u1, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

template <typename R>
__device__ __forceinline__ void normals4(uint4 w, R* z) {
    box_muller(w.x, w.y, z[0], z[1]);
    box_muller(w.z, w.w, z[2], z[3]);
}

}  // namespace mcd
