// Sampling kernels: the Monte Carlo estimator of Sec. 2.2 (Eq. 6-7) and, in
// the same pass, the sums that its derivative needs (Appendix A.3 proves the
// objective smooth; the estimators are the likelihood ratio and a
// sigmoid-smoothed indicator).
//
// A persistent grid takes tiles (design, draw range) from an atomic ticket.
// For one tile a block stages the design's Cholesky factor L (packed lower
// triangle) and t = b - mu in shared memory; each thread then walks groups of
// G draws whose d*G normals fill whole Philox calls, makes the normals in
// registers, forms y = L z, tests "y_i > t_i for some i" and counts hits.
// Counts are reduced per warp with redux.sync and added to the design's u64
// counter; gradient sums go through FP32 warp shuffles, FP64 across warps and
// fixed-point u64 atomics into the design's batch slot (order-independent,
// hence bit-reproducible).
#pragma once

#include <cstdint>

#include "mcd_internal.cuh"
#include "rng.cuh"

namespace mcd {

template <int D>
struct Shape {
    static constexpr int kG = (D % 4 == 0) ? 1 : ((D % 2 == 0) ? 2 : 4);  // draws per group
    static constexpr int kNZ = D * kG;                                     // normals per group
    static constexpr int kNC = kNZ / 4;                                    // Philox calls per group
    static constexpr int kTri = D * (D + 1) / 2;
    static constexpr bool kRegL = D <= 6;                                  // L and t in registers
};

// Row i of the lower factor starts at rowoff(i); rows are padded to whole
// 16-byte vectors so that a row is read with ld.shared.v4.f32 / v2.f64.
template <typename R>
struct LPad {
    static constexpr int V = 16 / static_cast<int>(sizeof(R));
    __host__ __device__ static constexpr int chunks(int i) { return (i + V) / V; }
    __host__ __device__ static constexpr int rowoff(int i) {
        int s = 0;
        for (int r = 0; r < i; ++r) s += chunks(r) * V;
        return s;
    }
};
constexpr int kMaxPad = LPad<float>::rowoff(kMaxD);   // 240 floats (220 doubles)

constexpr int kMaxWarps = 8;    // blocks of at most 256 threads

template <typename R>
struct TileShared {
    alignas(16) R L[kMaxPad];        // padded packed lower factor
    alignas(16) R t[kMaxD + 4];      // b - mu
    alignas(16) float tsc[kMaxD + 4];  // -t * log2(e) / h (negated, for the FMA y log2(e)/h + tsc)
    uint64_t start;
    uint64_t key;
    uint32_t n;
    uint32_t design;
    uint32_t batch;
    int32_t d;
    int32_t ok;
    int32_t scen;
    uint32_t tile;
    int64_t vec_off;
    int64_t acc_off;
};

template <int D, bool GRAD, typename R>
struct Acc {
    uint32_t cnt;
    R A[GRAD ? D : 1];
    R B[GRAD ? D : 1];
    R G[GRAD ? D : 1];
};

__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// Shared-memory vector loads that the compiler may not hoist out of the draw
// loop (volatile), so large factors are streamed from shared memory instead
// of being pinned in registers.
template <bool VOL>
__device__ __forceinline__ void lds_vec(const float* p, float* v) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    if constexpr (VOL)
        asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "r"(a));
    else
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "r"(a));
}
template <bool VOL>
__device__ __forceinline__ void lds_vec(const double* p, double* v) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    if constexpr (VOL)
        asm volatile("ld.volatile.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "r"(a));
    else
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "r"(a));
}
__device__ __forceinline__ float lds_one(const float* p) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    float v;
    asm volatile("ld.volatile.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ double lds_one(const double* p) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    double v;
    asm volatile("ld.volatile.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}

// The FP32 adjoint forms the sigmoid factors and the gradient sums two
// coordinates per packed instruction (one_draw), except at d = 16, 18, 20,
// whose one-block-per-SM kernels measured 7-11 % slower that way than with
// each row's factor formed right after its transform (64 designs x 4e6
// draws; 2-18 % faster at the other d, 20 % on the batched mixed-d kernel).
template <int D>
__host__ __device__ constexpr bool packed_adjoint() { return !(D == 16 || D == 18 || D == 20); }

// sigma((t - y)/h) = 1 / (1 + exp((y - t)/h)); ntsc = -t log2(e)/h.
__device__ __forceinline__ float smooth_keep(float y, float t, float ntsc, float hl2e, double) {
    return rcp_approx(1.0f + ex2_approx(fmadd(y, hl2e, ntsc)));
}
static __device__ __noinline__ double smooth_keep(double y, double t, float, float, double hinv) {
    return 1.0 / (1.0 + exp((y - t) * hinv));
}

// Above d = 6 the factor is read from shared memory for every draw.  Plain
// ld.shared lets the compiler share a load between the draws of a group and
// keep thresholds in registers; ld.volatile.shared makes every draw load
// again but frees those registers.  In the FP32 adjoint kernels the second
// form avoids register spills, and it measured faster on GB300 (64 designs
// x 2e6 draws, AR(1) factor) at d = 8..12 and 15..19 by 4-42 %; at d = 7,
// 13, 14 and 20, and in every forward kernel, the plain form is as fast or
// faster.
template <int D, bool GRAD, typename R>
__host__ __device__ constexpr bool volatile_loads() {
    return GRAD && sizeof(R) == 4 && ((D >= 8 && D <= 12) || (D >= 15 && D <= 19));
}

// Factor, thresholds and bandwidth of the current tile, as one draw sees them.
template <int D, typename R>
struct TileView {
    static constexpr bool kReg = Shape<D>::kRegL;
    R L[kReg ? LPad<R>::rowoff(D) : 1];
    R t[kReg ? D : 1];
    float tsc[kReg ? D : 1];
    const R* sL;
    const R* st;
    const float* stsc;
    float hl2e;
    double hinv;
};

// y_i = sum_{j <= i} L_ij z_j for row i.
template <int D, int I, bool VOL, typename R>
__device__ __forceinline__ R row_dot(const TileView<D, R>& v, const R* z) {
    constexpr int V = LPad<R>::V;
    constexpr int off = LPad<R>::rowoff(I);
    R s;
    if constexpr (TileView<D, R>::kReg) {
        s = v.L[off] * z[0];
#pragma unroll
        for (int j = 1; j <= I; ++j) s = fmadd(v.L[off + j], z[j], s);
    } else {
        R l[V];
        lds_vec<VOL>(v.sL + off, l);
        s = l[0] * z[0];
#pragma unroll
        for (int j = 1; j < V && j <= I; ++j) s = fmadd(l[j], z[j], s);
#pragma unroll
        for (int c = 1; c * V <= I; ++c) {
            lds_vec<VOL>(v.sL + off + c * V, l);
#pragma unroll
            for (int q = 0; q < V && c * V + q <= I; ++q) s = fmadd(l[q], z[c * V + q], s);
        }
    }
    return s;
}

template <int D, int I, bool GRAD, typename R>
struct Rows {
    // Walk rows I..D-1: hit test, and the smoothed-indicator factors.
    __device__ __forceinline__ static void run(const TileView<D, R>& v, const R* z, bool& hit,
                                               R* keep, R& prod, float* ntsc) {
        constexpr bool VOL = volatile_loads<D, GRAD, R>();
        const R y = row_dot<D, I, VOL, R>(v, z);
        R t;
        float tsc = 0.0f;
        if constexpr (TileView<D, R>::kReg) {
            t = v.t[I];
            if constexpr (GRAD) tsc = v.tsc[I];
        } else if constexpr (VOL) {
            t = lds_one(v.st + I);
            tsc = lds_one(v.stsc + I);
        } else {
            t = v.st[I];
            if constexpr (GRAD) tsc = v.stsc[I];
        }
        hit |= (y > t);
        if constexpr (GRAD) {
            if constexpr (sizeof(R) == 4 && packed_adjoint<D>()) {
                keep[I] = y;                                     // the sigmoid is formed in one_draw
                ntsc[I] = tsc;
            } else if (v.hl2e != 0.0f) {
                keep[I] = smooth_keep(y, t, tsc, v.hl2e, v.hinv);
                prod *= keep[I];
            }
        }
        if constexpr (I + 1 < D) Rows<D, I + 1, GRAD, R>::run(v, z, hit, keep, prod, ntsc);
    }
};

// a[i] = fma(s, x[i], a[i]) for i < D.  With PK, two coordinates per packed
// FMA (pairs (0, 1), (2, 3), ...: x and a then sit in aligned register
// pairs); each lane rounds exactly as the scalar FMA does.
template <int D, bool PK>
__device__ __forceinline__ void axpy(float (&a)[D], float s, const float* x) {
    if constexpr (PK) {
        const float2 s2 = make_float2(s, s);
#pragma unroll
        for (int i = 0; i + 1 < D; i += 2) {
            const float2 r = __ffma2_rn(s2, make_float2(x[i], x[i + 1]), make_float2(a[i], a[i + 1]));
            a[i] = r.x;
            a[i + 1] = r.y;
        }
        if constexpr (D % 2 != 0) a[D - 1] = __fmaf_rn(s, x[D - 1], a[D - 1]);
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) a[i] = __fmaf_rn(s, x[i], a[i]);
    }
}

// One draw: y = L z, hit = any(y_i > t_i), and the gradient sums.  In the
// FP32 adjoint (packed_adjoint) the sigmoid factors and the sums go two
// coordinates per packed instruction (fma.rn.f32x2 / add.rn.f32x2, rounded
// lane by lane as the scalar instructions, so the sums are bit-identical):
// always for the sigmoid and G (arrays of this draw), and for A and B when
// the draw's normals start at an even index of the group's array (zodd
// false), so that they pair with the accumulators without register moves.
template <int D, bool GRAD, bool ALL_VALID, typename R>
__device__ __forceinline__ void one_draw(const R* z, bool zodd, const TileView<D, R>& v, bool valid,
                                         Acc<D, GRAD, R>& acc) {
    bool hit = false;
    R keep[GRAD ? D : 1];
    float ntsc[GRAD ? D : 1];
    R prod = R(1);
    Rows<D, 0, GRAD, R>::run(v, z, hit, keep, prod, ntsc);
    const bool counted = ALL_VALID ? hit : (hit && valid);
    acc.cnt += counted ? 1u : 0u;
    if constexpr (GRAD && sizeof(R) == 4 && packed_adjoint<D>()) {
        const float hv = counted ? 1.0f : 0.0f;
        const float vv = (ALL_VALID || valid) ? 1.0f : 0.0f;
        if (!zodd) {
            axpy<D, true>(acc.A, hv, z);
            axpy<D, true>(acc.B, vv, z);
        } else {
            axpy<D, false>(acc.A, hv, z);
            axpy<D, false>(acc.B, vv, z);
        }
        if (v.hl2e != 0.0f) {
            // keep_i = 1 / (1 + 2^(y_i log2(e)/h - t_i log2(e)/h)); keep holds y
            const float2 h2 = make_float2(v.hl2e, v.hl2e), one2 = make_float2(1.0f, 1.0f);
#pragma unroll
            for (int i = 0; i + 1 < D; i += 2) {
                const float2 x = __ffma2_rn(make_float2(keep[i], keep[i + 1]), h2, make_float2(ntsc[i], ntsc[i + 1]));
                const float2 u = __fadd2_rn(one2, make_float2(ex2_approx(x.x), ex2_approx(x.y)));
                keep[i] = rcp_approx(u.x);
                keep[i + 1] = rcp_approx(u.y);
            }
            if constexpr (D % 2 != 0)
                keep[D - 1] = rcp_approx(1.0f + ex2_approx(__fmaf_rn(keep[D - 1], v.hl2e, ntsc[D - 1])));
#pragma unroll
            for (int i = 0; i < D; ++i) prod *= keep[i];
            prod *= vv;
            const float2 p2 = make_float2(prod, prod), m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
            for (int i = 0; i + 1 < D; i += 2) {
                const float2 omk = __ffma2_rn(make_float2(keep[i], keep[i + 1]), m1, one2);
                const float2 g = __ffma2_rn(p2, omk, make_float2(acc.G[i], acc.G[i + 1]));
                acc.G[i] = g.x;
                acc.G[i + 1] = g.y;
            }
            if constexpr (D % 2 != 0) acc.G[D - 1] = __fmaf_rn(prod, 1.0f - keep[D - 1], acc.G[D - 1]);
        }
    } else if constexpr (GRAD) {
        const R hv = counted ? R(1) : R(0);
#pragma unroll
        for (int i = 0; i < D; ++i) acc.A[i] = fmadd(hv, z[i], acc.A[i]);
        if constexpr (ALL_VALID) {
#pragma unroll
            for (int i = 0; i < D; ++i) acc.B[i] += z[i];
        } else {
            const R vv = valid ? R(1) : R(0);
#pragma unroll
            for (int i = 0; i < D; ++i) acc.B[i] = fmadd(vv, z[i], acc.B[i]);
            prod *= vv;
        }
        if (v.hl2e != 0.0f) {
#pragma unroll
            for (int i = 0; i < D; ++i) acc.G[i] = fmadd(prod, R(1) - keep[i], acc.G[i]);
        }
    }
}

// Draws of one group: the group's Philox calls are made in order and each
// draw is evaluated as soon as its last normal exists, so at most one draw's
// normals (plus one call's) are live.
template <int D, bool GRAD, bool FAST, bool ALL_VALID, typename R>
__device__ __forceinline__ void group_draws(uint32_t call_lo, uint64_t call, const Round1& r1,
                                            uint64_t key, const SampleParams& P, uint32_t base,
                                            uint32_t ofs, uint32_t n, const TileView<D, R>& v,
                                            Acc<D, GRAD, R>& acc) {
    using S = Shape<D>;
    R z[S::kNZ];
#pragma unroll
    for (int c = 0; c < S::kNC; ++c) {
        uint4 w;
        if constexpr (FAST) w = philox_fast(call_lo + c, r1, P.rk0, P.rk1);
        else w = philox_full(call + c, key, P.rk0, P.rk1);
        normals4<R>(w, &z[4 * c]);
#pragma unroll
        for (int g = 0; g < S::kG; ++g) {
            const int last = (g + 1) * D - 1;           // last normal of draw g
            if (last >= 4 * c && last < 4 * c + 4) {
                const bool valid = ALL_VALID || ((base + g - ofs) < n);
                one_draw<D, GRAD, ALL_VALID, R>(&z[g * D], ((g * D) & 1) != 0, v, valid, acc);
            }
        }
    }
}

// All draws of one tile that this thread owns.
template <int D, bool GRAD, bool FAST, typename R>
__device__ __forceinline__ void tile_draws(const TileShared<R>& ts, const SampleParams& P,
                                           Acc<D, GRAD, R>& acc) {
    using S = Shape<D>;
    const uint64_t g_first = ts.start / S::kG;
    const uint32_t ofs = static_cast<uint32_t>(ts.start - g_first * S::kG);
    const uint32_t end = ofs + ts.n;
    const uint32_t ngroups = (end + S::kG - 1) / S::kG;
    const uint64_t call_first = g_first * static_cast<uint64_t>(S::kNC);
    const Round1 r1 = round1_consts(static_cast<uint32_t>(call_first >> 32), ts.key, P.rk0, P.rk1);
    const uint32_t call_lo0 = static_cast<uint32_t>(call_first);

    TileView<D, R> v;
    if constexpr (TileView<D, R>::kReg) {
#pragma unroll
        for (int i = 0; i < LPad<R>::rowoff(D); ++i) v.L[i] = ts.L[i];
#pragma unroll
        for (int i = 0; i < D; ++i) { v.t[i] = ts.t[i]; v.tsc[i] = ts.tsc[i]; }
    }
    v.sL = ts.L;
    v.st = ts.t;
    v.stsc = ts.tsc;
    v.hl2e = GRAD ? P.hinv_log2e : 0.0f;
    v.hinv = P.hinv;

    for (uint32_t gi = threadIdx.x; gi < ngroups; gi += blockDim.x) {
        const uint32_t base = gi * S::kG;
        const uint32_t clo = call_lo0 + gi * S::kNC;
        const uint64_t call = call_first + static_cast<uint64_t>(gi) * S::kNC;
        if (base >= ofs && base + S::kG <= end)
            group_draws<D, GRAD, FAST, true, R>(clo, call, r1, ts.key, P, base, ofs, ts.n, v, acc);
        else
            group_draws<D, GRAD, FAST, false, R>(clo, call, r1, ts.key, P, base, ofs, ts.n, v, acc);
    }
}

__device__ __forceinline__ float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += shfl_xor(v, m);
    return v;
}

// Process one tile for dimension D and fold the block's sums into the outputs.
template <int D, bool GRAD, typename R, int DHI>
__device__ __forceinline__ void process_tile(TileShared<R>& ts, const SampleParams& P,
                                             uint32_t* cred, R (*gred)[GRAD ? 3 * DHI : 1]) {
    using S = Shape<D>;
    Acc<D, GRAD, R> acc;
    acc.cnt = 0;
    if constexpr (GRAD) {
#pragma unroll
        for (int i = 0; i < D; ++i) { acc.A[i] = R(0); acc.B[i] = R(0); acc.G[i] = R(0); }
    }
    // Call indices of the tile stay below one 2^32 boundary in all but
    // astronomically large streams; use the cheaper first round there.
    {
        const uint64_t g_first = ts.start / S::kG;
        const uint64_t g_last = (ts.start + ts.n + S::kG - 1) / S::kG;
        const uint64_t c0 = g_first * S::kNC, c1 = g_last * S::kNC;
        if ((c0 >> 32) == ((c1 - 1) >> 32)) tile_draws<D, GRAD, true, R>(ts, P, acc);
        else tile_draws<D, GRAD, false, R>(ts, P, acc);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wc = __reduce_add_sync(0xffffffffu, acc.cnt);
    if (lane == 0) cred[warp] = wc;
    if constexpr (GRAD) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const R a = warp_sum(acc.A[i]);
            const R b = warp_sum(acc.B[i]);
            const R g = warp_sum(acc.G[i]);
            if (lane == 0) { gred[warp][i] = a; gred[warp][D + i] = b; gred[warp][2 * D + i] = g; }
        }
    }
    __syncthreads();
    const int nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        unsigned long long total = 0;
        for (int w = 0; w < nwarps; ++w) total += cred[w];
        if (total) atomicAdd(&P.hits[ts.design], total);
    }
    if constexpr (GRAD) {
        if (threadIdx.x < 3 * D) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += static_cast<double>(gred[w][threadIdx.x]);
            const long long fx = __double2ll_rn(s * static_cast<double>(1ull << kGradFixBits));
            atomicAdd(&P.gacc[ts.acc_off + static_cast<int64_t>(ts.batch) * 3 * D + threadIdx.x],
                      static_cast<unsigned long long>(fx));
        }
    }
}

template <int DLO, int DHI, bool GRAD, typename R>
struct Dispatch {
    __device__ __forceinline__ static void run(int d, TileShared<R>& ts, const SampleParams& P,
                                               uint32_t* cred, R (*gred)[GRAD ? 3 * DHI : 1]) {
        if (d == DLO) process_tile<DLO, GRAD, R, DHI>(ts, P, cred, gred);
        else if constexpr (DLO < DHI) Dispatch<DLO + 1, DHI, GRAD, R>::run(d, ts, P, cred, gred);
    }
};

// The persistent loop over tiles (the body of both kernel wrappers below).
template <int DLO, int DHI, bool GRAD, typename R>
__device__ __forceinline__ void sample_body(const SampleParams& P) {
    __shared__ TileShared<R> ts;
    __shared__ uint32_t cred[kMaxWarps];
    __shared__ R gred[kMaxWarps][GRAD ? 3 * DHI : 1];

    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned int tk = atomicAdd(P.ticket, 1u);
            ts.tile = tk;
            if (static_cast<int64_t>(tk) < P.n_tiles) {
                const TileRec tr = P.tiles[tk];
                const DesignRec dr = P.designs[tr.design];
                ts.start = tr.start;
                ts.n = tr.n;
                ts.design = tr.design;
                ts.batch = tr.batch;
                ts.key = dr.key;
                ts.d = dr.d;
                ts.vec_off = dr.vec_off;
                ts.acc_off = dr.acc_off;
                ts.ok = P.scen_ok[dr.scen];
                ts.scen = dr.scen;
            }
        }
        __syncthreads();
        if (static_cast<int64_t>(ts.tile) >= P.n_tiles) break;
        const int d = ts.d;
        const int64_t loff = P.L_off[ts.scen];
        // row r of the packed factor goes to padded offset rowoff(r); pads are 0
        for (int r = threadIdx.x; r < d; r += blockDim.x) {
            const int po = LPad<R>::rowoff(r), pk = r * (r + 1) / 2;
            for (int q = 0; q < LPad<R>::chunks(r) * LPad<R>::V; ++q) {
                R val = R(0);
                if (q <= r) {
                    if constexpr (sizeof(R) == 4) val = P.L32[loff + pk + q];
                    else val = P.L64[loff + pk + q];
                }
                ts.L[po + q] = val;
            }
        }
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const double tt = P.b[ts.vec_off + i] - P.mu[ts.vec_off + i];
            if (tt != tt) set_status(P.status, MCD_ENAN, ts.design);
            ts.t[i] = static_cast<R>(tt);
            ts.tsc[i] = P.hinv_log2e != 0.0f ? -(static_cast<float>(tt) * P.hinv_log2e) : 0.0f;
        }
        __syncthreads();
        if (ts.ok) Dispatch<DLO, DHI, GRAD, R>::run(d, ts, P, cred, gred);
        __syncthreads();
    }
}

template <int DLO, int DHI, bool GRAD, typename R>
__global__ void __launch_bounds__(256) sample_kernel(const __grid_constant__ SampleParams P) {
    sample_body<DLO, DHI, GRAD, R>(P);
}

// Adjoint kernels of larger d carry 3d accumulators per thread; this variant
// asks the compiler for two resident 256-thread blocks (<= 128 registers) so
// that an SM keeps 16 warps to hide the Philox and MUFU latencies.
template <int DLO, int DHI, bool GRAD, typename R>
__global__ void __launch_bounds__(256, 2) sample_kernel_2b(const __grid_constant__ SampleParams P) {
    sample_body<DLO, DHI, GRAD, R>(P);
}

// Three (<= 85 registers) and four (<= 64) resident blocks per SM, for the
// kernels where that measured faster: the mixed-dimension forward kernel
// (d = 1..10 in one launch, 1.8 %) and the adjoint at d = 1 (25 %), d = 3
// (four blocks, 1.9 %) and d = 4 (3 %).
template <int DLO, int DHI, bool GRAD, typename R>
__global__ void __launch_bounds__(256, 3) sample_kernel_3b(const __grid_constant__ SampleParams P) {
    sample_body<DLO, DHI, GRAD, R>(P);
}

template <int DLO, int DHI, bool GRAD, typename R>
__global__ void __launch_bounds__(256, 4) sample_kernel_4b(const __grid_constant__ SampleParams P) {
    sample_body<DLO, DHI, GRAD, R>(P);
}

}  // namespace mcd
