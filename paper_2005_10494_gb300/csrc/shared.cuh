// Shared-draw sampling: designs with the same scenario, stream key and draw
// range see identical draws (common random numbers), so the draws need to be
// made only once for all of them.
//
// A tile is (chunk of up to 256 * kDpt designs of one sharing group, draw
// range).  For each batch of draws the block makes the normals and y = L z
// once, with the per-design kernel's Philox / Box-Muller / transform
// arithmetic, into shared memory; then every thread tests its designs against
// every draw of the batch (broadcast shared loads).  A design's indicator is
// the per-design kernel's FP32 comparison y_i > t_i, evaluated as the sign of
// the FP32 difference t_i - y_i (an exactly equivalent test), so hit counts
// are bit-identical to it; the gradient sums differ only in FP32 rounding
// (the order of additions, and the sigmoid's exponent formed from that
// difference).  Draws outside the tile's range enter as y = -inf, z = 0,
// which no region test counts and which add nothing to any sum.
//
// The paper's two-layer estimator (Sec. 2.2, Eq. 7) has this form too: its
// outer prior samples act as designs (thresholds b - S Delta_k) that share
// one inner stream of draws.
#pragma once

#include <cstdint>

#include "mcd_internal.cuh"
#include "rng.cuh"
#include "sample.cuh"

namespace mcd {

template <int D, bool GRAD>
struct SharedShape {
    static constexpr int kDP = (D + 3) / 4 * 4;                      // padded coordinates per draw
    // designs per thread: enough to amortise the shared loads, few enough to
    // keep t (and the gradient sums) in registers
    static constexpr int kDpt = GRAD ? (D <= 4 ? 4 : (D <= 8 ? 2 : 1)) : (D <= 10 ? 4 : 2);
    static constexpr int kBD = kSharedThreads * Shape<D>::kG;        // draws per batch (one group per thread)
    // adjoint at odd d: the z row carries 1 in its padding slot d for a
    // valid draw, so the packed sum over hits, whose last pair would
    // otherwise be a scalar add, counts them in A's slot d at no extra
    // instruction; a tile has at most 2^18 draws, so the FP32 count is exact
    static constexpr bool kCnt = GRAD && (D % 2 != 0);
    static constexpr int kDA = D + (kCnt ? 1 : 0);                   // sums of A per design
    // Register layout per d, chosen by timing each d on d-dimensional
    // common-random-number grids (2048 designs x 2e6 draws), forward and
    // adjoint, against the plain layout (G in registers, draw loop unrolled
    // 4 / 8 times, normals of a group made up front, no register bound):
    // - kWide (adjoint at d = 11, 14, 16, 18, 20): the sigmoid sums G in
    //   thread-private shared memory (touched only in the warp-draws that
    //   reach the sigmoid), the draw loop unrolled twice and the kernel held
    //   to 128 registers: two blocks per SM instead of one, 5-21 % faster;
    static constexpr bool kWide = GRAD && (D == 11 || D == 14 || D == 16 || D == 18 || D == 20);
    static constexpr int kUnroll = GRAD ? (kWide ? 2 : 4) : 8;
    // - kBound2: 128 registers (two blocks per SM) for kWide, and for the
    //   forward kernel at d >= 9 except 10 and 12 (which fit two blocks
    //   anyway): 2-13 % faster;
    static constexpr bool kBound2 = kWide || (!GRAD && D >= 9 && D != 10 && D != 12);
    // - kProg (odd d >= 9): each draw's normals made just before its
    //   transform (make_batch); a group holds four draws at odd d, whose
    //   4 d normals made up front need as many registers.  It lets the
    //   d = 9 adjoint fit two blocks per SM unbounded (28 % faster) and the
    //   bounded kernels above spill less.
    static constexpr bool kProg = D >= 9 && D % 2 != 0;
    static constexpr size_t kSmem = static_cast<size_t>(kBD) * kDP * sizeof(float) * (GRAD ? 2 : 1);
};

// The batch's draws: this thread makes group `gi` (kG draws) and writes y
// (and z for the adjoint) to shared memory; `bsum` gathers z of the valid
// draws.
template <int D, bool GRAD>
__device__ __forceinline__ void make_batch(const float* __restrict__ sL, uint64_t call, uint32_t call_lo,
                                           bool fast, const Round1& r1, uint64_t key, const SampleParams& P,
                                           uint32_t base, uint32_t ofs, uint32_t n, float* sy, float* sz,
                                           float* bsum) {
    using S = Shape<D>;
    constexpr int DP = SharedShape<D, GRAD>::kDP;
    constexpr bool kProg = SharedShape<D, GRAD>::kProg;
    float z[S::kNZ];
    if constexpr (!kProg) {
#pragma unroll
        for (int c = 0; c < S::kNC; ++c) {
            uint4 w;
            if (fast) w = philox_fast(call_lo + c, r1, P.rk0, P.rk1);
            else w = philox_full(call + c, key, P.rk0, P.rk1);
            normals4<float>(w, &z[4 * c]);
        }
    }
#pragma unroll
    for (int g = 0; g < S::kG; ++g) {
        if constexpr (kProg) {
            // the Philox calls whose normals draw g is the first to use
            // (draw g takes normals g d .. g d + d - 1, four per call), made
            // just before its transform so that the normals of earlier draws
            // are dead by then
#pragma unroll
            for (int c = (g * D + 3) / 4; c < ((g + 1) * D + 3) / 4; ++c) {
                uint4 w;
                if (fast) w = philox_fast(call_lo + c, r1, P.rk0, P.rk1);
                else w = philox_full(call + c, key, P.rk0, P.rk1);
                normals4<float>(w, &z[4 * c]);
            }
        }
        const bool valid = (base + g - ofs) < n;
        float y[DP], zz[DP];
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const int row = LPad<float>::rowoff(i);
            float s = sL[row] * z[g * D];
#pragma unroll
            for (int j = 1; j <= i; ++j) s = fmadd(sL[row + j], z[g * D + j], s);
            y[i] = valid ? s : -INFINITY;
            zz[i] = valid ? z[g * D + i] : 0.0f;
            if constexpr (GRAD) bsum[i] += zz[i];
        }
#pragma unroll
        for (int i = D; i < DP; ++i) {
            y[i] = -INFINITY;
            zz[i] = (SharedShape<D, GRAD>::kCnt && i == D && valid) ? 1.0f : 0.0f;
        }
        float4* yv = reinterpret_cast<float4*>(sy + (threadIdx.x * S::kG + g) * DP);
#pragma unroll
        for (int v = 0; v < DP / 4; ++v) yv[v] = make_float4(y[4 * v], y[4 * v + 1], y[4 * v + 2], y[4 * v + 3]);
        if constexpr (GRAD) {
            float4* zv = reinterpret_cast<float4*>(sz + (threadIdx.x * S::kG + g) * DP);
#pragma unroll
            for (int v = 0; v < DP / 4; ++v) zv[v] = make_float4(zz[4 * v], zz[4 * v + 1], zz[4 * v + 2], zz[4 * v + 3]);
        }
    }
}

// The sigmoid sums G of a thread's DPT designs: registers, or (SH)
// thread-private shared-memory slots strided by the block size (`s` points
// at the thread's first slot), so that a warp's accesses hit 32 banks.
template <int D, int DPT, bool SH>
struct GSums {
    float r[SH ? 1 : DPT][SH ? 1 : D];
    float* s;
    __device__ __forceinline__ float& operator()(int q, int i) {
        if constexpr (SH) return s[(q * D + i) * kSharedThreads];
        else return r[q][i];
    }
};

// Smallest of three floats in one instruction (three-input min).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// The differences t_i - y_i, two coordinates per packed FMA: fma(y, -1, t)
// rounds the exact t - y once, which is the FP32 subtraction bit for bit.
template <int D>
__device__ __forceinline__ void diffs(const float (&t)[D], const float* y, float (&dif)[D]) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int i = 0; i + 1 < D; i += 2) {
        const float2 r = __ffma2_rn(make_float2(y[i], y[i + 1]), m1, make_float2(t[i], t[i + 1]));
        dif[i] = r.x;
        dif[i + 1] = r.y;
    }
    if constexpr (D % 2 != 0) dif[D - 1] = __fsub_rn(t[D - 1], y[D - 1]);
}

template <int DP>
__device__ __forceinline__ void load_row(const float* p, float* v) {
#pragma unroll
    for (int q = 0; q < DP / 4; ++q) {
        const float4 f = reinterpret_cast<const float4*>(p)[q];
        v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
    }
}

// Test the batch's nb draws (y, and z for the adjoint, in shared memory)
// against this thread's first NQ designs.  y_i > t_i exactly when the FP32
// difference t_i - y_i is negative: two unequal floats never subtract to
// zero (gradual underflow), rounding keeps the sign, and the infinities
// (dropped tests, draws outside the range) give +inf.  The differences go
// two coordinates per packed FMA (diffs).  Forward: the hit is the sign bit
// of the or of the differences (one three-input or per three coordinates
// instead of a compare and a predicate merge per coordinate).  Adjoint: the
// hit is a negative smallest difference (three-input minima), the sum A
// over hits takes two coordinates per packed add, and the same minimum
// gives the largest sigmoid exponent (below); the minimum is formed one
// design ahead.  The draw loop is unrolled (8 draws forward, 4 or 2 with
// the adjoint's larger bodies, SharedShape::kUnroll).
template <int D, bool GRAD, int DPT, int NQ>
__device__ __forceinline__ void test_draws(const float* sy, const float* sz, int nb, const float (&t)[DPT][D],
                                           float nhl2e, float wsk, uint32_t (&cnt)[DPT],
                                           float (&A)[DPT][GRAD ? SharedShape<D, GRAD>::kDA : 1],
                                           GSums<D, DPT, SharedShape<D, GRAD>::kWide>& G) {
    constexpr int DP = SharedShape<D, GRAD>::kDP;
    constexpr int DA = SharedShape<D, GRAD>::kDA;
    constexpr int kUnroll = SharedShape<D, GRAD>::kUnroll;
#pragma unroll kUnroll
    for (int dn = 0; dn < nb; ++dn) {
        float y[DP];
        load_row<DP>(sy + dn * DP, y);
        float zz[GRAD ? DP : 4];
        if constexpr (GRAD) load_row<DP>(sz + dn * DP, zz);
        // adjoint: each design's smallest difference is formed one design
        // ahead (design q + 1's before design q's vote and branch), so that
        // two designs' dependent chains share a basic block
        float dnext = 0.0f;
        if constexpr (GRAD) {
            float d0[D];
            diffs<D>(t[0], y, d0);
            dnext = d0[0];
#pragma unroll
            for (int i = 1; i < D; i += 2) dnext = i + 1 < D ? fmin3(dnext, d0[i], d0[i + 1]) : fminf(dnext, d0[i]);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float dif[D];
            if constexpr (!GRAD) {
                diffs<D>(t[q], y, dif);
                uint32_t sgn = 0u;
#pragma unroll
                for (int i = 0; i < D; ++i) sgn |= __float_as_uint(dif[i]);
                cnt[q] += sgn >> 31;
            } else {
                const float dmin = dnext;
                if (q + 1 < NQ) {
                    float dn1[D];
                    diffs<D>(t[q + 1 < NQ ? q + 1 : q], y, dn1);   // (index kept in range for the compiler)
                    dnext = dn1[0];
#pragma unroll
                    for (int i = 1; i < D; i += 2) dnext = i + 1 < D ? fmin3(dnext, dn1[i], dn1[i + 1]) : fminf(dnext, dn1[i]);
                }
                const bool hit = dmin < 0.0f;
                if constexpr (!SharedShape<D, GRAD>::kCnt) cnt[q] += hit ? 1u : 0u;
                // sum A over the hits (adding z, or nothing, as the FMA
                // with a 0/1 factor does), and the count in slot d
                if (hit) {
#pragma unroll
                    for (int i = 0; i + 1 < DA; i += 2) {
                        const float2 a = __fadd2_rn(make_float2(A[q][i], A[q][i + 1]), make_float2(zz[i], zz[i + 1]));
                        A[q][i] = a.x;
                        A[q][i + 1] = a.y;
                    }
                    if constexpr (DA % 2 != 0) A[q][DA - 1] = __fadd_rn(A[q][DA - 1], zz[DA - 1]);
                }
                {
                    // x_i = (y_i - t_i) log2(e) / h = (t_i - y_i) nhl2e, the
                    // exponent of the sigmoid; the largest is xm = dmin nhl2e
                    // (nhl2e < 0).  wsk = 25.03 / |nhl2e| (to FP32
                    // rounding), so |dmin| >= wsk gives |xm| > 25.02.  When xm < -25 (dmin
                    // >= wsk) every x_i < -25 and the draw adds exactly zero
                    // to every G_i (2^x_i < 2^-25 vanishes in 1 + 2^x_i, so
                    // every keep_i = 1).  When xm > 25 (dmin <= -wsk), keep_k
                    // = 1 / (1 + 2^xm) < 2^-25 bounds the product, so every
                    // contribution prod (1 - keep_i) is below 3e-8: such
                    // draws are skipped too, which moves G / N by less than
                    // 3e-8 (the derivative by less than 3e-8 / h, far below
                    // its Monte Carlo error).  A warp takes the exponentials
                    // only when some lane's draw has |dmin| < wsk: one
                    // comparison of a magnitude.  wsk < 0 (no sigmoid sums)
                    // never passes.
                    if (__any_sync(0xffffffffu, fabsf(dmin) < wsk)) {
                        diffs<D>(t[q], y, dif);                    // again, in the rare branch
                        float keep[D], prod = 1.0f;
                        const float2 nh2 = make_float2(nhl2e, nhl2e), one2 = make_float2(1.0f, 1.0f);
#pragma unroll
                        for (int i = 0; i + 1 < D; i += 2) {
                            const float2 x = __fmul2_rn(make_float2(dif[i], dif[i + 1]), nh2);
                            const float2 u = __fadd2_rn(one2, make_float2(ex2_approx(x.x), ex2_approx(x.y)));
                            keep[i] = rcp_approx(u.x);
                            keep[i + 1] = rcp_approx(u.y);
                        }
                        if constexpr (D % 2 != 0) keep[D - 1] = rcp_approx(1.0f + ex2_approx(dif[D - 1] * nhl2e));
#pragma unroll
                        for (int i = 0; i < D; ++i) prod *= keep[i];
                        const float2 pr2 = make_float2(prod, prod), m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
                        for (int i = 0; i + 1 < D; i += 2) {
                            const float2 omk = __ffma2_rn(make_float2(keep[i], keep[i + 1]), m1, one2);
                            const float2 g = __ffma2_rn(pr2, omk, make_float2(G(q, i), G(q, i + 1)));
                            G(q, i) = g.x;
                            G(q, i + 1) = g.y;
                        }
                        if constexpr (D % 2 != 0) G(q, D - 1) = fmadd(prod, 1.0f - keep[D - 1], G(q, D - 1));
                    }
                }
            }
        }
    }
}

// The persistent loop over shared tiles (the body of both kernel wrappers below).
template <int D, bool GRAD>
__device__ __forceinline__ void shared_body(const SampleParams& P, const SharedTile* __restrict__ tiles,
                                            const uint32_t* __restrict__ list) {
    using S = Shape<D>;
    using SS = SharedShape<D, GRAD>;
    constexpr int DPT = SS::kDpt, DP = SS::kDP;
    extern __shared__ __align__(16) float sh[];
    float* sy = sh;                                   // [kBD][kDP]
    float* sz = sh + SS::kBD * DP;                    // [kBD][kDP], adjoint only
    __shared__ __align__(16) float sL[LPad<float>::rowoff(D) + 4];
    __shared__ float sB[kMaxWarps][GRAD ? D : 1];
    __shared__ unsigned int s_tile;
    __shared__ float sGw[SS::kWide ? kSharedThreads * DPT * D : 1];   // G slots (kWide)

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(P.ticket, 1u);
        __syncthreads();
        const unsigned int tk = s_tile;
        if (static_cast<int64_t>(tk) >= P.n_tiles) break;
        const SharedTile tl = tiles[tk];
        const int ok = P.scen_ok[tl.scen];
        const int64_t loff = P.L_off[tl.scen];
        for (int r = threadIdx.x; r < D; r += blockDim.x) {
            const int po = LPad<float>::rowoff(r), pk = r * (r + 1) / 2;
            for (int q = 0; q < LPad<float>::chunks(r) * LPad<float>::V; ++q)
                sL[po + q] = q <= r ? P.L32[loff + pk + q] : 0.0f;
        }
        // this thread's designs (list positions threadIdx.x + q * blockDim.x)
        // and their thresholds; a missing design gets t = +inf (never a hit)
        const int nq = static_cast<int>((tl.list_cnt + blockDim.x - 1) / blockDim.x);   // block-uniform
        int dsg[DPT];
        float t[DPT][D];
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const uint32_t li = threadIdx.x + q * blockDim.x;
            dsg[q] = li < tl.list_cnt ? static_cast<int>(list[tl.list_off + li]) : -1;
            const int64_t vo = dsg[q] >= 0 ? P.designs[dsg[q]].vec_off : 0;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const double tt = dsg[q] >= 0 ? P.b[vo + i] - P.mu[vo + i] : 0.0;
                if (dsg[q] >= 0 && tt != tt) set_status(P.status, MCD_ENAN, dsg[q]);
                t[q][i] = dsg[q] >= 0 ? static_cast<float>(tt) : INFINITY;
            }
        }
        __syncthreads();                              // sL complete
        if (!ok) continue;                            // block-uniform; the next ticket read is behind a barrier

        const uint64_t g_first = tl.start / S::kG;
        const uint32_t ofs = static_cast<uint32_t>(tl.start - g_first * S::kG);
        const uint32_t ngroups = (ofs + tl.n + S::kG - 1) / S::kG;
        const uint64_t call_first = g_first * static_cast<uint64_t>(S::kNC);
        const uint64_t call_last = (g_first + ngroups) * static_cast<uint64_t>(S::kNC) - 1;
        const bool fast = (call_first >> 32) == (call_last >> 32);
        // the sigmoid's exponent scale -log2(e)/h, and the half-width
        // 25.03 h / log2(e) of the window of differences in which its work
        // is taken (test_draws; -1 when the sigmoid sums are off)
        const float nhl2e = GRAD ? -P.hinv_log2e : 0.0f;
        const float wsk = GRAD ? P.sig_skip_w : -1.0f;
        const Round1 r1 = round1_consts(static_cast<uint32_t>(call_first >> 32), tl.key, P.rk0, P.rk1);

        uint32_t cnt[DPT];
        float A[DPT][GRAD ? SS::kDA : 1], bsum[GRAD ? D : 1];
        GSums<D, DPT, SS::kWide> G;
        G.s = sGw + threadIdx.x;
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            cnt[q] = 0;
#pragma unroll
            for (int i = 0; i < (GRAD ? SS::kDA : 1); ++i) A[q][i] = 0.0f;
#pragma unroll
            for (int i = 0; i < D; ++i)
                if constexpr (GRAD) G(q, i) = 0.0f;
        }
#pragma unroll
        for (int i = 0; i < (GRAD ? D : 1); ++i) bsum[i] = 0.0f;

        for (uint32_t g0 = 0; g0 < ngroups; g0 += blockDim.x) {
            const uint32_t gi = g0 + threadIdx.x;
            make_batch<D, GRAD>(sL, call_first + static_cast<uint64_t>(gi) * S::kNC,
                                static_cast<uint32_t>(call_first) + gi * S::kNC, fast, r1, tl.key, P,
                                gi * S::kG, ofs, gi < ngroups ? tl.n : 0u, sy, sz, bsum);
            __syncthreads();
            const int nb = static_cast<int>(min(static_cast<uint32_t>(SS::kBD), (ngroups - g0) * S::kG));
            // nq is block-uniform: one branch per batch picks the loop for
            // exactly nq designs per thread
            if (nq >= DPT) test_draws<D, GRAD, DPT, DPT>(sy, sz, nb, t, nhl2e, wsk, cnt, A, G);
            else if constexpr (DPT > 1) {
                if (nq == 1) test_draws<D, GRAD, DPT, 1>(sy, sz, nb, t, nhl2e, wsk, cnt, A, G);
                else if constexpr (DPT > 2) {
                    if (nq == 2) test_draws<D, GRAD, DPT, 2>(sy, sz, nb, t, nhl2e, wsk, cnt, A, G);
                    else if constexpr (DPT > 3) test_draws<D, GRAD, DPT, 3>(sy, sz, nb, t, nhl2e, wsk, cnt, A, G);
                }
            }
            __syncthreads();                          // the next batch rewrites sy / sz
        }

        // hits: each design of the tile belongs to exactly one thread
        if constexpr (SS::kCnt) {
#pragma unroll
            for (int q = 0; q < DPT; ++q) cnt[q] = static_cast<uint32_t>(A[q][D]);
        }
#pragma unroll
        for (int q = 0; q < DPT; ++q)
            if (dsg[q] >= 0 && cnt[q]) atomicAdd(&P.hits[dsg[q]], static_cast<unsigned long long>(cnt[q]));
        if constexpr (GRAD) {
            // the sum of z over the tile's draws is common to all its designs
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const float w = warp_sum(bsum[i]);
                if (lane == 0) sB[warp][i] = w;
            }
            __syncthreads();
            const double fix = static_cast<double>(1ull << kGradFixBits);
#pragma unroll
            for (int q = 0; q < DPT; ++q) {
                if (dsg[q] < 0) continue;
                unsigned long long* slot = P.gacc + P.designs[dsg[q]].acc_off + static_cast<int64_t>(tl.batch) * 3 * D;
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    double s = 0.0;
                    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += static_cast<double>(sB[w][i]);
                    atomicAdd(slot + i, static_cast<unsigned long long>(__double2ll_rn(static_cast<double>(A[q][i]) * fix)));
                    atomicAdd(slot + D + i, static_cast<unsigned long long>(__double2ll_rn(s * fix)));
                    atomicAdd(slot + 2 * D + i, static_cast<unsigned long long>(__double2ll_rn(static_cast<double>(G(q, i)) * fix)));
                }
            }
        }
        // the next iteration's ticket read sits behind a barrier, so sB and
        // the per-tile shared state are not overwritten early
    }
}

template <int D, bool GRAD>
__global__ void __launch_bounds__(kSharedThreads) shared_kernel(const __grid_constant__ SampleParams P,
                                                                const SharedTile* __restrict__ tiles,
                                                                const uint32_t* __restrict__ list) {
    shared_body<D, GRAD>(P, tiles, list);
}

// The adjoint at d <= 3 with three resident blocks per SM (at most 85
// registers a thread): 24 warps instead of 16 hide more of the exponential
// and shared-load latencies, which measured 8.7 % faster on the d=3 grid
// than two blocks although ptxas spills a few registers.
template <int D, bool GRAD>
__global__ void __launch_bounds__(kSharedThreads, 3) shared_kernel_3b(const __grid_constant__ SampleParams P,
                                                                      const SharedTile* __restrict__ tiles,
                                                                      const uint32_t* __restrict__ list) {
    shared_body<D, GRAD>(P, tiles, list);
}

// Two resident blocks per SM (at most 128 registers a thread), at the
// dimensions SharedShape::kBound2 lists.
template <int D, bool GRAD>
__global__ void __launch_bounds__(kSharedThreads, 2) shared_kernel_2b(const __grid_constant__ SampleParams P,
                                                                      const SharedTile* __restrict__ tiles,
                                                                      const uint32_t* __restrict__ list) {
    shared_body<D, GRAD>(P, tiles, list);
}

template <int D, bool GRAD>
const void* shared_fn() {
    if constexpr (GRAD && D <= 3) return reinterpret_cast<const void*>(&shared_kernel_3b<D, GRAD>);
    else if constexpr (SharedShape<D, GRAD>::kBound2) return reinterpret_cast<const void*>(&shared_kernel_2b<D, GRAD>);
    else return reinterpret_cast<const void*>(&shared_kernel<D, GRAD>);
}

template <int D, bool GRAD>
size_t shared_smem() { return SharedShape<D, GRAD>::kSmem; }

}  // namespace mcd
