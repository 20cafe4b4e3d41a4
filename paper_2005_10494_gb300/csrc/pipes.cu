// Instruction-throughput microbenchmarks: the issue rate of each instruction
// class the sampling kernels are built from (32x32->64 multiply, three-input
// logic, FP32 FMA, each MUFU function, broadcast shared-memory loads), in
// operations per SM clock.  Together with the per-draw operation counts of
// the estimator they give the min-over-pipes bound on draw-evaluations per
// second.
//
// Each thread runs independent dependency chains of the measured instruction
// (eight; four for the shared loads, two Philox states), written in inline
// PTX so that the class is fixed.  Enough warps are resident to hide latency
// (8 blocks of 256 threads per SM), and every block reads the SM's cycle
// counter after a barrier on both sides of the loop.  Operations per SM
// clock = (the blocks' operations on one SM) / (last end - first start on
// that SM), a figure that does not depend on the clock frequency.
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "mcd_internal.cuh"
#include "pipes.cuh"
#include "rng.cuh"

namespace mcd {

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ uint32_t sm_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

template <int OP>
__device__ __forceinline__ float mufu_op(float x) {
    float y;
    if constexpr (OP == MCD_PIPE_LG2) asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if constexpr (OP == MCD_PIPE_SQRT) asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if constexpr (OP == MCD_PIPE_SIN) asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if constexpr (OP == MCD_PIPE_COS) asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if constexpr (OP == MCD_PIPE_EX2) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void lop3_ring(uint32_t* x, int n, uint32_t m) {
    // x_i <- x_i ^ x_{i+1} ^ m: each chain feeds its neighbour, so no
    // algebraic cancellation is possible across steps.
#pragma unroll
    for (int i = 0; i < n; ++i)
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[i]) : "r"(x[(i + 1) % n]), "r"(m));
}

__device__ __forceinline__ void ffma_ring(float* f, int n, float c) {
#pragma unroll
    for (int i = 0; i < n; ++i)
        asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[i]) : "f"(c), "f"(f[(i + 1) % n]));
}

// The packed form: one fma.rn.f32x2 does two FP32 FMAs on a register pair.
__device__ __forceinline__ void ffma2_ring(unsigned long long* f, int n, unsigned long long c) {
#pragma unroll
    for (int i = 0; i < n; ++i)
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(f[i]) : "l"(c), "l"(f[(i + 1) % n]));
}

// Throughput kernel for instruction class OP; every step is kChains
// instructions of that class (MCD_PIPE_FFMA2 counts packed instructions,
// two FMAs each; MCD_PIPE_MIXED: half FFMA, half LOP3;
// MCD_PIPE_PHILOX: two calls' rounds 2..10, counted as their 36 wide
// multiplies).
template <int OP>
__global__ void __launch_bounds__(kPipeThreads, kPipeBlocksPerSM)
pipe_kernel(int iters, uint32_t m, float c, PipeKeys keys, uint32_t* __restrict__ sink, long long* __restrict__ t0,
            long long* __restrict__ t1, int* __restrict__ smid) {
    __shared__ uint32_t red[kPipeThreads];
    __shared__ __align__(16) uint32_t tab[64 * 4];
    const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t fold = 0;
    if constexpr (OP == MCD_PIPE_LDS128) {
        // 64 entries of 16 bytes; every word of entry e holds the shared
        // address of entry (7e + 1) mod 64, so a chain of loads stays inside
        // the table.
        const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(tab));
        for (int j = threadIdx.x; j < 64 * 4; j += blockDim.x)
            tab[j] = base + 16u * (((static_cast<uint32_t>(j) >> 2) * 7u + 1u) & 63u);
    }
    __syncthreads();
    const long long start = clock64();
    if constexpr (OP == MCD_PIPE_MUL_WIDE) {
        uint64_t a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = (static_cast<uint64_t>(gid) << 8 | i) * 0x9E3779B97F4A7C15ull + m;
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int i = 0; i < kChains; ++i)
                asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a[i]) : "r"(static_cast<uint32_t>(a[i])), "r"(m));
        }
#pragma unroll
        for (int i = 0; i < kChains; ++i) fold ^= static_cast<uint32_t>(a[i] >> 32) ^ static_cast<uint32_t>(a[i]);
    } else if constexpr (OP == MCD_PIPE_MAD_LO) {
        uint32_t x[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = gid * 8u + i + m;
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int i = 0; i < kChains; ++i)
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(m), "r"(x[(i + 1) % kChains]));
        }
#pragma unroll
        for (int i = 0; i < kChains; ++i) fold ^= x[i];
    } else if constexpr (OP == MCD_PIPE_LOP3) {
        uint32_t x[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = gid * 8u + i + m;
        for (int k = 0; k < iters; ++k) lop3_ring(x, kChains, m);
#pragma unroll
        for (int i = 0; i < kChains; ++i) fold ^= x[i];
    } else if constexpr (OP == MCD_PIPE_FFMA) {
        float f[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) f[i] = static_cast<float>(gid & 1023u) * 1e-3f + i;
        for (int k = 0; k < iters; ++k) ffma_ring(f, kChains, c);
#pragma unroll
        for (int i = 0; i < kChains; ++i) fold ^= __float_as_uint(f[i]);
    } else if constexpr (OP == MCD_PIPE_FFMA2) {
        unsigned long long f[kChains];
        const float c2[2] = {c, c};
        unsigned long long cc;
        memcpy(&cc, c2, 8);
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            const float v[2] = {static_cast<float>(gid & 1023u) * 1e-3f + i, static_cast<float>(i) - 0.5f};
            memcpy(&f[i], v, 8);
        }
        for (int k = 0; k < iters; ++k) ffma2_ring(f, kChains, cc);
#pragma unroll
        for (int i = 0; i < kChains; ++i) fold ^= static_cast<uint32_t>(f[i]) ^ static_cast<uint32_t>(f[i] >> 32);
    } else if constexpr (OP == MCD_PIPE_LDS128) {
        // warp-uniform addresses: each load is one broadcast transaction.
        // Four chains, two loads each per step (every load writes four
        // registers, so eight chains would not fit the register budget).
        constexpr int NC = kChains / 2;
        uint32_t a[NC];
        const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(tab));
#pragma unroll
        for (int i = 0; i < NC; ++i) a[i] = base + 16u * ((i * 5u + (m & 7u)) & 63u);
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int rep = 0; rep < 2; ++rep) {
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    uint32_t w1, w2, w3;
                    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                                 : "=r"(a[i]), "=r"(w1), "=r"(w2), "=r"(w3) : "r"(a[i]));
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NC; ++i) fold ^= a[i];
    } else if constexpr (OP == MCD_PIPE_PHILOX) {
        // rounds 2..10 of Philox4x32-10 exactly as the sampling kernels run
        // them (18 wide multiplies per call), on two independent states
        uint32_t x[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int q = 0; q < 4; ++q) x[h][q] = gid * 8u + 4u * h + q + m;
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint4 w = philox_rounds_2_10(x[h][0], x[h][1], x[h][2], x[h][3], keys.rk0, keys.rk1);
                x[h][0] = w.x; x[h][1] = w.y; x[h][2] = w.z; x[h][3] = w.w;
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) fold ^= x[h][0] ^ x[h][1] ^ x[h][2] ^ x[h][3];
    } else if constexpr (OP == MCD_PIPE_MIXED) {
        float f[kChains / 2];
        uint32_t x[kChains / 2];
#pragma unroll
        for (int i = 0; i < kChains / 2; ++i) {
            f[i] = static_cast<float>(gid & 1023u) * 1e-3f + i;
            x[i] = gid * 8u + i + m;
        }
        for (int k = 0; k < iters; ++k) {
            ffma_ring(f, kChains / 2, c);
            lop3_ring(x, kChains / 2, m);
        }
#pragma unroll
        for (int i = 0; i < kChains / 2; ++i) fold ^= __float_as_uint(f[i]) ^ x[i];
    } else {
        float f[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) f[i] = 0.25f + static_cast<float>(gid & 1023u) * 1e-4f + 0.01f * i;
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) {
                f[i] = mufu_op<OP>(f[i]);
                // rcp(rcp(x)) = x may be folded away: an FP32 add (on the
                // FMA pipe, far from limiting) after each rcp breaks the
                // involution.
                if constexpr (OP == MCD_PIPE_RCP) asm volatile("add.f32 %0, %0, %1;" : "+f"(f[i]) : "f"(c));
            }
        }
#pragma unroll
        for (int i = 0; i < kChains; ++i) fold ^= __float_as_uint(f[i]);
    }
    // The shared store orders the loop before the closing barrier and the
    // second clock read.
    red[threadIdx.x] = fold;
    __syncthreads();
    const long long end = clock64();
    if (threadIdx.x == 0) {
        t0[blockIdx.x] = start;
        t1[blockIdx.x] = end;
        smid[blockIdx.x] = static_cast<int>(sm_id());
    }
    sink[gid] = red[(threadIdx.x + 1) % kPipeThreads];
}

}  // namespace

int pipe_ops_per_step(int op) { return op == MCD_PIPE_PHILOX ? 2 * 18 : 8; }

cudaError_t launch_pipe(int op, int iters, int blocks, uint32_t m, float c, uint32_t* sink, long long* t0,
                        long long* t1, int* smid, cudaStream_t s) {
    const dim3 g(blocks), b(kPipeThreads);
    PipeKeys keys;
    for (int r = 0; r < 10; ++r) {
        keys.rk0[r] = m + static_cast<uint32_t>(r) * kPhiloxW0;
        keys.rk1[r] = ~m + static_cast<uint32_t>(r) * kPhiloxW1;
    }
    switch (op) {
        case MCD_PIPE_MUL_WIDE: pipe_kernel<MCD_PIPE_MUL_WIDE><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_MAD_LO: pipe_kernel<MCD_PIPE_MAD_LO><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_LOP3: pipe_kernel<MCD_PIPE_LOP3><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_FFMA: pipe_kernel<MCD_PIPE_FFMA><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_FFMA2: pipe_kernel<MCD_PIPE_FFMA2><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_LG2: pipe_kernel<MCD_PIPE_LG2><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_SQRT: pipe_kernel<MCD_PIPE_SQRT><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_SIN: pipe_kernel<MCD_PIPE_SIN><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_COS: pipe_kernel<MCD_PIPE_COS><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_EX2: pipe_kernel<MCD_PIPE_EX2><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_RCP: pipe_kernel<MCD_PIPE_RCP><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_MIXED: pipe_kernel<MCD_PIPE_MIXED><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_LDS128: pipe_kernel<MCD_PIPE_LDS128><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        case MCD_PIPE_PHILOX: pipe_kernel<MCD_PIPE_PHILOX><<<g, b, 0, s>>>(iters, m, c, keys, sink, t0, t1, smid); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mcd
