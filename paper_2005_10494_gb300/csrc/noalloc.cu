// mc_design_eval_noalloc: the estimate of mc_design_eval for the designs of
// one scenario, computed without allocating any memory.
//
// Some callers cannot allocate device memory when they evaluate designs:
// code that reserves all of the GPU's memory up front in its own pool (a
// stray cudaMalloc there can fail or fragment the pool), loops that must not
// take the implicit device synchronisation of cudaMalloc / cudaFree, and
// processes whose allocator is owned by another runtime.  For them this
// entry point keeps its scratch -- the per-design hit counters, the stream
// keys and the Cholesky factor -- in one fixed-size array in device memory
// that the library declares statically; every GPU that loads the library
// holds it until the process exits.
//
// The hits it returns are bit-identical to mc_design_eval's for the same
// inputs: the sampling of each tile is the same device code (sample.cuh),
// only the tile schedule is computed in the kernel instead of planned.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "mcd_internal.cuh"
#include "sample.cuh"

namespace mcd {

namespace {

constexpr int kNoAllocMaxDesigns = 16384;

// Scratch layout (bytes): hit counters | keys | FP32 factor | FP64 factor | flag.
struct NoAllocScratch {
    unsigned long long hits[kNoAllocMaxDesigns];
    uint64_t keys[kNoAllocMaxDesigns];
    float L32[kMaxTri];
    double L64[kMaxTri];
    int32_t ok;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Per device, looked up once: the device address of the scratch array, the
// SM count and the resident blocks per SM of each dimension's kernel.
NoAllocScratch* g_scratch_ptr[64] = {};
int g_sm_count[64] = {};
int g_blocks_per_sm[64][kMaxD + 1] = {};
std::mutex g_scratch_mu;

// Sigma = L L^T for the one scenario (FP64, lower triangle read), FP32 copy.
__global__ void noalloc_cholesky_kernel(const double* __restrict__ Sigma, int d, NoAllocScratch* sc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    bool good = true;
    for (int i = 0; i < d && good; ++i) {
        for (int j = 0; j <= i; ++j) {
            double sum = Sigma[i * d + j];
            for (int k = 0; k < j; ++k) sum -= sc->L64[i * (i + 1) / 2 + k] * sc->L64[j * (j + 1) / 2 + k];
            if (i == j) {
                if (!(sum > 0.0) || !isfinite(sum)) { good = false; break; }
                sc->L64[i * (i + 1) / 2 + i] = sqrt(sum);
            } else {
                sc->L64[i * (i + 1) / 2 + j] = sum / sc->L64[j * (j + 1) / 2 + j];
            }
        }
    }
    for (int q = 0; q < d * (d + 1) / 2; ++q) sc->L32[q] = static_cast<float>(sc->L64[q]);
    sc->ok = good ? 1 : 0;
}

// Persistent sampling over tiles numbered design-major: tile t covers draws
// [c T, min(N, (c+1) T)) of design t / tiles_per_design, c = t % tiles_per_design.
template <int D>
__global__ void __launch_bounds__(256) noalloc_sample_kernel(const __grid_constant__ SampleParams P,
                                                             NoAllocScratch* sc, int32_t n_design,
                                                             uint64_t n_draws, int64_t tile_draws,
                                                             int64_t tiles_per_design) {
    __shared__ TileShared<float> ts;
    __shared__ uint32_t cred[kMaxWarps];
    __shared__ float gred[kMaxWarps][1];
    const int64_t n_tiles = static_cast<int64_t>(n_design) * tiles_per_design;
    if (!sc->ok) return;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t j = t / tiles_per_design, c = t % tiles_per_design;
        if (threadIdx.x == 0) {
            ts.start = static_cast<uint64_t>(c) * tile_draws;
            const uint64_t rem = n_draws - ts.start;
            ts.n = static_cast<uint32_t>(rem < static_cast<uint64_t>(tile_draws) ? rem : tile_draws);
            ts.design = static_cast<uint32_t>(j);
            ts.batch = 0;
            ts.key = sc->keys[j];
            ts.d = D;
            ts.vec_off = j * D;
            ts.acc_off = 0;
            ts.ok = 1;
            ts.scen = 0;
        }
        for (int r = threadIdx.x; r < D; r += blockDim.x) {
            const int po = LPad<float>::rowoff(r), pk = r * (r + 1) / 2;
            for (int q = 0; q < LPad<float>::chunks(r) * LPad<float>::V; ++q)
                ts.L[po + q] = q <= r ? sc->L32[pk + q] : 0.0f;
        }
        for (int i = threadIdx.x; i < D; i += blockDim.x) {
            const double tt = P.b[j * D + i] - P.mu[j * D + i];
            ts.t[i] = static_cast<float>(tt);
            ts.tsc[i] = 0.0f;
        }
        __syncthreads();
        process_tile<D, false, float, D>(ts, P, cred, gred);
        __syncthreads();
    }
}

__global__ void noalloc_finalize_kernel(const NoAllocScratch* sc, int32_t n_design, int d, uint64_t N,
                                        const double* __restrict__ mu, const double* __restrict__ b,
                                        int32_t region, uint64_t* hits, double* p, double* se) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_design) return;
    bool bad = !sc->ok;
    for (int i = 0; i < d; ++i) {
        const double tt = b[static_cast<int64_t>(j) * d + i] - mu[static_cast<int64_t>(j) * d + i];
        if (tt != tt) bad = true;
    }
    const uint64_t h_any = sc->hits[j];
    const bool any = region == MCD_ANY_EXCEEDS;
    const double pa = N ? static_cast<double>(h_any) / static_cast<double>(N) : 0.0;
    const double pv = any ? pa : (N ? 1.0 - pa : 0.0);
    if (hits) hits[j] = bad ? 0 : (any ? h_any : N - h_any);
    if (p) p[j] = bad ? NAN : pv;
    if (se) se[j] = bad ? NAN : (N ? sqrt(pv * (1.0 - pv) / static_cast<double>(N)) : 0.0);
}

template <int D>
cudaError_t launch_noalloc_sample(const SampleParams& P, NoAllocScratch* sc, int32_t J, uint64_t N, int64_t T,
                                  int64_t tpd, int sms, int device, cudaStream_t stream) {
    int bps;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        bps = g_blocks_per_sm[device][D];
    }
    if (bps == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, noalloc_sample_kernel<D>, 256, 0);
        if (e != cudaSuccess) return e;
        bps = std::max(bps, 1);
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        g_blocks_per_sm[device][D] = bps;
    }
    const int64_t n_tiles = static_cast<int64_t>(J) * tpd;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(n_tiles, static_cast<int64_t>(std::max(bps, 1)) * sms));
    noalloc_sample_kernel<D><<<static_cast<unsigned>(grid), 256, 0, stream>>>(P, sc, J, N, T, tpd);
    return cudaGetLastError();
}

template <int D>
cudaError_t dispatch_noalloc(int d, const SampleParams& P, NoAllocScratch* sc, int32_t J, uint64_t N, int64_t T,
                             int64_t tpd, int sms, int device, cudaStream_t stream) {
    if (d == D) return launch_noalloc_sample<D>(P, sc, J, N, T, tpd, sms, device, stream);
    if constexpr (D < kMaxD) return dispatch_noalloc<D + 1>(d, P, sc, J, N, T, tpd, sms, device, stream);
    return cudaErrorInvalidValue;
}

}  // namespace

}  // namespace mcd

using namespace mcd;

extern "C" mcd_status mc_design_eval_noalloc(int device, const mcd_problem* prob, uint64_t seed, uint64_t* hits,
                                             double* p, double* se, mcd_stream stream) {
    if (!prob || device < 0 || device >= 64) return MCD_EINVAL;
    const int32_t J = prob->n_design;
    if (prob->n_scen != 1 || !prob->scen_d) return MCD_EINVAL;
    const int d = prob->scen_d[0];
    if (d < 1 || d > MCD_MAX_D) return MCD_EUNSUPPORTED;
    if (J < 0 || J > kNoAllocMaxDesigns) return MCD_EINVAL;      // scratch holds 16384 designs
    if (prob->region != MCD_ANY_EXCEEDS && prob->region != MCD_ALL_BELOW) return MCD_EINVAL;
    if (!prob->Sigma || (J > 0 && (!prob->mu || !prob->b || !prob->n_draws || !prob->key || !prob->design_scen)))
        return MCD_EINVAL;
    const uint64_t N = J > 0 ? prob->n_draws[0] : 0;
    for (int32_t j = 0; j < J; ++j) {
        if (prob->design_scen[j] != 0 || prob->n_draws[j] != N) return MCD_EINVAL;   // one scenario, equal N
        if (prob->draw_begin && prob->draw_begin[j] != 0) return MCD_EINVAL;
    }
    if (N > (1ull << 62) / static_cast<uint64_t>(d)) return MCD_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return MCD_ECUDA;
    // Set-up on the first call for this device: the device address of the
    // static scratch array (host code may not use the array's name directly)
    // and the SM count.
    NoAllocScratch* sc;
    int sms;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[device]) {
            void* ptr = nullptr;
            int count = 0;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr ||
                cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
                cudaGetLastError();
                return MCD_ECUDA;
            }
            g_sm_count[device] = std::max(count, 1);
            g_scratch_ptr[device] = static_cast<NoAllocScratch*>(ptr);
        }
        sc = g_scratch_ptr[device];
        sms = g_sm_count[device];
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (J == 0) return MCD_OK;
    // the counters must start at zero; the keys of this call replace the last call's
    char* base = reinterpret_cast<char*>(sc);
    unsigned long long* d_hits = reinterpret_cast<unsigned long long*>(base + offsetof(NoAllocScratch, hits));
    uint64_t* d_keys = reinterpret_cast<uint64_t*>(base + offsetof(NoAllocScratch, keys));
    if (cudaMemsetAsync(d_hits, 0, sizeof(unsigned long long) * J, s) != cudaSuccess) return MCD_ECUDA;
    if (cudaMemcpyAsync(d_keys, prob->key, sizeof(uint64_t) * J, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MCD_ECUDA;
    noalloc_cholesky_kernel<<<1, 32, 0, s>>>(prob->Sigma, d, sc);
    if (cudaGetLastError() != cudaSuccess) return MCD_ECUDA;
    if (N > 0) {
        SampleParams P;
        memset(&P, 0, sizeof(P));
        P.mu = prob->mu;
        P.b = prob->b;
        P.hits = d_hits;
        for (int r = 0; r < 10; ++r) {
            P.rk0[r] = static_cast<uint32_t>(seed) + static_cast<uint32_t>(r) * kPhiloxW0;
            P.rk1[r] = static_cast<uint32_t>(seed >> 32) + static_cast<uint32_t>(r) * kPhiloxW1;
        }
        const int g = (d % 4 == 0) ? 1 : ((d % 2 == 0) ? 2 : 4);
        const double cost = 17.0 * d + 0.5 * d * (d + 1) + 6.0;
        const int64_t T = std::max<int64_t>(1, std::llround(32768.0 / cost / g)) * g * 256;
        const int64_t tpd = static_cast<int64_t>((N + T - 1) / T);
        if (dispatch_noalloc<1>(d, P, sc, J, N, T, tpd, sms, device, s) != cudaSuccess) return MCD_ECUDA;
    }
    noalloc_finalize_kernel<<<(J + 127) / 128, 128, 0, s>>>(sc, J, d, N, prob->mu, prob->b, prob->region, hits, p, se);
    if (cudaGetLastError() != cudaSuccess) return MCD_ECUDA;
    return MCD_OK;
}
