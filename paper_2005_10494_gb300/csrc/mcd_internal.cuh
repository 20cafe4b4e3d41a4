// Internal declarations shared by the mcdesign CUDA sources (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mcdesign.h"

namespace mcd {

constexpr int kMaxD = MCD_MAX_D;
constexpr int kMaxTri = kMaxD * (kMaxD + 1) / 2;   // packed lower triangle
constexpr int kGradFixBits = 28;                   // fixed point of the gradient sums
constexpr int kMaxBatches = 32;                    // batch-means batches per design
constexpr int kMixedMaxD = 10;                     // one-launch mixed-dimension kernel covers 1..10

// Philox4x32-10 constants (Salmon, Moraes, Dror, Shaw, SC'11).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// One design as the sampling kernels see it.
struct DesignRec {
    uint64_t key;        // stream key
    int64_t  vec_off;    // offset of mu_j / b_j (and of the packed mu-space outputs)
    int32_t  scen;       // scenario
    int32_t  d;          // dimension
    int64_t  acc_off;    // offset of the gradient accumulators: 3 * vec_off * batches
};

// One unit of work: draws [start, start + n) of design `design`.
struct TileRec {
    uint64_t start;      // absolute draw index
    uint32_t n;          // draws in the tile
    uint32_t design;
    uint32_t batch;      // batch-means slot of this tile within its design
    uint32_t pad;
};

// One unit of work of the shared-draw kernel: draws [start, start + n) of
// one stream, tested against the designs list[list_off .. list_off + list_cnt).
struct SharedTile {
    uint64_t start;      // absolute draw index
    uint64_t key;        // stream key common to the listed designs
    uint32_t n;          // draws in the tile
    uint32_t list_off;
    uint32_t list_cnt;   // designs in the tile (<= kSharedThreads * designs per thread)
    uint32_t batch;      // batch-means slot of this draw range
    int32_t  scen;
    int32_t  pad;
};
constexpr int kSharedThreads = 256;    // block size of the shared-draw kernel

// Device status word: code and index of the first error.
struct DevStatus {
    int32_t code;
    int32_t pad;
    long long index;
};

// Parameters of the sampling kernels (kept in the constant bank).
struct SampleParams {
    const DesignRec* designs;
    const TileRec*   tiles;
    int64_t          n_tiles;
    unsigned int*    ticket;        // dynamic tile counter (reset before each launch)
    const float*     L32;           // packed lower factors, FP32
    const double*    L64;           // packed lower factors, FP64
    const int64_t*   L_off;         // per scenario offset into L32 / L64
    const int32_t*   scen_ok;       // per scenario: 1 when the factorisation succeeded
    const double*    mu;
    const double*    b;
    unsigned long long* hits;       // [J] hit accumulators (zeroed before each launch)
    unsigned long long* gacc;       // fixed-point gradient accumulators (grad launches)
    int32_t          batches;       // batch-means slots per design
    float            hinv_log2e;    // log2(e) / h for the smoothed indicator (0: off)
    float            sig_skip_w;    // 25.03 h / log2(e): shared-draw sigmoid window half-width (-1: off)
    double           hinv;          // 1 / h (FP64 path)
    uint32_t         rk0[10];       // Philox round keys (seed_lo + r W0)
    uint32_t         rk1[10];       // Philox round keys (seed_hi + r W1)
    DevStatus*       status;
};

// Host-side launchers (defined in the .cu files).
cudaError_t launch_sample(int d_lo, int d_hi, bool grad, bool fp64, const SampleParams& p,
                          int grid, int threads, cudaStream_t stream);
int  sample_kernel_regs(int d_lo, int d_hi, bool grad, bool fp64);
cudaError_t sample_occupancy(int d_lo, int d_hi, bool grad, bool fp64, int threads, int* blocks);

// Shared-draw kernel of dimension d (FP32 only).
cudaError_t launch_shared(int d, bool grad, const SampleParams& p, const SharedTile* tiles, const uint32_t* list,
                          int grid, cudaStream_t stream);
cudaError_t shared_occupancy(int d, bool grad, int* blocks);
int shared_designs_per_thread(int d, bool grad);
int shared_batch_draws(int d);

cudaError_t launch_cholesky(const double* Sigma, const int64_t* sig_off, const int32_t* scen_d,
                            const int64_t* L_off, int n_scen, float* L32, double* L64,
                            int32_t* scen_ok, DevStatus* status, cudaStream_t stream);

struct FinalizeParams {
    const DesignRec* designs;
    int32_t          n_design;
    const uint64_t*  n_draws;       // [J]
    const unsigned long long* hits; // [J]
    const unsigned long long* gacc;
    const uint64_t*  batch_draws;   // [J * batches] draws per batch slot
    int32_t          batches;
    const double*    L64;
    const int64_t*   L_off;
    const double*    jac;           // [J][d][k] or NULL
    int32_t          k;
    int32_t          region;
    double           hinv;          // 1/h, or 0 when the smoothed indicator is off
    uint64_t*        out_hits;
    double*          out_p;
    double*          out_se;
    double*          g_lr;
    double*          g_sig;
    double*          g_se;
};
cudaError_t launch_finalize(const FinalizeParams& p, bool grad, cudaStream_t stream);

cudaError_t launch_debug_normals(uint64_t seed, uint64_t key, uint64_t m_begin, uint64_t count,
                                 float* z32, double* z64, uint32_t* words, cudaStream_t stream);

cudaError_t smooth_argmax(int n_scen, int g1, int g2, const double* value, double bandwidth,
                          int degree, double* smoothed, int64_t* argmax_idx, double* argmax_val,
                          int64_t* raw_idx, double* raw_val, double* wbuf, float* wbuf32,
                          double* part_val, int64_t* part_idx, DevStatus* status, cudaStream_t stream);
size_t smooth_weight_count();
size_t smooth_candidate_count(int n_scen, int g1, int g2);

// Record the first error in the device status word.
__device__ __forceinline__ void set_status(DevStatus* st, int code, long long index) {
    if (atomicCAS(&st->code, 0, code) == 0) st->index = index;
}

}  // namespace mcd
