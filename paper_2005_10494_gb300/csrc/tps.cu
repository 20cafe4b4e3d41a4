// Thin-plate spline smoothing of scattered estimates and the maximiser of
// the fitted surface (Sec. 2.3: the N3 noisy P_hat(alpha) are smoothed by a
// TPS, whose maximum is found by a quasi-Newton method started at the best
// fitted point).
//
// Fit.  For points x_i in R^k (k = 1, 2, 3), values y_i and smoothing s >= 0
//   f(x) = sum_i c_i eta(|x - x_i|) + d_0 + sum_j d_j x_j,
//   (K + s I) c + P d = y,  P^T c = 0,  K_ij = eta(|x_i - x_j|),  P = [1, x],
// with eta(r) = r^3 (k = 1), r^2 log r (k = 2), -r (k = 3), the radial
// functions of the second-order spline in k dimensions.  The side condition
// is removed with the QR factorisation of P by m = k + 1 Householder
// reflections, Q^T P = [R; 0]: with B = Q^T (K + s I) Q and y~ = Q^T y, the
// trailing block B22 is positive definite and B22 w = y~_2 gives
// c = Q [0; w] and R d = y~_1 - B12 w.  B22 is factored by a blocked
// Cholesky in FP64 (diagonal block by one warp in registers, panel solve,
// trailing update), the two triangular systems by block substitution with
// one multi-block launch per 32 rows.  The fitted values at the data are
// y - s c.
//
// Maximiser.  One thread-block cluster of 8 CTAs per surface: projected
// BFGS on -f inside a box (Armijo backtracking along the projected path),
// started at the data point with the largest fitted value inside the box.
// f and its gradient are sums over the N centres, which the CTAs of the
// cluster split and combine through distributed shared memory (FP64 runs
// at about two FMAs per SM clock on this GPU, so one SM per surface left
// the search bound by that one SM); every CTA then takes the same step.
#include <cmath>
#include <cstdint>

#include <cooperative_groups.h>

#include "tps.cuh"

namespace mcd {

namespace {

constexpr int kNb = 32;            // Cholesky block

__device__ __forceinline__ double eta(double r, int k) {
    if (k == 1) return r * r * r;
    if (k == 2) return r > 0.0 ? r * r * log(r) : 0.0;
    return -r;
}

// eta'(r) / r, the factor of (x - x_i) in the gradient (0 at r = 0)
__device__ __forceinline__ double deta_over_r(double r, int k) {
    if (k == 1) return 3.0 * r;
    if (k == 2) return r > 0.0 ? 2.0 * log(r) + 1.0 : 0.0;
    return r > 0.0 ? -1.0 / r : 0.0;
}

template <int NT>
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    return s;
}

__global__ void assemble_kernel(double* __restrict__ A, const double* __restrict__ x, int N, int k, double s) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= N) return;
    double r2 = 0.0;
    for (int q = 0; q < k; ++q) {
        const double t = x[static_cast<int64_t>(i) * k + q] - x[static_cast<int64_t>(j) * k + q];
        r2 += t * t;
    }
    A[static_cast<int64_t>(i) * N + j] = eta(sqrt(r2), k) + (i == j ? s : 0.0);
}

// Householder QR of P = [1, x] (N x m) in one block: reflector j is
// v_j (zero above row j, stored in V[j][.]) with H_j = I - tau_j v_j v_j^T;
// R (m x m, row-major) and y~ = Q^T y.
constexpr int kQrThreads = 1024;
__global__ void __launch_bounds__(kQrThreads) qr_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                      int N, int k, double* __restrict__ Pw, double* __restrict__ V,
                                                      double* __restrict__ tau, double* __restrict__ R,
                                                      double* __restrict__ yt) {
    __shared__ double red[kQrThreads / 32];
    __shared__ double s_alpha;
    const int m = k + 1;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        Pw[i] = 1.0;
        for (int q = 0; q < k; ++q) Pw[static_cast<int64_t>(q + 1) * N + i] = x[static_cast<int64_t>(i) * k + q];
        yt[i] = y[i];
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        double* col = Pw + static_cast<int64_t>(j) * N;
        double loc = 0.0;
        for (int i = j + threadIdx.x; i < N; i += blockDim.x) loc += col[i] * col[i];
        const double nrm2 = block_sum<kQrThreads>(loc, red);
        if (threadIdx.x == 0) {
            const double a0 = col[j];
            s_alpha = a0 >= 0.0 ? -sqrt(nrm2) : sqrt(nrm2);
        }
        __syncthreads();
        const double alpha = s_alpha;
        double* v = V + static_cast<int64_t>(j) * N;
        for (int i = threadIdx.x; i < N; i += blockDim.x) v[i] = i < j ? 0.0 : (i == j ? col[i] - alpha : col[i]);
        __syncthreads();
        double lv = 0.0;
        for (int i = j + threadIdx.x; i < N; i += blockDim.x) lv += v[i] * v[i];
        const double vv = block_sum<kQrThreads>(lv, red);
        const double t = vv > 0.0 ? 2.0 / vv : 0.0;
        if (threadIdx.x == 0) { tau[j] = t; R[j * m + j] = alpha; }
        // apply H_j to the remaining columns and to y~
        for (int l = j + 1; l <= m; ++l) {
            double* u = l < m ? Pw + static_cast<int64_t>(l) * N : yt;
            double ld = 0.0;
            for (int i = j + threadIdx.x; i < N; i += blockDim.x) ld += v[i] * u[i];
            const double dot = block_sum<kQrThreads>(ld, red);
            for (int i = j + threadIdx.x; i < N; i += blockDim.x) u[i] -= t * dot * v[i];
            __syncthreads();
            if (l < m && threadIdx.x == 0) R[j * m + l] = u[j];
        }
        if (threadIdx.x < m && threadIdx.x < j) R[j * m + threadIdx.x] = 0.0;
        __syncthreads();
    }
}

// w = A v for the symmetric N x N matrix A (one warp per row).
__global__ void matvec_kernel(const double* __restrict__ A, const double* __restrict__ v, double* __restrict__ w, int N) {
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= N) return;
    const double* a = A + static_cast<int64_t>(row) * N;
    double s = 0.0;
    for (int j = lane; j < N; j += 32) s += a[j] * v[j];
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[row] = s;
}

// u = tau w - (tau^2 v^T w / 2) v, in place in w (one block).
__global__ void __launch_bounds__(1024) rank2_prep_kernel(const double* __restrict__ v, double* __restrict__ w,
                                                          const double* __restrict__ tau, int j, int N) {
    __shared__ double red[32];
    double l = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) l += v[i] * w[i];
    const double vw = block_sum<1024>(l, red);
    const double t = tau[j];
    for (int i = threadIdx.x; i < N; i += blockDim.x) w[i] = t * w[i] - 0.5 * t * t * vw * v[i];
}

// A <- H A H = A - v u^T - u v^T.
__global__ void rank2_kernel(double* __restrict__ A, const double* __restrict__ v, const double* __restrict__ u, int N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= N) return;
    A[static_cast<int64_t>(i) * N + j] -= v[i] * u[j] + u[i] * v[j];
}

// max |A_ij| (non-negative doubles order like their bit patterns).
__global__ void maxabs_kernel(const double* __restrict__ A, int64_t count, unsigned long long* __restrict__ out) {
    double m = 0.0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        m = fmax(m, fabs(A[i]));
    for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(m)));
}

// Cholesky of a b x b diagonal block held by one warp, lane i holding row i
// (a[j], j <= i) in registers, in place.  For column c the pivot comes from
// lane c by a shuffle, the lanes below it scale their entry by its
// reciprocal square root, and each later column j takes L_jc from lane j by
// a shuffle for the update A_ij -= L_ic L_jc (i >= j).  A pivot at or below
// floor_p (the projected system is singular to working precision, e.g.
// repeated points without smoothing) is replaced by 1 and reported.
__device__ __forceinline__ bool factor_rows(double (&a)[kNb], int b, double floor_p) {
    const int i = threadIdx.x & 31;
    bool failed = false;
#pragma unroll
    for (int c = 0; c < kNb; ++c) {
        if (c < b) {                                          // b is warp-uniform
            const double p = __shfl_sync(0xffffffffu, a[c], c);
            double r = 1.0, inv = 1.0;
            if (p > floor_p) { inv = rsqrt(p); r = p * inv; }
            else failed = true;
            if (i == c) a[c] = r;
            else if (i > c) a[c] *= inv;
#pragma unroll
            for (int j = c + 1; j < kNb; ++j) {
                const double ljc = __shfl_sync(0xffffffffu, a[c], j);
                if (i >= j) a[j] = fma(-a[c], ljc, a[j]);
            }
        }
    }
    return failed;
}

__device__ __forceinline__ double pivot_floor(int n, const unsigned long long* amax) {
    return static_cast<double>(n) * 2.220446049250313e-16 * __longlong_as_double(static_cast<long long>(*amax));
}

// The first diagonal block of the factorisation (G, leading dimension ld).
__global__ void __launch_bounds__(32) chol_diag_kernel(double* __restrict__ G, int64_t ld, int b, int n,
                                                      const unsigned long long* __restrict__ amax,
                                                      int* __restrict__ bad) {
    const int i = threadIdx.x;
    double a[kNb];
#pragma unroll
    for (int j = 0; j < kNb; ++j) a[j] = (i < b && j <= i) ? G[static_cast<int64_t>(i) * ld + j] : 0.0;
    if (factor_rows(a, b, pivot_floor(n, amax)) && i == 0) *bad = 1;
    if (i < b) {
#pragma unroll
        for (int j = 0; j < kNb; ++j)
            if (j <= i) G[static_cast<int64_t>(i) * ld + j] = a[j];
    }
}

// Look-ahead: the next diagonal block (the bn x bn block at T, leading
// dimension ld) receives its update from the current panel Pn (its first bn
// rows, b columns), by all 256 threads, and is then factored by one warp,
// while the trailing update of the rest of the matrix runs on another
// stream (chol_syrk_kernel skips this block).
constexpr int kNextThreads = 256;
__global__ void __launch_bounds__(kNextThreads) chol_next_diag_kernel(double* __restrict__ T,
                                                                     const double* __restrict__ Pn, int64_t ld,
                                                                     int b, int bn, int n,
                                                                     const unsigned long long* __restrict__ amax,
                                                                     int* __restrict__ bad) {
    __shared__ double pr[kNb][kNb + 1];
    __shared__ double tb[kNb][kNb + 1];
    for (int t = threadIdx.x; t < kNb * kNb; t += blockDim.x) {
        const int r = t / kNb, c = t % kNb;
        pr[r][c] = (r < bn && c < b) ? Pn[static_cast<int64_t>(r) * ld + c] : 0.0;
        tb[r][c] = (r < bn && c <= r) ? T[static_cast<int64_t>(r) * ld + c] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kNb * kNb; t += blockDim.x) {
        const int r = t / kNb, c = t % kNb;
        if (r < bn && c <= r) {
            double acc = 0.0;
#pragma unroll
            for (int l = 0; l < kNb; ++l) acc = fma(pr[r][l], pr[c][l], acc);
            tb[r][c] -= acc;
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int i = threadIdx.x;
    double a[kNb];
#pragma unroll
    for (int j = 0; j < kNb; ++j) a[j] = tb[i][j];
    if (factor_rows(a, bn, pivot_floor(n, amax)) && i == 0) *bad = 1;
    if (i < bn) {
#pragma unroll
        for (int j = 0; j < kNb; ++j)
            if (j <= i) T[static_cast<int64_t>(i) * ld + j] = a[j];
    }
}

// Rows below the diagonal block: X <- X L^{-T} for the n_rem x b panel at
// Pn (leading dimension ld), L the factored diagonal block at G; one row per
// thread.  Column by column, x_c = s_c / L_cc (the pivots' reciprocals
// formed once per block) and s_j -= x_c L_jc for the later columns, so the
// dependent chain is one multiply and one FMA per column and the updates of
// a column are independent.
constexpr int kTrsmThreads = 64;
__global__ void __launch_bounds__(kTrsmThreads) chol_trsm_kernel(const double* __restrict__ G,
                                                                 double* __restrict__ Pn, int64_t ld, int b,
                                                                 int n_rem) {
    __shared__ double L[kNb][kNb + 1];
    __shared__ double rd[kNb];
    for (int t = threadIdx.x; t < kNb * kNb; t += blockDim.x) {
        const int r = t / kNb, c = t % kNb;
        L[r][c] = (r < b && c <= r) ? G[static_cast<int64_t>(r) * ld + c] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < kNb) rd[threadIdx.x] = threadIdx.x < b ? 1.0 / L[threadIdx.x][threadIdx.x] : 0.0;
    __syncthreads();
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n_rem) return;
    double* p = Pn + static_cast<int64_t>(row) * ld;
    double x[kNb];
#pragma unroll
    for (int c = 0; c < kNb; ++c) x[c] = c < b ? p[c] : 0.0;
#pragma unroll
    for (int c = 0; c < kNb; ++c) {
        x[c] *= rd[c];
#pragma unroll
        for (int j2 = c + 1; j2 < kNb; ++j2) x[j2] = fma(-x[c], L[j2][c], x[j2]);
    }
#pragma unroll
    for (int c = 0; c < kNb; ++c)
        if (c < b) p[c] = x[c];
}

// Trailing update of the lower triangle: T[i][j] -= sum_l Pn[i][l] Pn[j][l],
// i >= j, for the n_rem x n_rem matrix at T and the n_rem x b panel at Pn.
// Block (bx, by): output tile rows by*TS.., columns bx*TS..; 256 threads,
// P x P outputs each (TS = 16 P).  64 x 64 tiles while there are enough of
// them to fill the GPU, 32 x 32 below that (a tile's FMAs run on one SM's
// FP64 units, about two a clock).  The leading skip x skip block (the next
// diagonal block, updated and factored by chol_next_diag_kernel meanwhile)
// is left alone.
template <int P>
__global__ void __launch_bounds__(256) chol_syrk_kernel(double* __restrict__ T, const double* __restrict__ Pn,
                                                        int64_t ld, int b, int n_rem, int skip) {
    constexpr int TS = 16 * P;
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (tj > ti) return;
    __shared__ double si[TS][kNb + 1];
    __shared__ double sj[TS][kNb + 1];
    const int r0 = ti * TS, c0 = tj * TS;
    for (int t = threadIdx.x; t < TS * kNb; t += blockDim.x) {
        const int r = t / kNb, l = t % kNb;
        si[r][l] = (r0 + r < n_rem && l < b) ? Pn[static_cast<int64_t>(r0 + r) * ld + l] : 0.0;
        sj[r][l] = (c0 + r < n_rem && l < b) ? Pn[static_cast<int64_t>(c0 + r) * ld + l] : 0.0;
    }
    __syncthreads();
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    double acc[P][P] = {};
    for (int l = 0; l < b; ++l) {
        double a[P], c[P];
#pragma unroll
        for (int q = 0; q < P; ++q) { a[q] = si[ty + 16 * q][l]; c[q] = sj[tx + 16 * q][l]; }
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
            for (int q = 0; q < P; ++q) acc[p][q] = fma(a[p], c[q], acc[p][q]);
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int i = r0 + ty + 16 * p, j = c0 + tx + 16 * q;
            if (i < n_rem && j < n_rem && j <= i && !(i < skip && j < skip))
                T[static_cast<int64_t>(i) * ld + j] -= acc[p][q];
        }
}

// Solve L z = r, then L^T w = z, for the n x n lower factor at L (leading
// dimension ld), right-looking, one launch per block of 32 rows so that
// every SM's FP64 units share the n^2 multiply-adds.  GB300 issues about two
// FP64 FMAs per SM clock; a single block doing all of them was bound by its
// one SM.
//   Forward step at rows i0..i0+b-1: every block solves the b x b diagonal
//   system L_bb z_b = r_b with one warp (lane q holds row q of L_bb, r_q
//   and 1 / L_qq in registers; column by column, z_c comes from lane c by
//   a shuffle and every lane subtracts L_qc z_c, so no step waits on a
//   memory load or a reduction) into shared memory, block 0 stores z_b,
//   then the block's warps update the later rows it owns, r_j -= L_j,b z_b,
//   one row per warp (its 32 entries of L contiguous).
//   Backward step: the transposed diagonal system L_bb^T w_b = z_b (lane q
//   holds column q of L_bb, from the last column back), then
//   z_j -= sum_c L_(i0+c),j w_c for the earlier rows, one per thread
//   (rows of L read contiguously across the warp).
// The right-hand side is read and updated in one array and the solution is
// written to another, so that no block reads an entry another block of the
// same launch writes.
constexpr int kSolveThreads = 256;
constexpr int kSolveMaxBlocks = 512;     // blocks per step (each re-solves the 32 x 32 diagonal)

__global__ void recip_diag_kernel(const double* __restrict__ L, int64_t ld, int n, double* __restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dinv[i] = 1.0 / L[static_cast<int64_t>(i) * ld + i];
}

__global__ void __launch_bounds__(kSolveThreads) solve_fwd_step_kernel(const double* __restrict__ L, int64_t ld,
                                                                      int n, int i0,
                                                                      const double* __restrict__ dinv,
                                                                      double* __restrict__ r,
                                                                      double* __restrict__ z) {
    __shared__ double zb[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = n - i0 < 32 ? n - i0 : 32;
    if (warp == 0) {
        // lane q: row q of the diagonal block left of the diagonal, its
        // right-hand side and reciprocal pivot, all loaded up front; then
        // column by column, z_c = r_c / L_cc from lane c and r_q -= L_qc z_c
        double lrow[32];
#pragma unroll
        for (int c = 0; c < 32; ++c)
            lrow[c] = (lane < b && c < lane) ? L[static_cast<int64_t>(i0 + lane) * ld + i0 + c] : 0.0;
        double rq = lane < b ? r[i0 + lane] : 0.0;
        const double dq = lane < b ? dinv[i0 + lane] : 0.0;
        double zq = 0.0;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            if (c < b) {                                         // b is warp-uniform
                const double zc = __shfl_sync(0xffffffffu, rq * dq, c);
                if (lane == c) zq = zc;
                rq = fma(-lrow[c], zc, rq);
            }
        }
        zb[lane] = zq;
        if (blockIdx.x == 0 && lane < b) z[i0 + lane] = zq;
    }
    __syncthreads();
    const int warps = blockDim.x >> 5;
    for (int j = i0 + b + blockIdx.x * warps + warp; j < n; j += gridDim.x * warps) {
        double t = lane < b ? L[static_cast<int64_t>(j) * ld + i0 + lane] * zb[lane] : 0.0;
        for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) r[j] -= t;
    }
}

__global__ void __launch_bounds__(kSolveThreads) solve_bwd_step_kernel(const double* __restrict__ L, int64_t ld,
                                                                      int n, int i0,
                                                                      const double* __restrict__ dinv,
                                                                      double* __restrict__ z,
                                                                      double* __restrict__ w) {
    __shared__ double wb[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = n - i0 < 32 ? n - i0 : 32;
    if (warp == 0) {
        // lane q: column q of the diagonal block below the diagonal (rows of
        // L read contiguously across the warp); then from the last column
        // back, w_c = z_c / L_cc from lane c and z_q -= L_cq w_c
        double lcol[32];
#pragma unroll
        for (int c = 0; c < 32; ++c)
            lcol[c] = (c < b && lane < c) ? L[static_cast<int64_t>(i0 + c) * ld + i0 + lane] : 0.0;
        double zq = lane < b ? z[i0 + lane] : 0.0;
        const double dq = lane < b ? dinv[i0 + lane] : 0.0;
        double wq = 0.0;
#pragma unroll
        for (int c = 31; c >= 0; --c) {
            if (c < b) {
                const double wc = __shfl_sync(0xffffffffu, zq * dq, c);
                if (lane == c) wq = wc;
                zq = fma(-lcol[c], wc, zq);
            }
        }
        wb[lane] = wq;
        if (blockIdx.x == 0 && lane < b) w[i0 + lane] = wq;
    }
    __syncthreads();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < i0; j += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int c = 0; c < b; ++c) t = fma(L[static_cast<int64_t>(i0 + c) * ld + j], wb[c], t);
        z[j] -= t;
    }
}

// The two triangular solves with L: the right-hand side in z on entry and
// the solution in z on return; r2 (n doubles) holds the intermediate
// solution and dinv (n doubles) the reciprocals of L's diagonal.
cudaError_t launch_solve(const double* L, int64_t ld, int n, double* z, double* r2, double* dinv,
                         cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    recip_diag_kernel<<<(n + 255) / 256, 256, 0, stream>>>(L, ld, n, dinv);
    const int nblk = (n + 31) / 32;
    for (int bi = 0; bi < nblk; ++bi) {
        const int i0 = bi * 32;
        const int rows = n - i0 - 32;                            // later rows to update
        const int warps = kSolveThreads / 32;
        int grid = rows > 0 ? (rows + warps - 1) / warps : 1;
        if (grid > kSolveMaxBlocks) grid = kSolveMaxBlocks;
        solve_fwd_step_kernel<<<grid, kSolveThreads, 0, stream>>>(L, ld, n, i0, dinv, z, r2);
    }
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int i0 = bi * 32;
        int grid = i0 > 0 ? (i0 + kSolveThreads - 1) / kSolveThreads : 1;
        if (grid > kSolveMaxBlocks) grid = kSolveMaxBlocks;
        solve_bwd_step_kernel<<<grid, kSolveThreads, 0, stream>>>(L, ld, n, i0, dinv, r2, z);
    }
    return cudaGetLastError();
}

// c = Q [0; w], R d = y~_1 - B12 w, fitted = y - s c; NaN when the
// factorisation failed.  One block.
__global__ void __launch_bounds__(1024) combine_kernel(const double* __restrict__ A, const double* __restrict__ V,
                                                       const double* __restrict__ tau, const double* __restrict__ R,
                                                       const double* __restrict__ yt, const double* __restrict__ w,
                                                       const double* __restrict__ y, int N, int k, double s,
                                                       const int* __restrict__ bad, double* __restrict__ coef,
                                                       double* __restrict__ fitted, DevStatus* status, int surf) {
    __shared__ double red[32];
    __shared__ double rhs[4];
    const int m = k + 1;
    const bool ok = *bad == 0;
    if (!ok) {
        if (threadIdx.x == 0) set_status(status, MCD_ENOTSPD, surf);
        for (int i = threadIdx.x; i < N + m; i += blockDim.x) coef[i] = NAN;
        if (fitted)
            for (int i = threadIdx.x; i < N; i += blockDim.x) fitted[i] = NAN;
        return;
    }
    // rhs_j = y~_j - sum_l B[j][m + l] w_l
    for (int j = 0; j < m; ++j) {
        double l = 0.0;
        for (int i = threadIdx.x; i < N - m; i += blockDim.x) l += A[static_cast<int64_t>(j) * N + m + i] * w[i];
        const double t = block_sum<1024>(l, red);
        if (threadIdx.x == 0) rhs[j] = yt[j] - t;
        __syncthreads();
    }
    // c = H_0 ... H_{m-1} [0; w]
    for (int i = threadIdx.x; i < N; i += blockDim.x) coef[i] = i < m ? 0.0 : w[i - m];
    __syncthreads();
    for (int j = m - 1; j >= 0; --j) {
        const double* v = V + static_cast<int64_t>(j) * N;
        double l = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) l += v[i] * coef[i];
        const double dot = block_sum<1024>(l, red);
        for (int i = threadIdx.x; i < N; i += blockDim.x) coef[i] -= tau[j] * dot * v[i];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double d[4];
        for (int j = m - 1; j >= 0; --j) {
            double t = rhs[j];
            for (int l = j + 1; l < m; ++l) t -= R[j * m + l] * d[l];
            d[j] = t / R[j * m + j];
        }
        for (int j = 0; j < m; ++j) coef[N + j] = d[j];
    }
    if (fitted)
        for (int i = threadIdx.x; i < N; i += blockDim.x) fitted[i] = y[i] - s * coef[i];
}

// ---- generalised cross-validation ------------------------------------------
// With T = Q2^T K Q2 (the projection at s = 0) and M = T + s I = L L^T,
// (I - A_s) y = s c with |c| = |w|, w = M^{-1} y~_2, and tr(I - A_s) =
// s tr(M^{-1}) = s |L^{-1}|_F^2, so V(s) = N |w|^2 / |L^{-1}|_F^4.

// dst (n x n, leading dimension n) = src (leading dimension lds) + s I,
// lower triangle and diagonal.
__global__ void shift_copy_kernel(const double* __restrict__ src, int64_t lds, double* __restrict__ dst, int n,
                                  double s) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j > i || i >= n) return;
    dst[static_cast<int64_t>(i) * n + j] = src[static_cast<int64_t>(i) * lds + j] + (i == j ? s : 0.0);
}

// Inverse of each b x b lower-triangular diagonal block of L (leading
// dimension n), into the same block of X; thread c makes column c.
__global__ void __launch_bounds__(kNb) tri_inv_diag_kernel(const double* __restrict__ L, double* __restrict__ X,
                                                          int n) {
    __shared__ double a[kNb][kNb + 1];
    __shared__ double x[kNb][kNb + 1];
    const int j0 = blockIdx.x * kNb;
    const int b = n - j0 < kNb ? n - j0 : kNb;
    const int c = threadIdx.x;
    for (int r = 0; r < kNb; ++r) a[r][c] = (r < b && c <= r) ? L[static_cast<int64_t>(j0 + r) * n + j0 + c] : 0.0;
    __syncthreads();
    if (c < b) {
        for (int r = 0; r < kNb; ++r) x[r][c] = 0.0;
        x[c][c] = 1.0 / a[c][c];
        for (int r = c + 1; r < b; ++r) {
            double t = 0.0;
            for (int l = c; l < r; ++l) t += a[r][l] * x[l][c];
            x[r][c] = -t / a[r][r];
        }
        for (int r = c; r < b; ++r) X[static_cast<int64_t>(j0 + r) * n + j0 + c] = x[r][c];
    }
}

// Block row i of X = L^{-1} (i >= 1): for every block column j < i,
// X_ij = -X_ii (sum_{l=j}^{i-1} L_il X_lj), 32 x 32 blocks, one block per j.
__global__ void __launch_bounds__(256) tri_inv_step_kernel(const double* __restrict__ L, double* __restrict__ X,
                                                           int n, int bi) {
    __shared__ double ls[kNb][kNb + 1];
    __shared__ double xs[kNb][kNb + 1];
    const int bj = blockIdx.x;
    const int i0 = bi * kNb, j0 = bj * kNb;
    const int tr = threadIdx.x / 8, tc0 = (threadIdx.x % 8) * 4;      // row tr, columns tc0 .. tc0 + 3
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int bl = bj; bl < bi; ++bl) {
        const int l0 = bl * kNb;
        for (int t = threadIdx.x; t < kNb * kNb; t += blockDim.x) {
            const int r = t / kNb, q = t % kNb;
            ls[r][q] = (i0 + r < n) ? L[static_cast<int64_t>(i0 + r) * n + l0 + q] : 0.0;
            xs[r][q] = (l0 + r >= j0 + q) ? X[static_cast<int64_t>(l0 + r) * n + j0 + q] : 0.0;   // lower part only
        }
        __syncthreads();
        for (int l = 0; l < kNb; ++l) {
            const double lv = ls[tr][l];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(lv, xs[l][tc0 + q], acc[q]);
        }
        __syncthreads();
    }
    // X_ij = -X_ii S: S through shared memory, X_ii from X
    for (int q = 0; q < 4; ++q) xs[tr][tc0 + q] = acc[q];
    for (int t = threadIdx.x; t < kNb * kNb; t += blockDim.x) {
        const int r = t / kNb, q = t % kNb;
        ls[r][q] = (i0 + r < n && i0 + q < n && q <= r) ? X[static_cast<int64_t>(i0 + r) * n + i0 + q] : 0.0;
    }
    __syncthreads();
    if (i0 + tr < n) {
        for (int q = 0; q < 4; ++q) {
            double v = 0.0;
            for (int l = 0; l <= tr; ++l) v += ls[tr][l] * xs[l][tc0 + q];
            X[static_cast<int64_t>(i0 + tr) * n + j0 + tc0 + q] = -v;
        }
    }
}

// |X|_F^2 over the lower triangle (n x n, leading dimension n).
__global__ void sumsq_lower_kernel(const double* __restrict__ X, int n, double* __restrict__ out) {
    const int i = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j <= i; j += blockDim.x) {
        const double v = X[static_cast<int64_t>(i) * n + j];
        s += v * v;
    }
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// V(s) = N |w|^2 / tr^2, NaN when the factorisation failed.
__global__ void __launch_bounds__(1024) gcv_score_kernel(const double* __restrict__ w, int n, const double* __restrict__ tr,
                                                         const int* __restrict__ bad, int N, double* __restrict__ out) {
    __shared__ double red[32];
    double l = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) l += w[i] * w[i];
    const double ww = block_sum<1024>(l, red);
    if (threadIdx.x == 0) *out = *bad ? NAN : static_cast<double>(N) * ww / (*tr * *tr);
}

// ---- maximiser ---------------------------------------------------------------
constexpr int kMaxThreads = 256;
constexpr int kArgmaxCluster = 8;    // CTAs per surface (a thread-block cluster)

// f and its gradient at z, the same values in every thread of the cluster.
// CTA `rank` sums the centres rank, rank + C, ... (C = kArgmaxCluster) in its
// threads; the block's four sums go to its slot part[parity]; after one
// cluster barrier every CTA adds the C slots, read through distributed
// shared memory, in rank order, so all CTAs hold bit-identical f and g (and
// take the same branches of the search).  The slots alternate with the
// parity of the evaluation, so a CTA that runs ahead writes the other slot
// while the rest still read this one; it cannot get two evaluations ahead,
// since each evaluation's barrier waits for every CTA.
__device__ void f_and_grad(const double* __restrict__ x, const double* __restrict__ coef, int N, int k,
                           const double* z, double& f, double* g, double (*red)[4], double (*part)[4],
                           int& parity) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = static_cast<int>(cluster.block_rank());
    double l4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = rank * blockDim.x + threadIdx.x; i < N; i += kArgmaxCluster * blockDim.x) {
        double diff[3], r2 = 0.0;
        for (int q = 0; q < k; ++q) {
            diff[q] = z[q] - x[static_cast<int64_t>(i) * k + q];
            r2 += diff[q] * diff[q];
        }
        const double r = sqrt(r2), c = coef[i];
        l4[0] += c * eta(r, k);
        const double fac = c * deta_over_r(r, k);
        for (int q = 0; q < k; ++q) l4[1 + q] += fac * diff[q];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < 4; ++v)
        for (int o = 16; o >= 1; o >>= 1) l4[v] += __shfl_xor_sync(0xffffffffu, l4[v], o);
    if (lane == 0) {
#pragma unroll
        for (int v = 0; v < 4; ++v) red[warp][v] = l4[v];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
        part[parity][threadIdx.x] = t;
    }
    cluster.sync();
    double tot[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r = 0; r < kArgmaxCluster; ++r) {
        const double* pr = cluster.map_shared_rank(&part[parity][0], r);
#pragma unroll
        for (int v = 0; v < 4; ++v) tot[v] += pr[v];
    }
    parity ^= 1;
    f = tot[0] + coef[N];
    for (int q = 0; q < k; ++q) f += coef[N + 1 + q] * z[q];
    for (int q = 0; q < 3; ++q) g[q] = q < k ? tot[1 + q] + coef[N + 1 + q] : 0.0;
}

__global__ void __cluster_dims__(kArgmaxCluster, 1, 1) __launch_bounds__(kMaxThreads)
argmax_tps_kernel(const double* __restrict__ x,
                                                                 const double* __restrict__ coef,
                                                                 const double* __restrict__ fitted, int N, int k,
                                                                 const double* __restrict__ lo,
                                                                 const double* __restrict__ hi, int iters,
                                                                 double* __restrict__ xbest,
                                                                 double* __restrict__ fbest) {
    __shared__ double red[kMaxThreads / 32][4];
    __shared__ double part[2][4];
    __shared__ double sbest[kMaxThreads];
    __shared__ int sidx[kMaxThreads];
    int parity = 0;
    const int surf = blockIdx.x / kArgmaxCluster;   // one cluster of CTAs per surface
    const double* X = x + static_cast<int64_t>(surf) * N * k;
    const double* C = coef + static_cast<int64_t>(surf) * (N + k + 1);
    const double* F = fitted + static_cast<int64_t>(surf) * N;
    // start: the data point inside the box with the largest fitted value
    // (lowest index on ties)
    double bv = -INFINITY;
    int bi = -1;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        bool in = true;
        for (int q = 0; q < k; ++q) {
            const double t = X[static_cast<int64_t>(i) * k + q];
            in = in && t >= lo[q] && t <= hi[q];
        }
        if (in && F[i] > bv) { bv = F[i]; bi = i; }
    }
    sbest[threadIdx.x] = bv;
    sidx[threadIdx.x] = bi;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < blockDim.x; ++t)
            if (sidx[t] >= 0 && (sidx[0] < 0 || sbest[t] > sbest[0] || (sbest[t] == sbest[0] && sidx[t] < sidx[0]))) {
                sbest[0] = sbest[t];
                sidx[0] = sidx[t];
            }
    }
    __syncthreads();
    const int start = sidx[0];
    double z[3] = {0, 0, 0}, g[3] = {0, 0, 0}, f;
    for (int q = 0; q < k; ++q) z[q] = start >= 0 ? X[static_cast<int64_t>(start) * k + q] : 0.5 * (lo[q] + hi[q]);
    f_and_grad(X, C, N, k, z, f, g, red, part, parity);
    // inverse-Hessian approximation of -f (ascent direction H g)
    double H[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double scale = 0.0;
    for (int q = 0; q < k; ++q) scale = fmax(scale, hi[q] - lo[q]);
    double gn0 = 0.0;
    for (int q = 0; q < k; ++q) gn0 += g[q] * g[q];
    for (int q = 0; q < k; ++q) H[q][q] = 0.1 * scale / fmax(1e-300, sqrt(gn0));
    for (int it = 0; it < iters; ++it) {
        double p[3] = {0, 0, 0};
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b) p[a] += H[a][b] * g[b];
        // components that would leave the box at an active bound are dropped
        for (int q = 0; q < k; ++q)
            if ((z[q] <= lo[q] && p[q] < 0.0) || (z[q] >= hi[q] && p[q] > 0.0)) p[q] = 0.0;
        double gp = 0.0;
        for (int q = 0; q < k; ++q) gp += g[q] * p[q];
        if (!(gp > 0.0)) {                                       // not an ascent direction: restart along g
            for (int a = 0; a < k; ++a)
                for (int b = 0; b < k; ++b) H[a][b] = a == b ? H[a][a] : 0.0;
            for (int q = 0; q < k; ++q) {
                p[q] = H[q][q] * g[q];
                if ((z[q] <= lo[q] && p[q] < 0.0) || (z[q] >= hi[q] && p[q] > 0.0)) p[q] = 0.0;
            }
            gp = 0.0;
            for (int q = 0; q < k; ++q) gp += g[q] * p[q];
            if (!(gp > 0.0)) break;                              // projected gradient is zero
        }
        double t = 1.0, zn[3] = {z[0], z[1], z[2]}, fn = f, gn[3] = {g[0], g[1], g[2]};
        bool moved = false;
        for (int ls = 0; ls < 60; ++ls) {
            for (int q = 0; q < k; ++q) zn[q] = fmin(fmax(z[q] + t * p[q], lo[q]), hi[q]);
            f_and_grad(X, C, N, k, zn, fn, gn, red, part, parity);
            double dz = 0.0, gz = 0.0;
            for (int q = 0; q < k; ++q) { dz += fabs(zn[q] - z[q]); gz += g[q] * (zn[q] - z[q]); }
            if (dz == 0.0) break;
            if (fn >= f + 1e-4 * gz) { moved = true; break; }
            t *= 0.5;
        }
        if (!moved) break;
        double s[3], yv[3], sy = 0.0;
        for (int q = 0; q < k; ++q) { s[q] = zn[q] - z[q]; yv[q] = -(gn[q] - g[q]); sy += s[q] * yv[q]; }
        for (int q = 0; q < k; ++q) { z[q] = zn[q]; g[q] = gn[q]; }
        const double df = fn - f;
        f = fn;
        if (sy > 1e-300) {                                       // BFGS update of the inverse Hessian of -f
            double Hy[3] = {0, 0, 0}, yHy = 0.0;
            for (int a = 0; a < k; ++a)
                for (int b = 0; b < k; ++b) Hy[a] += H[a][b] * yv[b];
            for (int a = 0; a < k; ++a) yHy += yv[a] * Hy[a];
            const double rho = 1.0 / sy;
            for (int a = 0; a < k; ++a)
                for (int b = 0; b < k; ++b)
                    H[a][b] += (1.0 + yHy * rho) * rho * s[a] * s[b] - rho * (Hy[a] * s[b] + s[a] * Hy[b]);
        }
        if (df <= 1e-16 * fmax(1.0, fabs(f))) break;
    }
    if (threadIdx.x == 0 && cooperative_groups::this_cluster().block_rank() == 0) {
        for (int q = 0; q < k; ++q) xbest[static_cast<int64_t>(surf) * k + q] = z[q];
        fbest[surf] = f;
    }
    // no CTA leaves while another may still read its partial sums
    cooperative_groups::this_cluster().sync();
}

}  // namespace

// Blocked Cholesky (lower, in place) of the n x n matrix at B (leading
// dimension ld), with one step of look-ahead: after the panel solve of
// block j, the next diagonal block is updated and factored on a second
// stream while the rest of the trailing update runs on `stream`; the two
// write disjoint parts of the matrix, and the next panel solve waits for
// both.  The factorisation of a diagonal block is a chain of 32 dependent
// FP64 pivots (about 1.5 us each on this GPU's FP64 units), which the
// trailing update now hides.
static cudaError_t chol_blocked(double* B, int64_t ld, int n, const unsigned long long* amax, int* bad,
                                cudaStream_t stream) {
    // 64 x 64 trailing-update tiles while their lower triangle has at least
    // one tile per SM, 32 x 32 after that
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_panel = nullptr, ev_diag = nullptr;
    int prio_lo = 0, prio_hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_panel, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_diag, cudaEventDisableTiming);
    if (e == cudaSuccess && n > 0) {
        const int b0 = n < kNb ? n : kNb;
        chol_diag_kernel<<<1, 32, 0, stream>>>(B, ld, b0, n, amax, bad);
    }
    for (int j0 = 0; e == cudaSuccess && j0 < n; j0 += kNb) {
        const int b = n - j0 < kNb ? n - j0 : kNb;
        double* G = B + j0 * ld + j0;
        const int rem = n - j0 - b;
        if (rem <= 0) break;
        double* Pn = G + b * ld;
        chol_trsm_kernel<<<(rem + kTrsmThreads - 1) / kTrsmThreads, kTrsmThreads, 0, stream>>>(G, Pn, ld, b, rem);
        const int bn = rem < kNb ? rem : kNb;
        if ((e = cudaEventRecord(ev_panel, stream)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(side, ev_panel, 0)) != cudaSuccess) break;
        chol_next_diag_kernel<<<1, kNextThreads, 0, side>>>(Pn + b, Pn, ld, b, bn, n, amax, bad);
        if ((e = cudaEventRecord(ev_diag, side)) != cudaSuccess) break;
        const int t64 = (rem + 63) / 64;
        if (t64 * (t64 + 1) / 2 >= sms) {
            chol_syrk_kernel<4><<<dim3(t64, t64), 256, 0, stream>>>(Pn + b, Pn, ld, b, rem, bn);
        } else {
            const int t32 = (rem + 31) / 32;
            chol_syrk_kernel<2><<<dim3(t32, t32), 256, 0, stream>>>(Pn + b, Pn, ld, b, rem, bn);
        }
        if ((e = cudaStreamWaitEvent(stream, ev_diag, 0)) != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    // destruction is deferred by the runtime until the queued work is done
    if (ev_diag) cudaEventDestroy(ev_diag);
    if (ev_panel) cudaEventDestroy(ev_panel);
    if (side) cudaStreamDestroy(side);
    return e;
}

// Workspace of one fit: A (N x N), V and Pw (m x N each), y~, w, z (N each),
// R (m x m), tau (m), then the reciprocals of the factor's diagonal (N).
static size_t tps_base_doubles(int N, int k) {
    const size_t m = static_cast<size_t>(k) + 1;
    return static_cast<size_t>(N) * N + 2 * m * N + 3 * static_cast<size_t>(N) + m * m + m + 8;
}

size_t tps_workspace_doubles(int N, int k) { return tps_base_doubles(N, k) + static_cast<size_t>(N); }

cudaError_t tps_fit_one(const double* x, const double* y, int N, int k, double s, double* coef, double* fitted,
                        double* ws, int* bad, unsigned long long* amax, DevStatus* status, int surf,
                        cudaStream_t stream) {
    const int m = k + 1;
    double* A = ws;
    double* V = A + static_cast<size_t>(N) * N;
    double* Pw = V + static_cast<size_t>(m) * N;
    double* yt = Pw + static_cast<size_t>(m) * N;
    double* w = yt + N;
    double* z = w + N;
    double* R = z + N;
    double* tau = R + m * m;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(amax, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    assemble_kernel<<<dim3((N + 255) / 256, N), 256, 0, stream>>>(A, x, N, k, s);
    qr_kernel<<<1, kQrThreads, 0, stream>>>(x, y, N, k, Pw, V, tau, R, yt);
    for (int j = 0; j < m; ++j) {
        const double* v = V + static_cast<size_t>(j) * N;
        matvec_kernel<<<(N + 7) / 8, 256, 0, stream>>>(A, v, w, N);
        rank2_prep_kernel<<<1, 1024, 0, stream>>>(v, w, tau, j, N);
        rank2_kernel<<<dim3((N + 255) / 256, N), 256, 0, stream>>>(A, v, w, N);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // blocked Cholesky of B22 = A[m:, m:]
    const int n = N - m;
    double* B = A + static_cast<size_t>(m) * N + m;
    maxabs_kernel<<<256, 256, 0, stream>>>(A, static_cast<int64_t>(N) * N, amax);
    if ((e = chol_blocked(B, N, n, amax, bad, stream)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(z, yt + m, sizeof(double) * n, cudaMemcpyDeviceToDevice, stream)) != cudaSuccess) return e;
    if ((e = launch_solve(B, N, n, z, w, ws + tps_base_doubles(N, k), stream)) != cudaSuccess) return e;
    combine_kernel<<<1, 1024, 0, stream>>>(A, V, tau, R, yt, z, y, N, k, s, bad, coef, fitted, status, surf);
    return cudaGetLastError();
}

size_t tps_gcv_workspace_doubles(int N, int k) {
    const size_t n = static_cast<size_t>(N) - (k + 1);
    return tps_workspace_doubles(N, k) + 2 * n * n + 8;
}

cudaError_t tps_gcv(const double* x, const double* y, int N, int k, const double* s_values, int n_s, double* score,
                    double* ws, int* bad, unsigned long long* amax, double* trace, cudaStream_t stream) {
    const int m = k + 1;
    const int n = N - m;
    double* A = ws;
    double* V = A + static_cast<size_t>(N) * N;
    double* Pw = V + static_cast<size_t>(m) * N;
    double* yt = Pw + static_cast<size_t>(m) * N;
    double* w = yt + N;
    double* z = w + N;
    double* R = z + N;
    double* tau = R + m * m;
    double* W = ws + tps_workspace_doubles(N, k);
    double* X = W + static_cast<size_t>(n) * n;
    // projection of K (s = 0) and y~
    assemble_kernel<<<dim3((N + 255) / 256, N), 256, 0, stream>>>(A, x, N, k, 0.0);
    qr_kernel<<<1, kQrThreads, 0, stream>>>(x, y, N, k, Pw, V, tau, R, yt);
    for (int j = 0; j < m; ++j) {
        const double* v = V + static_cast<size_t>(j) * N;
        matvec_kernel<<<(N + 7) / 8, 256, 0, stream>>>(A, v, w, N);
        rank2_prep_kernel<<<1, 1024, 0, stream>>>(v, w, tau, j, N);
        rank2_kernel<<<dim3((N + 255) / 256, N), 256, 0, stream>>>(A, v, w, N);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double* T22 = A + static_cast<size_t>(m) * N + m;
    const int nb = (n + kNb - 1) / kNb;
    for (int q = 0; q < n_s; ++q) {
        if ((e = cudaMemsetAsync(bad, 0, sizeof(int), stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(amax, 0, sizeof(unsigned long long), stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(trace, 0, sizeof(double), stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(X, 0, sizeof(double) * static_cast<size_t>(n) * n, stream)) != cudaSuccess) return e;
        shift_copy_kernel<<<dim3((n + 255) / 256, n), 256, 0, stream>>>(T22, N, W, n, s_values[q]);
        maxabs_kernel<<<256, 256, 0, stream>>>(W, static_cast<int64_t>(n) * n, amax);
        if ((e = chol_blocked(W, n, n, amax, bad, stream)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(z, yt + m, sizeof(double) * n, cudaMemcpyDeviceToDevice, stream)) != cudaSuccess)
            return e;
        if ((e = launch_solve(W, n, n, z, w, ws + tps_base_doubles(N, k), stream)) != cudaSuccess) return e;
        tri_inv_diag_kernel<<<nb, kNb, 0, stream>>>(W, X, n);
        for (int bi = 1; bi < nb; ++bi) tri_inv_step_kernel<<<bi, 256, 0, stream>>>(W, X, n, bi);
        sumsq_lower_kernel<<<n, 128, 0, stream>>>(X, n, trace);
        gcv_score_kernel<<<1, 1024, 0, stream>>>(z, n, trace, bad, N, score + q);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t tps_argmax(const double* x, const double* coef, const double* fitted, int n_surf, int N, int k,
                       const double* lo, const double* hi, int iters, double* xbest, double* fbest,
                       cudaStream_t stream) {
    argmax_tps_kernel<<<n_surf * kArgmaxCluster, kMaxThreads, 0, stream>>>(x, coef, fitted, N, k, lo, hi, iters, xbest,
                                                                          fbest);
    return cudaGetLastError();
}

}  // namespace mcd
