// Small FP64 kernels around the sampling pass: Cholesky factorisation of each
// scenario's Sigma, the count -> probability / gradient finalisation, and the
// unit-check normals.
#include <cmath>
#include <cstdint>

#include "mcd_internal.cuh"
#include "rng.cuh"

namespace mcd {

namespace {

__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// Sigma_s = L L^T (Cholesky-Banachiewicz, FP64, lower triangle of Sigma read).
__global__ void cholesky_kernel(const double* __restrict__ Sigma, const int64_t* __restrict__ sig_off,
                                const int32_t* __restrict__ scen_d, const int64_t* __restrict__ L_off,
                                int n_scen, float* __restrict__ L32, double* __restrict__ L64,
                                int32_t* __restrict__ scen_ok, DevStatus* status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_scen) return;
    const int d = scen_d[s];
    const double* A = Sigma + sig_off[s];
    double* L = L64 + L_off[s];
    float* Lf = L32 + L_off[s];
    bool good = true;
    for (int i = 0; i < d && good; ++i) {
        for (int j = 0; j <= i; ++j) {
            double sum = A[i * d + j];
            for (int k = 0; k < j; ++k) sum -= L[tri(i, k)] * L[tri(j, k)];
            if (i == j) {
                if (!(sum > 0.0) || !isfinite(sum)) { good = false; break; }
                L[tri(i, i)] = sqrt(sum);
            } else {
                L[tri(i, j)] = sum / L[tri(j, j)];
            }
        }
    }
    const int n = d * (d + 1) / 2;
    for (int i = 0; i < n; ++i) {
        if (!good) L[i] = 0.0;
        Lf[i] = static_cast<float>(L[i]);
    }
    scen_ok[s] = good ? 1 : 0;
    if (!good) set_status(status, MCD_ENOTSPD, s);
}

__device__ __forceinline__ double fix_to_double(unsigned long long v) {
    return static_cast<double>(static_cast<long long>(v)) * (1.0 / static_cast<double>(1ull << kGradFixBits));
}

// Solve L^T g = v in place (L packed lower, FP64), with the reciprocals
// rdiag[i] = 1 / L_ii computed once per design: FP64 division is a long
// sequence on this GPU, and the batch-means error below takes a solve per
// batch.
__device__ __forceinline__ void solve_lt(const double* L, const double* rdiag, int d, double* v) {
    for (int i = d - 1; i >= 0; --i) {
        double s = v[i];
        for (int k = i + 1; k < d; ++k) s -= L[tri(k, i)] * v[k];
        v[i] = s * rdiag[i];
    }
}

__global__ void finalize_kernel(const FinalizeParams P, bool grad) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.n_design) return;
    const DesignRec dr = P.designs[j];
    const uint64_t N = P.n_draws[j];
    const uint64_t h_any = P.hits[j];
    const bool any = (P.region == MCD_ANY_EXCEEDS);
    const double Nd = static_cast<double>(N);
    const double p_any = N ? static_cast<double>(h_any) / Nd : 0.0;
    const double p = any ? p_any : (N ? 1.0 - p_any : 0.0);
    if (P.out_hits) P.out_hits[j] = any ? h_any : N - h_any;
    if (P.out_p) P.out_p[j] = p;
    if (P.out_se) P.out_se[j] = N ? sqrt(p * (1.0 - p) / Nd) : 0.0;
    if (!grad) return;

    const int d = dr.d;
    const double sign = any ? 1.0 : -1.0;
    const double* L = P.L64 + P.L_off[dr.scen];
    const int k = P.k;
    const int nout = k > 0 ? k : d;
    const int64_t out_off = k > 0 ? static_cast<int64_t>(j) * k : dr.vec_off;
    const double* J = P.jac ? P.jac + dr.vec_off * k : nullptr;
    if (k > 0 && !J) return;   // the host rejects this; never dereference a missing Jacobian

    double rdiag[kMaxD];
    for (int i = 0; i < d; ++i) rdiag[i] = 1.0 / L[tri(i, i)];
    double A[kMaxD], B[kMaxD], G[kMaxD];
    for (int i = 0; i < d; ++i) { A[i] = 0.0; B[i] = 0.0; G[i] = 0.0; }
    const unsigned long long* acc = P.gacc + dr.acc_off;
    int nonempty = 0;
    for (int bt = 0; bt < P.batches; ++bt) {
        const unsigned long long* a = acc + static_cast<int64_t>(bt) * 3 * d;
        for (int i = 0; i < d; ++i) {
            A[i] += fix_to_double(a[i]);
            B[i] += fix_to_double(a[d + i]);
            G[i] += fix_to_double(a[2 * d + i]);
        }
        if (P.batch_draws[static_cast<int64_t>(j) * P.batches + bt] > 0) ++nonempty;
    }
    // likelihood ratio with the zero-mean control variate: L^-T (A - p B) / N
    double g[kMaxD], gs[kMaxD];
    const double rN = N ? 1.0 / Nd : 0.0;
    for (int i = 0; i < d; ++i) {
        g[i] = (A[i] - p_any * B[i]) * rN;
        gs[i] = P.hinv > 0.0 ? G[i] * P.hinv * rN : 0.0;
    }
    solve_lt(L, rdiag, d, g);
    double est[kMaxD], est_s[kMaxD];
    for (int m = 0; m < nout; ++m) {
        if (k > 0) {
            double s1 = 0.0, s2 = 0.0;
            for (int i = 0; i < d; ++i) { s1 -= J[i * k + m] * g[i]; s2 -= J[i * k + m] * gs[i]; }
            est[m] = sign * s1;
            est_s[m] = sign * s2;
        } else {
            est[m] = sign * g[m];
            est_s[m] = sign * gs[m];
        }
    }
    if (P.g_lr) for (int m = 0; m < nout; ++m) P.g_lr[out_off + m] = est[m];
    if (P.g_sig && P.hinv > 0.0) for (int m = 0; m < nout; ++m) P.g_sig[out_off + m] = est_s[m];
    if (!P.g_se) return;
    // batch means: per batch the same estimator on its own draws
    double ss[kMaxD];
    for (int m = 0; m < nout; ++m) ss[m] = 0.0;
    uint64_t nb_last = 0;
    double rnb = 0.0;                                 // 1 / nb, recomputed only when nb changes
    for (int bt = 0; bt < P.batches; ++bt) {
        const uint64_t nb = P.batch_draws[static_cast<int64_t>(j) * P.batches + bt];
        if (!nb) continue;
        if (nb != nb_last) { rnb = 1.0 / static_cast<double>(nb); nb_last = nb; }
        const unsigned long long* a = acc + static_cast<int64_t>(bt) * 3 * d;
        double v[kMaxD];
        for (int i = 0; i < d; ++i) v[i] = (fix_to_double(a[i]) - p_any * fix_to_double(a[d + i])) * rnb;
        solve_lt(L, rdiag, d, v);
        for (int m = 0; m < nout; ++m) {
            double c;
            if (k > 0) {
                c = 0.0;
                for (int i = 0; i < d; ++i) c -= J[i * k + m] * v[i];
                c *= sign;
            } else {
                c = sign * v[m];
            }
            const double dev = c - est[m];
            ss[m] += static_cast<double>(nb) * dev * dev;
        }
    }
    for (int m = 0; m < nout; ++m)
        P.g_se[out_off + m] = nonempty >= 2 ? sqrt(ss[m] / (Nd * (nonempty - 1))) : NAN;
}

__global__ void debug_normals_kernel(uint64_t seed, uint64_t key, uint64_t m_begin, uint64_t count,
                                     float* z32, double* z64, uint32_t* words) {
    uint32_t rk0[10], rk1[10];
    for (int r = 0; r < 10; ++r) {
        rk0[r] = static_cast<uint32_t>(seed) + static_cast<uint32_t>(r) * kPhiloxW0;
        rk1[r] = static_cast<uint32_t>(seed >> 32) + static_cast<uint32_t>(r) * kPhiloxW1;
    }
    const uint64_t first_call = m_begin >> 2;
    const uint64_t ncalls = count ? ((m_begin + count - 1) >> 2) - first_call + 1 : 0;
    const uint64_t idx = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx < count) {
        const uint64_t m = m_begin + idx;
        const uint4 w = philox_full(m >> 2, key, rk0, rk1);
        float f[4];
        double g[4];
        normals4<float>(w, f);
        normals4<double>(w, g);
        if (z32) z32[idx] = f[m & 3];
        if (z64) z64[idx] = g[m & 3];
    }
    if (words && idx < ncalls) {
        const uint4 w = philox_full(first_call + idx, key, rk0, rk1);
        words[4 * idx + 0] = w.x;
        words[4 * idx + 1] = w.y;
        words[4 * idx + 2] = w.z;
        words[4 * idx + 3] = w.w;
    }
}

}  // namespace

cudaError_t launch_cholesky(const double* Sigma, const int64_t* sig_off, const int32_t* scen_d,
                            const int64_t* L_off, int n_scen, float* L32, double* L64,
                            int32_t* scen_ok, DevStatus* status, cudaStream_t stream) {
    const int threads = 64;
    cholesky_kernel<<<(n_scen + threads - 1) / threads, threads, 0, stream>>>(
        Sigma, sig_off, scen_d, L_off, n_scen, L32, L64, scen_ok, status);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeParams& p, bool grad, cudaStream_t stream) {
    if (p.n_design == 0) return cudaSuccess;
    const int threads = 128;
    finalize_kernel<<<(p.n_design + threads - 1) / threads, threads, 0, stream>>>(p, grad);
    return cudaGetLastError();
}

cudaError_t launch_debug_normals(uint64_t seed, uint64_t key, uint64_t m_begin, uint64_t count,
                                 float* z32, double* z64, uint32_t* words, cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    const uint64_t ncalls = ((m_begin + count - 1) >> 2) - (m_begin >> 2) + 1;
    const uint64_t n = count > ncalls ? count : ncalls;
    const int threads = 256;
    debug_normals_kernel<<<static_cast<unsigned>((n + threads - 1) / threads), threads, 0, stream>>>(
        seed, key, m_begin, count, z32, z64, words);
    return cudaGetLastError();
}

}  // namespace mcd
