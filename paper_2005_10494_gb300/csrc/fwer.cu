// Calibration of an alpha split to the family-wise error rate, on the device
// (Eq. 2, with the reparametrisation of Sec. 2.1: the split w of the alpha
// budget is fixed and its scale s solved for, alpha = s w).
//
// Under the null hypothesis (mu = 0) the FWER of thresholds b_i =
// Z_{1 - s w_i} is 1 - Phi_Sigma(b(s)); it increases in s and lies between
// max_i s w_i and s sum_i w_i (Bonferroni), which brackets the solution of
// FWER(s) = alpha0 in [alpha0 / sum w, alpha0 / max w].  Each round the
// sampling kernels estimate the FWER of every design at its current s (the
// same draws every round, so the estimate is a nondecreasing step function of
// s); fwer_update_kernel then narrows the bracket and picks the next s by
// false position with the Illinois modification (when the same end is kept
// twice in a row, the other end's residual is halved).
#include <cmath>

#include "fwer.cuh"

namespace mcd {

namespace {

// b_i = Z_{1 - s w_i} = -Phi^{-1}(s w_i); a zero weight drops test i.
__device__ void write_thresholds(const double* __restrict__ w, double* __restrict__ b, int64_t off, int d,
                                 double s) {
    for (int i = 0; i < d; ++i) {
        const double a = s * w[off + i];
        b[off + i] = a > 0.0 ? -normcdfinv(a) : INFINITY;
    }
}

__global__ void fwer_init_kernel(int J, const DesignRec* __restrict__ dr, const double* __restrict__ w,
                                 double alpha0, FwerState* __restrict__ st, double* __restrict__ b,
                                 DevStatus* status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    const int64_t off = dr[j].vec_off;
    const int d = dr[j].d;
    double sum = 0.0, mx = 0.0;
    bool ok = true;
    for (int i = 0; i < d; ++i) {
        const double x = w[off + i];
        if (!(x >= 0.0) || x == INFINITY) ok = false;       // negative, NaN or infinite
        sum += x;
        mx = fmax(mx, x);
    }
    if (!ok || !(mx > 0.0)) {
        set_status(status, MCD_EINVAL, j);
        ok = false;
    }
    FwerState s;
    s.lo = ok ? alpha0 / sum : 0.0;
    s.hi = ok ? alpha0 / mx : 0.0;                         // every s w_i stays <= alpha0 < 1
    s.lo = fmin(s.lo, s.hi);
    s.f_lo = 0.0;
    s.f_hi = 1.0;
    s.s = s.lo;
    s.side = 0;
    s.ok = ok ? 1 : 0;
    st[j] = s;
    if (ok) write_thresholds(w, b, off, d, s.s);
    else
        for (int i = 0; i < d; ++i) b[off + i] = NAN;
}

// Round `round` has estimated the FWER p[j] of every design at its current
// scale.  Rounds 0 and 1 evaluate the two ends of the bracket; later rounds
// its interior.  After the last round the current scale and its estimate are
// the result (the thresholds in b already belong to it).
__global__ void fwer_update_kernel(int J, const DesignRec* __restrict__ dr, const double* __restrict__ w,
                                   const double* __restrict__ p, double alpha0, int round, int last,
                                   FwerState* __restrict__ st, double* __restrict__ b, double* __restrict__ scale,
                                   double* __restrict__ fwer) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    FwerState s = st[j];
    const double F = p[j];
    if (last || !s.ok) {
        if (last) {
            scale[j] = s.ok ? s.s : NAN;
            fwer[j] = s.ok ? F : NAN;
        }
        return;
    }
    if (round == 0) {
        s.f_lo = F;
    } else if (round == 1) {
        s.f_hi = F;
    } else if (F <= alpha0) {                  // the new point replaces the low end
        s.lo = s.s;
        s.f_lo = F;
        if (s.side < 0) s.f_hi = alpha0 + 0.5 * (s.f_hi - alpha0);
        s.side = -1;
    } else {                                   // ... or the high end
        s.hi = s.s;
        s.f_hi = F;
        if (s.side > 0) s.f_lo = alpha0 - 0.5 * (alpha0 - s.f_lo);
        s.side = 1;
    }
    double next;
    if (round == 0) {
        next = s.hi;
    } else if (s.f_lo >= alpha0) {             // the low end already reaches alpha0
        next = s.lo;
    } else if (s.f_hi <= alpha0) {             // the high end does not exceed it
        next = s.hi;
    } else {
        next = s.lo + (alpha0 - s.f_lo) * (s.hi - s.lo) / (s.f_hi - s.f_lo);
        next = fmin(fmax(next, s.lo), s.hi);
    }
    s.s = next;
    st[j] = s;
    write_thresholds(w, b, dr[j].vec_off, dr[j].d, next);
}

}  // namespace

cudaError_t launch_fwer_init(int J, const DesignRec* dr, const double* w, double alpha0, FwerState* st, double* b,
                             DevStatus* status, cudaStream_t stream) {
    if (J <= 0) return cudaSuccess;
    fwer_init_kernel<<<(J + 127) / 128, 128, 0, stream>>>(J, dr, w, alpha0, st, b, status);
    return cudaGetLastError();
}

cudaError_t launch_fwer_update(int J, const DesignRec* dr, const double* w, const double* p, double alpha0, int round,
                               bool last, FwerState* st, double* b, double* scale, double* fwer,
                               cudaStream_t stream) {
    if (J <= 0) return cudaSuccess;
    fwer_update_kernel<<<(J + 127) / 128, 128, 0, stream>>>(J, dr, w, p, alpha0, round, last ? 1 : 0, st, b, scale,
                                                             fwer);
    return cudaGetLastError();
}

}  // namespace mcd
