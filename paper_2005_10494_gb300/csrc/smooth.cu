// Local-polynomial smoothing of design-grid estimates and their argmax
// (Sec. 2.3: smooth the noisy P_hat surface, start the search from its best
// point; the paper fits thin-plate splines, this engine local polynomials on
// the regular grid).
//
// At grid point (i, j) the smoothed value is beta_0 of the weighted least
// squares fit of the monomials of (k - i, l - j) up to `degree` with tricube
// product weights w((k-i)/h) w((l-j)/h), w(u) = (1 - |u|^3)^3, over the window
// of points with positive weight, cut at the grid edges.  beta_0 is a fixed
// linear stencil for each pair of edge classes (distance to the low and high
// edge, capped at the reach R), so the FP64 solve runs once per class pair
// and the application over the grid is a stencil, HBM-bound, in FP32.
#include <algorithm>
#include <cmath>
#include <cstdint>


#include "mcd_internal.cuh"
#include "smooth.cuh"

namespace mcd {

namespace {

constexpr int kMaxReach = 3;
constexpr int kMaxTaps = (2 * kMaxReach + 1) * (2 * kMaxReach + 1);
constexpr int kRowsPerBlock = 32;     // output rows of one block (2-D)
constexpr int kColsPerBlock = 128;    // output columns of one block (2-D)
constexpr int kLine = 512;            // outputs of one block (1-D)
// The interior class's FP32 stencil is also stored compactly after the class
// table, 16-byte aligned, for vector loads (T*T of the first 64 floats),
// followed at kSepOff by its separable factors (see weights_kernel).
constexpr int kClassSlots = (kMaxReach + 1) * (kMaxReach + 1) * (kMaxReach + 1) * (kMaxReach + 1);
constexpr int kSepOff = 64;
constexpr int kIntSlot = kSepOff + 16;

__host__ __device__ inline int reach_of(double bw) {
    const double f = floor(bw);
    return (f == bw) ? static_cast<int>(bw) - 1 : static_cast<int>(f);
}

__device__ inline double tricube(double u) {
    const double a = fabs(u);
    if (a >= 1.0) return 0.0;
    const double c = 1.0 - a * a * a;
    return c * c * c;
}

// Monomials of (dx, dy) up to the degree ({1, x, y, x^2, xy, y^2}); 1-D drops y.
__device__ inline int basis(double dx, double dy, int degree, bool two_d, double* x) {
    int n = 0;
    x[n++] = 1.0;
    if (degree >= 1) { x[n++] = dx; if (two_d) x[n++] = dy; }
    if (degree >= 2) { x[n++] = dx * dx; if (two_d) { x[n++] = dx * dy; x[n++] = dy * dy; } }
    return n;
}

// One thread per class pair: stencil weights w[(dx+R)(2R+1) + (dy+R)] in FP64.
// Class of a position: lo = min(i, R) points below, hi = min(G-1-i, R) above;
// class id = lo (R+1) + hi.  1-D grids use only the x axis (classes in x).
__global__ void weights_kernel(int R, double bw, int degree, bool two_d, int gx, int gy,
                               double* w64, float* w32, DevStatus* status) {
    const int ncls = (R + 1) * (R + 1);
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (two_d ? ncls * ncls : ncls)) return;
    const int cx = two_d ? id / ncls : id, cy = two_d ? id % ncls : 0;
    const int xlo = cx / (R + 1), xhi = cx % (R + 1);
    const int ylo = two_d ? cy / (R + 1) : 0, yhi = two_d ? cy % (R + 1) : 0;
    const int T = 2 * R + 1;
    double* w = w64 + static_cast<int64_t>(id) * kMaxTaps;
    float* wf = w32 + static_cast<int64_t>(id) * kMaxTaps;
    // the thread of the interior class pair also fills the compact copy
    // (zeros when this grid has no interior point)
    float* wint = (xlo == R && xhi == R && (!two_d || (ylo == R && yhi == R)))
                      ? w32 + static_cast<int64_t>(kClassSlots) * kMaxTaps : nullptr;
    for (int q = 0; q < kMaxTaps; ++q) { w[q] = 0.0; wf[q] = 0.0f; }
    if (wint)
        for (int q = 0; q < kIntSlot; ++q) wint[q] = 0.0f;
    // classes that no position of this grid has are skipped
    if (xlo + xhi + 1 > gx || (xlo < R && xhi < R && xlo + xhi + 1 != gx)) return;
    if (two_d && (ylo + yhi + 1 > gy || (ylo < R && yhi < R && ylo + yhi + 1 != gy))) return;
    double M[6][6] = {};
    double x[6];
    int nb = 0;
    for (int dx = -xlo; dx <= xhi; ++dx) {
        for (int dy = -ylo; dy <= yhi; ++dy) {
            const double W = tricube(dx / bw) * (two_d ? tricube(dy / bw) : 1.0);
            nb = basis(dx, dy, degree, two_d, x);
            for (int a = 0; a < nb; ++a)
                for (int c = 0; c < nb; ++c) M[a][c] += W * x[a] * x[c];
        }
    }
    // u = M^-1 e_0 by Gaussian elimination with partial pivoting
    double u[6] = {1.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int col = 0; col < nb; ++col) {
        int piv = col;
        for (int r = col + 1; r < nb; ++r) if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (!(fabs(M[piv][col]) > 1e-12)) { set_status(status, MCD_EINVAL, id); return; }
        if (piv != col) {
            for (int c = 0; c < nb; ++c) { const double tmp = M[col][c]; M[col][c] = M[piv][c]; M[piv][c] = tmp; }
            const double tu = u[col]; u[col] = u[piv]; u[piv] = tu;
        }
        for (int r = 0; r < nb; ++r) {
            if (r == col) continue;
            const double f = M[r][col] / M[col][col];
            if (f == 0.0) continue;
            for (int c = col; c < nb; ++c) M[r][c] -= f * M[col][c];
            u[r] -= f * u[col];
        }
    }
    for (int r = 0; r < nb; ++r) u[r] /= M[r][r];
    for (int dx = -xlo; dx <= xhi; ++dx) {
        for (int dy = -ylo; dy <= yhi; ++dy) {
            const double W = tricube(dx / bw) * (two_d ? tricube(dy / bw) : 1.0);
            basis(dx, dy, degree, two_d, x);
            double s = 0.0;
            for (int a = 0; a < nb; ++a) s += x[a] * u[a];
            const int q = two_d ? (dx + R) * T + (dy + R) : (dx + R);
            w[q] = W * s;
            wf[q] = static_cast<float>(W * s);
            if (wint) wint[q] = wf[q];
        }
    }
    // The interior stencil in 2-D is separable into two rank-one parts.  With
    // symmetric product weights W(dx) W(dy), the coefficients of the odd
    // monomials (dx, dy, dx dy) vanish, so the stencil is
    //   W(dx) W(dy) (u_0 + u_x dx^2 + u_y dy^2)
    //     = [W(dx) (u_0 + u_x dx^2)] W(dy) + [W(dx) u_y] dy^2 W(dy).
    // The tile kernel applies it as two row filters (W(v), v^2 W(v)) and one
    // column pass with the weights W(u) (u_0 + u_x u^2) and W(u) u_y; for
    // degree 0 and 1, u_x = u_y = 0 (one rank-one part).
    if (wint && two_d) {
        const double ux = nb == 6 ? u[3] : 0.0, uy = nb == 6 ? u[5] : 0.0;
        for (int k = 0; k <= R; ++k) {
            const double wk = tricube(k / bw);
            wint[kSepOff + k] = static_cast<float>(wk);
            wint[kSepOff + 4 + k] = static_cast<float>(k * k * wk);
            wint[kSepOff + 8 + k] = static_cast<float>(wk * (u[0] + ux * k * k));
            wint[kSepOff + 12 + k] = static_cast<float>(wk * uy);
        }
    }
}

__device__ __forceinline__ int cls(int i, int G, int R) {
    const int lo = i < R ? i : R;
    const int hi = (G - 1 - i) < R ? (G - 1 - i) : R;
    return lo * (R + 1) + hi;
}

// GB300 has little FP64 throughput, so the stencil keeps FP64 only at its
// edges: values are converted between FP64 and FP32 and ordered for the
// argmax with integer operations on their bit patterns.

// FP64 -> FP32, truncating the dropped mantissa bits (error below one FP32
// ulp); magnitudes below the FP32 normal range become 0, above it infinity,
// NaN stays NaN.  The mantissa and exponent move together with one funnel
// shift: (hi:lo) << 3 puts the low 8 exponent bits and the top 23 mantissa
// bits in place, and subtracting (1023 - 127) << 23 rebiases.
__device__ __forceinline__ float d2f_bits(unsigned long long b) {
    const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
    const unsigned e = (hi >> 20) & 0x7ffu;
    unsigned mag = __funnelshift_l(lo, hi, 3) - (896u << 23);
    if (e - 897u >= 254u) {                                   // outside the FP32 normal range
        mag = e <= 896u ? 0u
            : ((e == 0x7ffu && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u);
    }
    return __uint_as_float((hi & 0x80000000u) | mag);
}

// FP32 -> FP64 bits, exact for normal numbers (FP32 subnormals flush to
// signed zero; infinity and NaN keep their class).
__device__ __forceinline__ unsigned long long f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ex = u & 0x7f800000u, sign = u & 0x80000000u;
    if (ex - 0x00800000u < 0x7f000000u) {                     // normal
        const unsigned hi = sign | (((u & 0x7fffffffu) >> 3) + (896u << 20));
        return (static_cast<unsigned long long>(hi) << 32) | (u << 29);
    }
    if (ex == 0u) return static_cast<unsigned long long>(sign) << 32;
    const unsigned hi = sign | 0x7ff00000u | ((u >> 3) & 0xfffffu);
    return (static_cast<unsigned long long>(hi) << 32) | (u << 29);
}

// Monotone map of FP64 bit patterns to unsigned keys (larger value, larger key).
__device__ __forceinline__ unsigned long long order_key(unsigned long long b) {
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ unsigned long long key_bits(unsigned long long k) {
    return (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
}
__device__ __forceinline__ bool nan_bits(unsigned long long b) {
    return (b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
}

// argmax on keys with the lowest index on ties; index -1 means "none"
__device__ __forceinline__ void amax(unsigned long long& k, long long& i, unsigned long long k2, long long i2) {
    if (i2 < 0) return;
    if (i < 0 || k2 > k || (k2 == k && i2 < i)) { k = k2; i = i2; }
}

__device__ __forceinline__ void amax_value(unsigned long long& k, long long& i, unsigned long long bits, long long idx) {
    if (!nan_bits(bits)) amax(k, i, order_key(bits), idx);
}

__device__ __forceinline__ void block_amax(unsigned long long& v, long long& i, unsigned long long* sv, long long* si) {
    for (int m = 16; m >= 1; m >>= 1) {
        const unsigned long long v2 = __shfl_xor_sync(0xffffffffu, v, m);
        const long long i2 = __shfl_xor_sync(0xffffffffu, i, m);
        amax(v, i, v2, i2);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sv[warp] = v; si[warp] = i; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) amax(v, i, sv[w], si[w]);
    }
}

// Exact running argmax of FP64 values visited in increasing index order: a
// cheap FP32 comparison first (rounding to FP32 is monotone, so a strictly
// larger FP32 value means a larger FP64 value and a smaller one a smaller),
// the exact key comparison only when the FP32 values tie.
struct RunMax {
    float f;
    unsigned long long key;
    long long idx;
    __device__ __forceinline__ void init() { f = -INFINITY; key = 0; idx = -1; }
    __device__ __forceinline__ void add(float x, unsigned long long bits, long long i) {
        if (x > f) {
            f = x; key = order_key(bits); idx = i;
        } else if (x == f && !nan_bits(bits)) {
            const unsigned long long k = order_key(bits);
            if (idx < 0 || k > key) { key = k; idx = i; }
        }
    }
};

// Element types of the grids: FP64 values are handled as their bit patterns
// (conversions and argmax keys are integer operations); FP32 values are
// read and written as they are, and their argmax keys are those of the
// exactly converted FP64 value.
template <typename Elem> struct GridWord;
template <> struct GridWord<double> { using W = unsigned long long; };
template <> struct GridWord<float> { using W = float; };

// Fast FP64 -> FP32 for exponents 897..1150 (the FP32 normal range): one
// funnel shift moves exponent and mantissa together, one subtraction
// rebiases, the sign is or-ed back; the result truncates like d2f_bits.
// `bad` collects values outside that range, which the caller converts again
// with d2f_bits.
__device__ __forceinline__ float d2f_fast(unsigned long long b, bool& bad) {
    const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
    bad |= ((hi & 0x7fffffffu) - 0x38100000u) >= 0x0fe00000u;
    const unsigned mag = __funnelshift_l(lo, hi, 3) - (896u << 23);
    return __uint_as_float((hi & 0x80000000u) | mag);
}

// Fast FP32 -> FP64 bits for normal, finite f (same result as f2d_bits):
// hi = (u >> 3) + 896 << 20 moves and rebiases the exponent, and for
// negative f the sign bit shifted to bit 28 is moved back to bit 31 by adding
// 0x70000000.  `bad` collects zeros, subnormals, infinities and NaNs.
__device__ __forceinline__ unsigned long long f2d_fast(float f, bool& bad) {
    const unsigned u = __float_as_uint(f);
    bad |= !(fabsf(f) >= 0x1p-126f && fabsf(f) <= 0x1.fffffep127f);
    const unsigned hi = (u >> 3) + 0x38000000u + ((u >> 31) ? 0x70000000u : 0u);
    return (static_cast<unsigned long long>(hi) << 32) | (u << 29);
}

// Store the pair (x0, x1) of staged row rr, pair slot m, at shared columns
// 2m - E + R and 2m - E + R + 1 (column -1 of odd R is not needed).
template <int R, int E, int NPR, int SR, int SCP>
__device__ __forceinline__ void store_pair(float (*tile)[SCP], int rr, int m, float x0, float x1) {
    if (rr >= SR || m >= NPR) return;
    const int sc = 2 * m - E + R;
    if constexpr (R % 2 == 0) {
        *reinterpret_cast<float2*>(&tile[rr][sc]) = make_float2(x0, x1);
    } else {
        if (sc >= 0) tile[rr][sc] = x0;
        tile[rr][sc + 1] = x1;
    }
}

// Staging of tile rows warp + 8 k, k in [K0, K1), into FP32 shared memory.
// Input column c0 - R sits at shared column 0.  Lane l takes the pairs of
// doubles l, l + 32, l + 64 of a row, pair m covering global columns
// c0 - E + 2m and c0 - E + 2m + 1 (E = R rounded up to even, so that with VEC
// every pair is one aligned 16-byte load).  All loads of the batch are issued
// before any value is converted.  Positions outside the grid hold 1.0: their
// weight in every stencil that reads them is zero, and a finite value keeps
// 0 * x = 0.
// FP32 grid: pairs of floats (one 8-byte load with VEC) straight into the
// tile, all loads of the batch in flight before the first store; raw argmax
// keys from the exact FP64 value.  Positions outside the grid hold 1.0.
template <int R, bool RAW, bool VEC, int K0, int K1, int SR, int SCP>
__device__ __forceinline__ void stage_rows_f32(const float* __restrict__ V, int g1, int g2, int r0, int c0,
                                               float (*tile)[SCP], RunMax& raw) {
    constexpr int E = (R + 1) / 2 * 2;
    constexpr int NPR = (kColsPerBlock + 2 * E) / 2;        // pairs per staged row
    constexpr int PPL = (NPR + 31) / 32;                    // pair slots per lane
    constexpr int NK = K1 - K0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 v[NK][PPL];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int rr = warp + 8 * (K0 + k);
        const int gr = r0 - R + rr;
        const bool row_in = rr < SR && gr >= 0 && gr < g1;
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
            const int m = lane + 32 * p;
            const int gc = c0 - E + 2 * m;
            v[k][p] = make_float2(1.0f, 1.0f);
            if (row_in && m < NPR) {
                const float* q = V + static_cast<int64_t>(gr) * g2 + gc;
                if constexpr (VEC) {
                    if (gc >= 0 && gc < g2) v[k][p] = __ldg(reinterpret_cast<const float2*>(q));
                } else {
                    if (gc >= 0 && gc < g2) v[k][p].x = __ldg(q);
                    if (gc + 1 >= 0 && gc + 1 < g2) v[k][p].y = __ldg(q + 1);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int rr = warp + 8 * (K0 + k);
        const int gr = r0 - R + rr;
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
            const int m = lane + 32 * p;
            const int gc = c0 - E + 2 * m;
            store_pair<R, E, NPR, SR, SCP>(tile, rr, m, v[k][p].x, v[k][p].y);
            if constexpr (RAW) {
                if (rr < SR && m < NPR && rr >= R && rr < R + kRowsPerBlock && gr >= 0 && gr < g1) {
                    if (gc >= c0 && gc < c0 + kColsPerBlock && gc < g2)
                        raw.add(v[k][p].x, f2d_bits(v[k][p].x), static_cast<long long>(gr) * g2 + gc);
                    if (gc + 1 >= c0 && gc + 1 < c0 + kColsPerBlock && gc + 1 < g2)
                        raw.add(v[k][p].y, f2d_bits(v[k][p].y), static_cast<long long>(gr) * g2 + gc + 1);
                }
            }
        }
    }
}

template <int R, bool RAW, bool VEC, int K0, int K1, int SR, int SCP>
__device__ __forceinline__ void stage_rows_f64(const unsigned long long* __restrict__ V, int g1, int g2, int r0,
                                               int c0, float (*tile)[SCP], RunMax& raw) {
    constexpr int E = (R + 1) / 2 * 2;
    constexpr int NPR = (kColsPerBlock + 2 * E) / 2;        // pairs per staged row
    constexpr int PPL = (NPR + 31) / 32;                    // pair slots per lane
    constexpr int NK = K1 - K0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr unsigned long long kOne = 0x3ff0000000000000ull;
    unsigned long long b0[NK][PPL], b1[NK][PPL];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int rr = warp + 8 * (K0 + k);
        const int gr = r0 - R + rr;
        const bool row_in = rr < SR && gr >= 0 && gr < g1;
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
            const int m = lane + 32 * p;
            const int gc = c0 - E + 2 * m;
            b0[k][p] = kOne;
            b1[k][p] = kOne;
            if (row_in && m < NPR) {
                const unsigned long long* q = V + static_cast<int64_t>(gr) * g2 + gc;
                if constexpr (VEC) {
                    if (gc >= 0 && gc < g2) {
                        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(q));
                        b0[k][p] = v.x;
                        b1[k][p] = v.y;
                    }
                } else {
                    if (gc >= 0 && gc < g2) b0[k][p] = __ldg(q);
                    if (gc + 1 >= 0 && gc + 1 < g2) b1[k][p] = __ldg(q + 1);
                }
            }
        }
    }
    // fast conversions go straight to shared memory; in the rare batch that
    // holds a value outside the fast range the warp converts and stores
    // every value again with the exact routine
    bool bad = false;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int rr = warp + 8 * (K0 + k);
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
            const float x0 = d2f_fast(b0[k][p], bad), x1 = d2f_fast(b1[k][p], bad);
            store_pair<R, E, NPR, SR, SCP>(tile, rr, lane + 32 * p, x0, x1);
        }
    }
    const bool slow = __any_sync(0xffffffffu, bad);
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int rr = warp + 8 * (K0 + k);
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
            const int m = lane + 32 * p;
            float x0 = 0.0f, x1 = 0.0f;
            if (slow || RAW) { x0 = d2f_bits(b0[k][p]); x1 = d2f_bits(b1[k][p]); }
            if (slow) store_pair<R, E, NPR, SR, SCP>(tile, rr, m, x0, x1);
            if constexpr (RAW) {
                const int gr = r0 - R + rr, gc = c0 - E + 2 * m;
                if (rr < SR && m < NPR && rr >= R && rr < R + kRowsPerBlock && gr < g1) {
                    if (gc >= c0 && gc < c0 + kColsPerBlock && gc < g2)
                        raw.add(x0, b0[k][p], static_cast<long long>(gr) * g2 + gc);
                    if (gc + 1 >= c0 && gc + 1 < c0 + kColsPerBlock && gc + 1 < g2)
                        raw.add(x1, b1[k][p], static_cast<long long>(gr) * g2 + gc + 1);
                }
            }
        }
    }
}

template <int R, bool RAW, bool VEC, int K0, int K1, int SR, int SCP, typename Elem>
__device__ __forceinline__ void stage_rows(const typename GridWord<Elem>::W* __restrict__ V, int g1, int g2, int r0,
                                           int c0, float (*tile)[SCP], RunMax& raw) {
    if constexpr (sizeof(Elem) == 4) stage_rows_f32<R, RAW, VEC, K0, K1, SR, SCP>(V, g1, g2, r0, c0, tile, raw);
    else stage_rows_f64<R, RAW, VEC, K0, K1, SR, SCP>(V, g1, g2, r0, c0, tile, raw);
}

// Shape constants of the 2-D kernels for reach R.
template <int R>
struct Tile2D {
    static constexpr int T = 2 * R + 1;
    static constexpr int SR = kRowsPerBlock + 2 * R;        // staged rows
    static constexpr int NV = (4 + 2 * R + 3) / 4;          // 16-byte loads per window row
    static constexpr int SCP = 4 * 31 + 4 * NV;             // FP32 tile row stride (floats)
    static constexpr int RPW = (SR + 7) / 8;                // staged rows per warp
};

constexpr int kWarps2D = 8;           // argmax candidates per 2-D tile (one per warp)

// Outputs of one staged tile (rows r0.., columns c0.. of scenario s): the
// interior stencil for every thread's 4 x 4 patch (thread (tx, ty) owns rows
// 4 ty.., columns 4 tx..; the 4 + 2R rows of its window stream through
// registers with 16-byte shared loads), kept where the edge class is
// interior; then the tile's edge outputs (fewer than R points to a grid
// edge), one per thread, with their class stencils; then the tile's argmax
// candidates (smoothed, and raw when RAW), one per warp, at slot `slot` of
// scenario s.
template <int R, bool RAW, typename Elem>
__device__ __forceinline__ void tile_outputs(float (*tile)[Tile2D<R>::SCP], int g1, int g2, int s, int r0, int c0,
                                             const float* __restrict__ w32, const float* __restrict__ wint,
                                             typename GridWord<Elem>::W* __restrict__ out, int nb, int slot,
                                             unsigned long long* part_v, long long* part_i,
                                             unsigned long long* rpart_v, long long* rpart_i,
                                             RunMax& raw) {
    constexpr int T = Tile2D<R>::T;
    constexpr int NV = Tile2D<R>::NV;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int orow = r0 + 4 * ty, ocol = c0 + 4 * tx;       // first output of this thread
    const int ncls = (R + 1) * (R + 1);
    typename GridWord<Elem>::W* O = out ? out + static_cast<int64_t>(s) * g1 * g2 : nullptr;
    // the largest interior output of the patch and its position i * 4 + j
    // (visited in row-major order, so a tie keeps the lowest index)
    float best = -INFINITY;
    int bsel = -1;
    // Interior stencil of every output of the patch, in its separable form
    // (weights_kernel): for each of the 4 + 2R window rows, the two row
    // filters H1 = sum_v W(v) x_(c+v) and H2 = sum_v v^2 W(v) x_(c+v) at the
    // patch's 4 columns, then every output row within reach adds
    // p(u) H1 + q(u) H2.  Adjacent columns go two per packed FP32
    // instruction: the window row's values sit in aligned register pairs
    // (16-byte shared loads), so a pair of symmetric taps whose first index
    // is even is one packed add, otherwise two scalar adds.
    float acc[4][4];
    {
        const float* sep = wint + kSepOff;
        float hw[R + 1], ha[R + 1], vp[R + 1], vq[R + 1];
#pragma unroll
        for (int k = 0; k <= R; ++k) {
            hw[k] = __ldg(sep + k);
            ha[k] = __ldg(sep + 4 + k);
            vp[k] = __ldg(sep + 8 + k);
            vq[k] = __ldg(sep + 12 + k);
        }
        float2 accp[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i) accp[i][0] = accp[i][1] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int ir = 0; ir < 4 + 2 * R; ++ir) {
            float in[4 * NV];
            const float4* src = reinterpret_cast<const float4*>(&tile[4 * ty + ir][4 * tx]);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float4 q = src[v];
                in[4 * v] = q.x; in[4 * v + 1] = q.y; in[4 * v + 2] = q.z; in[4 * v + 3] = q.w;
            }
            float2 h1[2], h2[2];
#pragma unroll
            for (int jp = 0; jp < 2; ++jp) {
                const int j = 2 * jp;
                float2 a1 = __fmul2_rn(make_float2(hw[0], hw[0]), make_float2(in[j + R], in[j + R + 1]));
                float2 a2 = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                    float2 sk;
                    if ((j + R - k) % 2 == 0) {
                        sk = __fadd2_rn(make_float2(in[j + R - k], in[j + R - k + 1]),
                                        make_float2(in[j + R + k], in[j + R + k + 1]));
                    } else {
                        sk = make_float2(in[j + R - k] + in[j + R + k], in[j + R - k + 1] + in[j + R + k + 1]);
                    }
                    a1 = __ffma2_rn(make_float2(hw[k], hw[k]), sk, a1);
                    a2 = k == 1 ? __fmul2_rn(make_float2(ha[k], ha[k]), sk)
                                : __ffma2_rn(make_float2(ha[k], ha[k]), sk, a2);
                }
                h1[jp] = a1;
                h2[jp] = a2;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int dx = ir - i;                      // window row of output row i
                if (dx < 0 || dx >= T) continue;
                const int u = dx < R ? R - dx : dx - R;
#pragma unroll
                for (int jp = 0; jp < 2; ++jp)
                    accp[i][jp] = __ffma2_rn(make_float2(vp[u], vp[u]), h1[jp],
                                             __ffma2_rn(make_float2(vq[u], vq[u]), h2[jp], accp[i][jp]));
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            acc[i][0] = accp[i][0].x; acc[i][1] = accp[i][0].y;
            acc[i][2] = accp[i][1].x; acc[i][3] = accp[i][1].y;
        }
    }
    {
        bool col_int[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) col_int[j] = ocol + j >= R && ocol + j <= g2 - 1 - R;
        const bool all_cols = col_int[0] && col_int[3];
        // 16-byte stores: pairs of doubles (even row length) or four floats
        // (row length a multiple of 4), from a 16-byte aligned output
        const bool vec_out = (g2 % (sizeof(Elem) == 4 ? 4 : 2)) == 0 && (reinterpret_cast<uintptr_t>(O) & 15u) == 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool row_int = orow + i >= R && orow + i <= g1 - 1 - R;
            const int64_t idx0 = static_cast<int64_t>(orow + i) * g2 + ocol;
            if constexpr (sizeof(Elem) == 4) {
                if (O && row_int) {
                    if (vec_out && all_cols) {
                        *reinterpret_cast<float4*>(O + idx0) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) if (col_int[j]) O[idx0 + j] = acc[i][j];
                    }
                }
            } else {
                unsigned long long o[4];
                bool bad = false;
#pragma unroll
                for (int j = 0; j < 4; ++j) o[j] = f2d_fast(acc[i][j], bad);
                if (__any_sync(0xffffffffu, bad)) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) o[j] = f2d_bits(acc[i][j]);
                }
                if (O && row_int) {
                    if (vec_out && all_cols) {
                        ulonglong2* dst = reinterpret_cast<ulonglong2*>(O + idx0);
                        dst[0] = make_ulonglong2(o[0], o[1]);
                        dst[1] = make_ulonglong2(o[2], o[3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) if (col_int[j]) O[idx0 + j] = o[j];
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float v = (row_int && col_int[j]) ? acc[i][j] : -INFINITY;
                if (v > best) { best = v; bsel = 4 * i + j; }
            }
        }
    }
    // The tile's edge outputs (fewer than R rows or columns to a grid edge),
    // one per thread, with the stencil of their edge class: edge columns (all
    // rows of the tile) first, then edge rows (the other columns).  They are
    // handed out from the last thread down: the last warps stage one row
    // fewer.
    float eb_v = -INFINITY;
    long long eb_i = -1;
    {
        const int nl = c0 == 0 ? min(R, g2) : 0;                           // left edge columns 0 .. nl-1
        const int cr0 = max(max(g2 - R, R), c0), cr1 = min(g2, c0 + kColsPerBlock);
        const int nr = max(0, cr1 - cr0);                                  // right edge columns cr0 ..
        const int nt = r0 == 0 ? min(R, g1) : 0;                           // top edge rows 0 .. nt-1
        const int rb0 = max(max(g1 - R, R), r0), rb1 = min(g1, r0 + kRowsPerBlock);
        const int nbm = max(0, rb1 - rb0);                                 // bottom edge rows rb0 ..
        const int nec = nl + nr, ner = nt + nbm;
        const int rows_here = min(kRowsPerBlock, g1 - r0);
        const int n1 = nec * rows_here, n2 = ner * kColsPerBlock;
        for (int t = static_cast<int>(blockDim.x) - 1 - static_cast<int>(threadIdx.x); t < n1 + n2; t += blockDim.x) {
            int r, c;
            if (t < n1) {
                const int e = t / rows_here;
                c = e < nl ? e : cr0 + (e - nl);
                r = r0 + t % rows_here;
            } else {
                const int e = (t - n1) / kColsPerBlock;
                r = e < nt ? e : rb0 + (e - nt);
                c = c0 + (t - n1) % kColsPerBlock;
                if (c >= g2 || c < R || c > g2 - 1 - R) continue;                // edge columns done above
            }
            const float* w = w32 + static_cast<int64_t>(cls(r, g1, R) * ncls + cls(c, g2, R)) * kMaxTaps;
            float a = 0.0f;
#pragma unroll
            for (int dx = 0; dx < T; ++dx)
#pragma unroll
                for (int dy = 0; dy < T; ++dy)
                    a = fmaf(__ldg(&w[dx * T + dy]), tile[r - r0 + dx][c - c0 + dy], a);
            const long long idx = static_cast<long long>(r) * g2 + c;
            if (O) {
                if constexpr (sizeof(Elem) == 4) O[idx] = a;
                else O[idx] = f2d_bits(a);
            }
            if (a > eb_v || (a == eb_v && idx < eb_i)) { eb_v = a; eb_i = idx; }
        }
    }
    // this thread's candidate: the interior best, or an edge output that is
    // larger, or equal at a lower index
    unsigned my_i = bsel >= 0 ? static_cast<unsigned>(orow + (bsel >> 2)) * static_cast<unsigned>(g2) +
                                    static_cast<unsigned>(ocol + (bsel & 3))
                              : 0xffffffffu;
    if (eb_i >= 0 && (eb_v > best || (eb_v == best && static_cast<unsigned>(eb_i) < my_i))) {
        best = eb_v;
        my_i = static_cast<unsigned>(eb_i);
    }
    // Argmax over the warp's outputs, without block barriers: the largest
    // value by max reductions, then the lowest index (within the grid,
    // below 2^31) holding it; one candidate per warp and tile, folded in
    // index order by argmax_kernel.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t q = (static_cast<int64_t>(s) * nb + slot) * kWarps2D + warp;
    {
        float m = best;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const unsigned cand = (best == m && m > -INFINITY) ? my_i : 0xffffffffu;
        const unsigned wi = __reduce_min_sync(0xffffffffu, cand);
        if (lane == 0) {
            part_v[q] = wi != 0xffffffffu ? order_key(f2d_bits(m)) : 0ull;
            part_i[q] = wi != 0xffffffffu ? static_cast<long long>(wi) : -1ll;
        }
    }
    if constexpr (RAW) {
        unsigned long long raw_k = raw.key;
        long long raw_i = raw.idx;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, raw_k, o);
            const long long i2 = __shfl_xor_sync(0xffffffffu, raw_i, o);
            amax(raw_k, raw_i, k2, i2);
        }
        if (lane == 0) { rpart_v[q] = raw_k; rpart_i[q] = raw_i; }
    }
}

// 2-D stencil, one block per tile of kRowsPerBlock x kColsPerBlock outputs,
// 256 threads.  The input window is staged as FP32 through registers
// (stage_rows, in three batches of rows, each with all its loads in flight
// at once), then tile_outputs.  VEC: g2 even and the input 16-byte aligned
// (pairs of doubles per load).
template <int R, bool RAW, bool VEC, typename Elem>
__global__ void __launch_bounds__(256, 4) smooth2d_kernel(const typename GridWord<Elem>::W* __restrict__ val, int g1,
                                                       int g2, const float* __restrict__ w32,
                                                       const float* __restrict__ wint,
                                                       typename GridWord<Elem>::W* __restrict__ out,
                                                       unsigned long long* part_v, long long* part_i,
                                                       unsigned long long* rpart_v, long long* rpart_i) {
    using TS = Tile2D<R>;
    __shared__ __align__(16) float tile[TS::SR][TS::SCP];
    const int s = blockIdx.z;
    const int r0 = blockIdx.y * kRowsPerBlock, c0 = blockIdx.x * kColsPerBlock;
    const typename GridWord<Elem>::W* V = val + static_cast<int64_t>(s) * g1 * g2;
    RunMax raw;
    raw.init();
    static_assert(TS::RPW == 5, "staging batches assume 5 rows per warp");
    stage_rows<R, RAW, VEC, 0, 2, TS::SR, TS::SCP, Elem>(V, g1, g2, r0, c0, tile, raw);
    stage_rows<R, RAW, VEC, 2, 4, TS::SR, TS::SCP, Elem>(V, g1, g2, r0, c0, tile, raw);
    stage_rows<R, RAW, VEC, 4, 5, TS::SR, TS::SCP, Elem>(V, g1, g2, r0, c0, tile, raw);
    __syncthreads();
    tile_outputs<R, RAW, Elem>(tile, g1, g2, s, r0, c0, w32, wint, out, gridDim.x * gridDim.y,
                            blockIdx.y * gridDim.x + blockIdx.x, part_v, part_i, rpart_v, rpart_i, raw);
}

// 1-D stencil along a line of n points.
template <int R, typename Elem>
__global__ void __launch_bounds__(256) smooth1d_kernel(const typename GridWord<Elem>::W* __restrict__ val, int n,
                                                       const float* __restrict__ w32,
                                                       typename GridWord<Elem>::W* __restrict__ out,
                                                       unsigned long long* part_v, long long* part_i,
                                                       unsigned long long* rpart_v, long long* rpart_i) {
    constexpr int T = 2 * R + 1;
    __shared__ float line[kLine + 2 * R];
    __shared__ unsigned long long sv[8];
    __shared__ long long si[8];
    const int s = blockIdx.y;
    const int c0 = blockIdx.x * kLine;
    const typename GridWord<Elem>::W* V = val + static_cast<int64_t>(s) * n;
    unsigned long long raw_v = 0;
    long long raw_i = -1;
    for (int q = threadIdx.x; q < kLine + 2 * R; q += blockDim.x) {
        const int g = c0 - R + q;
        float x = 0.0f;
        if (g >= 0 && g < n) {
            unsigned long long bits;
            if constexpr (sizeof(Elem) == 4) {
                x = __ldg(&V[g]);
                bits = f2d_bits(x);
            } else {
                bits = __ldg(&V[g]);
                x = d2f_bits(bits);
            }
            if (q >= R && q < R + kLine) amax_value(raw_v, raw_i, bits, g);
        }
        line[q] = x;
    }
    __syncthreads();
    unsigned long long best_v = 0;
    long long best_i = -1;
    for (int q = threadIdx.x; q < kLine; q += blockDim.x) {
        const int c = c0 + q;
        if (c >= n) break;
        const float* w = w32 + static_cast<int64_t>(cls(c, n, R)) * kMaxTaps;
        float acc = 0.0f;
#pragma unroll
        for (int dx = 0; dx < T; ++dx) acc = fmaf(__ldg(&w[dx]), line[q + dx], acc);
        const unsigned long long o = f2d_bits(acc);
        if (out) {
            if constexpr (sizeof(Elem) == 4) out[static_cast<int64_t>(s) * n + c] = acc;
            else out[static_cast<int64_t>(s) * n + c] = o;
        }
        amax_value(best_v, best_i, o, c);
    }
    const int nb = gridDim.x;
    block_amax(best_v, best_i, sv, si);
    if (threadIdx.x == 0) { part_v[static_cast<int64_t>(s) * nb + blockIdx.x] = best_v; part_i[static_cast<int64_t>(s) * nb + blockIdx.x] = best_i; }
    __syncthreads();
    block_amax(raw_v, raw_i, sv, si);
    if (threadIdx.x == 0) { rpart_v[static_cast<int64_t>(s) * nb + blockIdx.x] = raw_v; rpart_i[static_cast<int64_t>(s) * nb + blockIdx.x] = raw_i; }
}

// One block per scenario: fold its argmax candidates (largest key, then
// lowest index, so the order of the candidates does not matter).
template <typename Elem>
__global__ void argmax_kernel(int nb, const unsigned long long* part_v, const long long* part_i,
                              const unsigned long long* rpart_v, const long long* rpart_i, int64_t* idx,
                              Elem* v, int64_t* ridx, Elem* rv) {
    __shared__ unsigned long long sv[8];
    __shared__ long long si[8];
    const int s = blockIdx.x;
    unsigned long long bv = 0;
    long long bi = -1;
    for (int q = threadIdx.x; q < nb; q += blockDim.x)
        amax(bv, bi, part_v[static_cast<int64_t>(s) * nb + q], part_i[static_cast<int64_t>(s) * nb + q]);
    block_amax(bv, bi, sv, si);
    if (threadIdx.x == 0) {
        if (idx) idx[s] = bi;
        if (v) v[s] = static_cast<Elem>(bi >= 0 ? __longlong_as_double(static_cast<long long>(key_bits(bv))) : NAN);
    }
    if (!ridx && !rv) return;
    __syncthreads();
    bv = 0;
    bi = -1;
    for (int q = threadIdx.x; q < nb; q += blockDim.x)
        amax(bv, bi, rpart_v[static_cast<int64_t>(s) * nb + q], rpart_i[static_cast<int64_t>(s) * nb + q]);
    block_amax(bv, bi, sv, si);
    if (threadIdx.x == 0) {
        if (ridx) ridx[s] = bi;
        if (rv) rv[s] = static_cast<Elem>(bi >= 0 ? __longlong_as_double(static_cast<long long>(key_bits(bv))) : NAN);
    }
}

int blocks_per_scen(int g1, int g2);

// Argmax candidates of one scenario: one per block (1-D), one per warp and
// tile (2-D).
int candidates_per_scen(int g1, int g2) {
    return (g1 == 1 || g2 == 1) ? blocks_per_scen(g1, g2) : blocks_per_scen(g1, g2) * kWarps2D;
}

int blocks_per_scen(int g1, int g2) {
    if (g1 == 1 || g2 == 1) {
        const int n = g1 * g2;
        return (n + kLine - 1) / kLine;
    }
    return ((g2 + kColsPerBlock - 1) / kColsPerBlock) * ((g1 + kRowsPerBlock - 1) / kRowsPerBlock);
}

}  // namespace

const char* smooth_shape_error(int n_scen, int g1, int g2) {
    // launch limits: scenarios on gridDim.z (2-D) or gridDim.y (1-D), and
    // in 2-D the rows of blocks on gridDim.y, each at most 65535
    if (n_scen > 65535) return "at most 65535 scenarios per call";
    if (g1 > 1 && g2 > 1 && (g1 + kRowsPerBlock - 1) / kRowsPerBlock > 65535)
        return "g1 too large for the 2-D stencil (at most 65535 * 32 rows)";
    return nullptr;
}

size_t smooth_weight_count() {
    return static_cast<size_t>(kClassSlots) * kMaxTaps + kIntSlot;
}

// Argmax candidates: smoothed then raw, n_scen * candidates_per_scen each.
size_t smooth_candidate_count(int n_scen, int g1, int g2) {
    return 2 * static_cast<size_t>(n_scen) * candidates_per_scen(g1, g2);
}

namespace {

// wbuf / wbuf32: stencil weights (smooth_weight_count() each); part_val /
// part_idx: smooth_candidate_count() argmax candidates.
template <typename Elem>
cudaError_t smooth_argmax_t(int n_scen, int g1, int g2, const Elem* value, double bandwidth, int degree, Elem* smoothed,
                            int64_t* argmax_idx, Elem* argmax_val, int64_t* raw_idx, Elem* raw_val, double* wbuf,
                            float* wbuf32, double* part_val, int64_t* part_idx, DevStatus* status,
                            cudaStream_t stream) {
    using W = typename GridWord<Elem>::W;
    const int R = reach_of(bandwidth);
    const bool two_d = (g1 > 1 && g2 > 1);
    const int ncls = (R + 1) * (R + 1);
    const int nw = two_d ? ncls * ncls : ncls;
    const int gx = two_d ? g1 : g1 * g2;
    weights_kernel<<<(nw + 63) / 64, 64, 0, stream>>>(R, bandwidth, degree, two_d, gx, g2, wbuf, wbuf32,
                                                      status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb = blocks_per_scen(g1, g2);
    const int ncand = candidates_per_scen(g1, g2);
    unsigned long long* pv = reinterpret_cast<unsigned long long*>(part_val);
    long long* pi = reinterpret_cast<long long*>(part_idx);
    unsigned long long* rpv = pv + static_cast<size_t>(n_scen) * ncand;
    long long* rpi = pi + static_cast<size_t>(n_scen) * ncand;
    const W* vb = reinterpret_cast<const W*>(value);
    W* ob = reinterpret_cast<W*>(smoothed);
    if (two_d) {
        dim3 grid((g2 + kColsPerBlock - 1) / kColsPerBlock, (g1 + kRowsPerBlock - 1) / kRowsPerBlock, n_scen);
        const bool raw = raw_idx || raw_val;
        // one 16-byte (FP64) or 8-byte (FP32) load per pair of values when
        // every row starts on such a boundary
        const bool vec = (g2 % 2) == 0 && (reinterpret_cast<uintptr_t>(value) & (2 * sizeof(Elem) - 1)) == 0;
        const float* wint = wbuf32 + static_cast<size_t>(kClassSlots) * kMaxTaps;
        const int key = (R - 1) * 4 + (raw ? 2 : 0) + (vec ? 1 : 0);
        switch (key) {
#define MCD_SMOOTH2D(RR, RAW, VEC) \
            case (RR - 1) * 4 + (RAW ? 2 : 0) + (VEC ? 1 : 0): \
                smooth2d_kernel<RR, RAW, VEC, Elem><<<grid, 256, 0, stream>>>(vb, g1, g2, wbuf32, wint, ob, pv, pi, rpv, rpi); \
                break;
            MCD_SMOOTH2D(1, false, false) MCD_SMOOTH2D(1, false, true) MCD_SMOOTH2D(1, true, false) MCD_SMOOTH2D(1, true, true)
            MCD_SMOOTH2D(2, false, false) MCD_SMOOTH2D(2, false, true) MCD_SMOOTH2D(2, true, false) MCD_SMOOTH2D(2, true, true)
            MCD_SMOOTH2D(3, false, false) MCD_SMOOTH2D(3, false, true) MCD_SMOOTH2D(3, true, false) MCD_SMOOTH2D(3, true, true)
#undef MCD_SMOOTH2D
            default: return cudaErrorInvalidValue;
        }
    } else {
        dim3 grid(nb, n_scen);
        const int n = g1 * g2;
        if (R == 1) smooth1d_kernel<1, Elem><<<grid, 256, 0, stream>>>(vb, n, wbuf32, ob, pv, pi, rpv, rpi);
        else if (R == 2) smooth1d_kernel<2, Elem><<<grid, 256, 0, stream>>>(vb, n, wbuf32, ob, pv, pi, rpv, rpi);
        else smooth1d_kernel<3, Elem><<<grid, 256, 0, stream>>>(vb, n, wbuf32, ob, pv, pi, rpv, rpi);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    argmax_kernel<Elem><<<n_scen, 256, 0, stream>>>(ncand, pv, pi, rpv, rpi, argmax_idx, argmax_val, raw_idx, raw_val);
    return cudaGetLastError();
}

}  // namespace

cudaError_t smooth_argmax(int n_scen, int g1, int g2, const double* value, double bandwidth,
                          int degree, double* smoothed, int64_t* argmax_idx, double* argmax_val,
                          int64_t* raw_idx, double* raw_val, double* wbuf, float* wbuf32,
                          double* part_val, int64_t* part_idx, DevStatus* status, cudaStream_t stream) {
    return smooth_argmax_t<double>(n_scen, g1, g2, value, bandwidth, degree, smoothed, argmax_idx, argmax_val,
                                   raw_idx, raw_val, wbuf, wbuf32, part_val, part_idx, status, stream);
}

cudaError_t smooth_argmax_f32(int n_scen, int g1, int g2, const float* value, double bandwidth,
                              int degree, float* smoothed, int64_t* argmax_idx, float* argmax_val,
                              int64_t* raw_idx, float* raw_val, double* wbuf, float* wbuf32,
                              double* part_val, int64_t* part_idx, DevStatus* status, cudaStream_t stream) {
    return smooth_argmax_t<float>(n_scen, g1, g2, value, bandwidth, degree, smoothed, argmax_idx, argmax_val,
                                  raw_idx, raw_val, wbuf, wbuf32, part_val, part_idx, status, stream);
}

}  // namespace mcd
