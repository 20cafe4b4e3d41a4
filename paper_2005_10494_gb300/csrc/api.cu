// Host side of the C ABI declared in include/mcdesign.h: contexts, plans
// (tile schedule, workspace, autotuning, CUDA-graph replay), launches and
// argument validation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fwer.cuh"
#include "tps.cuh"
#include "mcd_internal.cuh"
#include "pipes.cuh"
#include "smooth.cuh"

using namespace mcd;

namespace {

// Launch shape of one sampling kernel: block size and tile size, the latter
// as a multiple of the default tile of each dimension.
struct LaunchCfg {
    int threads = 256;
    double scale = 1.0;
};

// Issued instructions per draw, roughly: Philox (~10 per normal), Box-Muller
// (~7 per normal), transform d(d+1)/2, compares and bookkeeping.
double draw_cost(int d) { return 17.0 * d + 0.5 * d * (d + 1) + 6.0; }

int group_of(int d) { return (d % 4 == 0) ? 1 : ((d % 2 == 0) ? 2 : 4); }

// Draws per tile: about 32k issued instructions per thread, a whole number
// of draw groups per thread.
int64_t tile_draws(int d, const LaunchCfg& c) {
    const double per_thread = c.scale * 32768.0 / draw_cost(d);
    const int g = group_of(d);
    int64_t groups = static_cast<int64_t>(std::llround(per_thread / g));
    if (groups < 1) groups = 1;
    return groups * g * c.threads;
}

// One persistent launch: the tiles [tile_begin, tile_begin + n_tiles) of the
// schedule, all of dimension d_lo..d_hi (d_lo < d_hi: the mixed kernel).
struct Segment {
    int d_lo = 0, d_hi = 0;
    int64_t tile_begin = 0, n_tiles = 0;
    LaunchCfg cfg;
    int grid = 0;
    int blocks_per_sm = 0;
};

// One launch of the shared-draw kernel: the shared tiles
// [tile_begin, tile_begin + n_tiles) of dimension d.
struct SharedSeg {
    int d = 0;
    int64_t tile_begin = 0, n_tiles = 0;
    int64_t tile_draws = 0;
    int grid = 0;
    int blocks_per_sm = 0;
};

// Which tiles a plan keeps (the autotuner times filtered plans).
struct TileFilter {
    int d_lo = 1, d_hi = MCD_MAX_D;
    int64_t stride = 1;
};

struct TuneKey {
    int d_lo, d_hi;
    bool grad, fp64;
    bool operator<(const TuneKey& o) const {
        return std::tie(d_lo, d_hi, grad, fp64) < std::tie(o.d_lo, o.d_hi, o.grad, o.fp64);
    }
};

}  // namespace

struct mcd_ctx {
    int device = 0;
    int sm_count = 0;
    std::string err = "no error";
    int64_t err_index = -1;
    DevStatus* d_status = nullptr;
    std::map<TuneKey, LaunchCfg> tuned;
    std::mutex mu;
    int inject = 0;                  // mcd_debug_fail_next: CUDA error of the next plan launch
};

struct mcd_plan {
    mcd_ctx* ctx = nullptr;
    int device = 0;                  // the context's GPU: destroy must not read *ctx (it may be gone)
    bool stream_ordered = false;     // one-shot plan: allocations on a stream
    cudaStream_t alloc_stream = nullptr;
    int32_t S = 0, J = 0, region = 0, k = 0, flags = 0;
    bool fp64 = false;
    std::vector<Segment> segs;       // sampling launches, in order
    std::vector<int> seg_of_d;       // segment index of each dimension, -1 if none
    std::vector<int64_t> tile_draws_of_d;  // per d
    int64_t n_tiles = 0;
    std::vector<SharedSeg> ssegs;    // shared-draw launches, after the per-design ones
    int64_t n_shared_tiles = 0;
    int batches = 1;
    const double* Sigma = nullptr;
    const double* mu = nullptr;
    const double* b = nullptr;
    // device
    DesignRec* d_designs = nullptr;
    TileRec* d_tiles = nullptr;
    int64_t* d_sig_off = nullptr;
    int32_t* d_scen_d = nullptr;
    int64_t* d_L_off = nullptr;
    float* d_L32 = nullptr;
    double* d_L64 = nullptr;
    int32_t* d_scen_ok = nullptr;
    uint64_t* d_n_draws = nullptr;
    uint64_t* d_batch_draws = nullptr;
    unsigned long long* d_hits = nullptr;
    unsigned long long* d_gacc = nullptr;
    unsigned int* d_ticket = nullptr;  // one tile counter per segment (per-design, then shared)
    SharedTile* d_stiles = nullptr;
    uint32_t* d_slist = nullptr;       // designs of the shared tiles, chunk by chunk
    size_t gacc_len = 0;
    std::vector<void*> owned;
    // CUDA graphs, one per launch kind (0 eval, 1 grad)
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    std::vector<uint64_t> gargs[2];
    // MCD_PLAN_TIMING: events around the sampling launches
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace {

// NVTX range around one entry point (a no-op unless a profiler is attached),
// so that traces show planning, launches, calibration and smoothing apart.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

mcd_status fail(mcd_ctx* ctx, mcd_status code, const std::string& msg, int64_t index = -1) {
    if (ctx) {
        ctx->err = msg;
        ctx->err_index = index;
    }
    return code;
}

mcd_status cuda_fail(mcd_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? MCD_ENOMEM : MCD_ECUDA, m);
}

#define MCD_CUDA(call, what)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
mcd_status plan_alloc(mcd_plan* pl, T** out, size_t count) {
    mcd_ctx* ctx = pl->ctx;
    *out = nullptr;
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaError_t e = pl->stream_ordered ? cudaMallocAsync(&p, count * sizeof(T), pl->alloc_stream)
                                       : cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device allocation");
    pl->owned.push_back(p);
    *out = static_cast<T*>(p);
    return MCD_OK;
}

template <typename T>
mcd_status plan_upload(mcd_plan* pl, T* dst, const std::vector<T>& src) {
    mcd_ctx* ctx = pl->ctx;
    if (src.empty()) return MCD_OK;
    cudaError_t e = pl->stream_ordered
                        ? cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, pl->alloc_stream)
                        : cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upload");
    // a pageable source has been staged when cudaMemcpyAsync returns, so the
    // host vector may be released afterwards
    return MCD_OK;
}

void plan_release(mcd_plan* pl) {
    for (int i = 0; i < 2; ++i) {
        if (pl->gexec[i]) cudaGraphExecDestroy(pl->gexec[i]);
        pl->gexec[i] = nullptr;
        if (pl->ev[i]) cudaEventDestroy(pl->ev[i]);
        pl->ev[i] = nullptr;
    }
    for (void* p : pl->owned) {
        if (pl->stream_ordered) cudaFreeAsync(p, pl->alloc_stream);
        else cudaFree(p);
    }
    pl->owned.clear();
}

mcd_status validate_problem(mcd_ctx* ctx, const mcd_problem* pr, int32_t k) {
    if (!pr) return fail(ctx, MCD_EINVAL, "problem is NULL");
    if (pr->n_scen < 1) return fail(ctx, MCD_EINVAL, "n_scen must be >= 1");
    if (pr->n_design < 0) return fail(ctx, MCD_EINVAL, "n_design must be >= 0");
    if (pr->region != MCD_ANY_EXCEEDS && pr->region != MCD_ALL_BELOW)
        return fail(ctx, MCD_EINVAL, "region must be MCD_ANY_EXCEEDS or MCD_ALL_BELOW");
    if (k < 0 || k > 8) return fail(ctx, MCD_EINVAL, "k must be in 0..8");
    if (!pr->scen_d) return fail(ctx, MCD_EINVAL, "scen_d is NULL");
    if (!pr->Sigma) return fail(ctx, MCD_EINVAL, "Sigma is NULL");
    if (!is_device_ptr(pr->Sigma)) return fail(ctx, MCD_EINVAL, "Sigma is not device memory");
    for (int s = 0; s < pr->n_scen; ++s) {
        const int d = pr->scen_d[s];
        if (d < 1) return fail(ctx, MCD_EINVAL, "scenario dimension must be >= 1", s);
        if (d > MCD_MAX_D) return fail(ctx, MCD_EUNSUPPORTED, "scenario dimension above MCD_MAX_D", s);
    }
    if (pr->n_design == 0) return MCD_OK;
    if (!pr->design_scen || !pr->n_draws || !pr->key)
        return fail(ctx, MCD_EINVAL, "design_scen, n_draws and key must not be NULL");
    if (!pr->mu || !pr->b) return fail(ctx, MCD_EINVAL, "mu and b must not be NULL");
    if (!is_device_ptr(pr->mu) || !is_device_ptr(pr->b))
        return fail(ctx, MCD_EINVAL, "mu and b must be device memory");
    for (int j = 0; j < pr->n_design; ++j) {
        const int s = pr->design_scen[j];
        if (s < 0 || s >= pr->n_scen) return fail(ctx, MCD_EINVAL, "design_scen out of range", j);
        const uint64_t d = static_cast<uint64_t>(pr->scen_d[s]);
        const uint64_t begin = pr->draw_begin ? pr->draw_begin[j] : 0;
        const uint64_t n = pr->n_draws[j];
        const uint64_t lim = (1ull << 62) / d;
        if (begin > lim || n > lim - begin)
            return fail(ctx, MCD_EINVAL, "(draw_begin + n_draws) * d must stay below 2^62", j);
    }
    return MCD_OK;
}

// Host-side planning: tiles, batch slots, offsets; uploads; workspace.
// The filter keeps only some designs' tiles (the autotuner's timing plans).
mcd_status plan_build(mcd_ctx* ctx, const mcd_problem* pr, int32_t flags, int32_t k, mcd_plan* pl,
                      const TileFilter& filt = TileFilter()) {
    pl->ctx = ctx;
    pl->device = ctx->device;
    pl->S = pr->n_scen;
    pl->J = pr->n_design;
    pl->region = pr->region;
    pl->k = k;
    pl->flags = flags;
    pl->fp64 = (flags & MCD_PLAN_FP64) != 0;
    pl->Sigma = pr->Sigma;
    pl->mu = pr->mu;
    pl->b = pr->b;
    const int S = pl->S, J = pl->J;
    const bool grad_kernel = (flags & MCD_PLAN_GRAD) != 0;

    // common-random-number groups for the shared-draw kernel
    std::vector<char> is_shared(J, 0);
    std::vector<std::vector<int>> groups;
    if (flags & MCD_PLAN_SHARED) {
        if (pl->fp64) return fail(ctx, MCD_EUNSUPPORTED, "MCD_PLAN_SHARED is not available with MCD_PLAN_FP64");
        std::map<std::tuple<int, uint64_t, uint64_t, uint64_t>, std::vector<int>> by;
        for (int j = 0; j < J; ++j) {
            const uint64_t begin = pr->draw_begin ? pr->draw_begin[j] : 0;
            if (pr->n_draws[j] == 0) continue;
            by[std::make_tuple(pr->design_scen[j], pr->key[j], begin, pr->n_draws[j])].push_back(j);
        }
        for (auto& kv : by) {
            if (static_cast<int>(kv.second.size()) < MCD_SHARED_MIN) continue;
            for (int j : kv.second) is_shared[j] = 1;
            groups.push_back(std::move(kv.second));
        }
    }

    std::vector<int64_t> sig_off(S), L_off(S);
    std::vector<int32_t> scen_d(pr->scen_d, pr->scen_d + S);
    int64_t so = 0, lo = 0;
    for (int s = 0; s < S; ++s) {
        sig_off[s] = so;
        L_off[s] = lo;
        so += static_cast<int64_t>(scen_d[s]) * scen_d[s];
        lo += static_cast<int64_t>(scen_d[s]) * (scen_d[s] + 1) / 2;
    }
    // segments: all d <= kMixedMaxD in one launch (the mixed kernel when
    // they differ), each larger d in its own launch
    std::vector<int> present(MCD_MAX_D + 1, 0);
    for (int j = 0; j < J; ++j)
        if (!is_shared[j]) present[scen_d[pr->design_scen[j]]] = 1;
    int n_small = 0, small_lo = MCD_MAX_D + 1;
    for (int d = 1; d <= kMixedMaxD; ++d)
        if (present[d]) { ++n_small; small_lo = std::min(small_lo, d); }
    if (pl->fp64) {
        int n_present = 0;
        for (int d = 1; d <= MCD_MAX_D; ++d) n_present += present[d];
        if (n_present > 1) return fail(ctx, MCD_EUNSUPPORTED, "the FP64 path needs designs of one dimension");
    }
    pl->seg_of_d.assign(MCD_MAX_D + 1, -1);
    pl->segs.clear();
    if (n_small > 0) {
        Segment sg;
        sg.d_lo = (n_small == 1) ? small_lo : 1;
        sg.d_hi = (n_small == 1) ? small_lo : kMixedMaxD;
        for (int d = 1; d <= kMixedMaxD; ++d) if (present[d]) pl->seg_of_d[d] = 0;
        pl->segs.push_back(sg);
    }
    for (int d = kMixedMaxD + 1; d <= MCD_MAX_D; ++d) {
        if (!present[d]) continue;
        Segment sg;
        sg.d_lo = sg.d_hi = d;
        pl->seg_of_d[d] = static_cast<int>(pl->segs.size());
        pl->segs.push_back(sg);
    }
    pl->tile_draws_of_d.assign(MCD_MAX_D + 1, 0);
    for (auto& sg : pl->segs) {
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            auto it = ctx->tuned.find({sg.d_lo, sg.d_hi, grad_kernel, pl->fp64});
            if (it != ctx->tuned.end()) sg.cfg = it->second;
        }
        for (int d = sg.d_lo; d <= sg.d_hi; ++d) pl->tile_draws_of_d[d] = tile_draws(d, sg.cfg);
    }

    // designs, tiles and batch slots
    std::vector<DesignRec> designs(J);
    std::vector<uint64_t> n_draws(pr->n_draws, pr->n_draws + J);
    int64_t vo = 0, total_tiles = 0, max_tiles = 1;
    std::vector<int64_t> tiles_of(J);
    for (int j = 0; j < J; ++j) {
        const int s = pr->design_scen[j];
        const int d = scen_d[s];
        designs[j].key = pr->key[j];
        designs[j].vec_off = vo;
        designs[j].scen = s;
        designs[j].d = d;
        vo += d;
        const int64_t T = pl->tile_draws_of_d[d];
        const bool keep = !is_shared[j] && (j % filt.stride == 0) && d >= filt.d_lo && d <= filt.d_hi;
        tiles_of[j] = keep ? static_cast<int64_t>((n_draws[j] + T - 1) / T) : 0;
        total_tiles += tiles_of[j];
        max_tiles = std::max(max_tiles, tiles_of[j]);
    }

    // shared-draw schedule: per dimension one launch; a group is cut into
    // chunks of at most kSharedThreads * (designs per thread) designs of
    // balanced size, and its draw range into tiles of whole batches sized so
    // that each launch has about 16 tiles per resident block
    struct SChunk { int g; size_t first, cnt; };
    std::vector<SChunk> chunks;
    std::vector<int64_t> stile_draws(MCD_MAX_D + 1, 0);
    pl->ssegs.clear();
    {
        std::vector<double> chunk_draws(MCD_MAX_D + 1, 0.0);
        for (size_t g = 0; g < groups.size(); ++g) {
            const int d = scen_d[pr->design_scen[groups[g][0]]];
            const size_t cap = static_cast<size_t>(kSharedThreads) * shared_designs_per_thread(d, grad_kernel);
            const size_t m = groups[g].size(), nch = (m + cap - 1) / cap, per = (m + nch - 1) / nch;
            for (size_t c = 0; c < m; c += per) chunks.push_back({static_cast<int>(g), c, std::min(per, m - c)});
            chunk_draws[d] += static_cast<double>(nch) * static_cast<double>(n_draws[groups[g][0]]);
        }
        for (int d = 1; d <= MCD_MAX_D; ++d) {
            if (chunk_draws[d] == 0.0) continue;
            SharedSeg sg;
            sg.d = d;
            int bps = 0;
            cudaError_t e = shared_occupancy(d, grad_kernel, &bps);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy query");
            sg.blocks_per_sm = std::max(1, bps);
            const double bd = shared_batch_draws(d);
            const double want = chunk_draws[d] / (16.0 * ctx->sm_count * sg.blocks_per_sm);
            const int64_t mult = std::max<int64_t>(1, std::min<int64_t>(256, std::llround(want / bd)));
            sg.tile_draws = mult * static_cast<int64_t>(bd);
            stile_draws[d] = sg.tile_draws;
            pl->ssegs.push_back(sg);
        }
        for (const SChunk& c : chunks) {
            const int j0 = groups[c.g][0];
            const int64_t T = stile_draws[scen_d[pr->design_scen[j0]]];
            max_tiles = std::max<int64_t>(max_tiles, static_cast<int64_t>((n_draws[j0] + T - 1) / T));
        }
    }
    if (total_tiles >= (1ll << 31)) return fail(ctx, MCD_EINVAL, "too many tiles (reduce n_draws)");
    pl->n_tiles = total_tiles;
    pl->batches = static_cast<int>(std::min<int64_t>(kMaxBatches, max_tiles));
    const int B = pl->batches;
    // A gradient slot is a signed 64-bit fixed-point sum at 2^-28 of |z| <=
    // sqrt(48 ln 2) < 5.8 per draw; at most 2^32 draws per slot keep it
    // below 5.8 * 2^60 < 2^63.
    constexpr uint64_t kMaxSlotDraws = 1ull << 32;
    if (grad_kernel) {
        for (int j = 0; j < J; ++j) {
            const int64_t T = pl->tile_draws_of_d[designs[j].d];
            const uint64_t per = static_cast<uint64_t>((tiles_of[j] + B - 1) / B) * static_cast<uint64_t>(T);
            if (per > kMaxSlotDraws)
                return fail(ctx, MCD_EINVAL, "n_draws too large for a gradient plan (2^32 draws per batch slot, 32 slots)", j);
        }
        for (const SChunk& c : chunks) {
            const int j0 = groups[c.g][0];
            const int64_t T = stile_draws[scen_d[pr->design_scen[j0]]];
            const uint64_t ranges = (n_draws[j0] + T - 1) / T;
            if ((ranges + B - 1) / B * static_cast<uint64_t>(T) > kMaxSlotDraws)
                return fail(ctx, MCD_EINVAL, "n_draws too large for a gradient plan (2^32 draws per batch slot, 32 slots)", j0);
        }
    }
    for (int j = 0; j < J; ++j) designs[j].acc_off = 3 * designs[j].vec_off * B;
    pl->gacc_len = static_cast<size_t>(3) * vo * B;

    std::vector<TileRec> tiles;
    tiles.reserve(static_cast<size_t>(total_tiles));
    std::vector<uint64_t> batch_draws(static_cast<size_t>(J) * B, 0);
    for (int j = 0; j < J; ++j) {
        const int d = designs[j].d;
        const int64_t T = pl->tile_draws_of_d[d];
        const uint64_t begin = pr->draw_begin ? pr->draw_begin[j] : 0;
        for (int64_t t = 0; t < tiles_of[j]; ++t) {
            TileRec tr;
            tr.start = begin + static_cast<uint64_t>(t) * T;
            const uint64_t rem = n_draws[j] - static_cast<uint64_t>(t) * T;
            tr.n = static_cast<uint32_t>(std::min<uint64_t>(rem, static_cast<uint64_t>(T)));
            tr.design = static_cast<uint32_t>(j);
            tr.batch = static_cast<uint32_t>(t % B);
            tr.pad = 0;
            batch_draws[static_cast<size_t>(j) * B + tr.batch] += tr.n;
            tiles.push_back(tr);
        }
    }
    // shared tiles and their design lists
    std::vector<SharedTile> stiles;
    std::vector<uint32_t> slist;
    for (const SChunk& c : chunks) {
        const std::vector<int>& gr = groups[c.g];
        const int j0 = gr[c.first];
        const int d = scen_d[pr->design_scen[j0]];
        const int64_t T = stile_draws[d];
        const uint64_t begin = pr->draw_begin ? pr->draw_begin[j0] : 0;
        const uint64_t n = n_draws[j0];
        const uint32_t off = static_cast<uint32_t>(slist.size());
        for (size_t q = 0; q < c.cnt; ++q) slist.push_back(static_cast<uint32_t>(gr[c.first + q]));
        const int64_t ranges = static_cast<int64_t>((n + T - 1) / T);
        // draws the chunk's tiles add to each batch slot, added to each of
        // its designs once (not once per tile and design)
        std::vector<uint64_t> chunk_batch(static_cast<size_t>(B), 0);
        for (int64_t r = 0; r < ranges; ++r) {
            SharedTile st;
            st.start = begin + static_cast<uint64_t>(r) * T;
            st.n = static_cast<uint32_t>(std::min<uint64_t>(n - static_cast<uint64_t>(r) * T, static_cast<uint64_t>(T)));
            st.key = pr->key[j0];
            st.list_off = off;
            st.list_cnt = static_cast<uint32_t>(c.cnt);
            st.batch = static_cast<uint32_t>(r % B);
            st.scen = pr->design_scen[j0];
            st.pad = 0;
            chunk_batch[st.batch] += st.n;
            stiles.push_back(st);
        }
        for (size_t q = 0; q < c.cnt; ++q)
            for (int bb = 0; bb < B; ++bb)
                batch_draws[static_cast<size_t>(gr[c.first + q]) * B + bb] += chunk_batch[static_cast<size_t>(bb)];
    }
    if (static_cast<int64_t>(stiles.size()) + total_tiles >= (1ll << 31))
        return fail(ctx, MCD_EINVAL, "too many tiles (reduce n_draws)");
    std::stable_sort(stiles.begin(), stiles.end(), [&](const SharedTile& a, const SharedTile& c) {
        const int da = scen_d[a.scen], dc = scen_d[c.scen];
        if (da != dc) return da < dc;
        return static_cast<double>(a.list_cnt) * a.n > static_cast<double>(c.list_cnt) * c.n;
    });
    {
        int64_t pos = 0;
        for (SharedSeg& sg : pl->ssegs) {
            sg.tile_begin = pos;
            while (pos < static_cast<int64_t>(stiles.size()) && scen_d[stiles[pos].scen] == sg.d) ++pos;
            sg.n_tiles = pos - sg.tile_begin;
            const int64_t g = static_cast<int64_t>(sg.blocks_per_sm) * ctx->sm_count;
            sg.grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, sg.n_tiles)));
        }
    }
    pl->n_shared_tiles = static_cast<int64_t>(stiles.size());

    // by segment, and within a segment the costliest tiles first: the
    // dynamic ticket then leaves only small tiles for the tail
    std::stable_sort(tiles.begin(), tiles.end(), [&](const TileRec& a, const TileRec& c) {
        const int sa = pl->seg_of_d[designs[a.design].d], sc = pl->seg_of_d[designs[c.design].d];
        if (sa != sc) return sa < sc;
        const double ca = draw_cost(designs[a.design].d) * a.n, cc = draw_cost(designs[c.design].d) * c.n;
        return ca > cc;
    });
    {
        int64_t pos = 0;
        for (size_t q = 0; q < pl->segs.size(); ++q) {
            Segment& sg = pl->segs[q];
            sg.tile_begin = pos;
            while (pos < static_cast<int64_t>(tiles.size()) && pl->seg_of_d[designs[tiles[pos].design].d] == static_cast<int>(q)) ++pos;
            sg.n_tiles = pos - sg.tile_begin;
        }
    }

    mcd_status st;
    if ((st = plan_alloc(pl, &pl->d_designs, J)) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_tiles, tiles.size())) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_sig_off, S)) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_scen_d, S)) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_L_off, S)) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_L32, lo)) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_L64, lo)) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_scen_ok, S)) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_n_draws, J)) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_batch_draws, batch_draws.size())) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_hits, J)) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_ticket, std::max<size_t>(1, pl->segs.size() + pl->ssegs.size()))) != MCD_OK)
        return st;
    if ((st = plan_alloc(pl, &pl->d_stiles, stiles.size())) != MCD_OK) return st;
    if ((st = plan_alloc(pl, &pl->d_slist, slist.size())) != MCD_OK) return st;
    if (grad_kernel && (st = plan_alloc(pl, &pl->d_gacc, pl->gacc_len)) != MCD_OK) return st;

    if ((st = plan_upload(pl, pl->d_designs, designs)) != MCD_OK) return st;
    if ((st = plan_upload(pl, pl->d_tiles, tiles)) != MCD_OK) return st;
    if ((st = plan_upload(pl, pl->d_sig_off, sig_off)) != MCD_OK) return st;
    if ((st = plan_upload(pl, pl->d_scen_d, scen_d)) != MCD_OK) return st;
    if ((st = plan_upload(pl, pl->d_L_off, L_off)) != MCD_OK) return st;
    if ((st = plan_upload(pl, pl->d_n_draws, n_draws)) != MCD_OK) return st;
    if ((st = plan_upload(pl, pl->d_batch_draws, batch_draws)) != MCD_OK) return st;
    if ((st = plan_upload(pl, pl->d_stiles, stiles)) != MCD_OK) return st;
    if ((st = plan_upload(pl, pl->d_slist, slist)) != MCD_OK) return st;

    if (flags & MCD_PLAN_TIMING) {
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = cudaEventCreate(&pl->ev[i]);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "event create");
        }
    }
    // persistent grids: resident blocks per SM x SMs
    for (auto& sg : pl->segs) {
        int bps = 0;
        cudaError_t e = sample_occupancy(sg.d_lo, sg.d_hi, grad_kernel, pl->fp64, sg.cfg.threads, &bps);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy query");
        if (bps < 1) bps = 1;
        sg.blocks_per_sm = bps;
        const int64_t g = static_cast<int64_t>(bps) * ctx->sm_count;
        sg.grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, std::max<int64_t>(1, sg.n_tiles))));
    }
    return MCD_OK;
}

void fill_round_keys(uint64_t seed, SampleParams& sp) {
    for (int r = 0; r < 10; ++r) {
        sp.rk0[r] = static_cast<uint32_t>(seed) + static_cast<uint32_t>(r) * kPhiloxW0;
        sp.rk1[r] = static_cast<uint32_t>(seed >> 32) + static_cast<uint32_t>(r) * kPhiloxW1;
    }
}

struct LaunchArgs {
    bool grad = false;
    uint64_t seed = 0;
    const double* jac = nullptr;
    double h = 0.0;
    uint64_t* hits = nullptr;
    double* p = nullptr;
    double* se = nullptr;
    double* g_lr = nullptr;
    double* g_sig = nullptr;
    double* g_se = nullptr;
};

// The whole launch sequence of one evaluation on `stream`.
mcd_status enqueue(mcd_plan* pl, const LaunchArgs& a, cudaStream_t stream) {
    {
        // host-side fault injection: report the chosen CUDA error, queue nothing
        mcd_ctx* c = pl->ctx;
        std::lock_guard<std::mutex> lk(c->mu);
        if (c->inject != 0) {
            const cudaError_t e = static_cast<cudaError_t>(c->inject);
            c->inject = 0;
            c->err = std::string("launch: ") + cudaGetErrorString(e) + " (injected by mcd_debug_fail_next)";
            c->err_index = -1;
            return MCD_ECUDA;
        }
    }
    mcd_ctx* ctx = pl->ctx;
    if (a.grad && (pl->k > 0) != (a.jac != nullptr))
        return fail(ctx, MCD_EINVAL, "the Jacobian must be given exactly when the plan has k > 0");
    if (a.grad && !pl->d_gacc && pl->gacc_len) return fail(ctx, MCD_EINVAL, "plan has no gradient workspace");
    MCD_CUDA(cudaMemsetAsync(pl->d_ticket, 0,
                             sizeof(unsigned int) * std::max<size_t>(1, pl->segs.size() + pl->ssegs.size()), stream),
             "memset");
    if (pl->J > 0) MCD_CUDA(cudaMemsetAsync(pl->d_hits, 0, sizeof(unsigned long long) * pl->J, stream), "memset");
    if (a.grad && pl->gacc_len)
        MCD_CUDA(cudaMemsetAsync(pl->d_gacc, 0, sizeof(unsigned long long) * pl->gacc_len, stream), "memset");
    MCD_CUDA(launch_cholesky(pl->Sigma, pl->d_sig_off, pl->d_scen_d, pl->d_L_off, pl->S, pl->d_L32, pl->d_L64,
                             pl->d_scen_ok, ctx->d_status, stream), "cholesky launch");
    // under stream capture the timing events must become event-record nodes
    // of the graph (cudaEventRecordExternal), not capture-internal joins
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    MCD_CUDA(cudaStreamIsCapturing(stream, &capturing), "cudaStreamIsCapturing");
    const unsigned ev_flags = capturing == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (pl->ev[0]) MCD_CUDA(cudaEventRecordWithFlags(pl->ev[0], stream, ev_flags), "event record");
    auto base_params = [&](SampleParams& sp) {
        std::memset(&sp, 0, sizeof(sp));
        sp.designs = pl->d_designs;
        sp.L32 = pl->d_L32;
        sp.L64 = pl->d_L64;
        sp.L_off = pl->d_L_off;
        sp.scen_ok = pl->d_scen_ok;
        sp.mu = pl->mu;
        sp.b = pl->b;
        sp.hits = pl->d_hits;
        sp.gacc = pl->d_gacc;
        sp.batches = pl->batches;
        sp.hinv_log2e = (a.grad && a.h > 0.0) ? static_cast<float>(1.4426950408889634 / a.h) : 0.0f;
        sp.sig_skip_w = (a.grad && a.h > 0.0) ? static_cast<float>(25.03 * a.h / 1.4426950408889634) : -1.0f;
        sp.hinv = (a.grad && a.h > 0.0) ? 1.0 / a.h : 0.0;
        sp.status = ctx->d_status;
        fill_round_keys(a.seed, sp);
    };
    for (size_t q = 0; q < pl->ssegs.size(); ++q) {
        const SharedSeg& sg = pl->ssegs[q];
        if (sg.n_tiles == 0) continue;
        SampleParams sp;
        base_params(sp);
        sp.n_tiles = sg.n_tiles;
        sp.ticket = pl->d_ticket + pl->segs.size() + q;
        MCD_CUDA(launch_shared(sg.d, a.grad, sp, pl->d_stiles + sg.tile_begin, pl->d_slist, sg.grid, stream),
                 "shared-draw launch");
    }
    for (size_t q = 0; q < pl->segs.size(); ++q) {
        const Segment& sg = pl->segs[q];
        if (sg.n_tiles == 0) continue;
        SampleParams sp;
        base_params(sp);
        sp.tiles = pl->d_tiles + sg.tile_begin;
        sp.n_tiles = sg.n_tiles;
        sp.ticket = pl->d_ticket + q;
        MCD_CUDA(launch_sample(sg.d_lo, sg.d_hi, a.grad, pl->fp64, sp, sg.grid, sg.cfg.threads, stream),
                 "sampling launch");
    }
    if (pl->ev[1]) MCD_CUDA(cudaEventRecordWithFlags(pl->ev[1], stream, ev_flags), "event record");
    FinalizeParams fp;
    std::memset(&fp, 0, sizeof(fp));
    fp.designs = pl->d_designs;
    fp.n_design = pl->J;
    fp.n_draws = pl->d_n_draws;
    fp.hits = pl->d_hits;
    fp.gacc = pl->d_gacc;
    fp.batch_draws = pl->d_batch_draws;
    fp.batches = pl->batches;
    fp.L64 = pl->d_L64;
    fp.L_off = pl->d_L_off;
    fp.jac = a.jac;
    fp.k = pl->k;
    fp.region = pl->region;
    fp.hinv = (a.grad && a.h > 0.0) ? 1.0 / a.h : 0.0;
    fp.out_hits = a.hits;
    fp.out_p = a.p;
    fp.out_se = a.se;
    fp.g_lr = a.g_lr;
    fp.g_sig = a.g_sig;
    fp.g_se = a.g_se;
    MCD_CUDA(launch_finalize(fp, a.grad, stream), "finalize launch");
    return MCD_OK;
}

std::vector<uint64_t> graph_key(const LaunchArgs& a) {
    return {a.grad, a.seed, reinterpret_cast<uint64_t>(a.jac), static_cast<uint64_t>(std::llround(a.h * 1e15)),
            reinterpret_cast<uint64_t>(a.hits), reinterpret_cast<uint64_t>(a.p), reinterpret_cast<uint64_t>(a.se),
            reinterpret_cast<uint64_t>(a.g_lr), reinterpret_cast<uint64_t>(a.g_sig), reinterpret_cast<uint64_t>(a.g_se)};
}

// Run through a captured graph when the plan asks for it and the stream can
// be captured (not the legacy default stream); re-capture when the
// arguments change.
mcd_status launch(mcd_plan* pl, const LaunchArgs& a, cudaStream_t stream) {
    mcd_ctx* ctx = pl->ctx;
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MCD_CUDA(cudaStreamIsCapturing(stream, &cs), "cudaStreamIsCapturing");
    const bool use_graph = (pl->flags & MCD_PLAN_GRAPH) && stream != nullptr && cs == cudaStreamCaptureStatusNone;
    if (!use_graph) return enqueue(pl, a, stream);
    const int kind = a.grad ? 1 : 0;
    const std::vector<uint64_t> key = graph_key(a);
    if (!pl->gexec[kind] || pl->gargs[kind] != key) {
        cudaGraph_t graph = nullptr;
        MCD_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        mcd_status st = enqueue(pl, a, stream);
        cudaError_t e = cudaStreamEndCapture(stream, &graph);
        if (st != MCD_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
        bool updated = false;
        if (pl->gexec[kind]) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(pl->gexec[kind], graph, &info) == cudaSuccess) updated = true;
            else { cudaGetLastError(); cudaGraphExecDestroy(pl->gexec[kind]); pl->gexec[kind] = nullptr; }
        }
        if (!updated) {
            e = cudaGraphInstantiate(&pl->gexec[kind], graph, 0);
            if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(ctx, e, "graph instantiate"); }
        }
        cudaGraphDestroy(graph);
        pl->gargs[kind] = key;
    }
    MCD_CUDA(cudaGraphLaunch(pl->gexec[kind], stream), "graph launch");
    return MCD_OK;
}

// Autotuner: for each launch segment of the plan, time the whole launch
// sequence on every stride-th design of that segment (about 30 ms of work)
// over candidate block and tile sizes, and keep the fastest per draw.
mcd_status autotune(mcd_ctx* ctx, const mcd_problem* pr, int32_t flags, int32_t k, const mcd_plan* shape) {
    const bool grad = (flags & MCD_PLAN_GRAD) != 0;
    for (const Segment& seg : shape->segs) {
        const TuneKey key{seg.d_lo, seg.d_hi, grad, shape->fp64};
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            if (ctx->tuned.count(key)) continue;
        }
        double total = 0.0;
        for (int j = 0; j < pr->n_design; ++j) {
            const int d = pr->scen_d[pr->design_scen[j]];
            if (d >= seg.d_lo && d <= seg.d_hi) total += static_cast<double>(pr->n_draws[j]);
        }
        TileFilter filt;
        filt.d_lo = seg.d_lo;
        filt.d_hi = seg.d_hi;
        filt.stride = std::max<int64_t>(1, static_cast<int64_t>(total / (1e12 / draw_cost(seg.d_hi))));
        double draws = 0.0;
        for (int j = 0; j < pr->n_design; j += static_cast<int>(filt.stride)) {
            const int d = pr->scen_d[pr->design_scen[j]];
            if (d >= seg.d_lo && d <= seg.d_hi) draws += static_cast<double>(pr->n_draws[j]);
        }
        cudaStream_t s;
        MCD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        LaunchCfg best;
        double best_rate = -1.0;
        mcd_status st = MCD_OK;
        for (int threads : {128, 256}) {
            for (double f : {0.25, 0.5, 1.0, 2.0}) {
                LaunchCfg c;
                c.threads = threads;
                c.scale = f;
                {
                    std::lock_guard<std::mutex> lk(ctx->mu);
                    ctx->tuned[key] = c;
                }
                mcd_plan trial;
                // timing plans take no Jacobian (k = 0): the finalisation is
                // the same per-design work either way
                st = plan_build(ctx, pr, flags & ~(MCD_PLAN_GRAPH | MCD_PLAN_TIMING | MCD_PLAN_SHARED), 0, &trial,
                                filt);
                LaunchArgs la;
                la.grad = grad;
                la.h = grad ? 0.01 : 0.0;
                double best_ms = 1e30;
                for (int rep = 0; rep < 5 && st == MCD_OK; ++rep) {   // two warm-ups, best of three
                    cudaEventRecord(e0, s);
                    st = enqueue(&trial, la, s);
                    cudaEventRecord(e1, s);
                    if (st != MCD_OK) break;
                    cudaError_t ce = cudaEventSynchronize(e1);
                    if (ce != cudaSuccess) { st = cuda_fail(ctx, ce, "autotune run"); break; }
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep >= 2) best_ms = std::min(best_ms, static_cast<double>(ms));
                }
                plan_release(&trial);
                if (st != MCD_OK) break;
                const double rate = draws / best_ms;
                if (rate > best_rate) { best_rate = rate; best = c; }
            }
            if (st != MCD_OK) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(s);
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (st != MCD_OK) { ctx->tuned.erase(key); return st; }
        ctx->tuned[key] = best;
    }
    return MCD_OK;
}

}  // namespace

// ============================================================== C ABI ======
extern "C" {

mcd_status mcd_create(mcd_ctx** out, int device) {
    if (!out) return MCD_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return MCD_EINVAL;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return MCD_ECUDA;
    if (prop.major * 10 + prop.minor != 103) return MCD_EUNSUPPORTED;
    mcd_ctx* ctx = new (std::nothrow) mcd_ctx;
    if (!ctx) return MCD_ENOMEM;
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&ctx->d_status, sizeof(DevStatus)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(DevStatus)) != cudaSuccess) {
        delete ctx;
        return MCD_ECUDA;
    }
    *out = ctx;
    return MCD_OK;
}

void mcd_destroy(mcd_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaFree(ctx->d_status);
    delete ctx;
    cudaGetLastError();              // a void call leaves no error for the next one
}

const char* mcd_last_error(const mcd_ctx* ctx) { return ctx ? ctx->err.c_str() : "context is NULL"; }

int64_t mcd_error_index(const mcd_ctx* ctx) { return ctx ? ctx->err_index : -1; }

mcd_status mcd_sync_status(mcd_ctx* ctx, mcd_stream stream) {
    if (!ctx) return MCD_EINVAL;
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    MCD_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)), "stream synchronize");
    DevStatus st;
    MCD_CUDA(cudaMemcpy(&st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost), "status read");
    MCD_CUDA(cudaMemset(ctx->d_status, 0, sizeof(DevStatus)), "status clear");
    if (st.code == MCD_OK) return MCD_OK;
    const char* what = st.code == MCD_ENOTSPD ? "Sigma is not positive definite (scenario index)"
                       : st.code == MCD_ENAN  ? "NaN in mu or b (design index)"
                                              : "invalid device input: smoothing window (class index) or allocation split (design index)";
    return fail(ctx, st.code, what, st.index);
}

mcd_status mcd_plan_create(mcd_ctx* ctx, const mcd_problem* prob, int32_t flags, int32_t k, mcd_plan** plan) {
    NvtxRange nvtx_("mcd_plan_create");
    if (!ctx || !plan) return fail(ctx, MCD_EINVAL, "ctx and plan must not be NULL");
    *plan = nullptr;
    if (flags & ~(MCD_PLAN_GRAD | MCD_PLAN_AUTOTUNE | MCD_PLAN_GRAPH | MCD_PLAN_FP64 | MCD_PLAN_TIMING |
                  MCD_PLAN_SHARED))
        return fail(ctx, MCD_EINVAL, "unknown plan flags");
    mcd_status st = validate_problem(ctx, prob, k);
    if (st != MCD_OK) return st;
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    mcd_plan* pl = new (std::nothrow) mcd_plan;
    if (!pl) return fail(ctx, MCD_ENOMEM, "host allocation");
    if (flags & MCD_PLAN_AUTOTUNE) {
        mcd_plan probe;                                  // segments for the tuner
        TileFilter none;
        none.d_lo = MCD_MAX_D + 1;                       // no tiles: shape only
        st = plan_build(ctx, prob, flags, k, &probe, none);
        plan_release(&probe);
        if (st == MCD_OK) st = autotune(ctx, prob, flags, k, &probe);
        if (st != MCD_OK) { delete pl; return st; }
    }
    st = plan_build(ctx, prob, flags, k, pl);
    if (st != MCD_OK) {
        plan_release(pl);
        delete pl;
        return st;
    }
    *plan = pl;
    return MCD_OK;
}

void mcd_plan_destroy(mcd_plan* plan) {
    if (!plan) return;
    // the plan's own device index: its context may already be destroyed
    // (e.g. a garbage collector finalising both in either order)
    cudaSetDevice(plan->device);
    plan_release(plan);
    delete plan;
    cudaGetLastError();              // a void call leaves no error for the next one
}

mcd_status mcd_plan_eval(mcd_plan* plan, uint64_t seed, uint64_t* hits, double* p, double* se, mcd_stream stream) {
    NvtxRange nvtx_("mcd_plan_eval");
    if (!plan) return MCD_EINVAL;
    LaunchArgs a;
    a.seed = seed;
    a.hits = hits;
    a.p = p;
    a.se = se;
    return launch(plan, a, reinterpret_cast<cudaStream_t>(stream));
}

mcd_status mcd_plan_grad(mcd_plan* plan, uint64_t seed, const double* dt_dtheta, double h_sigmoid, uint64_t* hits,
                         double* p, double* grad_lr, double* grad_sig, double* grad_se, mcd_stream stream) {
    NvtxRange nvtx_("mcd_plan_grad");
    if (!plan) return MCD_EINVAL;
    mcd_ctx* ctx = plan->ctx;
    if (!(plan->flags & MCD_PLAN_GRAD)) return fail(ctx, MCD_EINVAL, "plan was created without MCD_PLAN_GRAD");
    if (plan->k > 0 && !dt_dtheta) return fail(ctx, MCD_EINVAL, "plan has k > 0 but dt_dtheta is NULL");
    if (plan->k == 0 && dt_dtheta) return fail(ctx, MCD_EINVAL, "plan has k = 0 but dt_dtheta is given");
    if (!(h_sigmoid == h_sigmoid)) return fail(ctx, MCD_EINVAL, "h_sigmoid is NaN");
    LaunchArgs a;
    a.grad = true;
    a.seed = seed;
    a.jac = dt_dtheta;
    a.h = h_sigmoid > 0.0 ? h_sigmoid : 0.0;
    a.hits = hits;
    a.p = p;
    a.g_lr = grad_lr;
    a.g_sig = grad_sig;
    a.g_se = grad_se;
    return launch(plan, a, reinterpret_cast<cudaStream_t>(stream));
}

mcd_status mcd_plan_config(const mcd_plan* plan, int32_t d, int32_t* threads, int64_t* tile_draws,
                           int32_t* blocks_per_sm) {
    if (!plan || d < 1 || d > MCD_MAX_D) return MCD_EINVAL;
    if (plan->seg_of_d[d] < 0) {
        for (const SharedSeg& sg : plan->ssegs) {
            if (sg.d != d) continue;
            if (threads) *threads = kSharedThreads;
            if (tile_draws) *tile_draws = sg.tile_draws;
            if (blocks_per_sm) *blocks_per_sm = sg.blocks_per_sm;
            return MCD_OK;
        }
        return MCD_EINVAL;
    }
    const Segment& sg = plan->segs[plan->seg_of_d[d]];
    if (threads) *threads = sg.cfg.threads;
    if (tile_draws) *tile_draws = plan->tile_draws_of_d[d];
    if (blocks_per_sm) *blocks_per_sm = sg.blocks_per_sm;
    return MCD_OK;
}

int64_t mcd_plan_tiles(const mcd_plan* plan) { return plan ? plan->n_tiles + plan->n_shared_tiles : -1; }

mcd_status mcd_plan_kernel_ms(mcd_plan* plan, float* ms) {
    if (!plan || !ms) return MCD_EINVAL;
    mcd_ctx* ctx = plan->ctx;
    if (!plan->ev[0]) return fail(ctx, MCD_EINVAL, "plan was created without MCD_PLAN_TIMING");
    MCD_CUDA(cudaEventSynchronize(plan->ev[1]), "event synchronize");
    MCD_CUDA(cudaEventElapsedTime(ms, plan->ev[0], plan->ev[1]), "event elapsed");
    return MCD_OK;
}

static mcd_status one_shot(mcd_ctx* ctx, const mcd_problem* prob, int32_t k, bool grad, const LaunchArgs& a,
                           mcd_stream stream) {
    NvtxRange nvtx_("mc_design_eval/grad");
    if (!ctx) return MCD_EINVAL;
    mcd_status st = validate_problem(ctx, prob, k);
    if (st != MCD_OK) return st;
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MCD_CUDA(cudaStreamIsCapturing(s, &cs), "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone) return fail(ctx, MCD_EINVAL, "one-shot calls cannot be captured; use a plan");
    mcd_plan pl;
    pl.stream_ordered = true;
    pl.alloc_stream = s;
    st = plan_build(ctx, prob, grad ? MCD_PLAN_GRAD : 0, k, &pl);
    if (st == MCD_OK) st = enqueue(&pl, a, s);
    plan_release(&pl);
    return st;
}

mcd_status mc_design_eval(mcd_ctx* ctx, const mcd_problem* prob, uint64_t seed, uint64_t* hits, double* p,
                          double* se, mcd_stream stream) {
    LaunchArgs a;
    a.seed = seed;
    a.hits = hits;
    a.p = p;
    a.se = se;
    return one_shot(ctx, prob, 0, false, a, stream);
}

mcd_status mc_design_grad(mcd_ctx* ctx, const mcd_problem* prob, uint64_t seed, int32_t k, const double* dt_dtheta,
                          double h_sigmoid, uint64_t* hits, double* p, double* grad_lr, double* grad_sig,
                          double* grad_se, mcd_stream stream) {
    if (!ctx) return MCD_EINVAL;
    if (k > 0 && !dt_dtheta) return fail(ctx, MCD_EINVAL, "k > 0 needs dt_dtheta");
    if (k == 0 && dt_dtheta) return fail(ctx, MCD_EINVAL, "dt_dtheta given with k = 0");
    if (!(h_sigmoid == h_sigmoid)) return fail(ctx, MCD_EINVAL, "h_sigmoid is NaN");
    LaunchArgs a;
    a.grad = true;
    a.seed = seed;
    a.jac = dt_dtheta;
    a.h = h_sigmoid > 0.0 ? h_sigmoid : 0.0;
    a.hits = hits;
    a.p = p;
    a.g_lr = grad_lr;
    a.g_sig = grad_sig;
    a.g_se = grad_se;
    return one_shot(ctx, prob, k, true, a, stream);
}

mcd_status mc_fwer_calibrate(mcd_ctx* ctx, const mcd_problem* prob, const double* w, double alpha0, int32_t rounds,
                             uint64_t seed, double* scale, double* b, double* fwer, mcd_stream stream) {
    NvtxRange nvtx_("mc_fwer_calibrate");
    if (!ctx) return MCD_EINVAL;
    if (!prob) return fail(ctx, MCD_EINVAL, "problem is NULL");
    if (!(alpha0 > 0.0 && alpha0 < 1.0)) return fail(ctx, MCD_EINVAL, "alpha0 must be in (0, 1)");
    if (rounds < 2 || rounds > 200) return fail(ctx, MCD_EINVAL, "rounds must be in 2..200");
    if (prob->region != MCD_ANY_EXCEEDS)
        return fail(ctx, MCD_EINVAL, "the FWER is the probability that some test rejects: region must be MCD_ANY_EXCEEDS");
    if (prob->n_design == 0) return MCD_OK;
    if (!w || !scale || !b || !fwer) return fail(ctx, MCD_EINVAL, "w, scale, b and fwer must not be NULL");
    if (!is_device_ptr(w) || !is_device_ptr(scale) || !is_device_ptr(b) || !is_device_ptr(fwer))
        return fail(ctx, MCD_EINVAL, "w, scale, b and fwer must be device memory");
    if (!prob->scen_d || !prob->design_scen) return fail(ctx, MCD_EINVAL, "scen_d and design_scen must not be NULL");
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MCD_CUDA(cudaStreamIsCapturing(s, &cs), "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone) return fail(ctx, MCD_EINVAL, "mc_fwer_calibrate cannot be captured");
    const int J = prob->n_design;
    size_t vec_len = 0;
    for (int j = 0; j < J; ++j) {
        const int sc = prob->design_scen[j];
        if (sc < 0 || sc >= prob->n_scen) return fail(ctx, MCD_EINVAL, "design_scen out of range", j);
        vec_len += static_cast<size_t>(prob->scen_d[sc]);
    }
    // the sampler sees mu = 0 (the null hypothesis) and reads its thresholds
    // from the output array b, which every round rewrites
    double* mu0 = nullptr;
    FwerState* st = nullptr;
    uint64_t* hits = nullptr;
    double* p = nullptr;
    MCD_CUDA(cudaMallocAsync(&mu0, sizeof(double) * vec_len, s), "calibration workspace");
    cudaError_t e = cudaMallocAsync(&st, sizeof(FwerState) * J, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&hits, sizeof(uint64_t) * J, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&p, sizeof(double) * J, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mu0, 0, sizeof(double) * vec_len, s);
    mcd_status rc = e == cudaSuccess ? MCD_OK : cuda_fail(ctx, e, "calibration workspace");
    mcd_problem q = *prob;
    q.mu = mu0;
    q.b = b;
    if (rc == MCD_OK) rc = validate_problem(ctx, &q, 0);
    mcd_plan pl;
    pl.stream_ordered = true;
    pl.alloc_stream = s;
    if (rc == MCD_OK) rc = plan_build(ctx, &q, MCD_PLAN_SHARED, 0, &pl);
    if (rc == MCD_OK) {
        e = launch_fwer_init(J, pl.d_designs, w, alpha0, st, b, ctx->d_status, s);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "calibration launch");
    }
    for (int r = 0; r < rounds && rc == MCD_OK; ++r) {
        LaunchArgs a;
        a.seed = seed;
        a.hits = hits;
        a.p = p;
        rc = enqueue(&pl, a, s);
        if (rc != MCD_OK) break;
        e = launch_fwer_update(J, pl.d_designs, w, p, alpha0, r, r == rounds - 1, st, b, scale, fwer, s);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "calibration launch");
    }
    plan_release(&pl);
    for (void* x : {static_cast<void*>(p), static_cast<void*>(hits), static_cast<void*>(st), static_cast<void*>(mu0)})
        if (x) cudaFreeAsync(x, s);
    return rc;
}

mcd_status mc_tps_fit(mcd_ctx* ctx, int32_t n_surf, int32_t n_pts, int32_t k, const double* x, const double* y,
                      double smoothing, double* coef, double* fitted, mcd_stream stream) {
    NvtxRange nvtx_("mc_tps_fit");
    if (!ctx) return MCD_EINVAL;
    if (n_surf < 1) return fail(ctx, MCD_EINVAL, "n_surf must be >= 1");
    if (k < 1 || k > 3) return fail(ctx, MCD_EINVAL, "k must be 1, 2 or 3");
    if (n_pts < k + 2 || n_pts > 16384) return fail(ctx, MCD_EINVAL, "n_pts must be in k + 2 .. 16384");
    if (!(smoothing >= 0.0) || smoothing == INFINITY) return fail(ctx, MCD_EINVAL, "smoothing must be finite and >= 0");
    if (!x || !y || !coef) return fail(ctx, MCD_EINVAL, "x, y and coef must not be NULL");
    if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(coef) || (fitted && !is_device_ptr(fitted)))
        return fail(ctx, MCD_EINVAL, "x, y, coef and fitted must be device memory");
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MCD_CUDA(cudaStreamIsCapturing(s, &cs), "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone) return fail(ctx, MCD_EINVAL, "mc_tps_fit cannot be captured");
    // Surfaces are independent fits whose time is mostly dependent chains
    // (pivots, triangular solves), so up to kTpsWorkers of them run at once,
    // each worker stream fitting its share in turn with a workspace of its
    // own; the workers start after the work already queued on `s` and `s`
    // waits for all of them.  The number of workers is also held to about
    // 4 GB of workspace.
    constexpr int kTpsWorkers = 4;
    const size_t nws = tps_workspace_doubles(n_pts, k);
    const size_t per_worker = nws + 2;
    int workers = n_surf < kTpsWorkers ? n_surf : kTpsWorkers;
    while (workers > 1 && per_worker * sizeof(double) * workers > (static_cast<size_t>(4) << 30)) --workers;
    double* ws = nullptr;
    MCD_CUDA(cudaMallocAsync(&ws, sizeof(double) * per_worker * workers, s), "spline workspace");
    mcd_status rc = MCD_OK;
    const int64_t m = k + 1;
    cudaStream_t wstream[kTpsWorkers] = {};
    cudaEvent_t ev_start = nullptr, ev_done[kTpsWorkers] = {};
    cudaError_t e = cudaSuccess;
    if (workers > 1) {
        e = cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
        for (int w = 0; w < workers && e == cudaSuccess; ++w) {
            e = cudaStreamCreateWithFlags(&wstream[w], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_done[w], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_start, s);
        for (int w = 0; w < workers && e == cudaSuccess; ++w) e = cudaStreamWaitEvent(wstream[w], ev_start, 0);
    } else {
        wstream[0] = s;
    }
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "spline streams");
    for (int q = 0; q < n_surf && rc == MCD_OK; ++q) {
        const int w = q % workers;
        double* wsw = ws + per_worker * w;
        int* bad = reinterpret_cast<int*>(wsw + nws);
        unsigned long long* amax = reinterpret_cast<unsigned long long*>(wsw + nws + 1);
        e = tps_fit_one(x + static_cast<int64_t>(q) * n_pts * k, y + static_cast<int64_t>(q) * n_pts, n_pts, k,
                        smoothing, coef + static_cast<int64_t>(q) * (n_pts + m),
                        fitted ? fitted + static_cast<int64_t>(q) * n_pts : nullptr, wsw, bad, amax, ctx->d_status, q,
                        wstream[w]);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "spline launch");
    }
    if (workers > 1) {
        // join every worker that was created, whatever happened above
        for (int w = 0; w < workers; ++w) {
            if (wstream[w] && ev_done[w] && cudaEventRecord(ev_done[w], wstream[w]) == cudaSuccess)
                cudaStreamWaitEvent(s, ev_done[w], 0);
        }
        for (int w = 0; w < workers; ++w) {
            if (ev_done[w]) cudaEventDestroy(ev_done[w]);
            if (wstream[w]) cudaStreamDestroy(wstream[w]);
        }
        if (ev_start) cudaEventDestroy(ev_start);
    }
    cudaFreeAsync(ws, s);
    return rc;
}

mcd_status mc_tps_gcv(mcd_ctx* ctx, int32_t n_pts, int32_t k, const double* x, const double* y, int32_t n_s,
                      const double* s_values, double* score, mcd_stream stream) {
    NvtxRange nvtx_("mc_tps_gcv");
    if (!ctx) return MCD_EINVAL;
    if (k < 1 || k > 3) return fail(ctx, MCD_EINVAL, "k must be 1, 2 or 3");
    if (n_pts < k + 2 || n_pts > 16384) return fail(ctx, MCD_EINVAL, "n_pts must be in k + 2 .. 16384");
    if (n_s < 1 || n_s > 256 || !s_values) return fail(ctx, MCD_EINVAL, "n_s must be in 1..256 with s_values given");
    for (int q = 0; q < n_s; ++q)
        if (!(s_values[q] > 0.0) || s_values[q] == INFINITY)
            return fail(ctx, MCD_EINVAL, "smoothing values must be finite and > 0", q);
    if (!x || !y || !score) return fail(ctx, MCD_EINVAL, "x, y and score must not be NULL");
    if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(score))
        return fail(ctx, MCD_EINVAL, "x, y and score must be device memory");
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MCD_CUDA(cudaStreamIsCapturing(s, &cs), "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone) return fail(ctx, MCD_EINVAL, "mc_tps_gcv cannot be captured");
    const size_t nws = tps_gcv_workspace_doubles(n_pts, k);
    double* ws = nullptr;
    MCD_CUDA(cudaMallocAsync(&ws, sizeof(double) * (nws + 4), s), "spline workspace");
    int* bad = reinterpret_cast<int*>(ws + nws);
    unsigned long long* amax = reinterpret_cast<unsigned long long*>(ws + nws + 1);
    double* trace = ws + nws + 2;
    cudaError_t e = tps_gcv(x, y, n_pts, k, s_values, n_s, score, ws, bad, amax, trace, s);
    cudaFreeAsync(ws, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "spline GCV launch");
    return MCD_OK;
}

mcd_status mc_tps_argmax(mcd_ctx* ctx, int32_t n_surf, int32_t n_pts, int32_t k, const double* x, const double* coef,
                         const double* fitted, const double* lo, const double* hi, int32_t iters, double* x_best,
                         double* f_best, mcd_stream stream) {
    NvtxRange nvtx_("mc_tps_argmax");
    if (!ctx) return MCD_EINVAL;
    if (n_surf < 1) return fail(ctx, MCD_EINVAL, "n_surf must be >= 1");
    if (k < 1 || k > 3) return fail(ctx, MCD_EINVAL, "k must be 1, 2 or 3");
    if (n_pts < k + 2 || n_pts > 16384) return fail(ctx, MCD_EINVAL, "n_pts must be in k + 2 .. 16384");
    if (iters < 0 || iters > 100000) return fail(ctx, MCD_EINVAL, "iters must be in 0 .. 100000");
    const void* ptrs[] = {x, coef, fitted, lo, hi, x_best, f_best};
    for (const void* p : ptrs) {
        if (!p) return fail(ctx, MCD_EINVAL, "x, coef, fitted, lo, hi, x_best and f_best must not be NULL");
        if (!is_device_ptr(p)) return fail(ctx, MCD_EINVAL, "x, coef, fitted, lo, hi, x_best and f_best must be device memory");
    }
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    MCD_CUDA(tps_argmax(x, coef, fitted, n_surf, n_pts, k, lo, hi, iters, x_best, f_best,
                        reinterpret_cast<cudaStream_t>(stream)), "spline maximiser launch");
    return MCD_OK;
}

}  // extern "C"

namespace {

template <typename T>
mcd_status smooth_call(const char* name, mcd_ctx* ctx, int32_t n_scen, int32_t g1, int32_t g2, const T* value,
                       double bandwidth, int32_t degree, T* smoothed, int64_t* argmax_idx, T* argmax_val,
                       int64_t* raw_idx, T* raw_val, mcd_stream stream) {
    NvtxRange nvtx_(name);
    if (!ctx) return MCD_EINVAL;
    if (n_scen < 1 || g1 < 1 || g2 < 1) return fail(ctx, MCD_EINVAL, "n_scen, g1, g2 must be >= 1");
    if (static_cast<int64_t>(g1) * g2 >= (1ll << 31)) return fail(ctx, MCD_EINVAL, "grid too large");
    if (const char* why = smooth_shape_error(n_scen, g1, g2)) return fail(ctx, MCD_EINVAL, why);
    if (!(bandwidth > 1.0 && bandwidth <= 4.0)) return fail(ctx, MCD_EINVAL, "bandwidth must be in (1, 4]");
    if (degree < 0 || degree > 2) return fail(ctx, MCD_EINVAL, "degree must be 0, 1 or 2");
    if (!value || !argmax_idx || !argmax_val) return fail(ctx, MCD_EINVAL, "value, argmax_idx, argmax_val must not be NULL");
    if (!is_device_ptr(value)) return fail(ctx, MCD_EINVAL, "value is not device memory");
    const int n1 = (g1 == 1 || g2 == 1) ? g1 * g2 : std::min(g1, g2);
    if (n1 < degree + 1) return fail(ctx, MCD_EINVAL, "grid too small for the degree");
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t nw = smooth_weight_count();
    const size_t nc = smooth_candidate_count(n_scen, g1, g2);
    void* ws = nullptr;
    // layout: FP64 weights | FP32 weights | candidate values | candidate indices
    const size_t bytes = nw * sizeof(double) + nw * sizeof(float) + nc * (sizeof(double) + sizeof(int64_t)) + 64;
    MCD_CUDA(cudaMallocAsync(&ws, bytes, s), "smoothing workspace");
    double* w64 = static_cast<double*>(ws);
    float* w32 = reinterpret_cast<float*>(w64 + nw);
    double* pv = reinterpret_cast<double*>(reinterpret_cast<char*>(w32) + ((nw * sizeof(float) + 15) / 16) * 16);
    int64_t* pi = reinterpret_cast<int64_t*>(pv + nc);
    cudaError_t e;
    if constexpr (sizeof(T) == 8)
        e = smooth_argmax(n_scen, g1, g2, value, bandwidth, degree, smoothed, argmax_idx, argmax_val, raw_idx, raw_val,
                          w64, w32, pv, pi, ctx->d_status, s);
    else
        e = smooth_argmax_f32(n_scen, g1, g2, value, bandwidth, degree, smoothed, argmax_idx, argmax_val, raw_idx,
                              raw_val, w64, w32, pv, pi, ctx->d_status, s);
    cudaFreeAsync(ws, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "smoothing launch");
    return MCD_OK;
}

}  // namespace

extern "C" {

mcd_status mc_smooth_argmax(mcd_ctx* ctx, int32_t n_scen, int32_t g1, int32_t g2, const double* value,
                            double bandwidth, int32_t degree, double* smoothed, int64_t* argmax_idx,
                            double* argmax_val, int64_t* raw_idx, double* raw_val, mcd_stream stream) {
    return smooth_call<double>("mc_smooth_argmax", ctx, n_scen, g1, g2, value, bandwidth, degree, smoothed,
                               argmax_idx, argmax_val, raw_idx, raw_val, stream);
}

mcd_status mc_smooth_argmax_f32(mcd_ctx* ctx, int32_t n_scen, int32_t g1, int32_t g2, const float* value,
                                double bandwidth, int32_t degree, float* smoothed, int64_t* argmax_idx,
                                float* argmax_val, int64_t* raw_idx, float* raw_val, mcd_stream stream) {
    return smooth_call<float>("mc_smooth_argmax_f32", ctx, n_scen, g1, g2, value, bandwidth, degree, smoothed,
                              argmax_idx, argmax_val, raw_idx, raw_val, stream);
}

mcd_status mcd_debug_normals(mcd_ctx* ctx, uint64_t seed, uint64_t key, uint64_t m_begin, uint64_t count, float* z32,
                             double* z64, uint32_t* words, mcd_stream stream) {
    if (!ctx) return MCD_EINVAL;
    if (m_begin > (1ull << 62) || count > (1ull << 32)) return fail(ctx, MCD_EINVAL, "range too large");
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    MCD_CUDA(launch_debug_normals(seed, key, m_begin, count, z32, z64, words, reinterpret_cast<cudaStream_t>(stream)),
             "debug launch");
    return MCD_OK;
}

mcd_status mcd_debug_fail_next(mcd_ctx* ctx, int32_t cuda_error) {
    if (!ctx) return MCD_EINVAL;
    if (cuda_error < 0) return fail(ctx, MCD_EINVAL, "cuda_error must be >= 0");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->inject = cuda_error;
    return MCD_OK;
}

mcd_status mcd_pipe_rate(mcd_ctx* ctx, int32_t op, int32_t iters, double* rate, mcd_stream stream) {
    if (!ctx) return MCD_EINVAL;
    if (!rate || op < 0 || op >= MCD_PIPE_COUNT || iters < 1 || iters > (1 << 20))
        return fail(ctx, MCD_EINVAL, "pipe rate: unknown op, iters outside [1, 2^20] or NULL rate");
    NvtxRange nv("mcd_pipe_rate");
    MCD_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int blocks = ctx->sm_count * kPipeBlocksPerSM;
    // t0 | t1 (i64 per block) | smid (i32 per block, padded) | sink (u32 per thread)
    const size_t off_smid = 16 * static_cast<size_t>(blocks);
    const size_t off_sink = off_smid + ((4 * static_cast<size_t>(blocks) + 15) / 16) * 16;
    const size_t bytes = off_sink + 4 * static_cast<size_t>(blocks) * kPipeThreads;
    char* ws = nullptr;
    MCD_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&ws), bytes, s), "pipe workspace");
    long long* t0 = reinterpret_cast<long long*>(ws);
    long long* t1 = t0 + blocks;
    int* smid = reinterpret_cast<int*>(ws + off_smid);
    uint32_t* sink = reinterpret_cast<uint32_t*>(ws + off_sink);
    std::vector<long long> h0(blocks), h1(blocks);
    std::vector<int> hs(blocks);
    // a short warm-up launch, then the timed one
    cudaError_t e = launch_pipe(op, std::min(iters, 64), blocks, kPhiloxM0, 0.5f, sink, t0, t1, smid, s);
    if (e == cudaSuccess) e = launch_pipe(op, iters, blocks, kPhiloxM0, 0.5f, sink, t0, t1, smid, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h0.data(), t0, 8 * static_cast<size_t>(blocks), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h1.data(), t1, 8 * static_cast<size_t>(blocks), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), smid, 4 * static_cast<size_t>(blocks), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(ws, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pipe microbenchmark");
    // per SM: first start, last end, blocks
    std::vector<long long> lo(ctx->sm_count, 0), hi(ctx->sm_count, 0);
    std::vector<int> nb(ctx->sm_count, 0);
    for (int b = 0; b < blocks; ++b) {
        const int m = hs[b];
        if (m < 0 || m >= ctx->sm_count) continue;
        if (nb[m] == 0 || h0[b] < lo[m]) lo[m] = h0[b];
        if (nb[m] == 0 || h1[b] > hi[m]) hi[m] = h1[b];
        ++nb[m];
    }
    std::vector<double> r;
    const double ops_per_block = static_cast<double>(kPipeThreads) * pipe_ops_per_step(op) * iters;
    for (int m = 0; m < ctx->sm_count; ++m)
        if (nb[m] > 0 && hi[m] > lo[m]) r.push_back(ops_per_block * nb[m] / static_cast<double>(hi[m] - lo[m]));
    if (r.empty()) return fail(ctx, MCD_ECUDA, "pipe microbenchmark: no SM reported a positive cycle count");
    std::sort(r.begin(), r.end());
    *rate = (r.size() % 2) ? r[r.size() / 2] : 0.5 * (r[r.size() / 2 - 1] + r[r.size() / 2]);
    return MCD_OK;
}

}  // extern "C"
