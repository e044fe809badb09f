// Fused FP32 apply of one sub-BF in two launches (front: V, H levels, switch;
// back: G levels, U), phases read from the tables; the batched persistent
// kernel; configuration and launchers.  The tile bodies are in bf_f32_tile.h.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "bf_f32_tile.h"

namespace bfi {
namespace {

template <int R, int NV>
__global__ void __launch_bounds__(kThreads, 2) front_f32(FrontArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    front_tile<R, NV>(A, blockIdx.x, smem_raw);
}

template <int R, int NU>
__global__ void __launch_bounds__(kThreads, 2) back_f32(BackArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    back_tile<R, NU>(A, blockIdx.x, smem_raw);
}

template <int R>
cudaError_t launch_r(const FrontArgs& fa, const BackArgs& ba, size_t sf, size_t sb, int64_t nfront, int64_t nback,
                     cudaStream_t st)
{
    constexpr int NV = nv_of<R>();
    cudaError_t e = cudaFuncSetAttribute(front_f32<R, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(back_f32<R, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps("front_f32", st);
        front_f32<R, NV><<<(unsigned)nfront, kThreads, sf, st>>>(fa);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        ProfScope ps("back_f32", st);
        back_f32<R, NV><<<(unsigned)nback, kThreads, sb, st>>>(ba);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- batched --
// Out-of-line copies of the tile bodies for the persistent kernel, so that each
// body gets its own register allocation instead of the union of both.
template <int R, int NV>
__device__ __noinline__ void front_tile_ool(const FrontArgs& A, int64_t work, unsigned char* smem)
{
    front_tile<R, NV>(A, work, smem);
}
template <int R, int NV>
__device__ __noinline__ void back_tile_ool(const BackArgs& A, int64_t work, unsigned char* smem)
{
    back_tile<R, NV>(A, work, smem);
}

// One persistent launch over the front and back tiles of many operators.
// Work items are handed out by an atomic counter in segment order (off[],
// seg[]): each operator's front segment, and its back segment a little later
// (after about a thousand more work items, so that its fronts have usually
// finished while its switch-level workspace is still in L2).  Every front tile
// is claimed, by a running CTA, before any back tile of the same operator; a
// back tile waits until all front tiles of its operator are done (bounded
// spin; on time-out it sets *err and skips the tile).
template <int R, int NV>
__global__ void __launch_bounds__(kThreads, 2)
    batch_f32(const BatchItem* items, int nitems, const int64_t* off, const int* seg, int64_t total,
              unsigned long long* counter, int* done, int* err, long long spin_limit, int wait_extra)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_w;
    __shared__ int s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_w = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long w = s_w;
        __syncthreads();
        if (w >= total) break;
        int j = 0;  // segment of work item w
        while (j + 1 < 2 * nitems && off[j + 1] <= w) ++j;
        const int i = seg[j] >> 1;
        const long long local = w - off[j];
        if ((seg[j] & 1) == 0) {
            front_tile_ool<R, NV>(items[i].fa, local, smem_raw);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&done[i], 1);
            }
        } else {
            if (threadIdx.x == 0) {
                long long n = 0;
                int ok = 1;
                while (atomicAdd(&done[i], 0) < (int)items[i].nfront + wait_extra) {
                    if (++n > spin_limit) {
                        atomicExch(err, 2);
                        ok = 0;
                        break;
                    }
                    __nanosleep(128);
                }
                __threadfence();
                s_ok = ok;
            }
            __syncthreads();
            if (s_ok) back_tile_ool<R, NV>(items[i].ba, local, smem_raw);
        }
    }
}

// The batch in two phase launches: every operator's front tiles in one launch, then every
// back tile in a second one (no hand-off waits: the launch boundary orders them).  One CTA per
// work item, the tile bodies inlined, each launch with its own shared-memory size.
template <int R, int NV, int BACK>
__global__ void __launch_bounds__(kThreads, 2)
    batch_phase_f32(const BatchItem* items, const int* ord, const int64_t* off, int nitems)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t w = blockIdx.x;
    int lo = 0, hi = nitems - 1;  // the last k with off[k] <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= w) lo = mid;
        else hi = mid - 1;
    }
    const BatchItem& it = items[__ldg(ord + lo)];
    const int64_t local = w - __ldg(off + lo);
    if (BACK) back_tile<R, NV>(it.ba, local, smem_raw);
    else front_tile<R, NV>(it.fa, local, smem_raw);
}

template <int R>
cudaError_t batch_phases_r(const BatchLaunch& bl, cudaStream_t st, bool set_attr)
{
    constexpr int NV = nv_of<R>();
    if (set_attr) {
        cudaError_t e = cudaFuncSetAttribute(batch_phase_f32<R, NV, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bl.smem_f);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(batch_phase_f32<R, NV, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bl.smem_b);
    }
    if (bl.total_f < 1 || bl.total_b < 1 || bl.total_f >= (1ll << 31) || bl.total_b >= (1ll << 31))
        return cudaErrorInvalidConfiguration;
    {
        ProfScope ps("batch_front_f32", st);
        batch_phase_f32<R, NV, 0><<<(unsigned)bl.total_f, kThreads, bl.smem_f, st>>>(bl.items, bl.ord, bl.off_f,
                                                                                    bl.nitems);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        ProfScope ps("batch_back_f32", st);
        batch_phase_f32<R, NV, 1><<<(unsigned)bl.total_b, kThreads, bl.smem_b, st>>>(bl.items, bl.ord, bl.off_b,
                                                                                   bl.nitems);
    }
    return cudaGetLastError();
}

template <int R>
cudaError_t batch_launch_r(const BatchLaunch& bl, cudaStream_t st, bool set_attr, int* grid_out)
{
    constexpr int NV = nv_of<R>();
    if (set_attr)  // configuration only, no launch
        return cudaFuncSetAttribute(batch_f32<R, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bl.smem);
    if (grid_out) {
        int per_sm = 0, dev = 0, nsm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_f32<R, NV>, kThreads, bl.smem);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        *grid_out = per_sm * nsm;
        return cudaSuccess;
    }
    ProfScope ps("batch_f32", st);
    batch_f32<R, NV><<<bl.grid, kThreads, bl.smem, st>>>(bl.items, bl.nitems, bl.off, bl.seg, bl.total, bl.counter,
                                                          bl.done, bl.err, bl.spin_limit, bl.wait_extra);
    return cudaGetLastError();
}

}  // namespace

bool fused_f32_supported(int r) { return r == 6 || r == 8 || r == 10 || r == 12 || r == 14 || r == 16; }

namespace {

// Level passes of the plain apply.  A tile of 2^k pairs closes k levels; beyond
// kSplitAbove levels (kSplitAboveOtf with evaluated phases, whose last H pass also
// keeps [2^k][r][r] switch blocks) the shared memory of one tile leaves too few
// columns per tile, so the plain apply splits the kH H levels and the kG G levels
// into passes of at most kPassMax levels (as even as possible), linked through HBM
// workspaces.  The batched and sharded applies keep one pass per side.
constexpr int kSplitAbove = 5, kSplitAboveOtf = 4, kPassMax = 4;

std::vector<int> split_levels(int k, bool split, bool otf, int kpass = 0)
{
    if (!split || (kpass > 0 ? k <= kpass : k <= (otf ? kSplitAboveOtf : kSplitAbove))) return {k};
    const int pm = kpass > 0 ? kpass : kPassMax;
    const int n = (k + pm - 1) / pm, base = k / n, extra = k % n;
    std::vector<int> v;
    for (int i = 0; i < n; ++i) v.push_back(base + (i < extra ? 1 : 0));
    return v;
}

struct Passes {
    std::vector<int> hs;  // H pass sizes in level order; hs[0] includes V, the last one the switch
    std::vector<int> gs;  // G pass sizes in level order; the last one includes U
    bool split() const { return hs.size() > 1 || gs.size() > 1; }
    int kmax() const
    {
        int k = 0;
        for (int v : hs) k = std::max(k, v);
        for (int v : gs) k = std::max(k, v);
        return k;
    }
};

Passes passes_of(const Geo& g, bool split, int hint = 0)
{
    const int kp = tune_kpass(hint);
    return Passes{split_levels(g.kH, split, g.otf, kp), split_levels(g.kG, split, g.otf, kp)};
}

// largest shared memory of any pass for (mr, CTp) with one tile per CTA
size_t passes_smem(const Geo& g, const Passes& ps, int NV, int CTp, int mr)
{
    const int R = g.r;
    size_t s = std::max(front_smem(g, ps.hs[0], ps.hs.size() == 1, R, NV, CTp, mr, 1),
                        back_smem(g, ps.gs.back(), R, NV, CTp, mr, 1));
    for (size_t i = 1; i < ps.hs.size(); ++i) s = std::max(s, mid_smem(g, ps.hs[i], i + 1 == ps.hs.size(), R, CTp, 1));
    for (size_t i = 0; i + 1 < ps.gs.size(); ++i) s = std::max(s, mid_smem(g, ps.gs[i], false, R, CTp, 1));
    return s;
}

// tiles per CTA of a pass of k levels with `tiles` tiles per column slice: up to one
// (tile, group, column) item per thread and level, two CTAs per SM
template <typename SmemFn>
int tiles_per_cta(int k, int CTp, int64_t tiles, SmemFn smem)
{
    const int items = std::max(1, (1 << k) / 2) * CTp;
    int tpc = 1;
    while (tpc < 16 && 2 * tpc <= tiles && 2 * tpc * items <= kThreads && smem(2 * tpc) <= 113 * 1024) tpc *= 2;
    return tpc;
}

FusedCfg config_of(const Geo& g, int64_t m, int hint, const Passes& ps)
{
    const int mr_hint = tune_mr(hint);
    const int Tmax = 1 << ps.kmax();
    const int ra = g.ra > 0 ? g.ra : 1;
    const int NV = g.nv;
    auto smem = [&](int mr) { return passes_smem(g, ps, NV, 1 << ilog2(ra * mr), mr); };
    int mr;
    if (mr_hint > 0 && (mr_hint & (mr_hint - 1)) == 0 && (1 << ilog2(ra * mr_hint)) <= 256 &&
        smem(mr_hint) <= 200 * 1024) {
        mr = mr_hint;
    } else {
        // largest power-of-two mr with at most 512 (group, column) items per level
        // that keeps two CTAs resident per SM (shared memory <= 113 KB)
        mr = 64;
        while (mr > 1) {
            const int CTp = 1 << ilog2(ra * mr);
            if ((Tmax / 2) * CTp <= 512 && CTp <= 256 && smem(mr) <= 113 * 1024) break;
            mr >>= 1;
        }
        while (mr > 1 && (int64_t)(mr / 2) >= m) mr >>= 1;
    }
    FusedCfg c;
    c.mr = mr;
    c.nslice = (int)((m + mr - 1) / mr);
    // with few columns per tile, several front tiles (back chunks) per CTA
    const int CTp = 1 << ilog2(ra * mr);
    const int kf = ps.hs[0], kb = ps.gs.back();
    const bool lastf = ps.hs.size() == 1;
    c.tpc_f = tiles_per_cta(kf, CTp, (int64_t)1 << (g.L - kf),
                            [&](int t) { return front_smem(g, kf, lastf, g.r, NV, CTp, mr, t); });
    c.tpc_b = tiles_per_cta(kb, CTp, (int64_t)1 << g.l1, [&](int t) { return back_smem(g, kb, g.r, NV, CTp, mr, t); });
    // the autotuner's tiles per CTA, where they fit (at most 16, within the tile counts and
    // the two-CTAs-per-SM shared-memory limit)
    const int tf = tune_tpc_f(hint), tb = tune_tpc_b(hint);
    if (tf > 0 && tf <= 16 && (int64_t)tf <= ((int64_t)1 << (g.L - kf)) &&
        front_smem(g, kf, lastf, g.r, NV, CTp, mr, tf) <= 113 * 1024)
        c.tpc_f = tf;
    if (tb > 0 && tb <= 16 && tb <= (1 << g.l1) && back_smem(g, kb, g.r, NV, CTp, mr, tb) <= 113 * 1024) c.tpc_b = tb;
    c.kpass = ps.kmax();
    return c;
}

// Front and back argument blocks of the first H pass and the last G pass.  ws holds
// W (the switch-level coefficients) and, for a split plan, one more buffer of the
// same size for the coefficients between passes.  s_stage: a front pass that applies the
// switch copies its tiles' switch blocks, and then b_k, into shared memory when they fit
// beside the chosen tiles (two CTAs per SM); the arithmetic is the same either way.
bool make_args(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws, int mr_hint,
               const Passes& ps, FrontArgs* fa, BackArgs* ba, size_t* sf, size_t* sb, int64_t* nfront,
               int64_t* nback, bool s_stage = false)
{
    const Geo& g = B.g;
    if (!fused_f32_supported(g.r)) return false;
    const int NV = (g.r < 8) ? 8 : (g.r < 16 ? 16 : 32);
    if (g.nv != NV || g.ra < 1) return false;
    const FusedCfg cfg = config_of(g, m, mr_hint, ps);
    const int CTp = 1 << ilog2(g.ra * cfg.mr);
    const int kf = ps.hs[0], kb = ps.gs.back();
    fa->g = g;
    fa->F = F;
    fa->m = m;
    fa->mr = cfg.mr;
    fa->lmr = ilog2(cfg.mr);
    fa->CTp = CTp;
    fa->lct = ilog2(CTp);
    fa->nslice = cfg.nslice;
    fa->tpc = cfg.tpc_f;
    fa->bk = B.f32.b;
    fa->MvT = B.f32.Mv;
    fa->EV = B.f32.EV;
    fa->MHT = B.f32.MH;
    fa->EH = B.f32.EH;
    fa->S = B.f32.S;
    fa->W = ws;
    fa->wl = WLayout{g.h, g.L - g.h, 0, 0, g.P};
    fa->c0_lo = 0;
    fa->xi_lo = 0;
    fa->ph = B.ph;
    fa->K = kf;
    fa->last = ps.hs.size() == 1;
    fa->Wo = nullptr;
    fa->wlo = WLayout{g.l1 + kf, g.L - g.l1 - kf, 0, 0, g.P};
    ba->g = g;
    ba->m = m;
    ba->mr = cfg.mr;
    ba->lmr = fa->lmr;
    ba->CTp = CTp;
    ba->lct = fa->lct;
    ba->nslice = cfg.nslice;
    ba->tpc = cfg.tpc_b;
    ba->W = ws;
    ba->wl = fa->wl;
    ba->pp_lo = 0;
    ba->x_lo = 0;
    ba->MGT = B.f32.MG;
    ba->FG = B.f32.FG;
    ba->MU = B.f32.MU;
    ba->EU = B.f32.EU;
    ba->ak = B.f32.a;
    ba->G = G;
    ba->beta = beta;
    ba->ph = B.ph;
    ba->K = kb;
    ba->lb = g.L - g.l1 - kb;
    if (ba->lb != g.h) ba->wl = WLayout{ba->lb, g.L - ba->lb, 0, 0, g.P};
    *sf = front_smem(g, kf, fa->last, g.r, NV, CTp, cfg.mr, cfg.tpc_f);
    if (s_stage) {
        // two CTAs per SM need dynamic + static shared memory (the tile's small index
        // tables) + the 1 KB the SM reserves per CTA within 114 KB: stay 1 KB below 113 KB
        constexpr size_t kStageLimit = 112 * 1024;
        auto fs = [&](bool s, bool b) { return front_smem(g, kf, fa->last, g.r, NV, CTp, cfg.mr, cfg.tpc_f, s, b); };
        if (fa->last && !g.otf && fs(true, false) <= kStageLimit) fa->s_smem = 1;
        if (fs(fa->s_smem, true) <= kStageLimit) fa->bk_smem = 1;
        *sf = fs(fa->s_smem, fa->bk_smem);
    }
    *sb = back_smem(g, kb, g.r, NV, CTp, cfg.mr, cfg.tpc_b);
    *nfront = ((int64_t)1 << (g.L - kf)) * cfg.nslice / cfg.tpc_f;
    *nback = ((int64_t)1 << ba->lb) * cfg.nslice;
    return true;
}

}  // namespace

FusedCfg fused_f32_config(const Geo& g, int64_t m, int mr_hint, bool split)
{
    return config_of(g, m, mr_hint, passes_of(g, split, mr_hint));
}

size_t fused_f32_ws_bytes(const Geo& g, int64_t m, int mr_hint, bool split)
{
    const Passes ps = passes_of(g, split, mr_hint);
    const FusedCfg c = config_of(g, m, mr_hint, ps);
    const int CTp = 1 << ilog2((g.ra > 0 ? g.ra : 1) * c.mr);
    const size_t w = (size_t)c.nslice * g.P * g.r * CTp * sizeof(float2);
    return ps.split() ? 2 * w : w;
}

bool fused_make_args(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws, int mr_hint,
                     FrontArgs* fa, BackArgs* ba, size_t* sf, size_t* sb, int64_t* nfront, int64_t* nback)
{
    return make_args(B, F, m, G, beta, ws, mr_hint, passes_of(B.g, false, mr_hint), fa, ba, sf, sb, nfront, nback);
}

template <int R>
cudaError_t launch_part_r(const FrontArgs* fa, const BackArgs* ba, size_t smem, int64_t nblocks, cudaStream_t st)
{
    constexpr int NV = nv_of<R>();
    cudaError_t e;
    if (fa) {
        if ((e = cudaFuncSetAttribute(front_f32<R, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        ProfScope ps("front_f32", st);
        front_f32<R, NV><<<(unsigned)nblocks, kThreads, smem, st>>>(*fa);
    } else {
        if ((e = cudaFuncSetAttribute(back_f32<R, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        ProfScope ps("back_f32", st);
        back_f32<R, NV><<<(unsigned)nblocks, kThreads, smem, st>>>(*ba);
    }
    return cudaGetLastError();
}

cudaError_t launch_part(int r, const FrontArgs* fa, const BackArgs* ba, size_t smem, int64_t nblocks, cudaStream_t st)
{
    if (nblocks < 1) return cudaSuccess;
    if (fa ? fa->g.otf : ba->g.otf) return launch_part_otf(r, fa, ba, smem, nblocks, st);
    switch (r) {
    case 6: return launch_part_r<6>(fa, ba, smem, nblocks, st);
    case 8: return launch_part_r<8>(fa, ba, smem, nblocks, st);
    case 10: return launch_part_r<10>(fa, ba, smem, nblocks, st);
    case 12: return launch_part_r<12>(fa, ba, smem, nblocks, st);
    case 14: return launch_part_r<14>(fa, ba, smem, nblocks, st);
    case 16: return launch_part_r<16>(fa, ba, smem, nblocks, st);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_f32_front(int r, const FrontArgs& fa, size_t smem, int64_t nblocks, cudaStream_t st)
{
    return launch_part(r, &fa, nullptr, smem, nblocks, st);
}
cudaError_t launch_f32_back(int r, const BackArgs& ba, size_t smem, int64_t nblocks, cudaStream_t st)
{
    return launch_part(r, nullptr, &ba, smem, nblocks, st);
}

cudaError_t launch_fused_f32(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws,
                             cudaStream_t st, int mr_hint)
{
    if (B.g.ra == 0) {
        if (!beta) return cudaMemsetAsync(G, 0, (size_t)B.g.N * m * sizeof(float2), st);
        return cudaSuccess;
    }
    const Geo& g = B.g;
    const Passes ps = passes_of(g, true, mr_hint);
    FrontArgs fa;
    BackArgs ba;
    size_t sf, sb;
    int64_t nf, nb;
    if (!make_args(B, F, m, G, beta, ws, mr_hint, ps, &fa, &ba, &sf, &sb, &nf, &nb, true))
        return cudaErrorNotSupported;
    if (!ps.split()) {
        if (g.otf) {
            const cudaError_t e = launch_part(g.r, &fa, nullptr, sf, nf, st);
            return e != cudaSuccess ? e : launch_part(g.r, nullptr, &ba, sb, nb, st);
        }
        switch (g.r) {
        case 6: return launch_r<6>(fa, ba, sf, sb, nf, nb, st);
        case 8: return launch_r<8>(fa, ba, sf, sb, nf, nb, st);
        case 10: return launch_r<10>(fa, ba, sf, sb, nf, nb, st);
        case 12: return launch_r<12>(fa, ba, sf, sb, nf, nb, st);
        case 14: return launch_r<14>(fa, ba, sf, sb, nf, nb, st);
        case 16: return launch_r<16>(fa, ba, sf, sb, nf, nb, st);
        default: return cudaErrorNotSupported;
        }
    }
    // Split level ranges: ws = W | X, one more buffer of W's size.  A pass reads the
    // buffer the previous one wrote and writes the other: the last H pass writes W
    // (after the switch), so H pass i of nh writes X if nh - 2 - i is even, else W;
    // G pass j (of the middle ones) reads W or X and writes X if j is even, else W.
    // Order: front (V + first H pass) -> middle H passes -> middle G passes -> back.
    const size_t w = (size_t)fa.nslice * g.P * g.r * fa.CTp;
    float2* X = ws + w;
    auto plain = [&](int l) { return WLayout{l, g.L - l, 0, 0, g.P}; };
    MidArgs ma{};
    ma.g = g;
    ma.mr = fa.mr;
    ma.lmr = fa.lmr;
    ma.CTp = fa.CTp;
    ma.lct = fa.lct;
    ma.nslice = fa.nslice;
    ma.ph = B.ph;
    auto run_mid = [&]() {
        const bool last = ma.gkind == 0 && ma.last;
        ma.tpc = tiles_per_cta(ma.K, ma.CTp, (int64_t)1 << (g.L - ma.K),
                               [&](int t) { return mid_smem(g, ma.K, last, g.r, ma.CTp, t); });
        const size_t smem = mid_smem(g, ma.K, last, g.r, ma.CTp, ma.tpc);
        const int64_t nblocks = ((int64_t)1 << (g.L - ma.K)) * ma.nslice / ma.tpc;
        return g.otf ? launch_mid_otf(g.r, ma, smem, nblocks, st) : launch_mid(g.r, ma, smem, nblocks, st);
    };
    const int nh = (int)ps.hs.size();
    auto h_out = [&](int i) { return i == nh - 1 ? ws : (((nh - 2 - i) & 1) == 0 ? X : ws); };
    int lvl = g.l1 + ps.hs[0];
    if (!fa.last) fa.Wo = h_out(0);
    cudaError_t e = launch_part(g.r, &fa, nullptr, sf, nf, st);
    for (int i = 1; i < nh && e == cudaSuccess; ++i) {
        const bool last = i == nh - 1;
        ma.gkind = 0;
        ma.la = lvl;
        ma.K = ps.hs[(size_t)i];
        ma.last = last;
        ma.Wi = h_out(i - 1);
        ma.wli = plain(lvl);
        ma.Wo = h_out(i);
        ma.wlo = last ? fa.wl : plain(lvl + ma.K);
        ma.MT = B.f32.MH;
        ma.E = B.f32.EH;
        ma.e0 = lvl - g.l1;
        ma.S = B.f32.S;
        e = run_mid();
        lvl += ma.K;
    }
    const float2* src = ws;  // G side: from W at level h
    WLayout wsrc = fa.wl;
    lvl = g.h;
    for (size_t j = 0; j + 1 < ps.gs.size() && e == cudaSuccess; ++j) {
        ma.gkind = 1;
        ma.la = lvl;
        ma.K = ps.gs[j];
        ma.last = 0;
        ma.Wi = src;
        ma.wli = wsrc;
        ma.Wo = (j & 1) == 0 ? X : ws;
        ma.wlo = plain(lvl + ma.K);
        ma.MT = B.f32.MG;
        ma.E = B.f32.FG;
        ma.e0 = lvl - g.h;
        ma.S = nullptr;
        e = run_mid();
        src = ma.Wo;
        wsrc = ma.wlo;
        lvl += ma.K;
    }
    if (e != cudaSuccess) return e;
    ba.W = src;
    ba.wl = wsrc;
    return launch_part(g.r, nullptr, &ba, sb, nb, st);
}

// Row ranges of a single-pass apply (one front and one back pass): nch front launches over
// consecutive ranges of T_Omega chunks and nch back launches over consecutive ranges of
// x-nodes.  Front launch k reads F rows [k N/nch, (k+1) N/nch) only; back launch k writes
// G rows [k N/nch, (k+1) N/nch) only.  Same tiles, same arithmetic as launch_fused_f32.
static bool chunk_args(const DevBlock& B, const float2* F, int64_t m, float2* G, float2* ws, int mr_hint, int nch,
                       FrontArgs* fa, BackArgs* ba, size_t* sf, size_t* sb, int64_t* nf, int64_t* nb)
{
    const Geo& g = B.g;
    if (g.ra == 0 || nch < 1 || (nch & (nch - 1))) return false;
    const Passes ps = passes_of(g, true, mr_hint);
    if (ps.split()) return false;
    if (!make_args(B, F, m, G, 0, ws, mr_hint, ps, fa, ba, sf, sb, nf, nb, true)) return false;
    const int64_t nc0 = (g.N / g.n0) >> (fa->K + g.l1);  // T_Omega chunks c0 (tiles per x-node)
    const int64_t npp = (int64_t)1 << ba->lb;             // back x-nodes
    if (nc0 % nch || npp % nch) return false;
    if (((nc0 / nch) << g.l1) * fa->nslice % fa->tpc) return false;
    *nf /= nch;
    *nb /= nch;
    return true;
}

bool fused_f32_chunkable(const DevBlock& B, int64_t m, int mr_hint, int nch)
{
    FrontArgs fa;
    BackArgs ba;
    size_t sf, sb;
    int64_t nf, nb;
    return chunk_args(B, nullptr, m, nullptr, nullptr, mr_hint, nch, &fa, &ba, &sf, &sb, &nf, &nb);
}

cudaError_t launch_fused_f32_chunked(const DevBlock& B, const float2* F, int64_t m, float2* G, float2* ws,
                                     cudaStream_t st, cudaStream_t st2, int mr_hint, int nch, const cudaEvent_t* fready,
                                     const cudaEvent_t* gdone, const cudaEvent_t* join)
{
    FrontArgs fa;
    BackArgs ba;
    size_t sf, sb;
    int64_t nf, nb;
    if (!chunk_args(B, F, m, G, ws, mr_hint, nch, &fa, &ba, &sf, &sb, &nf, &nb)) return cudaErrorNotSupported;
    const int64_t nc0 = (B.g.N / B.g.n0) >> (fa.K + B.g.l1), npp = (int64_t)1 << ba.lb;
    // range k runs on stream k mod 2, so that a range's CTAs start while the previous
    // range's last wave drains; st2 starts after the caller's earlier work on st
    cudaStream_t S[2] = {st, st2};
    cudaError_t e = cudaEventRecord(join[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st2, join[0], 0);
    for (int k = 0; k < nch && e == cudaSuccess; ++k) {
        if ((e = cudaStreamWaitEvent(S[k & 1], fready[k], 0)) != cudaSuccess) break;
        fa.c0_lo = k * (nc0 / nch);
        e = launch_part(B.g.r, &fa, nullptr, sf, nf, S[k & 1]);
    }
    // every back range reads the switch-level pairs of all front ranges: join both streams
    if (e == cudaSuccess) e = cudaEventRecord(join[1], st2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join[1], 0);
    if (e == cudaSuccess) e = cudaEventRecord(join[2], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st2, join[2], 0);
    for (int k = 0; k < nch && e == cudaSuccess; ++k) {
        ba.pp_lo = k * (npp / nch);
        if ((e = launch_part(B.g.r, nullptr, &ba, sb, nb, S[k & 1])) != cudaSuccess) break;
        e = cudaEventRecord(gdone[k], S[k & 1]);
    }
    // st ends after all back ranges
    if (e == cudaSuccess) e = cudaEventRecord(join[3], st2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join[3], 0);
    return e;
}

cudaError_t batch_phases_f32(int r, const BatchLaunch& bl, cudaStream_t st, bool set_attr)
{
    switch (r) {
    case 6: return batch_phases_r<6>(bl, st, set_attr);
    case 8: return batch_phases_r<8>(bl, st, set_attr);
    case 10: return batch_phases_r<10>(bl, st, set_attr);
    case 12: return batch_phases_r<12>(bl, st, set_attr);
    case 14: return batch_phases_r<14>(bl, st, set_attr);
    case 16: return batch_phases_r<16>(bl, st, set_attr);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t batch_launch_f32(int r, const BatchLaunch& bl, cudaStream_t st, bool set_attr, int* grid_out)
{
    switch (r) {
    case 6: return batch_launch_r<6>(bl, st, set_attr, grid_out);
    case 8: return batch_launch_r<8>(bl, st, set_attr, grid_out);
    case 10: return batch_launch_r<10>(bl, st, set_attr, grid_out);
    case 12: return batch_launch_r<12>(bl, st, set_attr, grid_out);
    case 14: return batch_launch_r<14>(bl, st, set_attr, grid_out);
    case 16: return batch_launch_r<16>(bl, st, set_attr, grid_out);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace bfi
