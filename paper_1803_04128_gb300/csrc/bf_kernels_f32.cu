// Fused FP32 apply of one sub-BF in two launches (front: V, H levels, switch;
// back: G levels, U), phases read from the tables; the batched persistent
// kernel; configuration and launchers.  The tile bodies are in bf_f32_tile.h.
#include <algorithm>
#include <cstdio>

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

FusedCfg fused_f32_config(const Geo& g, int64_t m, int mr_hint)
{
    const int Tmax = 1 << (g.kG > g.kH ? g.kG : g.kH);
    const int ra = g.ra > 0 ? g.ra : 1;
    const int NV = g.nv;
    auto smem = [&](int mr) {
        const int CTp = 1 << ilog2(ra * mr);
        return std::max(front_smem(g, g.r, NV, CTp, mr, 1), back_smem(g, g.r, NV, CTp, mr, 1));
    };
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
    // with few columns per tile, several front tiles (back chunks) per CTA: up to one
    // (tile, group, column) item per thread and level, two CTAs per SM
    const int CTp = 1 << ilog2(ra * mr);
    const int itemsH = std::max(1, (1 << g.kH) / 2) * CTp, itemsG = std::max(1, (1 << g.kG) / 2) * CTp;
    const int64_t maxf = (int64_t)1 << (g.l1 + g.L - g.h), maxb = (int64_t)1 << g.l1;
    c.tpc_f = 1;
    while (c.tpc_f < 16 && 2 * c.tpc_f <= maxf && 2 * c.tpc_f * itemsH <= kThreads &&
           front_smem(g, g.r, NV, CTp, mr, 2 * c.tpc_f) <= 113 * 1024)
        c.tpc_f *= 2;
    c.tpc_b = 1;
    while (c.tpc_b < 16 && 2 * c.tpc_b <= maxb && 2 * c.tpc_b * itemsG <= kThreads &&
           back_smem(g, g.r, NV, CTp, mr, 2 * c.tpc_b) <= 113 * 1024)
        c.tpc_b *= 2;
    return c;
}

size_t fused_f32_ws_bytes(const Geo& g, int64_t m, int mr_hint)
{
    const FusedCfg c = fused_f32_config(g, m, mr_hint);
    const int CTp = 1 << ilog2((g.ra > 0 ? g.ra : 1) * c.mr);
    return (size_t)c.nslice * g.P * g.r * CTp * sizeof(float2);
}

bool fused_make_args(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws, int mr_hint,
                     FrontArgs* fa, BackArgs* ba, size_t* sf, size_t* sb, int64_t* nfront, int64_t* nback)
{
    const Geo& g = B.g;
    if (!fused_f32_supported(g.r)) return false;
    const int NV = (g.r < 8) ? 8 : (g.r < 16 ? 16 : 32);
    if (g.nv != NV || g.ra < 1) return false;
    const FusedCfg cfg = fused_f32_config(g, m, mr_hint);
    const int CTp = 1 << ilog2(g.ra * cfg.mr);
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
    *sf = front_smem(g, g.r, NV, CTp, cfg.mr, cfg.tpc_f);
    *sb = back_smem(g, g.r, NV, CTp, cfg.mr, cfg.tpc_b);
    *nfront = ((int64_t)1 << g.l1) * ((int64_t)1 << (g.L - g.h)) * cfg.nslice / cfg.tpc_f;
    *nback = ((int64_t)1 << g.h) * cfg.nslice;
    return true;
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
    FrontArgs fa;
    BackArgs ba;
    size_t sf, sb;
    int64_t nf, nb;
    if (!fused_make_args(B, F, m, G, beta, ws, mr_hint, &fa, &ba, &sf, &sb, &nf, &nb)) return cudaErrorNotSupported;
    if (B.g.otf) {
        const cudaError_t e = launch_part(B.g.r, &fa, nullptr, sf, nf, st);
        return e != cudaSuccess ? e : launch_part(B.g.r, nullptr, &ba, sb, nb, st);
    }
    switch (B.g.r) {
    case 6: return launch_r<6>(fa, ba, sf, sb, nf, nb, st);
    case 8: return launch_r<8>(fa, ba, sf, sb, nf, nb, st);
    case 10: return launch_r<10>(fa, ba, sf, sb, nf, nb, st);
    case 12: return launch_r<12>(fa, ba, sf, sb, nf, nb, st);
    case 14: return launch_r<14>(fa, ba, sf, sb, nf, nb, st);
    case 16: return launch_r<16>(fa, ba, sf, sb, nf, nb, st);
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
