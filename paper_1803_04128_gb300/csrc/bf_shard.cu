// Sharded apply of one operator: the front half (xi side) and the back half
// (x side) of the fused FP32 kernels on 1/G of the tiles each, with the
// switch-level workspace laid out in per-peer blocks for an all-to-all.
#include <algorithm>

#include "bf_device.h"
#include "bf_fused.h"
#include "bf_internal.h"
#include "bf_shard.h"

namespace bfi {
namespace {

int log2i(int64_t v)
{
    int l = 0;
    while (((int64_t)1 << l) < v) ++l;
    return l;
}

struct ShardCfg {
    FrontArgs fa;
    BackArgs ba;
    size_t sf = 0, sb = 0;
    int64_t nfront = 0, nback = 0, chunk_pairs = 0, chunk_elems = 0;
    int r = 0;
};

bf_status shard_setup(bf_plan* p, int G, int64_t m, ShardCfg& c, const char* who)
{
    if (!p || m < 1 || G < 1 || (G & (G - 1)) != 0) {
        set_error("%s: NULL plan, m < 1 or G not a power of two", who);
        return BF_ERR_ARG;
    }
    bf_status st = bf_upload(p);
    if (st != BF_OK) return st;
    if (p->dev->blocks.size() != 1) {
        set_error("%s: split plans are not sharded", who);
        return BF_ERR_UNSUPPORTED;
    }
    const DevBlock& B = p->dev->blocks[0];
    const Geo& g = B.g;
    const int lg = log2i(G);
    if (lg > g.l1 || lg > g.h) {
        set_error("%s: G = %d exceeds min(2^l1, 2^h) = %lld", who, G, (long long)std::min(1 << g.l1, 1 << g.h));
        return BF_ERR_ARG;
    }
    if (!fused_make_args(B, nullptr, m, nullptr, 0, nullptr, p->mr_hint(m), &c.fa, &c.ba, &c.sf, &c.sb, &c.nfront,
                         &c.nback)) {
        set_error("%s: no fused FP32 kernels for r = %d", who, g.r);
        return BF_ERR_UNSUPPORTED;
    }
    const int la = g.h - lg, lb = (g.L - g.h) - lg;
    const int64_t nslice = c.fa.nslice;
    c.chunk_pairs = nslice << (la + lb);
    c.chunk_elems = c.chunk_pairs * (int64_t)g.r * c.fa.CTp;
    c.fa.wl = WLayout{la, lb, c.chunk_pairs, 0, (int64_t)1 << (la + lb)};
    c.ba.wl = WLayout{la, lb, 0, c.chunk_pairs, (int64_t)1 << (la + lb)};
    const int64_t tiles = ((int64_t)1 << (g.l1 + lb)) * nslice;  // front tiles of one shard
    while (c.fa.tpc > 1 && tiles % c.fa.tpc != 0) c.fa.tpc >>= 1;
    c.nfront = tiles / c.fa.tpc;
    c.nback = ((int64_t)1 << la) * nslice;
    c.r = g.r;
    return BF_OK;
}

}  // namespace
}  // namespace bfi

using namespace bfi;

extern "C" {

bf_status bf_shard_info(bf_plan* p, int G, int64_t m, int64_t* chunk_elems)
{
    ShardCfg c;
    bf_status st = shard_setup(p, G, m, c, "bf_shard_info");
    if (st != BF_OK) return st;
    if (chunk_elems) *chunk_elems = c.chunk_elems;
    return BF_OK;
}

bf_status bf_apply_shard_front(bf_plan* p, int G, int s, const void* F_rows, int64_t m, void* W_send, void* stream)
{
    ShardCfg c;
    bf_status st = shard_setup(p, G, m, c, "bf_apply_shard_front");
    if (st != BF_OK) return st;
    if (s < 0 || s >= G || !F_rows || !W_send) {
        set_error("bf_apply_shard_front: shard out of range or NULL buffer");
        return BF_ERR_ARG;
    }
    const Geo& g = p->dev->blocks[0].g;
    c.fa.F = (const float2*)F_rows;
    c.fa.W = (float2*)W_send;
    c.fa.c0_lo = (int64_t)s << c.fa.wl.lb;
    c.fa.xi_lo = (int64_t)s * (g.N / G);
    cudaError_t e = cudaSetDevice(p->dev->device);
    if (e == cudaSuccess) e = launch_f32_front(c.r, c.fa, c.sf, c.nfront, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("bf_apply_shard_front: %s", cudaGetErrorString(e));
        return BF_ERR_CUDA;
    }
    return BF_OK;
}

bf_status bf_apply_shard_back(bf_plan* p, int G, int d, const void* W_recv, int64_t m, void* G_rows, void* stream)
{
    ShardCfg c;
    bf_status st = shard_setup(p, G, m, c, "bf_apply_shard_back");
    if (st != BF_OK) return st;
    if (d < 0 || d >= G || !W_recv || !G_rows) {
        set_error("bf_apply_shard_back: shard out of range or NULL buffer");
        return BF_ERR_ARG;
    }
    const Geo& g = p->dev->blocks[0].g;
    c.ba.W = (const float2*)W_recv;
    c.ba.G = (float2*)G_rows;
    c.ba.beta = 0;
    c.ba.pp_lo = (int64_t)d << c.ba.wl.la;
    c.ba.x_lo = (int64_t)d * (g.N / G);
    cudaError_t e = cudaSetDevice(p->dev->device);
    if (e == cudaSuccess) e = launch_f32_back(c.r, c.ba, c.sb, c.nback, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("bf_apply_shard_back: %s", cudaGetErrorString(e));
        return BF_ERR_CUDA;
    }
    return BF_OK;
}

}  // extern "C"
