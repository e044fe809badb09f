// Batched uneven apply (many operators of different N and m in one persistent
// launch, optionally captured in a CUDA graph) and the column-slice autotuner.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bf_batch.h"
#include "bf_fused.h"

using namespace bfi;

namespace {
constexpr int kStreams = 4;  // mode 2's streams
// one operator of mode 2: its own fused apply, as bf_apply launches it
struct SoloItem {
    const DevBlock* B = nullptr;
    const float2* F = nullptr;
    float2* G = nullptr;
    int64_t m = 0;
    float2* ws = nullptr;
    int hint = 0;
    int stream = 0;
};
}  // namespace

struct bf_batch {
    int device = 0;
    int r = 0;
    BatchLaunch bl;
    std::vector<BatchItem> items;
    // mode 2: the operators' own applies on kStreams streams (decreasing work, each on the
    // stream with the least work so far), forked from and joined to the caller's stream
    std::vector<SoloItem> solo;
    cudaStream_t ss[kStreams] = {};
    cudaEvent_t fork = nullptr, join[kStreams] = {};
    double tune_ms[3] = {0, 0, 0};
    void* dmem = nullptr;  // items, offsets, counter/done, err
    size_t dmem_bytes = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    unsigned char* reset_ptr = nullptr;  // counter + done, cleared before each launch
    size_t reset_bytes = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

namespace {

constexpr size_t kTwoCtaSmem = 113 * 1024;

bf_status cuda_fail(const char* where, cudaError_t e)
{
    set_error("%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA;
}

void free_batch(bf_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (int k = 0; k < kStreams; ++k) {
        if (b->ss[k]) cudaStreamDestroy(b->ss[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->dmem) cudaFree(b->dmem);
    if (b->ws) cudaFree(b->ws);
    delete b;
}

bf_status enqueue(bf_batch* b, cudaStream_t st)
{
    cudaError_t e;
    if (b->bl.mode == 2) {
        if ((e = cudaEventRecord(b->fork, st)) != cudaSuccess) return cuda_fail("bf_batch: fork", e);
        for (int k = 0; k < kStreams; ++k)
            if ((e = cudaStreamWaitEvent(b->ss[k], b->fork, 0)) != cudaSuccess) return cuda_fail("bf_batch: fork", e);
        for (const SoloItem& it : b->solo)
            if ((e = launch_fused_f32(*it.B, it.F, it.m, it.G, 0, it.ws, b->ss[it.stream], it.hint)) != cudaSuccess)
                return cuda_fail("bf_batch: launch", e);
        for (int k = 0; k < kStreams; ++k)
            if ((e = cudaEventRecord(b->join[k], b->ss[k])) != cudaSuccess ||
                (e = cudaStreamWaitEvent(st, b->join[k], 0)) != cudaSuccess)
                return cuda_fail("bf_batch: join", e);
        return BF_OK;
    }
    if (b->bl.grid < 1) {
        set_error("bf_batch: no persistent grid configured");
        return BF_ERR_STATE;
    }
    if (b->bl.mode == 1) {
        e = batch_phases_f32(b->r, b->bl, st, false);
        if (e != cudaSuccess) return cuda_fail("bf_batch: phase launches", e);
        return BF_OK;
    }
    e = cudaMemsetAsync(b->reset_ptr, 0, b->reset_bytes, st);
    if (e != cudaSuccess) return cuda_fail("bf_batch: reset", e);
    e = batch_launch_f32(b->r, b->bl, st, false, nullptr);
    if (e != cudaSuccess) return cuda_fail("bf_batch: launch", e);
    return BF_OK;
}

}  // namespace

extern "C" {

bf_status bf_batch_create(const bf_batch_item* in, int n, bf_batch** out)
{
    if (!in || n < 1 || !out) {
        set_error("bf_batch_create: need n >= 1 items and an output pointer");
        return BF_ERR_ARG;
    }
    *out = nullptr;
    bf_batch* b = new (std::nothrow) bf_batch();
    if (!b) {
        set_error("bf_batch_create: out of host memory");
        return BF_ERR_NOMEM;
    }
    // validate and upload
    for (int i = 0; i < n; ++i) {
        const bf_batch_item& it = in[i];
        if (!it.plan || !it.F || !it.G || it.m < 1 || it.F == it.G) {
            free_batch(b);
            set_error("bf_batch_create: item %d: NULL plan/buffer, m < 1 or G aliasing F", i);
            return BF_ERR_ARG;
        }
        bf_status st = bf_upload(it.plan);
        if (st != BF_OK) {
            free_batch(b);
            return st;
        }
        if (it.plan->otf) {
            free_batch(b);
            set_error("bf_batch_create: item %d: plans factored by bf_factor_otf are not batched (use bf_apply)", i);
            return BF_ERR_UNSUPPORTED;
        }
        if (it.plan->blocks.size() != 1) {
            free_batch(b);
            set_error("bf_batch_create: item %d: split plans are not batched (apply them with bf_apply)", i);
            return BF_ERR_UNSUPPORTED;
        }
        const int r = it.plan->r;
        if (i == 0) {
            b->r = r;
            b->device = it.plan->dev->device;
        } else if (r != b->r || it.plan->dev->device != b->device) {
            free_batch(b);
            set_error("bf_batch_create: item %d: all items must share r and device (got r=%d vs %d)", i, r, b->r);
            return BF_ERR_UNSUPPORTED;
        }
        if (it.plan->dev->blocks[0].g.ra < 1) {
            free_batch(b);
            set_error("bf_batch_create: item %d: zero amplitude", i);
            return BF_ERR_UNSUPPORTED;
        }
    }
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail("bf_batch_create: cudaSetDevice", e);
    }
    // workspaces (one per item, packed) and argument blocks
    std::vector<size_t> ws_off((size_t)n);
    size_t ws_total = 0;
    for (int i = 0; i < n; ++i) {
        const DevBlock& B = in[i].plan->dev->blocks[0];
        ws_off[(size_t)i] = ws_total;
        // the persistent kernels' one pass per side, and (mode 2) the plan's own apply, whose
        // long level ranges may run in passes
        const int hint = in[i].plan->mr_hint(in[i].m);
        ws_total += (std::max({fused_f32_ws_bytes(B.g, in[i].m, hint, false), fused_f32_ws_bytes(B.g, in[i].m, 0, false),
                               fused_f32_ws_bytes(B.g, in[i].m, hint)}) + 255) & ~(size_t)255;
    }
    if ((e = cudaMalloc(&b->ws, std::max<size_t>(ws_total, 256))) != cudaSuccess) {
        free_batch(b);
        return cuda_fail("bf_batch_create: workspace", e);
    }
    b->ws_bytes = ws_total;
    b->items.resize((size_t)n);
    std::vector<int64_t> off((size_t)(2 * n));
    int64_t tot = 0;
    size_t smem = 0, smem_f = 0, smem_b = 0;
    for (int i = 0; i < n; ++i) {
        const DevBlock& B = in[i].plan->dev->blocks[0];
        BatchItem& bi = b->items[(size_t)i];
        size_t sf, sb;
        // keep every item within the shared memory of two resident CTAs per SM: the
        // persistent launch runs all items at the occupancy of the largest one
        int hint = in[i].plan->mr_hint(in[i].m);
        bool ok = fused_make_args(B, (const float2*)in[i].F, in[i].m, (float2*)in[i].G, 0,
                                  (float2*)((unsigned char*)b->ws + ws_off[(size_t)i]), hint, &bi.fa, &bi.ba, &sf,
                                  &sb, &bi.nfront, &bi.nback);
        if (ok && hint != 0 && std::max(sf, sb) > kTwoCtaSmem)
            ok = fused_make_args(B, (const float2*)in[i].F, in[i].m, (float2*)in[i].G, 0,
                                 (float2*)((unsigned char*)b->ws + ws_off[(size_t)i]), 0, &bi.fa, &bi.ba, &sf, &sb,
                                 &bi.nfront, &bi.nback);
        if (!ok) {
            free_batch(b);
            set_error("bf_batch_create: item %d: no fused FP32 kernels for r=%d", i, B.g.r);
            return BF_ERR_UNSUPPORTED;
        }
        smem = std::max(smem, std::max(sf, sb));
        smem_f = std::max(smem_f, sf);
        smem_b = std::max(smem_b, sb);
    }
    // mode 1's order: operators by decreasing work (front + back CTAs), so that the small ones
    // fill the last wave of each phase
    std::vector<int> ord((size_t)n);
    for (int i = 0; i < n; ++i) ord[(size_t)i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
        const BatchItem &a = b->items[(size_t)x], &c = b->items[(size_t)y];
        return a.nfront + a.nback > c.nfront + c.nback;
    });
    // mode 2: operators by decreasing work, each on the stream with the least work so far
    {
        int64_t load[kStreams] = {};
        b->solo.resize((size_t)n);
        for (int k = 0; k < n; ++k) {
            const int i = ord[(size_t)k];
            const BatchItem& bi = b->items[(size_t)i];
            int best = 0;
            for (int q = 1; q < kStreams; ++q)
                if (load[q] < load[best]) best = q;
            load[best] += bi.nfront + bi.nback;
            SoloItem& so = b->solo[(size_t)k];
            so.B = &in[i].plan->dev->blocks[0];
            so.F = (const float2*)in[i].F;
            so.G = (float2*)in[i].G;
            so.m = in[i].m;
            so.ws = (float2*)((unsigned char*)b->ws + ws_off[(size_t)i]);
            so.hint = in[i].plan->mr_hint(in[i].m);
            so.stream = best;
        }
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int q = 0; q < kStreams && e == cudaSuccess; ++q) {
            e = cudaStreamCreateWithFlags(&b->ss[q], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[q], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            free_batch(b);
            return cuda_fail("bf_batch_create: streams", e);
        }
    }
    std::vector<int64_t> off_f((size_t)n + 1, 0), off_b((size_t)n + 1, 0);
    for (int k = 0; k < n; ++k) {
        off_f[(size_t)k + 1] = off_f[(size_t)k] + b->items[(size_t)ord[(size_t)k]].nfront;
        off_b[(size_t)k + 1] = off_b[(size_t)k] + b->items[(size_t)ord[(size_t)k]].nback;
    }
    // Work order: each operator's front segment, and its back segment once at
    // least kBackLag work items have been queued after that front segment (or
    // at the end), so that a back tile rarely finds its operator's fronts still
    // running.  Every front of an operator precedes all of its backs, so a back
    // tile's wait always ends.
    std::vector<int> seg((size_t)(2 * n));
    {
        constexpr int64_t kBackLag = 1024;
        std::vector<std::pair<int, int64_t>> pending;  // (op, position after its fronts)
        size_t head = 0, k = 0;
        auto put = [&](int op, bool back) {
            off[k] = tot;
            seg[k++] = (op << 1) | (back ? 1 : 0);
            tot += back ? b->items[(size_t)op].nback : b->items[(size_t)op].nfront;
        };
        for (int i = 0; i < n; ++i) {
            put(i, false);
            pending.emplace_back(i, tot);
            while (head < pending.size() && tot - pending[head].second >= kBackLag) put(pending[head++].first, true);
        }
        while (head < pending.size()) put(pending[head++].first, true);
    }
    if (smem > 227 * 1024) {
        free_batch(b);
        set_error("bf_batch_create: a tile needs %zu bytes of shared memory", smem);
        return BF_ERR_UNSUPPORTED;
    }
    // device copies: items | off[2n] | seg[2n] | counter | done[n] | err | ord[n] | off_f[n+1] | off_b[n+1]
    const size_t s_items = ((size_t)n * sizeof(BatchItem) + 255) & ~(size_t)255;
    const size_t s_off = ((size_t)(2 * n) * sizeof(int64_t) + 255) & ~(size_t)255;
    const size_t s_seg = ((size_t)(2 * n) * sizeof(int) + 255) & ~(size_t)255;
    const size_t s_reset = ((sizeof(unsigned long long) + (size_t)n * sizeof(int)) + 255) & ~(size_t)255;
    const size_t s_ord = ((size_t)n * sizeof(int) + 255) & ~(size_t)255;
    const size_t s_offp = ((size_t)(n + 1) * sizeof(int64_t) + 255) & ~(size_t)255;
    const size_t o_phase = s_items + s_off + s_seg + s_reset + 256;
    b->dmem_bytes = o_phase + s_ord + 2 * s_offp;
    if ((e = cudaMalloc(&b->dmem, b->dmem_bytes)) != cudaSuccess) {
        free_batch(b);
        return cuda_fail("bf_batch_create: descriptors", e);
    }
    unsigned char* base = (unsigned char*)b->dmem;
    std::vector<unsigned char> host(b->dmem_bytes, 0);
    std::memcpy(host.data(), b->items.data(), (size_t)n * sizeof(BatchItem));
    std::memcpy(host.data() + s_items, off.data(), (size_t)(2 * n) * sizeof(int64_t));
    std::memcpy(host.data() + s_items + s_off, seg.data(), (size_t)(2 * n) * sizeof(int));
    std::memcpy(host.data() + o_phase, ord.data(), (size_t)n * sizeof(int));
    std::memcpy(host.data() + o_phase + s_ord, off_f.data(), (size_t)(n + 1) * sizeof(int64_t));
    std::memcpy(host.data() + o_phase + s_ord + s_offp, off_b.data(), (size_t)(n + 1) * sizeof(int64_t));
    if ((e = cudaMemcpy(base, host.data(), b->dmem_bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
        free_batch(b);
        return cuda_fail("bf_batch_create: upload", e);
    }
    b->bl.items = (const BatchItem*)base;
    b->bl.nitems = n;
    b->bl.off = (const int64_t*)(base + s_items);
    b->bl.seg = (const int*)(base + s_items + s_off);
    b->reset_ptr = base + s_items + s_off + s_seg;
    b->reset_bytes = s_reset;
    b->bl.counter = (unsigned long long*)b->reset_ptr;
    b->bl.done = (int*)(b->reset_ptr + sizeof(unsigned long long));
    b->bl.err = (int*)(b->reset_ptr + s_reset);
    b->bl.total = tot;
    b->bl.smem = smem;
    b->bl.ord = (const int*)(base + o_phase);
    b->bl.off_f = (const int64_t*)(base + o_phase + s_ord);
    b->bl.off_b = (const int64_t*)(base + o_phase + s_ord + s_offp);
    b->bl.smem_f = smem_f;
    b->bl.smem_b = smem_b;
    b->bl.total_f = off_f[(size_t)n];
    b->bl.total_b = off_b[(size_t)n];
    b->bl.mode = 0;
    e = batch_launch_f32(b->r, b->bl, nullptr, true, nullptr);
    if (e == cudaSuccess) e = batch_phases_f32(b->r, b->bl, nullptr, true);
    if (e == cudaSuccess) e = batch_launch_f32(b->r, b->bl, nullptr, false, &b->bl.grid);
    if (e != cudaSuccess || b->bl.grid < 1) {
        free_batch(b);
        return cuda_fail("bf_batch_create: occupancy", e == cudaSuccess ? cudaErrorInvalidConfiguration : e);
    }
    *out = b;
    return BF_OK;
}

bf_status bf_batch_run(bf_batch* b, void* stream)
{
    if (!b) {
        set_error("bf_batch_run: NULL batch");
        return BF_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return cuda_fail("bf_batch_run: cudaSetDevice", e);
    return enqueue(b, (cudaStream_t)stream);
}

bf_status bf_batch_capture_graph(bf_batch* b, void* stream)
{
    if (!b || !stream) {
        set_error("bf_batch_capture_graph: NULL batch or default stream (capture needs a created stream)");
        return BF_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return cuda_fail("bf_batch_capture_graph: cudaSetDevice", e);
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail("bf_batch_capture_graph: begin", e);
    bf_status s = enqueue(b, st);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (s != BF_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail("bf_batch_capture_graph: end", e);
    b->graph = g;
    if ((e = cudaGraphInstantiate(&b->exec, g, 0)) != cudaSuccess) return cuda_fail("bf_batch_capture_graph: instantiate", e);
    return BF_OK;
}

bf_status bf_batch_replay(bf_batch* b, void* stream)
{
    if (!b || !b->exec) {
        set_error("bf_batch_replay: NULL batch or no captured graph");
        return BF_ERR_STATE;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail("bf_batch_replay", e);
    return BF_OK;
}

bf_status bf_batch_status(bf_batch* b, void* stream)
{
    if (!b) {
        set_error("bf_batch_status: NULL batch");
        return BF_ERR_ARG;
    }
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail("bf_batch_status: sync", e);
    int h = 0;
    if ((e = cudaMemcpy(&h, b->bl.err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail("bf_batch_status: read", e);
    if (h) {
        cudaMemset(b->bl.err, 0, sizeof(int));
        set_error("bf_batch: a back tile gave up waiting for its front tiles (code %d)", h);
        return BF_ERR_TIMEOUT;
    }
    return BF_OK;
}

bf_status bf_batch_get_info(const bf_batch* b, int64_t* work_items, int* grid, int64_t* ws_bytes, int64_t* smem)
{
    if (!b) {
        set_error("bf_batch_get_info: NULL batch");
        return BF_ERR_ARG;
    }
    if (work_items) *work_items = b->bl.total;
    if (grid) *grid = b->bl.grid;
    if (ws_bytes) *ws_bytes = (int64_t)b->ws_bytes;
    if (smem) *smem = (int64_t)b->bl.smem;
    return BF_OK;
}

bf_status bf_batch_set_mode(bf_batch* b, int mode)
{
    if (!b || mode < 0 || mode > 2) {
        set_error("bf_batch_set_mode: NULL batch or mode not 0, 1 or 2");
        return BF_ERR_ARG;
    }
    if (b->bl.mode != mode && b->exec) {
        cudaGraphExecDestroy(b->exec);  // a captured graph holds the other mode's launches
        b->exec = nullptr;
        if (b->graph) cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    b->bl.mode = mode;
    return BF_OK;
}

bf_status bf_batch_get_mode(const bf_batch* b, int* mode)
{
    if (!b || !mode) {
        set_error("bf_batch_get_mode: NULL argument");
        return BF_ERR_ARG;
    }
    *mode = b->bl.mode;
    return BF_OK;
}

bf_status bf_batch_tune(bf_batch* b, void* stream, int* mode_out, double* ms_out)
{
    if (!b) {
        set_error("bf_batch_tune: NULL batch");
        return BF_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return cuda_fail("bf_batch_tune: cudaSetDevice", e);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail("bf_batch_tune: events", e);
    }
    const int keep = b->bl.mode;
    double best = 1e30, ms[3] = {0, 0, 0};
    int bm = keep;
    bf_status rs = BF_OK;
    for (int mode = 0; mode < 3 && rs == BF_OK; ++mode) {
        b->bl.mode = mode;
        double tot = 0;
        for (int rep = 0; rep < 4 && rs == BF_OK; ++rep) {  // one warm-up, three timed
            cudaEventRecord(e0, st);
            rs = enqueue(b, st);
            cudaEventRecord(e1, st);
            if (rs == BF_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) rs = cuda_fail("bf_batch_tune: run", e);
            float t = 0;
            if (rs == BF_OK) cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) tot += t;
        }
        ms[mode] = tot / 3;
        if (rs == BF_OK && ms[mode] < best) {
            best = ms[mode];
            bm = mode;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->bl.mode = keep;
    if (rs != BF_OK) return rs;
    rs = bf_batch_set_mode(b, bm);
    for (int k = 0; k < 3; ++k) b->tune_ms[k] = ms[k];
    if (mode_out) *mode_out = bm;
    if (ms_out) {
        ms_out[0] = ms[0];
        ms_out[1] = ms[1];
    }
    return rs;
}

bf_status bf_batch_tune_times(const bf_batch* b, double* ms, int n)
{
    if (!b || !ms || n < 1) {
        set_error("bf_batch_tune_times: NULL argument or n < 1");
        return BF_ERR_ARG;
    }
    for (int k = 0; k < n && k < 3; ++k) ms[k] = b->tune_ms[k];
    return BF_OK;
}

bf_status bf_batch_set_spin_limit(bf_batch* b, long long polls)
{
    if (!b || polls < 1) {
        set_error("bf_batch_set_spin_limit: NULL batch or polls < 1");
        return BF_ERR_ARG;
    }
    b->bl.spin_limit = polls;
    return BF_OK;
}

bf_status bf_batch_debug_hold(bf_batch* b, int on)
{
    if (!b) {
        set_error("bf_batch_debug_hold: NULL batch");
        return BF_ERR_ARG;
    }
    b->bl.wait_extra = on ? 1 : 0;
    return BF_OK;
}

void bf_batch_destroy(bf_batch* b) { free_batch(b); }

// ---------------------------------------------------------- one-call form --
namespace {
struct KeptBatch {
    std::vector<const bf_plan*> plans;
    std::vector<int64_t> ms;
    bf_batch* b = nullptr;  // not freed at thread exit (the CUDA context may be gone)
};
thread_local KeptBatch tl_kept;
}  // namespace

bf_status bf_apply_batched(bf_plan* const* plans, const bf_apply_item* items, int n, void* stream)
{
    if (!plans || !items || n < 1) {
        set_error("bf_apply_batched: NULL arguments or n_items < 1");
        return BF_ERR_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (!plans[i] || !items[i].F || !items[i].G || items[i].m < 1) {
            set_error("bf_apply_batched: item %d: NULL plan/F/G or m < 1", i);
            return BF_ERR_ARG;
        }
    KeptBatch& k = tl_kept;
    bool same = k.b && (int)k.plans.size() == n;
    for (int i = 0; same && i < n; ++i) same = k.plans[(size_t)i] == plans[i] && k.ms[(size_t)i] == items[i].m;
    if (same) {
        bf_batch* b = k.b;
        for (int i = 0; i < n; ++i) {
            b->items[(size_t)i].fa.F = (const float2*)items[i].F;
            b->items[(size_t)i].ba.G = (float2*)items[i].G;
        }
        cudaError_t e = cudaSetDevice(b->device);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->dmem, b->items.data(), (size_t)n * sizeof(BatchItem), cudaMemcpyHostToDevice,
                                (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail("bf_apply_batched: descriptor upload", e);
        return enqueue(b, (cudaStream_t)stream);
    }
    bf_apply_batched_release();
    std::vector<bf_batch_item> in((size_t)n);
    for (int i = 0; i < n; ++i) in[(size_t)i] = bf_batch_item{plans[i], items[i].F, items[i].G, items[i].m};
    bf_batch* b = nullptr;
    bf_status st = bf_batch_create(in.data(), n, &b);
    if (st != BF_OK) return st;
    k.b = b;
    k.plans.assign(plans, plans + n);
    k.ms.resize((size_t)n);
    for (int i = 0; i < n; ++i) k.ms[(size_t)i] = items[i].m;
    return bf_batch_run(b, stream);
}

void bf_apply_batched_release(void)
{
    KeptBatch& k = tl_kept;
    if (k.b) free_batch(k.b);
    k.b = nullptr;
    k.plans.clear();
    k.ms.clear();
}

// ---------------------------------------------------------------- autotune --
bf_status bf_autotune(bf_plan* p, int64_t m, const char* cache_path, int* mr_out)
{
    if (!p || m < 1) {
        set_error("bf_autotune: NULL plan or m < 1");
        return BF_ERR_ARG;
    }
    bf_status st = bf_upload(p);
    if (st != BF_OK) return st;
    DeviceState* ds = p->dev;
    const Geo& g0 = ds->blocks[0].g;
    char key[160];
    snprintf(key, sizeof(key), "N=%lld r=%d ra=%d split=%d m=%lld", (long long)p->N, p->r, g0.ra, p->opt.split,
             (long long)m);
    if (cache_path) {
        FILE* f = fopen(cache_path, "r");
        if (f) {
            char line[256];
            while (fgets(line, sizeof(line), f)) {
                const size_t kl = strlen(key);
                if (strncmp(line, key, kl) == 0 && line[kl] == ' ') {
                    int word = atoi(line + kl + 4);  // " mr=<v>"
                    const char* c = strstr(line + kl, " cfg=");
                    if (c) word = atoi(c + 5);       // the full tuning word, where recorded
                    if (tune_mr(word) > 0) {
                        p->tuned_mr[m] = word;
                        if (mr_out) *mr_out = tune_mr(word);
                        fclose(f);
                        return BF_OK;
                    }
                }
            }
            fclose(f);
        }
    }
    cudaError_t e = cudaSetDevice(ds->device);
    if (e != cudaSuccess) return cuda_fail("bf_autotune: cudaSetDevice", e);
    // candidate tuning words, searched one field at a time: the column-slice width mr, then
    // the most levels per pass of split level ranges, then the front tiles per CTA, then the
    // back chunks per CTA; each field keeps the best of its candidates (and 0, the built-in
    // rule) before the next is searched.  Every candidate computes the same result bitwise.
    auto cfg_of = [&](int w) { return fused_f32_config(g0, m, w); };
    auto same = [&](int a, int b) {
        const FusedCfg x = cfg_of(a), y = cfg_of(b);
        return x.mr == y.mr && x.tpc_f == y.tpc_f && x.tpc_b == y.tpc_b && x.kpass == y.kpass;
    };
    const int mr0 = cfg_of(0).mr;
    std::vector<int> mrs;
    for (int mr = 1; mr <= 128; mr *= 2)
        if (mr >= mr0 / 4 && mr <= mr0 * 4 && (int64_t)mr <= 2 * m && cfg_of(mr).mr == mr) mrs.push_back(mr);
    if (mrs.empty()) mrs.push_back(mr0);
    std::vector<int> kps = {0};
    if (std::max(g0.kH, g0.kG) > 2)
        for (int kp = 2; kp <= 6; ++kp) kps.push_back(kp);
    const int tlogs[] = {0, 1, 2, 3, 4, 5};  // 0: the rule; v: 2^(v - 1) tiles per CTA
    // workspace for every candidate: the largest over mr and pass splits (tiles per CTA do
    // not change it)
    size_t wsmax = 0;
    for (int mr : mrs)
        for (int kp : kps)
            for (auto& B : ds->blocks) wsmax = std::max(wsmax, fused_f32_ws_bytes(B.g, m, tune_word(mr, kp, 0, 0)));
    void *F = nullptr, *G = nullptr, *ws = nullptr;
    const size_t nb = (size_t)p->N * m * sizeof(float2);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (F) cudaFree(F);
        if (G) cudaFree(G);
        if (ws) cudaFree(ws);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    };
    if ((e = cudaMalloc(&F, nb)) != cudaSuccess || (e = cudaMalloc(&G, nb)) != cudaSuccess ||
        (e = cudaMalloc(&ws, wsmax)) != cudaSuccess || (e = cudaMemset(F, 0, nb)) != cudaSuccess ||
        (e = cudaStreamCreate(&s)) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
        (e = cudaEventCreate(&e1)) != cudaSuccess) {
        cleanup();
        return cuda_fail("bf_autotune: set-up", e);
    }
    // time one candidate: 4 applies after one warm-up
    auto trial = [&](int w, float* out_ms) -> cudaError_t {
        float tot = 0;
        for (int rep = 0; rep < 5; ++rep) {
            cudaEventRecord(e0, s);
            for (size_t i = 0; i < ds->blocks.size(); ++i) {
                const DevBlock& B = ds->blocks[i];
                const int beta = (p->opt.split == 2 && (i % 2) == 1) ? 1 : 0;
                const cudaError_t le = launch_fused_f32(B, (const float2*)F + B.col0 * m, m,
                                                        (float2*)G + B.row0 * m, beta, (float2*)ws, s, w);
                if (le != cudaSuccess) return le;
            }
            cudaEventRecord(e1, s);
            const cudaError_t se = cudaEventSynchronize(e1);
            if (se != cudaSuccess) return se;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep >= 1) tot += ms;  // the first run warms up
        }
        *out_ms = tot;
        return cudaSuccess;
    };
    int best = tune_word(mrs[0], 0, 0, 0);
    float best_ms = 1e30f;
    std::vector<int> tried;
    auto consider = [&](int w) -> cudaError_t {
        for (int t : tried)
            if (same(t, w)) return cudaSuccess;  // the same effective configuration
        tried.push_back(w);
        float ms = 0;
        const cudaError_t te = trial(w, &ms);
        if (te != cudaSuccess) return te;
        if (ms < best_ms) {
            best_ms = ms;
            best = w;
        }
        return cudaSuccess;
    };
    for (int mr : mrs)
        if ((e = consider(tune_word(mr, 0, 0, 0))) != cudaSuccess) break;
    const int mrb = tune_mr(best);
    for (size_t i = 0; i < kps.size() && e == cudaSuccess; ++i) e = consider(tune_word(mrb, kps[i], 0, 0));
    const int kpb = tune_kpass(best);
    for (int v : tlogs)
        if (e == cudaSuccess) e = consider(tune_word(mrb, kpb, v, 0));
    const int tfb = (best >> 12) & 0xF;
    for (int v : tlogs)
        if (e == cudaSuccess) e = consider(tune_word(mrb, kpb, tfb, v));
    cleanup();
    if (e != cudaSuccess) return cuda_fail("bf_autotune: trial", e);
    p->tuned_mr[m] = best;
    if (mr_out) *mr_out = tune_mr(best);
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s mr=%d cfg=%d ms=%.4f\n", key, tune_mr(best), best, best_ms / 4);
            fclose(f);
        }
    }
    return BF_OK;
}

bf_status bf_autotune_get(const bf_plan* p, int64_t m, int* mr, int* levels_per_pass, int* tpc_front, int* tpc_back)
{
    if (!p || m < 1) {
        set_error("bf_autotune_get: NULL plan or m < 1");
        return BF_ERR_ARG;
    }
    if (!p->dev || p->dev->blocks.empty()) {
        set_error("bf_autotune_get: plan not uploaded");
        return BF_ERR_STATE;
    }
    const FusedCfg c = fused_f32_config(p->dev->blocks[0].g, m, p->mr_hint(m));
    if (mr) *mr = c.mr;
    if (levels_per_pass) *levels_per_pass = c.kpass;
    if (tpc_front) *tpc_front = c.tpc_f;
    if (tpc_back) *tpc_back = c.tpc_b;
    return BF_OK;
}


}  // extern "C"
