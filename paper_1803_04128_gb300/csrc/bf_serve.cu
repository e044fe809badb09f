// Continuous-batching request loop (host runtime) over resident operators.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bf_internal.h"
#include "bf_serve.h"

using namespace bfi;

namespace {

using Clock = std::chrono::steady_clock;
// device intervals kept for the busy / overlap statistics (per reset; later batches are not counted)
constexpr size_t kMaxSpans = (size_t)1 << 20;
// batches of 2..kMaxSegs requests and at most kMaxCols columns move each request's rows as one
// contiguous copy and interleave them on the device (a host copy with rows of m elements is
// slow for small m); others copy each request's column block with a 2-D copy
constexpr int kMaxSegs = 64, kMaxCols = 1024;

// Column blocks of a batch: request k owns columns [c0[k], c0[k + 1]) of the [N][M] batch
// and, in the contiguous staging buffer, the N x m_k rows from element c0[k] * N on.
struct Segs {
    int n;
    int c0[kMaxSegs + 1];
};

// GATHER: dst[x][col] = staging of col's request (x, col - c0);  else the reverse.  A block
// takes chunks of about 4096 consecutive batch elements (whole rows of [N][M]), one thread
// per element, so the batch side is coalesced and each request's side walks its rows
// contiguously.
template <typename T, bool GATHER>
__global__ void interleave(const T* __restrict__ src, T* __restrict__ dst, int64_t N, int M, Segs sg)
{
    __shared__ short seg_of[kMaxCols];
    for (int k = 0; k < sg.n; ++k)
        for (int c = sg.c0[k] + (int)threadIdx.x; c < sg.c0[k + 1]; c += blockDim.x) seg_of[c] = (short)k;
    __syncthreads();
    const int rows = M >= 4096 ? 1 : 4096 / M;
    const int64_t nchunks = (N + rows - 1) / rows;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t x0 = ch * rows;
        const int nr = (int)(N - x0 < rows ? N - x0 : rows);
        for (int i = threadIdx.x; i < nr * M; i += blockDim.x) {
            const int xl = i / M, col = i - xl * M, k = seg_of[col], c0 = sg.c0[k], mk = sg.c0[k + 1] - c0;
            const int64_t e = x0 * M + i, st = (int64_t)c0 * N + (x0 + xl) * mk + (col - c0);
            if (GATHER) dst[e] = src[st];
            else dst[st] = src[e];
        }
    }
}

cudaError_t launch_interleave(bool gather, size_t elt, const void* src, void* dst, int64_t N, int M, const Segs& sg,
                              int nsm, cudaStream_t st)
{
    const int64_t chunks = (N + (4096 / M) - 1) / (4096 / M);  // M <= kMaxCols < 4096
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)nsm * 8));
    if (elt == sizeof(float2)) {
        if (gather) interleave<float2, true><<<grid, 256, 0, st>>>((const float2*)src, (float2*)dst, N, M, sg);
        else interleave<float2, false><<<grid, 256, 0, st>>>((const float2*)src, (float2*)dst, N, M, sg);
    } else {
        if (gather) interleave<double2, true><<<grid, 256, 0, st>>>((const double2*)src, (double2*)dst, N, M, sg);
        else interleave<double2, false><<<grid, 256, 0, st>>>((const double2*)src, (double2*)dst, N, M, sg);
    }
    return cudaGetLastError();
}

double ms_since(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Req {
    int op = 0;
    const void* F = nullptr;
    void* G = nullptr;
    int64_t m = 0;
    Clock::time_point t_submit, t_done;
    bool done = false;
    bf_status status = BF_OK;
};

struct Op {
    bf_plan* plan = nullptr;
    int64_t N = 0;
    int64_t cap = 0;  // right-hand sides per batch
    bool nufft = false;  // evaluated by the NUFFT of Eq. tg3 (method = auto and the phase allows it)
    std::deque<uint64_t> pending;
};

// A single large NUFFT request runs in kChunks column chunks, so that its host copies overlap
// its kernels: chunk k's copy in, its apply and its copy out are on three streams.
constexpr int kChunks = 2;
constexpr int64_t kChunkMinCols = 32, kChunkMinUnits = (int64_t)1 << 20;

struct Slot {
    cudaStream_t st = nullptr;
    bool hi = false;  // highest-priority stream, small batches only
    cudaEvent_t ev = nullptr;
    cudaEvent_t ev0 = nullptr;  // recorded before the batch's first copy (device-time accounting)
    cudaStream_t up = nullptr, down = nullptr;           // chunked requests: copies in / out
    cudaEvent_t in_ready[kChunks] = {}, done[kChunks] = {}, joined = nullptr;
    void* F = nullptr;
    void* G = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool busy = false;
    std::vector<uint64_t> reqs;
    int op = -1;
    int64_t cols = 0;
};

}  // namespace

struct bf_server {
    bf_server_options opt{};
    size_t elt = sizeof(float2);
    std::vector<Op> ops;
    std::vector<Slot> slots;
    int64_t factor_bytes = 0;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_id = 1;
    std::thread thr;
    bool started = false, stop = false;
    // statistics
    std::vector<double> lat;
    int64_t submitted = 0, completed = 0, launches = 0, batch_cols = 0;
    double units_done = 0;
    Clock::time_point t0 = Clock::now();
    // device intervals [start, end) of completed batches, ms after the base event
    cudaEvent_t base = nullptr;
    std::vector<std::pair<double, double>> spans;
    int nsm = 1;  // SMs of the device (grid of the interleave kernels)
};

namespace {

void reap(bf_server* s)
{
    for (auto& sl : s->slots) {
        if (!sl.busy) continue;
        cudaError_t e = cudaEventQuery(sl.ev);
        if (e == cudaErrorNotReady) continue;
        const auto now = Clock::now();
        if (e == cudaSuccess) {
            float a = 0.f, b = 0.f;
            if (s->spans.size() < kMaxSpans && cudaEventElapsedTime(&a, s->base, sl.ev0) == cudaSuccess &&
                cudaEventElapsedTime(&b, s->base, sl.ev) == cudaSuccess)
                s->spans.emplace_back((double)a, (double)b);
        }
        for (uint64_t id : sl.reqs) {
            auto it = s->reqs.find(id);
            if (it == s->reqs.end()) continue;
            Req& r = it->second;
            r.done = true;
            r.t_done = now;
            r.status = e == cudaSuccess ? BF_OK : BF_ERR_CUDA;
            if (e == cudaSuccess) {
                s->lat.push_back(ms_since(r.t_submit, now));
                s->completed += 1;
                s->units_done += (double)s->ops[(size_t)r.op].N * (double)r.m;
            }
        }
        sl.reqs.clear();
        sl.busy = false;
        s->cv_done.notify_all();
    }
}

// Enqueue one batch on a slot (called without the lock; the slot is owned).
bf_status enqueue_batch(bf_server* s, Slot& sl, Op& op, std::vector<Req*>& rs, bool idle_queue)
{
    const int64_t N = op.N, M = sl.cols;
    const size_t elt = s->elt;
    cudaError_t e = cudaEventRecord(sl.ev0, sl.st);
    if (e != cudaSuccess) return BF_ERR_CUDA;
    if (idle_queue && op.nufft && rs.size() == 1 && M >= kChunkMinCols && M % kChunks == 0 &&
        N * M >= kChunkMinUnits) {
        // one request in column chunks: every column is computed on its own, so the chunks
        // give the request's result exactly; the copies of one chunk overlap the kernels of
        // the other (strided host rows of M / kChunks elements).  Only with no other request
        // waiting: under a backlog the other slots' work overlaps the copies already, and
        // the NUFFT costs more per column at half the columns.
        const Req* r = rs[0];
        const int64_t mc = M / kChunks;
        const size_t w = (size_t)mc * elt, pitch = (size_t)M * elt, blk = (size_t)N * w;
        if ((e = cudaStreamWaitEvent(sl.up, sl.ev0, 0)) != cudaSuccess) return BF_ERR_CUDA;
        for (int k = 0; k < kChunks; ++k) {
            if ((e = cudaMemcpy2DAsync((unsigned char*)sl.F + k * blk, w, (const unsigned char*)r->F + k * w, pitch, w,
                                       (size_t)N, cudaMemcpyHostToDevice, sl.up)) != cudaSuccess ||
                (e = cudaEventRecord(sl.in_ready[k], sl.up)) != cudaSuccess)
                return BF_ERR_CUDA;
        }
        for (int k = 0; k < kChunks; ++k) {
            if ((e = cudaStreamWaitEvent(sl.st, sl.in_ready[k], 0)) != cudaSuccess) return BF_ERR_CUDA;
            const bf_status st = nufft_apply_ws(op.plan, (unsigned char*)sl.F + k * blk, mc,
                                                (unsigned char*)sl.G + k * blk, sl.st, sl.ws, sl.ws_bytes);
            if (st != BF_OK) return st;
            if ((e = cudaEventRecord(sl.done[k], sl.st)) != cudaSuccess) return BF_ERR_CUDA;
        }
        for (int k = 0; k < kChunks; ++k) {
            if ((e = cudaStreamWaitEvent(sl.down, sl.done[k], 0)) != cudaSuccess ||
                (e = cudaMemcpy2DAsync((unsigned char*)r->G + k * w, pitch, (unsigned char*)sl.G + k * blk, w, w,
                                       (size_t)N, cudaMemcpyDeviceToHost, sl.down)) != cudaSuccess)
                return BF_ERR_CUDA;
        }
        if ((e = cudaEventRecord(sl.joined, sl.down)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(sl.st, sl.joined, 0)) != cudaSuccess || (e = cudaEventRecord(sl.ev, sl.st)) != cudaSuccess)
            return BF_ERR_CUDA;
        return BF_OK;
    }
    // staged: each request's rows in one contiguous copy into sl.G (free until the apply
    // writes it), interleaved into sl.F; after the apply, G de-interleaved into sl.F (free
    // again) and copied out per request
    const bool staged = rs.size() > 1 && rs.size() <= (size_t)kMaxSegs && M <= kMaxCols;
    Segs sg{};
    int64_t c = 0;
    for (Req* r : rs) {
        if (staged) {
            sg.c0[sg.n++] = (int)c;
            e = cudaMemcpyAsync((unsigned char*)sl.G + (size_t)c * N * elt, r->F, (size_t)N * r->m * elt,
                                cudaMemcpyHostToDevice, sl.st);
        } else {
            e = cudaMemcpy2DAsync((unsigned char*)sl.F + c * elt, (size_t)M * elt, r->F, (size_t)r->m * elt,
                                  (size_t)r->m * elt, (size_t)N, cudaMemcpyHostToDevice, sl.st);
        }
        if (e != cudaSuccess) return BF_ERR_CUDA;
        c += r->m;
    }
    sg.c0[sg.n] = (int)c;
    if (staged && launch_interleave(true, elt, sl.G, sl.F, N, (int)M, sg, s->nsm, sl.st) != cudaSuccess)
        return BF_ERR_CUDA;
    bf_status st = op.nufft ? nufft_apply_ws(op.plan, sl.F, M, sl.G, sl.st, sl.ws, sl.ws_bytes)
                            : device_apply_ws(op.plan, (bf_precision)s->opt.precision, sl.F, M, sl.G, sl.st, sl.ws,
                                              sl.ws_bytes);
    if (st != BF_OK) return st;
    if (staged && launch_interleave(false, elt, sl.G, sl.F, N, (int)M, sg, s->nsm, sl.st) != cudaSuccess)
        return BF_ERR_CUDA;
    c = 0;
    for (Req* r : rs) {
        if (staged)
            e = cudaMemcpyAsync(r->G, (unsigned char*)sl.F + (size_t)c * N * elt, (size_t)N * r->m * elt,
                                cudaMemcpyDeviceToHost, sl.st);
        else
            e = cudaMemcpy2DAsync(r->G, (size_t)r->m * elt, (unsigned char*)sl.G + c * elt, (size_t)M * elt,
                                  (size_t)r->m * elt, (size_t)N, cudaMemcpyDeviceToHost, sl.st);
        if (e != cudaSuccess) return BF_ERR_CUDA;
        c += r->m;
    }
    e = cudaEventRecord(sl.ev, sl.st);
    return e == cudaSuccess ? BF_OK : BF_ERR_CUDA;
}

void scheduler(bf_server* s)
{
    cudaSetDevice(s->opt.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        reap(s);
        bool launched = false;
        for (auto& sl : s->slots) {
            if (sl.busy) continue;
            // operator of the oldest pending request (a priority slot: of the oldest small one)
            const int64_t small = s->opt.small_units > 0 ? s->opt.small_units : ((int64_t)1 << 21);
            int best = -1;
            Clock::time_point bt{};
            for (size_t i = 0; i < s->ops.size(); ++i) {
                auto& q = s->ops[i].pending;
                if (q.empty()) continue;
                const Req& fr = s->reqs[q.front()];
                if (sl.hi && s->ops[i].N * fr.m > small) continue;
                if (best < 0 || fr.t_submit < bt) {
                    best = (int)i;
                    bt = fr.t_submit;
                }
            }
            if (best < 0) continue;
            Op& op = s->ops[(size_t)best];
            const int64_t cap = sl.hi ? std::max<int64_t>(1, std::min(op.cap, small / op.N)) : op.cap;
            std::vector<Req*> rs;
            int64_t cols = 0;
            while (!op.pending.empty()) {
                Req& r = s->reqs[op.pending.front()];
                if (cols + r.m > cap && !rs.empty()) break;
                if (cols + r.m > op.cap) break;
                cols += r.m;
                sl.reqs.push_back(op.pending.front());
                rs.push_back(&r);
                op.pending.pop_front();
                if (s->opt.per_request) break;
            }
            if (rs.empty()) break;
            sl.busy = true;
            sl.op = best;
            sl.cols = cols;
            s->launches += 1;
            s->batch_cols += cols;
            bool idle_queue = true;
            for (const Op& o : s->ops) idle_queue = idle_queue && o.pending.empty();
            lk.unlock();  // Req objects stay put: only this thread erases them after completion
            bf_status st = enqueue_batch(s, sl, op, rs, idle_queue);
            lk.lock();
            if (st != BF_OK) {
                const auto now = Clock::now();
                for (uint64_t id : sl.reqs) {
                    auto it = s->reqs.find(id);
                    if (it != s->reqs.end()) {
                        it->second.done = true;
                        it->second.t_done = now;
                        it->second.status = st;
                    }
                }
                cudaStreamSynchronize(sl.up);
                cudaStreamSynchronize(sl.st);
                cudaStreamSynchronize(sl.down);
                sl.reqs.clear();
                sl.busy = false;
                s->cv_done.notify_all();
            }
            launched = true;
        }
        bool any_busy = false;
        for (auto& sl : s->slots) any_busy = any_busy || sl.busy;
        if (s->stop && !any_busy) break;
        if (!launched) s->cv_sched.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 2000));
    }
}

size_t op_ws_bytes(const bf_server* s, const Op& op, int64_t m)
{
    return op.nufft ? nufft_ws_bytes(op.plan, m) : device_ws_bytes(op.plan, (bf_precision)s->opt.precision, m);
}

int64_t per_col_bytes(const bf_server* s, const Op& op, int64_t m)
{
    return (int64_t)(2 * (size_t)op.N * (size_t)m * s->elt + op_ws_bytes(s, op, m));
}

}  // namespace

extern "C" {

bf_status bf_server_default_options(bf_server_options* o)
{
    if (!o) {
        set_error("bf_server_default_options: NULL");
        return BF_ERR_ARG;
    }
    std::memset(o, 0, sizeof(*o));
    o->n_slots = 4;
    o->hbm_budget = 0;
    o->max_batch_rhs = 256;
    o->precision = BF_PREC_F32;
    o->per_request = 0;
    o->device = 0;
    o->n_priority_slots = -1;  // n_slots / 2
    o->small_units = 0;        // 2^21
    o->method = 0;             // the butterfly apply for every operator
    o->nufft_eps = 1e-6;
    return BF_OK;
}

bf_status bf_server_create(const bf_server_options* opt, bf_server** out)
{
    if (!out) {
        set_error("bf_server_create: NULL output");
        return BF_ERR_ARG;
    }
    *out = nullptr;
    bf_server* s = new (std::nothrow) bf_server();
    if (!s) {
        set_error("bf_server_create: out of host memory");
        return BF_ERR_NOMEM;
    }
    if (opt) s->opt = *opt; else bf_server_default_options(&s->opt);
    if (s->opt.n_slots < 1) s->opt.n_slots = 1;
    if (s->opt.max_batch_rhs < 1) s->opt.max_batch_rhs = 256;
    if (s->opt.precision != BF_PREC_F32 && s->opt.precision != BF_PREC_F64) {
        delete s;
        set_error("bf_server_create: precision must be BF_PREC_F32 or BF_PREC_F64");
        return BF_ERR_ARG;
    }
    s->elt = s->opt.precision == BF_PREC_F64 ? sizeof(double2) : sizeof(float2);
    if (cudaSetDevice(s->opt.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->opt.device) != cudaSuccess) {
        delete s;
        set_error("bf_server_create: cannot use device %d", s->opt.device);
        return BF_ERR_CUDA;
    }
    if (s->opt.hbm_budget <= 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete s;
            set_error("bf_server_create: cudaMemGetInfo failed");
            return BF_ERR_CUDA;
        }
        s->opt.hbm_budget = (int64_t)(0.6 * (double)fr);
    }
    *out = s;
    return BF_OK;
}

bf_status bf_server_add_operator(bf_server* s, bf_plan* plan, int* op_id)
{
    if (!s || !plan) {
        set_error("bf_server_add_operator: NULL argument");
        return BF_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->started) {
        set_error("bf_server_add_operator: add operators before bf_server_start");
        return BF_ERR_STATE;
    }
    if (!plan->factored) {
        set_error("bf_server_add_operator: plan not factored");
        return BF_ERR_STATE;
    }
    if (plan->otf) {
        set_error("bf_server_add_operator: plans factored by bf_factor_otf are not served");
        return BF_ERR_UNSUPPORTED;
    }
    if (plan->opt.device != s->opt.device) {
        set_error("bf_server_add_operator: plan is on device %d, server on %d", plan->opt.device, s->opt.device);
        return BF_ERR_ARG;
    }
    bf_plan_info info;
    const bool was_up = plan->dev != nullptr;
    if (!was_up) {
        // admission: estimate the device factor bytes from the host factors (both arenas)
        int64_t est = 0;
        for (auto& B : plan->blocks) est += (int64_t)(B.host_bytes() * 3 / 2);
        if (s->factor_bytes + est > s->opt.hbm_budget) {
            set_error("bf_server_add_operator: factors (%lld bytes) exceed the remaining HBM budget (%lld)",
                      (long long)est, (long long)(s->opt.hbm_budget - s->factor_bytes));
            return BF_ERR_NOMEM;
        }
    }
    bf_status st = bf_upload(plan);
    if (st != BF_OK) return st;
    bf_plan_get_info(plan, &info);
    s->factor_bytes += info.dev_bytes_f32 + info.dev_bytes_f64;
    if (s->factor_bytes > s->opt.hbm_budget) {
        s->factor_bytes -= info.dev_bytes_f32 + info.dev_bytes_f64;
        set_error("bf_server_add_operator: factors exceed the HBM budget");
        return BF_ERR_NOMEM;
    }
    Op op;
    op.plan = plan;
    op.N = plan->N;
    if (s->opt.method == 1 && s->opt.precision == BF_PREC_F32 && !s->opt.per_request) {
        // Sec. 3's choice: the NUFFT of Eq. tg3 where the phase is rank 1 on the column halves
        // (bf_nufft_prepare accepts it), the butterfly otherwise
        if (plan->nufft || bf_nufft_prepare(plan, s->opt.nufft_eps > 0 ? s->opt.nufft_eps : 1e-6, nullptr) == BF_OK)
            op.nufft = true;
    }
    s->ops.push_back(op);
    if (op_id) *op_id = (int)s->ops.size() - 1;
    return BF_OK;
}

bf_status bf_server_start(bf_server* s)
{
    if (!s) {
        set_error("bf_server_start: NULL server");
        return BF_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->started) return BF_OK;
    if (s->ops.empty()) {
        set_error("bf_server_start: no operators");
        return BF_ERR_STATE;
    }
    if (cudaSetDevice(s->opt.device) != cudaSuccess) {
        set_error("bf_server_start: cudaSetDevice failed");
        return BF_ERR_CUDA;
    }
    const int64_t per_slot = (s->opt.hbm_budget - s->factor_bytes) / s->opt.n_slots;
    size_t slab = 0, ws = 0;
    for (auto& op : s->ops) {
        int64_t m = s->opt.max_batch_rhs;
        while (m > 1 && per_col_bytes(s, op, m) > per_slot) m = m * 3 / 4;
        if (per_col_bytes(s, op, m) > per_slot) {
            set_error("bf_server_start: one right-hand side of N=%lld does not fit a slot (%lld bytes)",
                      (long long)op.N, (long long)per_slot);
            return BF_ERR_NOMEM;
        }
        op.cap = m;
        slab = std::max(slab, (size_t)op.N * (size_t)m * s->elt);
        ws = std::max(ws, op_ws_bytes(s, op, m));
    }
    s->slots.resize((size_t)s->opt.n_slots);
    int pri_lo = 0, pri_hi = 0;
    cudaDeviceGetStreamPriorityRange(&pri_lo, &pri_hi);
    const int nhi = s->opt.n_priority_slots < 0 ? s->opt.n_slots / 2 : std::min(s->opt.n_priority_slots, s->opt.n_slots);
    for (size_t i = 0; i < s->slots.size(); ++i) {
        Slot& sl = s->slots[i];
        sl.hi = (int)i < nhi;
        cudaError_t e;
        if ((e = cudaStreamCreateWithPriority(&sl.st, cudaStreamNonBlocking, sl.hi ? pri_hi : pri_lo)) != cudaSuccess ||
            (e = cudaStreamCreateWithPriority(&sl.up, cudaStreamNonBlocking, sl.hi ? pri_hi : pri_lo)) != cudaSuccess ||
            (e = cudaStreamCreateWithPriority(&sl.down, cudaStreamNonBlocking, sl.hi ? pri_hi : pri_lo)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&sl.joined, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreate(&sl.ev)) != cudaSuccess || (e = cudaEventCreate(&sl.ev0)) != cudaSuccess ||
            (e = cudaMalloc(&sl.F, slab)) != cudaSuccess || (e = cudaMalloc(&sl.G, slab)) != cudaSuccess ||
            (e = cudaMalloc(&sl.ws, ws)) != cudaSuccess) {
            set_error("bf_server_start: slot allocation: %s", cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA;
        }
        for (int k = 0; k < kChunks; ++k)
            if ((e = cudaEventCreateWithFlags(&sl.in_ready[k], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&sl.done[k], cudaEventDisableTiming)) != cudaSuccess) {
                set_error("bf_server_start: slot events: %s", cudaGetErrorString(e));
                return BF_ERR_CUDA;
            }
        sl.ws_bytes = ws;
    }
    if (cudaEventCreate(&s->base) != cudaSuccess || cudaEventRecord(s->base, s->slots[0].st) != cudaSuccess ||
        cudaEventSynchronize(s->base) != cudaSuccess) {
        set_error("bf_server_start: base event");
        return BF_ERR_CUDA;
    }
    s->t0 = Clock::now();
    s->started = true;
    s->thr = std::thread(scheduler, s);
    return BF_OK;
}

bf_status bf_server_submit(bf_server* s, int op_id, const void* F, int64_t m, void* G, uint64_t* req_id)
{
    if (!s || !F || !G || m < 1) {
        set_error("bf_server_submit: NULL argument or m < 1");
        return BF_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->started || s->stop) {
        set_error("bf_server_submit: server not running");
        return BF_ERR_STATE;
    }
    if (op_id < 0 || op_id >= (int)s->ops.size()) {
        set_error("bf_server_submit: unknown operator %d", op_id);
        return BF_ERR_ARG;
    }
    Op& op = s->ops[(size_t)op_id];
    if (m > op.cap) {
        set_error("bf_server_submit: m=%lld exceeds the batch width %lld of operator %d", (long long)m,
                  (long long)op.cap, op_id);
        return BF_ERR_ARG;
    }
    const uint64_t id = s->next_id++;
    Req r;
    r.op = op_id;
    r.F = F;
    r.G = G;
    r.m = m;
    r.t_submit = Clock::now();
    s->reqs.emplace(id, r);
    op.pending.push_back(id);
    s->submitted += 1;
    if (req_id) *req_id = id;
    s->cv_sched.notify_one();
    return BF_OK;
}

bf_status bf_server_wait(bf_server* s, uint64_t id, double timeout_ms, double* latency_ms)
{
    if (!s) {
        set_error("bf_server_wait: NULL server");
        return BF_ERR_ARG;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        set_error("bf_server_wait: unknown request %llu", (unsigned long long)id);
        return BF_ERR_ARG;
    }
    auto pred = [&] { return s->reqs[id].done; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, pred);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred)) {
        set_error("bf_server_wait: request %llu not done after %.1f ms", (unsigned long long)id, timeout_ms);
        return BF_ERR_TIMEOUT;
    }
    Req r = s->reqs[id];
    s->reqs.erase(id);
    if (latency_ms) *latency_ms = ms_since(r.t_submit, r.t_done);
    if (r.status != BF_OK) set_error("bf_server_wait: request %llu failed", (unsigned long long)id);
    return r.status;
}

bf_status bf_server_drain(bf_server* s, double timeout_ms)
{
    if (!s) {
        set_error("bf_server_drain: NULL server");
        return BF_ERR_ARG;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto pred = [&] {
        for (auto& kv : s->reqs)
            if (!kv.second.done) return false;
        return true;
    };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, pred);
        return BF_OK;
    }
    if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred)) {
        set_error("bf_server_drain: requests still pending after %.1f ms", timeout_ms);
        return BF_ERR_TIMEOUT;
    }
    return BF_OK;
}

bf_status bf_server_get_stats(bf_server* s, bf_server_stats* out)
{
    if (!s || !out) {
        set_error("bf_server_get_stats: NULL argument");
        return BF_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    int64_t pend = 0, fl = 0;
    for (auto& op : s->ops) pend += (int64_t)op.pending.size();
    for (auto& sl : s->slots) fl += (int64_t)sl.reqs.size();
    out->pending = pend;
    out->in_flight = fl;
    out->launches = s->launches;
    out->mean_batch_rhs = s->launches ? (double)s->batch_cols / (double)s->launches : 0.0;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto q = [&](double p) { return v[(size_t)std::min((double)v.size() - 1, p * (double)(v.size() - 1) + 0.5)]; };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / (double)v.size();
        out->max_ms = v.back();
    }
    out->wall_s = ms_since(s->t0, Clock::now()) / 1e3;
    out->units_per_s = out->wall_s > 0 ? s->units_done / out->wall_s : 0.0;
    // device time of the completed batches: covered by at least one slot, and by two or more
    std::vector<std::pair<double, int>> ev;
    for (auto& sp : s->spans) {
        ev.emplace_back(sp.first, +1);
        ev.emplace_back(sp.second, -1);
    }
    std::sort(ev.begin(), ev.end());
    int depth = 0;
    double prev = 0;
    for (auto& e : ev) {
        if (depth >= 1) out->device_busy_ms += e.first - prev;
        if (depth >= 2) out->overlap_ms += e.first - prev;
        depth += e.second;
        prev = e.first;
    }
    int64_t nn = 0;
    for (auto& op : s->ops) nn += op.nufft ? 1 : 0;
    out->nufft_operators = nn;
    return BF_OK;
}

bf_status bf_server_reset_stats(bf_server* s)
{
    if (!s) {
        set_error("bf_server_reset_stats: NULL server");
        return BF_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat.clear();
    s->completed = 0;
    s->submitted = 0;
    s->launches = 0;
    s->batch_cols = 0;
    s->units_done = 0;
    s->spans.clear();
    s->t0 = Clock::now();
    return BF_OK;
}

void bf_server_destroy(bf_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // pending (not yet launched) requests are dropped
        for (auto& op : s->ops) op.pending.clear();
        s->cv_sched.notify_all();
    }
    if (s->thr.joinable()) s->thr.join();
    cudaSetDevice(s->opt.device);
    for (auto& sl : s->slots) {
        if (sl.up) cudaStreamSynchronize(sl.up);
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.down) cudaStreamSynchronize(sl.down);
        cudaFree(sl.F);
        cudaFree(sl.G);
        cudaFree(sl.ws);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.ev0) cudaEventDestroy(sl.ev0);
        for (int k = 0; k < kChunks; ++k) {
            if (sl.in_ready[k]) cudaEventDestroy(sl.in_ready[k]);
            if (sl.done[k]) cudaEventDestroy(sl.done[k]);
        }
        if (sl.joined) cudaEventDestroy(sl.joined);
        if (sl.up) cudaStreamDestroy(sl.up);
        if (sl.down) cudaStreamDestroy(sl.down);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    if (s->base) cudaEventDestroy(s->base);
    delete s;
}

}  // extern "C"
