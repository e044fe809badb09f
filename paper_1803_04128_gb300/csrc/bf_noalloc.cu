// Allocation-free variant of the fused FP32 apply.
//
// Some callers cannot allocate device memory at apply time: code that runs
// under a fixed device-memory budget owned by someone else (an inference
// server or a host application that hands out all GPU memory from its own
// pool), code that must not call into the CUDA allocator on its latency path
// (cudaMalloc can synchronise the device and take milliseconds), and plugins
// whose rules forbid allocating outside their set-up phase.  bf_apply needs a
// workspace for the switch-level coefficients and grows it with cudaMalloc;
// bf_apply_f32_noalloc instead uses one fixed scratch array compiled into the
// library, so it never allocates.
//
// The scratch is a file-scope __device__ array of kNoallocScratchBytes
// (32 MiB).  Every GPU that loads this library holds it until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; make that first call before any
// stream capture.  The cache is not refreshed: a cudaDeviceReset, which
// re-creates the primary context and reloads the module, leaves the cached
// address stale, so this entry point is not for processes that reset devices.  All calls share the array and it keeps the last call's
// contents: the front kernel writes every element the back kernel reads, so
// nothing needs clearing, but calls that overlap on the GPU (different
// streams, or different plans on one device) race on it.
#include <mutex>

#include "bf_device.h"

namespace bfi {
namespace {

constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 256;
void* g_addr[kMaxDevices] = {};

}  // namespace
}  // namespace bfi

using namespace bfi;

extern "C" bf_status bf_apply_f32_noalloc(bf_plan* p, const void* F, int64_t m, void* G, void* stream)
{
    if (!p || !F || !G || m < 1) {
        set_error("bf_apply_f32_noalloc: NULL plan/buffer or m < 1");
        return BF_ERR_ARG;
    }
    if (F == G) {
        set_error("bf_apply_f32_noalloc: G must not alias F");
        return BF_ERR_ARG;
    }
    if (!p->dev) {
        set_error("bf_apply_f32_noalloc: plan not uploaded (call bf_upload first; this entry point allocates nothing)");
        return BF_ERR_STATE;
    }
    if (prof_active()) {
        set_error("bf_apply_f32_noalloc: not available while bf_profile timing is on (it creates events)");
        return BF_ERR_STATE;
    }
    DeviceState* ds = p->dev;
    for (auto& B : ds->blocks) {
        if (!fused_f32_supported(B.g.r) || B.g.nv > 2 * B.g.r) {
            set_error("bf_apply_f32_noalloc: no fused FP32 kernels for r=%d", B.g.r);
            return BF_ERR_UNSUPPORTED;
        }
        const size_t need = fused_f32_ws_bytes(B.g, m);
        if (need > kNoallocScratchBytes) {
            set_error("bf_apply_f32_noalloc: N=%lld, m=%lld needs %zu bytes of scratch, more than the fixed %zu "
                      "(use bf_apply, or fewer right-hand sides per call)",
                      (long long)B.g.N, (long long)m, need, kNoallocScratchBytes);
            return BF_ERR_ARG;
        }
    }
    if (ds->device < 0 || ds->device >= kMaxDevices) {
        set_error("bf_apply_f32_noalloc: device ordinal %d out of range", ds->device);
        return BF_ERR_ARG;
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        set_error("bf_apply_f32_noalloc: cudaGetDevice failed");
        return BF_ERR_CUDA;
    }
    if (cur != ds->device && cudaSetDevice(ds->device) != cudaSuccess) {
        set_error("bf_apply_f32_noalloc: cudaSetDevice(%d) failed", ds->device);
        return BF_ERR_CUDA;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[ds->device]) {
            void* a = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
            if (e != cudaSuccess || !a) {
                set_error("bf_apply_f32_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                if (cur != ds->device) cudaSetDevice(cur);
                return BF_ERR_CUDA;
            }
            g_addr[ds->device] = a;
        }
        scratch = g_addr[ds->device];
    }
    bf_status st = BF_OK;
    const int sp = p->opt.split;
    for (size_t i = 0; i < ds->blocks.size(); ++i) {
        const DevBlock& B = ds->blocks[i];
        const int beta = (sp == 2 && (i % 2) == 1) ? 1 : 0;
        const float2* Fb = (const float2*)F + B.col0 * m;
        float2* Gb = (float2*)G + B.row0 * m;
        cudaError_t e = launch_fused_f32(B, Fb, m, Gb, beta, (float2*)scratch, (cudaStream_t)stream);
        if (e != cudaSuccess) {
            set_error("bf_apply_f32_noalloc: kernel launch failed: %s", cudaGetErrorString(e));
            st = BF_ERR_CUDA;
            break;
        }
    }
    if (cur != ds->device) cudaSetDevice(cur);
    return st;
}
