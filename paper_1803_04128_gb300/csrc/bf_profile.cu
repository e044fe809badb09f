// Per-kernel CUDA-event timing of the library's own launches (measurement aid).
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bf_device.h"

namespace bfi {
namespace {
struct Rec {
    const char* name;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<std::pair<std::string, std::pair<int64_t, double>>> g_agg;
thread_local bool t_suppress = false;
}  // namespace

void prof_suppress(bool on) { t_suppress = on; }

void prof_start(const char* name, cudaStream_t st, void** tok)
{
    *tok = nullptr;
    if (t_suppress) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    Rec r{name, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
    cudaEventRecord(r.a, st);
    g_recs.push_back(r);
    *tok = (void*)(intptr_t)g_recs.size();
}

bool prof_active()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_on;
}

void prof_stop(void* tok, cudaStream_t st)
{
    if (!tok) return;
    std::lock_guard<std::mutex> lk(g_mu);
    size_t i = (size_t)(intptr_t)tok - 1;
    if (i < g_recs.size()) cudaEventRecord(g_recs[i].b, st);
}

// Register-only FP32 FMA loop: 8 independent chains per thread, so every
// scheduler always has an FMA ready.  The multipliers are close to 1 and the
// addends small, so the values stay normal and finite; the result is stored
// only when it is impossible (never), which keeps the loop alive.
constexpr int kPeakIters = 2048;
__global__ void __launch_bounds__(256) ffma_peak_kernel(float* sink, float seed)
{
    float a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = seed + 1e-3f * (float)(threadIdx.x + c);
    const float b = 0.9999999f, d = 1e-7f;
    for (int i = 0; i < kPeakIters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = fmaf(a[c], b, d);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == -1.0f) sink[blockIdx.x] = s;
}

// The same loop in FP64 (DFMA).
__global__ void __launch_bounds__(256) dfma_peak_kernel(double* sink, double seed, int iters)
{
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = seed + 1e-3 * (double)(threadIdx.x + c);
    const double b = 0.9999999999, d = 1e-10;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = fma(a[c], b, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace bfi

using namespace bfi;

extern "C" {

bf_status bf_fp64_peak(int device, double* tflops)
{
    if (!tflops) {
        set_error("bf_fp64_peak: NULL output");
        return BF_ERR_ARG;
    }
    int cur = -1, sms = 0, per_sm = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        set_error("bf_fp64_peak: cannot select device %d", device);
        return BF_ERR_CUDA;
    }
    bf_status st = BF_OK;
    double* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    double best = 0.0;
    const int iters = 256;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess ||
        cudaMalloc(&sink, sizeof(double) * 65536) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("bf_fp64_peak: CUDA set-up failed");
        st = BF_ERR_CUDA;
    } else {
        const int blocks = sms * (per_sm / 256);
        const double flops = (double)blocks * 256 * iters * 8 * 2;
        for (int rep = 0; rep < 6 && st == BF_OK; ++rep) {
            cudaEventRecord(e0, s);
            dfma_peak_kernel<<<blocks, 256, 0, s>>>(sink, 1.0 + 1e-3 * rep, iters);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                set_error("bf_fp64_peak: kernel or timing failed");
                st = BF_ERR_CUDA;
            } else if (rep > 0 && ms > 0.f) {
                best = std::max(best, flops / (ms * 1e-3) / 1e12);
            }
        }
    }
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    cudaSetDevice(cur);
    *tflops = best;
    return st;
}

bf_status bf_fp32_peak(int device, int* sm_count, double* tflops)
{
    if (!sm_count || !tflops) {
        set_error("bf_fp32_peak: NULL output");
        return BF_ERR_ARG;
    }
    int cur = -1, sms = 0, per_sm = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        set_error("bf_fp32_peak: cannot select device %d", device);
        return BF_ERR_CUDA;
    }
    bf_status st = BF_OK;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    double best = 0.0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess ||
        cudaMalloc(&sink, sizeof(float) * 65536) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("bf_fp32_peak: CUDA set-up failed");
        st = BF_ERR_CUDA;
    } else {
        const int blocks = sms * (per_sm / 256);
        const double flops = (double)blocks * 256 * kPeakIters * 8 * 2;
        for (int rep = 0; rep < 6 && st == BF_OK; ++rep) {
            cudaEventRecord(e0, s);
            ffma_peak_kernel<<<blocks, 256, 0, s>>>(sink, 1.0f + 1e-3f * rep);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                set_error("bf_fp32_peak: kernel or timing failed");
                st = BF_ERR_CUDA;
            } else if (rep > 0 && ms > 0.f) {   // the first launch is a warm-up
                best = std::max(best, flops / (ms * 1e-3) / 1e12);
            }
        }
    }
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    cudaSetDevice(cur);
    *sm_count = sms;
    *tflops = best;
    return st;
}

bf_status bf_profile_begin(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = true;
    return BF_OK;
}

bf_status bf_profile_end(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = false;
    std::map<std::string, std::pair<int64_t, double>> agg;
    bf_status st = BF_OK;
    for (auto& r : g_recs) {
        float ms = 0;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            set_error("bf_profile_end: event timing failed");
            st = BF_ERR_CUDA;
        }
        auto& e = agg[r.name];
        e.first += 1;
        e.second += ms;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
    g_agg.assign(agg.begin(), agg.end());
    return st;
}

int bf_profile_count(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return (int)g_agg.size();
}

bf_status bf_profile_get(int i, const char** name, int64_t* launches, double* total_ms)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (i < 0 || i >= (int)g_agg.size() || !name || !launches || !total_ms) {
        set_error("bf_profile_get: bad index or NULL output");
        return BF_ERR_ARG;
    }
    *name = g_agg[(size_t)i].first.c_str();
    *launches = g_agg[(size_t)i].second.first;
    *total_ms = g_agg[(size_t)i].second.second;
    return BF_OK;
}

}  // extern "C"
