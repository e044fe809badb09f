// Per-kernel CUDA-event timing of the library's own launches (measurement aid).
#include <cuda_runtime.h>

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

}  // namespace bfi

using namespace bfi;

extern "C" {

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
