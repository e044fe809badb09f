// Device-side layouts of the IBF-MAT factors and the launch interfaces.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "bf_internal.h"

namespace bfi {

// Geometry of one sub-BF, as the kernels see it.
struct Geo {
    int64_t N;   // block size
    int64_t P;   // pairs per level = N / n0 = 2^L
    int r, n0, L, h, l1, nv;  // nv = n0 * 2^l1 (V and U leaf size)
    int kH, kG;               // number of H and G levels
    int ra;                   // amplitude rank
    int otf = 0;              // 1: no phase tables, the kernels evaluate the phases (OtfPhase)
};

// Phases evaluated inside the apply kernels (bf_factor_otf).  Every entry of
// the phase tables is e^{2 pi i (sum of +-Phi at grid points)} (Sec. 4, Eqs. 1,
// 2, 3, bf3 and the switch step of Algorithm 4.1), and for the built-in kinds
// Phi(x_i, xi_j) mod 1 at global grid indices (i, j), xi = j - Ng/2, is
//   xxi * (i xi mod Ng) / Ng + kappa_i |xi| + rho_i + sq * (xi^2 mod 4 Ng) / (4 Ng).
// The kernels hold it as an unsigned 32-bit count of 2^-32 turns, so sums and
// differences of phases wrap mod 1 exactly: the integer residues are exact,
// kappa_i |xi| is a 64-bit fixed-point product (K_i = frac(kappa_i) 2^64).
struct OtfPhase {
    const uint4* rows = nullptr;  // [Ng] per global row i: (K_i low word, K_i high word, round(frac(rho_i) 2^32), 0)
    const int* grids = nullptr;   // [lN + 1][16]: interpolation indices of a node of 2^e points (grid_rel)
    int row0 = 0, col0 = 0;       // block origin in global indices (Ng <= 2^30)
    int half = 0;                 // Ng / 2
    int lN = 0;                   // log2 of the block size
    int sh1 = -1;                 // 32 - log2 Ng if the x xi term is present, else -1
    int sh2 = -1;                 // 30 - log2 Ng if the xi^2 term is present, else -1
};

// Factor arrays of one sub-BF in one precision; T = float or double, C = float2/double2.
// Layouts (all row-major):
//   a, b  [ra][N]          Mv [r][nv]            EV [2^l1][N]
//   MH    [kH][r][2r]      EH [kH][P][2][r]      S  [P][r][r]
//   MG    [kG][2][r][r]    FG [kG][P][2][r]      MU [nv][r]      EU [2^l1][N]
// where a pair index at level l is q = a * 2^(L-l) + b (A = node a of T_X at
// level l, B = node b of T_Omega at level L-l).
template <typename T, typename C>
struct DevFactors {
    C *a = nullptr, *b = nullptr;
    T* Mv = nullptr;
    C* EV = nullptr;
    T* MH = nullptr;
    C* EH = nullptr;
    C* S = nullptr;
    T* MG = nullptr;
    C* FG = nullptr;
    T* MU = nullptr;
    C* EU = nullptr;
};

struct DevBlock {
    Geo g{};
    int64_t row0 = 0, col0 = 0;
    OtfPhase ph;  // g.otf = 1 only
    DevFactors<double, double2> f64;
    DevFactors<float, float2> f32;
};

struct DeviceState {
    int device = 0;
    std::vector<DevBlock> blocks;
    void* arena64 = nullptr;
    void* arena32 = nullptr;
    size_t bytes64 = 0, bytes32 = 0;
    // workspaces
    void* ws64 = nullptr;
    size_t ws64_bytes = 0;
    void* ws32 = nullptr;
    size_t ws32_bytes = 0;
    void* stage = nullptr;  // F/G staging for bf_apply_host
    size_t stage_bytes = 0;
    // bf_apply_host's copy stream, second compute stream and events (row ranges copied
    // while others compute)
    cudaStream_t copy = nullptr, comp2 = nullptr;
    static constexpr int kHostChunks = 4;
    cudaEvent_t hev[2 * kHostChunks + 6] = {};
    int* err = nullptr;     // device error word (0 = ok)
    bool otf = false;       // factored by bf_factor_otf: no phase tables, FP32 apply only
    void* otf_data = nullptr;  // OtfPhase rows and grids
    // the plain FP64 apply (one launch per stage) replayed from a CUDA graph
    // captured for the last (F, G, m, workspace)
    cudaStream_t cap = nullptr;
    cudaGraphExec_t g64 = nullptr;
    const void* g64_F = nullptr;
    void* g64_G = nullptr;
    int64_t g64_m = 0;
    void* g64_ws = nullptr;
};

// ---- construction of the phase tables on the device (bf_construct.cu) ----
cudaError_t construct_tables(const BlockFactors& B, int phase_kind, double phase_param, int64_t n_global,
                             const DevFactors<double, double2>& f64, const DevFactors<float, float2>& f32,
                             cudaStream_t st);

// ---- launchers (return cudaGetLastError() of the last launch) ----
// Plain FP64 form: one kernel per butterfly stage, state through global memory.
cudaError_t launch_plain_f64(const DevBlock& B, const double2* F, int64_t m, double2* G, int beta,
                             double2* ws0, double2* ws1, cudaStream_t st);
size_t plain_f64_ws_bytes(const Geo& g, int64_t m);  // bytes of ONE of the two state buffers

// Fused FP32 form: front pass (V + H levels + switch) and back pass (G levels + U).
struct FusedCfg {
    int mr;       // right-hand sides per column slice
    int nslice;   // ceil(m / mr)
    int tpc_f;    // front tiles per CTA
    int tpc_b;    // T_Omega chunks a back CTA processes together
    int kpass;    // most levels per pass (the largest pass of the H and G ranges)
};
inline int tune_word(int mr, int kpass, int tpc_f_log1, int tpc_b_log1)
{
    return (mr & 0xFF) | ((kpass & 0xF) << 8) | ((tpc_f_log1 & 0xF) << 12) | ((tpc_b_log1 & 0xF) << 16);
}
inline int tune_mr(int w) { return w & 0xFF; }
inline int tune_kpass(int w) { return (w >> 8) & 0xF; }
inline int tune_tpc_f(int w) { return ((w >> 12) & 0xF) ? 1 << (((w >> 12) & 0xF) - 1) : 0; }
inline int tune_tpc_b(int w) { return ((w >> 16) & 0xF) ? 1 << (((w >> 16) & 0xF) - 1) : 0; }
// mr_hint: the autotuner's tuning word (0 = built-in rules everywhere):
//   bits 0..7   mr, right-hand sides per column slice (a power of two)
//   bits 8..11  most levels per pass of the plain apply's split level ranges
//   bits 12..15 front tiles per CTA, as log2 + 1
//   bits 16..19 T_Omega chunks a back CTA processes together, as log2 + 1
// A field outside what fits (shared memory, tile counts) falls back to the built-in rule.
// Every choice gives the same tiles' arithmetic per column: results are bitwise equal.
// split: the plain apply's level passes (long H or G ranges in several passes); false: one pass per
// side, as the batched and sharded applies run them
FusedCfg fused_f32_config(const Geo& g, int64_t m, int mr_hint = 0, bool split = true);
size_t fused_f32_ws_bytes(const Geo& g, int64_t m, int mr_hint = 0, bool split = true);
// The same apply in nch row ranges (a power of two), for copies that overlap the kernels:
// front launch k waits for fready[k] (F rows [k N/nch, (k+1) N/nch) on the device); gdone[k]
// is recorded after back launch k (G rows [k N/nch, (k+1) N/nch) final).  Range k runs on
// st (k even) or st2 (k odd); join[0..3] order st2 after st's earlier work, the backs
// after all fronts, and st after everything.  Only plans that run one front and one back
// pass and split evenly (fused_f32_chunkable).
bool fused_f32_chunkable(const DevBlock& B, int64_t m, int mr_hint, int nch);
cudaError_t launch_fused_f32_chunked(const DevBlock& B, const float2* F, int64_t m, float2* G, float2* ws,
                                     cudaStream_t st, cudaStream_t st2, int mr_hint, int nch, const cudaEvent_t* fready,
                                     const cudaEvent_t* gdone, const cudaEvent_t* join);
cudaError_t launch_fused_f32(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta,
                             float2* ws, cudaStream_t st, int mr_hint = 0);
bool fused_f32_supported(int r);

// Split-BF16 tensor-core apply (bf_kernels_tc.cu)
bool tc_supported(const Geo& g, const char** why);
size_t tc_ws_bytes(const Geo& g, int64_t m);
cudaError_t launch_tc(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws, int* err,
                      cudaStream_t st);

// per-launch event timing (bf_profile_*); no-ops unless profiling is on
void prof_start(const char* name, cudaStream_t st, void** tok);
void prof_stop(void* tok, cudaStream_t st);
bool prof_active();
// no timing records from this thread while on (launches being captured into a graph)
void prof_suppress(bool on);
struct ProfScope {
    void* tok;
    cudaStream_t st;
    ProfScope(const char* name, cudaStream_t s) : st(s) { prof_start(name, s, &tok); }
    ~ProfScope() { prof_stop(tok, st); }
};

}  // namespace bfi
