// Argument blocks of the fused FP32 kernels (shared by the single-operator and
// batched launchers).
#pragma once

#include "bf_device.h"

namespace bfi {

struct FrontArgs {
    Geo g;
    const float2* F;  // [N][m]
    int64_t m;
    int mr, lmr, CTp, lct, nslice;
    int tpc;           // tiles per CTA (consecutive work indices)
    const float2* bk;  // [ra][N]
    const float* MvT;  // [nv][R]
    const float2* EV;  // [2^l1][N]
    const float* MHT;  // [kH][2R][R]
    const float2* EH;  // [kH][P][2][R]
    const float2* S;   // [P][R][R]
    float2* W;         // [nslice][P][R][CTp]
};

struct BackArgs {
    Geo g;
    int64_t m;
    int mr, lmr, CTp, lct, nslice;
    int tpc;           // T_Omega chunks processed together (divides 2^l1)
    const float2* W;
    const float* MGT;  // [kG][2][R][R]  (pos, s, t)
    const float2* FG;  // [kG][P][2][R]
    const float* MU;   // [nv][R]
    const float2* EU;  // [2^l1][N]
    const float2* ak;  // [ra][N]
    float2* G;         // [N][m]
    int beta;
};

// One operator of a batched launch: its front and back argument blocks and work counts.
struct BatchItem {
    FrontArgs fa;
    BackArgs ba;
    int64_t nfront, nback;
};

// Device-side description of a batched launch.
struct BatchLaunch {
    const BatchItem* items = nullptr;
    int nitems = 0;
    const int64_t* off = nullptr;  // [2 nitems] start of each segment in the work order (increasing)
    const int* seg = nullptr;      // [2 nitems] segment -> (op << 1) | (1 for its back tiles, 0 for its fronts)
    int64_t total = 0;
    unsigned long long* counter = nullptr;
    int* done = nullptr;  // [nitems]
    int* err = nullptr;
    long long spin_limit = 1ll << 24;
    int wait_extra = 0;  // test hook: extra front completions a back tile waits for (never arrive)
    size_t smem = 0;
    int grid = 0;
};

bool fused_make_args(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws, int mr_hint,
                     FrontArgs* fa, BackArgs* ba, size_t* sf, size_t* sb, int64_t* nfront, int64_t* nback);
// set_attr: only set the kernel's shared-memory limit to bl.smem (no launch);
// grid_out != NULL: only compute the persistent grid (occupancy x SMs) for bl.smem;
// otherwise launch (bl.grid CTAs).
cudaError_t batch_launch_f32(int r, const BatchLaunch& bl, cudaStream_t st, bool set_attr, int* grid_out);

}  // namespace bfi
