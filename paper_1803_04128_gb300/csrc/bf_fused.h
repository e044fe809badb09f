// Argument blocks of the fused FP32 kernels (shared by the single-operator and
// batched launchers).
#pragma once

#include "bf_device.h"

namespace bfi {

// Layout of the switch-level workspace W, in units of pairs (each R x CTp c64).
// Pair (a, b) of column slice sl (a: x-node at level h, b: T_Omega node at level
// L-h) is at  d * sD + s * sS + sl * slice + (a_loc << lb) + b_loc  with
// d = a >> la, a_loc = a mod 2^la, s = b >> lb, b_loc = b mod 2^lb.  One shard
// (the default): la = h, lb = L-h, sD = sS = 0, slice = P, i.e. a * 2^(L-h) + b.
// G shards: la = h - log2 G, lb = L-h - log2 G; a front's send buffer has
// sD = nslice * 2^(la+lb), sS = 0; a back's receive buffer sS = that, sD = 0.
struct WLayout {
    int la, lb;
    int64_t sD, sS, slice;
};

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
    float2* W;         // switch-level coefficients, layout wl
    WLayout wl;
    int64_t c0_lo;     // first T_Omega node (level L-h) of this shard's tiles
    int64_t xi_lo;     // F holds rows xi_lo ..: row xi at F + (xi - xi_lo) * m
    OtfPhase ph;       // g.otf = 1: phases evaluated in the kernel (EV, EH, S unused)
    int K;             // H levels of this pass, l1+1 .. l1+K (tiles of 2^K pairs): kH unless split
    int last;          // 1: the pass reaches level h: apply the switch and write W (layout wl)
    float2* Wo;        // last = 0: the coefficients at level l1 + K, layout wlo
    WLayout wlo;
    int s_smem = 0;    // last = 1, tables: copy each tile's switch blocks into shared memory
    int bk_smem = 0;   // copy each tile's b_k values into shared memory
};

struct BackArgs {
    Geo g;
    int64_t m;
    int mr, lmr, CTp, lct, nslice;
    int tpc;           // T_Omega chunks processed together (divides 2^l1)
    const float2* W;   // layout wl
    WLayout wl;
    int64_t pp_lo;     // first x-node (level h) of this shard
    int64_t x_lo;      // G holds rows x_lo ..: row x at G + (x - x_lo) * m
    const float* MGT;  // [kG][2][R][R]  (pos, s, t)
    const float2* FG;  // [kG][P][2][R]
    const float* MU;   // [nv][R]
    const float2* EU;  // [2^l1][N]
    const float2* ak;  // [ra][N]
    float2* G;         // [N][m]
    int beta;
    OtfPhase ph;       // g.otf = 1: phases evaluated in the kernel (FG, EU unused)
    int K;             // G levels of this pass, lb+1 .. lb+K = L-l1: kG unless split
    int lb;            // level of the input pairs in W (layout wl): h unless split
};

// A middle pass of a split level range: tiles of 2^K pairs read at level la
// (layout wli), K levels of H (Eq. 2) or G (Eq. 3) applied in shared memory,
// written at level la + K (layout wlo); an H pass that reaches level h applies
// the switch first.  A tile is (p: x-node at level la, c: chunk of 2^K
// consecutive T_Omega nodes at level L-la, column slice), as in the front.
struct MidArgs {
    Geo g;
    int mr, lmr, CTp, lct, nslice;
    int tpc;           // tiles per CTA
    int gkind;         // 0: H levels, 1: G levels
    int la, K;
    int last;          // H only: la + K = h
    const float2* Wi;  // input pairs, layout wli
    WLayout wli;
    float2* Wo;        // output pairs, layout wlo
    WLayout wlo;
    const float* MT;   // MH^T [kH][2R][R] or MG^T [kG][2][R][R] (all levels of that kind)
    const float2* E;   // EH or FG [k][P][2][R] (null with g.otf)
    int e0;            // index of level la + 1 in MT and E
    const float2* S;   // switch blocks [P][R][R] (last; null with g.otf)
    OtfPhase ph;
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
    // mode 1 (two phase launches): one launch over every operator's front tiles, then one over
    // every back tile, each CTA one work item; operators in the order ord (largest work first),
    // work item w of a phase belongs to ord[k] with off_x[k] <= w < off_x[k + 1]
    int mode = 0;
    const int* ord = nullptr;      // [nitems]
    const int64_t* off_f = nullptr;  // [nitems + 1]
    const int64_t* off_b = nullptr;  // [nitems + 1]
    size_t smem_f = 0, smem_b = 0;
    int64_t total_f = 0, total_b = 0;  // work items (CTAs) of each phase
};

// one front and one back pass over all kH and kG levels (the batched and sharded applies)
bool fused_make_args(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws, int mr_hint,
                     FrontArgs* fa, BackArgs* ba, size_t* sf, size_t* sb, int64_t* nfront, int64_t* nback);
// one of the two fused FP32 kernels with prepared arguments (nblocks CTAs)
cudaError_t launch_f32_front(int r, const FrontArgs& fa, size_t smem, int64_t nblocks, cudaStream_t st);
cudaError_t launch_f32_back(int r, const BackArgs& ba, size_t smem, int64_t nblocks, cudaStream_t st);
// the same with the phases evaluated in the kernel (bf_kernels_otf.cu; args with g.otf = 1)
cudaError_t launch_part_otf(int r, const FrontArgs* fa, const BackArgs* ba, size_t smem, int64_t nblocks,
                            cudaStream_t st);
// one middle pass (table phases or, with g.otf, evaluated ones)
cudaError_t launch_mid(int r, const MidArgs& ma, size_t smem, int64_t nblocks, cudaStream_t st);
cudaError_t launch_mid_otf(int r, const MidArgs& ma, size_t smem, int64_t nblocks, cudaStream_t st);
// set_attr: only set the kernel's shared-memory limit to bl.smem (no launch);
// grid_out != NULL: only compute the persistent grid (occupancy x SMs) for bl.smem;
// otherwise launch (bl.grid CTAs).
cudaError_t batch_launch_f32(int r, const BatchLaunch& bl, cudaStream_t st, bool set_attr, int* grid_out);
// mode 1: the two phase launches (set_attr: configure the kernels' shared memory only)
cudaError_t batch_phases_f32(int r, const BatchLaunch& bl, cudaStream_t st, bool set_attr);

}  // namespace bfi
