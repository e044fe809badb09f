// Split-BF16 tensor-core apply of one sub-BF (BF_PREC_BF16X3), two launches.
//
// Same tiles and level recursions as the fused FP32 kernels (front: V, H
// levels of Eq. 2, switch; back: G levels of Eq. 3, U of Eq. bf3), but every
// level product runs on the 5th-generation tensor cores:
//
//  * the tile's coefficients stay resident in tensor memory: pair slot s
//    holds, for each of the 128 right-hand-side rows (TMEM lanes), the 2r
//    real components (t, re/im) in columns [s * SLOT, s * SLOT + 2r);
//  * a level group (two input pairs -> two output pairs) is one dense complex
//    2r x 2r block W, built on the fly in shared memory from the factored
//    form (the real Lagrange matrix of the level times the pair's phases) as
//    its real embedding [[Re W, -Im W], [Im W, Re W]];
//  * operands are split x = hi + lo into BF16 (hi = bf16(x), lo = bf16(x - hi));
//    D = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 in TMEM by
//    tcgen05.mma (M = 128 rows, N = SLOT, K = 16 per instruction), issued by
//    one thread and tracked by an mbarrier;
//  * D is written in place over the two input slots it consumed.
//
// Rows are right-hand-side columns interleaved with amplitude terms:
// row = c * r_alpha + k (RHS c of the slice, amplitude term k), so the sum
// over k in Eq. (tg) is a warp shuffle.  The U stage accumulates each CTA's
// own rows of G in place (no other CTA touches them).
#include <cstdio>

#include "bf_device.h"
#include "bf_tc.h"

namespace bfi {
namespace {

constexpr int kTcThreads = 256;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ unsigned brev(unsigned v, int bits) { return bits == 0 ? 0u : (__brev(v) >> (32 - bits)); }

__device__ __forceinline__ void cp16(void* dst, const void* src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp8(void* dst, const void* src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit_wait()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void stage_matrix(float* dst, const float* src, int rows, int cols, int c4, int tid)
{
    const int half = cols / 2;
    for (int e = tid; e < rows * half; e += kTcThreads) {
        const int rr = e / half, cc = e - rr * half;
        cp8(dst + rr * c4 + 2 * cc, src + rr * cols + 2 * cc);
    }
}

template <int R>
struct Shape {
    static constexpr int D2 = 2 * R;                      // real components per pair
    static constexpr int SLOT = D2 <= 16 ? 16 : 32;       // TMEM columns per pair = MMA N
    static constexpr int KS = (D2 + 7) / 8 * 8;           // K rows per input pair in a group
    static constexpr int KG = 2 * KS;                     // K of a group MMA chain
    static constexpr int KP = (D2 + 15) / 16 * 16;        // K of a single-pair (switch) chain
    static constexpr int R4 = (R + 3) & ~3;
    static constexpr int SBO = (KG / 8) * 128;            // 8-row-group stride of the operands
    static constexpr int A_BYTES = 128 * KG * 2;          // one of A_hi / A_lo
    static constexpr int B_BYTES = SLOT * KG * 2;         // one B matrix (hi or lo, one output pair)
    static constexpr int BUF = 2 * A_BYTES + 4 * B_BYTES; // A_hi | A_lo | B_hi0 | B_hi1 | B_lo0 | B_lo1
};

struct TcArgs {
    Geo g;
    int64_t m;
    int mr, nslice;
    const float2* F;
    const float2* bk;
    const float* MvT;   // [nv][R]
    const float2* EV;
    const float* MHT;   // [kH][2R][R]
    const float2* EH;
    const float2* S;
    float2* W;          // [nslice][P][128][R]
    const float* MGT;   // [kG][2][R][R]
    const float2* FG;
    const float* MU;    // [nv][R]
    const float2* EU;
    const float2* ak;
    float2* G;
    int beta;
    int* err;
    long long spin;
};

__device__ __forceinline__ int opnd_off(int row, int k, int sbo)
{
    return (row >> 3) * sbo + (k >> 3) * 128 + (row & 7) * 16;  // byte offset of 8 K-values of a row
}

// A of a level group: this thread converts its row of input slot hw (K offset hw * KS)
template <int R>
__device__ __forceinline__ void build_A_group(unsigned char* buf, uint32_t tlane, int s0, int s1, int hw, int row)
{
    using S = Shape<R>;
    float v[S::KS];
#pragma unroll
    for (int d = S::D2; d < S::KS; ++d) v[d] = 0.f;
    tc::ld_dims<S::D2>(tlane + (uint32_t)((hw ? s1 : s0) * S::SLOT), v);
    tc::wait_ld();
    unsigned char* Ah = buf;
    unsigned char* Al = buf + S::A_BYTES;
#pragma unroll
    for (int ch = 0; ch < S::KS / 8; ++ch) {
        uint4 h, l;
        tc::split2(v[8 * ch + 0], v[8 * ch + 1], h.x, l.x);
        tc::split2(v[8 * ch + 2], v[8 * ch + 3], h.y, l.y);
        tc::split2(v[8 * ch + 4], v[8 * ch + 5], h.z, l.z);
        tc::split2(v[8 * ch + 6], v[8 * ch + 7], h.w, l.w);
        const int off = opnd_off(row, hw * S::KS + 8 * ch, S::SBO);
        *reinterpret_cast<uint4*>(Ah + off) = h;
        *reinterpret_cast<uint4*>(Al + off) = l;
    }
}

// A of a single pair (switch): K = KP; warps of half 0 do it
template <int R>
__device__ __forceinline__ void build_A_single(unsigned char* buf, uint32_t tlane, int slot, int row)
{
    using S = Shape<R>;
    constexpr int SBO1 = (S::KP / 8) * 128;
    float v[S::KP];
#pragma unroll
    for (int d = S::D2; d < S::KP; ++d) v[d] = 0.f;
    tc::ld_dims<S::D2>(tlane + (uint32_t)(slot * S::SLOT), v);
    tc::wait_ld();
#pragma unroll
    for (int ch = 0; ch < S::KP / 8; ++ch) {
        uint4 h, l;
        tc::split2(v[8 * ch + 0], v[8 * ch + 1], h.x, l.x);
        tc::split2(v[8 * ch + 2], v[8 * ch + 3], h.y, l.y);
        tc::split2(v[8 * ch + 4], v[8 * ch + 5], h.z, l.z);
        tc::split2(v[8 * ch + 6], v[8 * ch + 7], h.w, l.w);
        const int off = opnd_off(row, 8 * ch, SBO1);
        *reinterpret_cast<uint4*>(buf + off) = h;
        *reinterpret_cast<uint4*>(buf + S::A_BYTES + off) = l;
    }
}

// value of the real embedding of complex W at (n = 2t + ro, component ri)
__device__ __forceinline__ float embed(float2 w, int ro, int ri) { return ro == ri ? w.x : (ro ? w.y : -w.y); }

// B of a level group: two matrices (output pairs s = 0, 1) of SLOT x KG.
// kind 0 (H, Eq. 2): W_s[t][(c, s')] = MH[t][c r + s'] * E_s[c][s'].
// kind 1 (G, Eq. 3): W_s[t][(c, s')] = FG_s[c][t] * MG_s[t][s'].
template <int R, int KIND>
__device__ __forceinline__ void build_B_group(unsigned char* buf, const float* Mt, const float2* P0, const float2* P1,
                                              int tid)
{
    using S = Shape<R>;
    constexpr int NCH = S::KG / 8;
    unsigned char* Bh = buf + 2 * S::A_BYTES;
    unsigned char* Bl = Bh + 2 * S::B_BYTES;
    for (int it = tid; it < 2 * S::SLOT * NCH; it += kTcThreads) {
        const int s = it / (S::SLOT * NCH);
        const int rem = it - s * S::SLOT * NCH;
        const int n = rem / NCH, ch = rem - n * NCH;
        const float2* Pp = s ? P1 : P0;
        float vals[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = 8 * ch + e;
            const int c = k >= S::KS ? 1 : 0;
            const int kr = k - c * S::KS;
            float val = 0.f;
            if (n < S::D2 && kr < S::D2) {
                const int t = n >> 1, ro = n & 1, sp = kr >> 1, ri = kr & 1;
                float2 w;
                if (KIND == 0) {
                    const float mv = Mt[(c * R + sp) * S::R4 + t];  // MH^T[(c, s')][t]
                    const float2 ph = Pp[c * R + sp];              // E_s[c][s']
                    w = make_float2(mv * ph.x, mv * ph.y);
                } else {
                    const float mv = Mt[(s * R + sp) * S::R4 + t];  // MG^T[pos][s'][t]
                    const float2 ph = Pp[c * R + t];               // FG_pos[c][t]
                    w = make_float2(mv * ph.x, mv * ph.y);
                }
                val = embed(w, ro, ri);
            }
            vals[e] = val;
        }
        uint4 h, l;
        tc::split2(vals[0], vals[1], h.x, l.x);
        tc::split2(vals[2], vals[3], h.y, l.y);
        tc::split2(vals[4], vals[5], h.z, l.z);
        tc::split2(vals[6], vals[7], h.w, l.w);
        const int off = s * S::B_BYTES + opnd_off(n, 8 * ch, S::SBO);
        *reinterpret_cast<uint4*>(Bh + off) = h;
        *reinterpret_cast<uint4*>(Bl + off) = l;
    }
}

// B of the switch of one pair: W[t][s'] = S[t][s'] (complex, global), SLOT x KP
template <int R>
__device__ __forceinline__ void build_B_switch(unsigned char* buf, const float2* Sq, int tid)
{
    using S = Shape<R>;
    constexpr int NCH = S::KP / 8;
    constexpr int SBO1 = (S::KP / 8) * 128;
    unsigned char* Bh = buf + 2 * S::A_BYTES;
    unsigned char* Bl = Bh + 2 * S::B_BYTES;
    for (int it = tid; it < S::SLOT * NCH; it += kTcThreads) {
        const int n = it / NCH, ch = it - n * NCH;
        float vals[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = 8 * ch + e;
            float val = 0.f;
            if (n < S::D2 && k < S::D2) val = embed(__ldg(Sq + (n >> 1) * R + (k >> 1)), n & 1, k & 1);
            vals[e] = val;
        }
        uint4 h, l;
        tc::split2(vals[0], vals[1], h.x, l.x);
        tc::split2(vals[2], vals[3], h.y, l.y);
        tc::split2(vals[4], vals[5], h.z, l.z);
        tc::split2(vals[6], vals[7], h.w, l.w);
        const int off = opnd_off(n, 8 * ch, SBO1);
        *reinterpret_cast<uint4*>(Bh + off) = h;
        *reinterpret_cast<uint4*>(Bl + off) = l;
    }
}

// D(d_tmem) = A_hi B_hi + A_hi B_lo + A_lo B_hi over K (one thread)
__device__ __forceinline__ void issue_chain(uint32_t d_tmem, const unsigned char* Ah, const unsigned char* Al,
                                            const unsigned char* Bh, const unsigned char* Bl, int K, int sbo,
                                            uint32_t idesc)
{
    const int nks = K / 16;
    for (int ks = 0; ks < nks; ++ks)
        tc::mma_bf16(d_tmem, tc::desc(Ah + ks * 256, 128, sbo), tc::desc(Bh + ks * 256, 128, sbo), idesc, ks > 0);
    for (int ks = 0; ks < nks; ++ks)
        tc::mma_bf16(d_tmem, tc::desc(Ah + ks * 256, 128, sbo), tc::desc(Bl + ks * 256, 128, sbo), idesc, 1);
    for (int ks = 0; ks < nks; ++ks)
        tc::mma_bf16(d_tmem, tc::desc(Al + ks * 256, 128, sbo), tc::desc(Bh + ks * 256, 128, sbo), idesc, 1);
}

// double-buffered group pipeline state
struct Pipe {
    int pend[2];
    uint32_t ph[2];
    int n;
    bool ok;
    __device__ void init()
    {
        pend[0] = pend[1] = 0;
        ph[0] = ph[1] = 0;
        n = 0;
        ok = true;
    }
};

__device__ __forceinline__ void pipe_acquire(Pipe& pp, uint64_t* mbar, int b, long long spin)
{
    if (pp.pend[b]) {
        pp.ok = tc::mbar_wait(&mbar[b], pp.ph[b], spin) && pp.ok;
        pp.ph[b] ^= 1u;
        pp.pend[b] = 0;
        tc::fence_after();
    }
}
__device__ __forceinline__ void pipe_drain(Pipe& pp, uint64_t* mbar, long long spin)
{
    for (int b = 0; b < 2; ++b) pipe_acquire(pp, mbar, b, spin);
}
__device__ __forceinline__ void publish_operands()
{
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// level groups of one tile level (kind 0: H with phases Pl; kind 1: G with phases Pl)
template <int R, int KIND>
__device__ __forceinline__ void tc_level(unsigned char* bufs, Pipe& pp, uint64_t* mbar, uint32_t tbase, uint32_t tlane,
                                         int K, int j, const float* Mt, const float2* Pl, int hw, int row, int tid,
                                         long long spin)
{
    using S = Shape<R>;
    const int kj = K - j, half = 1 << kj, T = 1 << K;
    for (int grp = 0; grp < T / 2; ++grp) {
        const int b = pp.n & 1;
        pipe_acquire(pp, mbar, b, spin);
        unsigned char* buf = bufs + b * S::BUF;
        const int a = grp >> kj, bp = grp & (half - 1);
        const int s0 = (bp << j) + (int)brev((unsigned)a, j - 1), s1 = s0 + (1 << (j - 1));
        build_A_group<R>(buf, tlane, s0, s1, hw, row);
        build_B_group<R, KIND>(buf, Mt, Pl + (size_t)((2 * a) * half + bp) * S::D2,
                               Pl + (size_t)((2 * a + 1) * half + bp) * S::D2, tid);
        publish_operands();
        if (tid == 0) {
            const unsigned char* Ah = buf;
            const unsigned char* Al = buf + S::A_BYTES;
            const unsigned char* Bh = buf + 2 * S::A_BYTES;
            const unsigned char* Bl = Bh + 2 * S::B_BYTES;
            constexpr uint32_t id = tc::idesc_bf16(128, S::SLOT);
            issue_chain(tbase + (uint32_t)(s0 * S::SLOT), Ah, Al, Bh, Bl, S::KG, S::SBO, id);
            issue_chain(tbase + (uint32_t)(s1 * S::SLOT), Ah, Al, Bh + S::B_BYTES, Bl + S::B_BYTES, S::KG, S::SBO, id);
            tc::commit(&mbar[b]);
        }
        pp.pend[b] = 1;
        ++pp.n;
    }
    pipe_drain(pp, mbar, spin);
}

template <int R>
size_t front_tc_smem(const Geo& g, int NV)
{
    using S = Shape<R>;
    const size_t T = (size_t)1 << g.kH;
    size_t s = 2 * (size_t)S::BUF + sizeof(float2) * ((size_t)g.kH * T * S::D2 + T * NV) +
               sizeof(float) * ((size_t)NV * S::R4 + (size_t)g.kH * 2 * R * S::R4);
    return std::max<size_t>(s, 120 * 1024);  // one CTA per SM: the tile holds all 512 TMEM columns
}

template <int R>
size_t back_tc_smem(const Geo& g, int NU)
{
    using S = Shape<R>;
    const size_t T = (size_t)1 << g.kG;
    size_t s = 2 * (size_t)S::BUF + sizeof(float2) * ((size_t)g.kG * T * S::D2 + T * NU) +
               sizeof(float) * ((size_t)g.kG * 2 * R * S::R4 + (size_t)NU * S::R4);
    return std::max<size_t>(s, 120 * 1024);
}

// ------------------------------------------------------------------ front --
template <int R, int NV>
__global__ void __launch_bounds__(kTcThreads, 1) front_tc(TcArgs A)
{
    using S = Shape<R>;
    constexpr int R4 = S::R4;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[2];
    const Geo& g = A.g;
    const int K = g.kH, T = 1 << K, ra = g.ra, mr = A.mr;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, qd = warp & 3, hw = warp >> 2;
    const int row = 32 * qd + lane;
    const int slice = (int)(blockIdx.x % A.nslice);
    const int64_t tile = blockIdx.x / A.nslice;
    const int nP = 1 << g.l1;
    const int64_t p = tile & (nP - 1), c0 = tile >> g.l1;
    const int64_t nBh = (int64_t)1 << (g.L - g.h);
    const int64_t xi_base = c0 * T * NV;
    const int64_t N = g.N, P = g.P;

    unsigned char* bufs = smem;
    float2* EHs = reinterpret_cast<float2*>(smem + 2 * S::BUF);  // [K][T][2R]
    float2* EVs = EHs + (size_t)K * T * S::D2;                   // [T*NV]
    float* MvTs = reinterpret_cast<float*>(EVs + (size_t)T * NV); // [NV][R4]
    float* MHTs = MvTs + NV * R4;                                 // [K][2R][R4]

    if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
    if (tid == 0) {
        tc::mbar_init(&s_mbar[0], 1);
        tc::mbar_init(&s_mbar[1], 1);
    }
    stage_matrix(MvTs, A.MvT, NV, R, R4, tid);
    stage_matrix(MHTs, A.MHT, K * 2 * R, R, R4, tid);
    {
        const float2* ev = A.EV + p * N + xi_base;
        for (int e = tid; e < T * NV / 2; e += kTcThreads) cp16(EVs + 2 * e, ev + 2 * e);
    }
    for (int j = 1; j <= K; ++j) {
        const int64_t nBl = (int64_t)1 << (g.L - g.l1 - j);
        const float2* eh = A.EH + (size_t)(j - 1) * P * 2 * R;
        for (int e = tid; e < T * R; e += kTcThreads) {
            const int lp = e / R, w = e - lp * R;
            const int64_t ap = (p << j) + (lp >> (K - j));
            const int64_t bp = (c0 << (K - j)) + (lp & ((1 << (K - j)) - 1));
            cp16(EHs + ((size_t)(j - 1) * T + lp) * 2 * R + 2 * w, eh + (ap * nBl + bp) * 2 * R + 2 * w);
        }
    }
    cp_commit_wait();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_tmem;
    const uint32_t tlane = tbase + ((uint32_t)(32 * qd) << 16);

    // ---- V (Eq. 1): this thread's row (c, k) of slots hw, hw + 2, ...
    {
        const int c = row / ra, k = row - (row / ra) * ra;
        const int64_t cg = (int64_t)slice * mr + c;
        const bool valid = c < mr && cg < A.m;
        const float2* bk = A.bk + (size_t)(k < ra ? k : 0) * N;
        for (int j = hw; j < T; j += 2) {
            float v[S::D2];
#pragma unroll
            for (int d = 0; d < S::D2; ++d) v[d] = 0.f;
            const int64_t xi0 = xi_base + (int64_t)j * NV;
#pragma unroll 4
            for (int x = 0; x < NV; ++x) {
                const float2 f = valid ? __ldg(A.F + (xi0 + x) * A.m + cg) : make_float2(0.f, 0.f);
                const float2 z = cmulf(EVs[j * NV + x], cmulf(__ldg(bk + xi0 + x), f));
                const float* mv = MvTs + x * R4;
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    v[2 * t] = fmaf(mv[t], z.x, v[2 * t]);
                    v[2 * t + 1] = fmaf(mv[t], z.y, v[2 * t + 1]);
                }
            }
            tc::st_dims<S::D2>(tlane + (uint32_t)(j * S::SLOT), v);
        }
        tc::wait_st();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();

    Pipe pp;
    pp.init();
    for (int j = 1; j <= K; ++j)
        tc_level<R, 0>(bufs, pp, s_mbar, tbase, tlane, K, j, MHTs + (size_t)(j - 1) * 2 * R * R4,
                       EHs + (size_t)(j - 1) * T * S::D2, hw, row, tid, A.spin);

    // ---- switch (step 4), one pair per MMA chain
    for (int lp = 0; lp < T; ++lp) {
        const int b = pp.n & 1;
        pipe_acquire(pp, s_mbar, b, A.spin);
        unsigned char* buf = bufs + b * S::BUF;
        const int slot = (int)brev((unsigned)lp, K);
        const int64_t qg = ((p << K) + lp) * nBh + c0;
        if (hw == 0) build_A_single<R>(buf, tlane, slot, row);
        build_B_switch<R>(buf, A.S + qg * R * R, tid);
        publish_operands();
        if (tid == 0) {
            constexpr uint32_t id = tc::idesc_bf16(128, S::SLOT);
            constexpr int SBO1 = (S::KP / 8) * 128;
            const unsigned char* Bh = buf + 2 * S::A_BYTES;
            issue_chain(tbase + (uint32_t)(slot * S::SLOT), buf, buf + S::A_BYTES, Bh, Bh + 2 * S::B_BYTES, S::KP, SBO1,
                        id);
            tc::commit(&s_mbar[b]);
        }
        pp.pend[b] = 1;
        ++pp.n;
    }
    pipe_drain(pp, s_mbar, A.spin);

    // ---- write the switch-level coefficients: W[slice][q][row][R]
    float2* Wout = A.W + (size_t)slice * P * 128 * R;
    for (int lp = hw; lp < T; lp += 2) {
        const int slot = (int)brev((unsigned)lp, K);
        const int64_t qg = ((p << K) + lp) * nBh + c0;
        float v[S::D2];
        tc::ld_dims<S::D2>(tlane + (uint32_t)(slot * S::SLOT), v);
        tc::wait_ld();
        float4* dst = reinterpret_cast<float4*>(Wout + ((size_t)qg * 128 + row) * R);
#pragma unroll
        for (int i = 0; i < S::D2 / 4; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
    if (!pp.ok && tid == 0) atomicExch(A.err, 3);
}

// ------------------------------------------------------------------- back --
template <int R, int NU>
__global__ void __launch_bounds__(kTcThreads, 1) back_tc(TcArgs A)
{
    using S = Shape<R>;
    constexpr int R4 = S::R4;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[2];
    const Geo& g = A.g;
    const int K = g.kG, T = 1 << K, ra = g.ra, mr = A.mr;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, qd = warp & 3, hw = warp >> 2;
    const int row = 32 * qd + lane;
    const int slice = (int)(blockIdx.x % A.nslice);
    const int64_t pp_x = blockIdx.x / A.nslice;  // x-node at level h
    const int nC = 1 << g.l1;
    const int64_t nBh = (int64_t)1 << (g.L - g.h);
    const int XN = T * NU;
    const int64_t N = g.N, P = g.P, x0g = pp_x * XN;

    unsigned char* bufs = smem;
    float2* FGs = reinterpret_cast<float2*>(smem + 2 * S::BUF);  // [K][T][2R]
    float2* EUs = FGs + (size_t)K * T * S::D2;                   // [XN]
    float* MGTs = reinterpret_cast<float*>(EUs + XN);            // [K][2][R][R4]
    float* MUs = MGTs + (size_t)K * 2 * R * R4;                  // [NU][R4]

    if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
    if (tid == 0) {
        tc::mbar_init(&s_mbar[0], 1);
        tc::mbar_init(&s_mbar[1], 1);
    }
    stage_matrix(MGTs, A.MGT, K * 2 * R, R, R4, tid);
    stage_matrix(MUs, A.MU, NU, R, R4, tid);
    cp_commit_wait();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_tmem;
    const uint32_t tlane = tbase + ((uint32_t)(32 * qd) << 16);
    const int c = row / ra, k = row - (row / ra) * ra;
    const int64_t cg = (int64_t)slice * mr + c;
    const bool valid = c < mr && cg < A.m;
    const float2* akk = A.ak + (size_t)(k < ra ? k : 0) * N;
    const float2* Win = A.W + (size_t)slice * P * 128 * R;
    Pipe pp;
    pp.init();

    for (int c0 = 0; c0 < nC; ++c0) {
        // switch-level pairs (pp_x, c0 T + j) -> TMEM slots j
        for (int j = hw; j < T; j += 2) {
            const float4* src = reinterpret_cast<const float4*>(Win + ((size_t)(pp_x * nBh + (int64_t)c0 * T + j) * 128 + row) * R);
            float v[S::D2];
#pragma unroll
            for (int i = 0; i < S::D2 / 4; ++i) {
                const float4 w4 = __ldg(src + i);
                v[4 * i] = w4.x;
                v[4 * i + 1] = w4.y;
                v[4 * i + 2] = w4.z;
                v[4 * i + 3] = w4.w;
            }
            tc::st_dims<S::D2>(tlane + (uint32_t)(j * S::SLOT), v);
        }
        for (int jl = 1; jl <= K; ++jl) {
            const int64_t nBl = (int64_t)1 << (g.L - g.h - jl);
            const float2* fg = A.FG + (size_t)(jl - 1) * P * 2 * R;
            for (int e = tid; e < T * R; e += kTcThreads) {
                const int lp = e / R, w = e - lp * R;
                const int64_t ap = (pp_x << jl) + (lp >> (K - jl));
                const int64_t bp = ((int64_t)c0 << (K - jl)) + (lp & ((1 << (K - jl)) - 1));
                cp16(FGs + ((size_t)(jl - 1) * T + lp) * 2 * R + 2 * w, fg + (ap * nBl + bp) * 2 * R + 2 * w);
            }
        }
        for (int e = tid; e < XN / 2; e += kTcThreads) cp16(EUs + 2 * e, A.EU + (size_t)c0 * N + x0g + 2 * e);
        cp_commit_wait();
        tc::wait_st();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();

        for (int j = 1; j <= K; ++j)
            tc_level<R, 1>(bufs, pp, s_mbar, tbase, tlane, K, j, MGTs + (size_t)(j - 1) * 2 * R * R4,
                           FGs + (size_t)(j - 1) * T * S::D2, hw, row, tid, A.spin);

        // ---- U (Eq. bf3) of T_Omega node c0, summed over k, accumulated into this CTA's rows of G
        for (int lp = hw; lp < T; lp += 2) {
            const int slot = (int)brev((unsigned)lp, K);
            float v[S::D2];
            tc::ld_dims<S::D2>(tlane + (uint32_t)(slot * S::SLOT), v);
            tc::wait_ld();
            for (int i = 0; i < NU; ++i) {
                float2 w = make_float2(0.f, 0.f);
                const float* mu = MUs + i * R4;
#pragma unroll
                for (int s = 0; s < R; ++s) {
                    w.x = fmaf(mu[s], v[2 * s], w.x);
                    w.y = fmaf(mu[s], v[2 * s + 1], w.y);
                }
                const int64_t x = x0g + lp * NU + i;
                float2 ctb = cmulf(cmulf(__ldg(akk + x), EUs[lp * NU + i]), w);
                for (int o = 1; o < ra; o <<= 1) {
                    ctb.x += __shfl_xor_sync(0xffffffffu, ctb.x, o);
                    ctb.y += __shfl_xor_sync(0xffffffffu, ctb.y, o);
                }
                if (k == 0 && valid) {
                    float2* gp = A.G + x * A.m + cg;
                    if (c0 > 0 || A.beta) {
                        const float2 o = *gp;
                        ctb.x += o.x;
                        ctb.y += o.y;
                    }
                    *gp = ctb;
                }
            }
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
    if (!pp.ok && tid == 0) atomicExch(A.err, 3);
}

template <int R>
cudaError_t launch_tc_r(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws, int* err,
                        cudaStream_t st)
{
    constexpr int NV = (R < 8) ? 8 : (R < 16 ? 16 : 32);
    const Geo& g = B.g;
    TcArgs a;
    a.g = g;
    a.m = m;
    a.mr = 128 / g.ra;
    a.nslice = (int)((m + a.mr - 1) / a.mr);
    a.F = F;
    a.bk = B.f32.b;
    a.MvT = B.f32.Mv;
    a.EV = B.f32.EV;
    a.MHT = B.f32.MH;
    a.EH = B.f32.EH;
    a.S = B.f32.S;
    a.W = ws;
    a.MGT = B.f32.MG;
    a.FG = B.f32.FG;
    a.MU = B.f32.MU;
    a.EU = B.f32.EU;
    a.ak = B.f32.a;
    a.G = G;
    a.beta = beta;
    a.err = err;
    a.spin = 1ll << 20;
    const size_t sf = front_tc_smem<R>(g, NV), sb = back_tc_smem<R>(g, NV);
    cudaError_t e = cudaFuncSetAttribute(front_tc<R, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(back_tc<R, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    if (e != cudaSuccess) return e;
    const int64_t nfront = ((int64_t)1 << g.l1) * ((int64_t)1 << (g.L - g.h)) * a.nslice;
    const int64_t nback = ((int64_t)1 << g.h) * a.nslice;
    {
        ProfScope ps("front_tc", st);
        front_tc<R, NV><<<(unsigned)nfront, kTcThreads, sf, st>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        ProfScope ps("back_tc", st);
        back_tc<R, NV><<<(unsigned)nback, kTcThreads, sb, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

bool tc_supported(const Geo& g, const char** why)
{
    const int r = g.r;
    if (r != 8 && r != 10 && r != 12) {
        if (why) *why = "split-BF16 kernels are built for r = 8, 10, 12";
        return false;
    }
    const int NV = r < 16 ? 16 : 32;
    if (g.nv != NV) {
        if (why) *why = "split-BF16 kernels need n0 <= r";
        return false;
    }
    if (g.ra != 1 && g.ra != 2 && g.ra != 4) {
        if (why) *why = "split-BF16 kernels need an amplitude rank of 1, 2 or 4";
        return false;
    }
    const int slot = 2 * r <= 16 ? 16 : 32;
    const int T = 1 << (g.kH > g.kG ? g.kH : g.kG);
    if (T * slot > 512) {
        if (why) *why = "tile does not fit tensor memory (2^kH or 2^kG pairs x TMEM columns per pair > 512); use a "
                        "larger tolerance (r = 8) or split the operator";
        return false;
    }
    return true;
}

size_t tc_ws_bytes(const Geo& g, int64_t m)
{
    const int ra = g.ra > 0 ? g.ra : 1;
    const int mr = 128 / ra;
    const int64_t nslice = (m + mr - 1) / mr;
    return (size_t)nslice * g.P * 128 * g.r * sizeof(float2);
}

cudaError_t launch_tc(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws, int* err,
                      cudaStream_t st)
{
    if (B.g.ra == 0) {
        if (!beta) return cudaMemsetAsync(G, 0, (size_t)B.g.N * m * sizeof(float2), st);
        return cudaSuccess;
    }
    switch (B.g.r) {
    case 8: return launch_tc_r<8>(B, F, m, G, beta, ws, err, st);
    case 10: return launch_tc_r<10>(B, F, m, G, beta, ws, err, st);
    case 12: return launch_tc_r<12>(B, F, m, G, beta, ws, err, st);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace bfi
