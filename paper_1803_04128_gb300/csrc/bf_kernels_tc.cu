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

constexpr int kTcThreads = 288;  // 8 builder warps + 1 MMA-issue warp

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

constexpr int NBUF = 4;  // operand buffers in flight between the builders and the MMA issuer

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
    return (row >> 3) * sbo + (k >> 3) * 128 + (row & 7) * 16;  // byte offset of the 8-value chunk of (row, k)
}

// Warps 0..7 build operands ("builders"); warp 8 issues the MMAs.  Hand-over
// per double-buffer b: ready[b] (256 builder arrivals: operands of the item in
// b written) and done[b] (tcgen05.commit: its MMAs finished).
constexpr int kBuilders = 256;

__device__ __forceinline__ void builders_sync() { asm volatile("bar.sync 1, 256;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::smem_u32(mbar)) : "memory");
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

// A of a single pair (switch), same operand layout, K = KP; builder warps of half 0
template <int R>
__device__ __forceinline__ void build_A_single(unsigned char* buf, uint32_t tlane, int slot, int row)
{
    using S = Shape<R>;
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
        const int off = opnd_off(row, 8 * ch, S::SBO);
        *reinterpret_cast<uint4*>(buf + off) = h;
        *reinterpret_cast<uint4*>(buf + S::A_BYTES + off) = l;
    }
}

// One 16-byte chunk of B (hi and lo): row rho of the real embedding of four
// consecutive complex weights w[0..3] at K offset k0 (a multiple of 8).  Row
// 2t (real part of output t) holds (Re w, -Im w) per weight, row 2t + 1 (the
// imaginary part) holds (Im w, Re w).
template <int R>
__device__ __forceinline__ void put_chunk(unsigned char* Bh, unsigned char* Bl, int rho, int k0, const float2* w)
{
    using S = Shape<R>;
    uint4 h, l;
    if ((rho & 1) == 0) {
        tc::split2(w[0].x, -w[0].y, h.x, l.x);
        tc::split2(w[1].x, -w[1].y, h.y, l.y);
        tc::split2(w[2].x, -w[2].y, h.z, l.z);
        tc::split2(w[3].x, -w[3].y, h.w, l.w);
    } else {
        tc::split2(w[0].y, w[0].x, h.x, l.x);
        tc::split2(w[1].y, w[1].x, h.y, l.y);
        tc::split2(w[2].y, w[2].x, h.z, l.z);
        tc::split2(w[3].y, w[3].x, h.w, l.w);
    }
    const int off = opnd_off(rho, k0, S::SBO);
    *reinterpret_cast<uint4*>(Bh + off) = h;
    *reinterpret_cast<uint4*>(Bl + off) = l;
}

// B of a level group: two matrices (output pairs s = 0, 1).  Item = (row rho,
// input pair c, chunk q of four weights s' = 4q..4q+3, output pair s); weights
// with s' >= r are the zero padding of K.
// kind 0 (H, Eq. 2): W_s[t][(c, s')] = MH[t][c r + s'] * E_s[c][s'].
// kind 1 (G, Eq. 3): W_s[t][(c, s')] = FG_s[c][t] * MG_s[t][s'].
template <int R, int KIND>
__device__ __forceinline__ void build_B_group(unsigned char* buf, const float* Mt, const float2* P0, const float2* P1,
                                              int tid)
{
    using S = Shape<R>;
    constexpr int NQ = S::KS / 8;
    constexpr int ITEMS = S::D2 * NQ * 4;
    unsigned char* Bh = buf + 2 * S::A_BYTES;
    unsigned char* Bl = Bh + 2 * S::B_BYTES;
    for (int it = tid; it < ITEMS; it += kBuilders) {
        const int rho = it % S::D2;
        const int rest = it / S::D2;
        const int q = rest % NQ;
        const int c = (rest / NQ) & 1;
        const int s = rest / (2 * NQ);
        const int t = rho >> 1;
        const float2* Pp = s ? P1 : P0;
        float2 w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int sp = 4 * q + e;
            if (sp < R) {
                float mv;
                float2 ph;
                if (KIND == 0) {
                    mv = Mt[(c * R + sp) * S::R4 + t];
                    ph = Pp[c * R + sp];
                } else {
                    mv = Mt[(s * R + sp) * S::R4 + t];
                    ph = Pp[c * R + t];
                }
                w[e] = make_float2(mv * ph.x, mv * ph.y);
            } else {
                w[e] = make_float2(0.f, 0.f);
            }
        }
        put_chunk<R>(Bh + s * S::B_BYTES, Bl + s * S::B_BYTES, rho, c * S::KS + 8 * q, w);
    }
}

// B of the switch of one pair: W[t][s'] = S[t][s'] (complex, staged in shared memory)
template <int R>
__device__ __forceinline__ void build_B_switch(unsigned char* buf, const float2* Sq, int tid)
{
    using S = Shape<R>;
    constexpr int NQ = (R + 3) / 4;
    unsigned char* Bh = buf + 2 * S::A_BYTES;
    unsigned char* Bl = Bh + 2 * S::B_BYTES;
    for (int it = tid; it < S::D2 * NQ; it += kBuilders) {
        const int rho = it % S::D2, q = it / S::D2, t = rho >> 1;
        float2 w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int sp = 4 * q + e;
            w[e] = sp < R ? Sq[t * R + sp] : make_float2(0.f, 0.f);
        }
        put_chunk<R>(Bh, Bl, rho, 8 * q, w);
    }
}

// matrix descriptors of one buffer: A_hi, A_lo, B_hi(s = 0, 1), B_lo(s = 0, 1); k-step ks adds 256 bytes
template <int R>
struct BufDesc {
    uint64_t ah, al, bh0, bh1, bl0, bl1;
    __device__ void init(const unsigned char* buf)
    {
        using S = Shape<R>;
        ah = tc::desc(buf, 128, S::SBO);
        al = tc::desc(buf + S::A_BYTES, 128, S::SBO);
        bh0 = tc::desc(buf + 2 * S::A_BYTES, 128, S::SBO);
        bh1 = tc::desc(buf + 2 * S::A_BYTES + S::B_BYTES, 128, S::SBO);
        bl0 = tc::desc(buf + 2 * S::A_BYTES + 2 * S::B_BYTES, 128, S::SBO);
        bl1 = tc::desc(buf + 2 * S::A_BYTES + 3 * S::B_BYTES, 128, S::SBO);
    }
};

// D(d_tmem) = A_hi B_hi + A_hi B_lo + A_lo B_hi over K
__device__ __forceinline__ void issue_chain(uint32_t d_tmem, uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl, int K,
                                            uint32_t idesc)
{
    const int nks = K / 16;
    for (int ks = 0; ks < nks; ++ks) tc::mma_bf16(d_tmem, ah + 16 * ks, bh + 16 * ks, idesc, ks > 0);
    for (int ks = 0; ks < nks; ++ks) tc::mma_bf16(d_tmem, ah + 16 * ks, bl + 16 * ks, idesc, 1);
    for (int ks = 0; ks < nks; ++ks) tc::mma_bf16(d_tmem, al + 16 * ks, bh + 16 * ks, idesc, 1);
}

__device__ __forceinline__ void group_slots(int K, int j, int grp, int& s0, int& s1, int& lo0, int& lo1)
{
    const int kj = K - j, half = 1 << kj;
    const int a = grp >> kj, bp = grp & (half - 1);
    s0 = (bp << j) + (int)brev((unsigned)a, j - 1);
    s1 = s0 + (1 << (j - 1));
    lo0 = (2 * a) * half + bp;      // logical output pairs (phase rows)
    lo1 = (2 * a + 1) * half + bp;
}

// builder-side pipeline bookkeeping (identical in every builder thread)
struct BPipe {
    int n;       // items handed over so far
    bool ok;
};

// completion of item i (buffer i % NBUF, its (i / NBUF)-th use); a no-op for i < 0.  The
// barrier cannot be two phases past the awaited one: item i + NBUF is built only
// after every builder has passed this wait.
__device__ __forceinline__ void builders_wait_item(uint64_t* done, int item, long long spin, bool& ok)
{
    if (item < 0) return;
    ok = tc::mbar_wait(&done[item % NBUF], (uint32_t)((item / NBUF) & 1), spin) && ok;
}

// builders: acquire the buffer of item n (its previous use finished) and, at a
// level start, the previous item's outputs (one commit covers all earlier MMAs)
__device__ __forceinline__ unsigned char* builders_begin(unsigned char* bufs, int BUF, uint64_t* done, BPipe& bp,
                                                         bool level_start, long long spin)
{
    if (level_start) builders_wait_item(done, bp.n - 1, spin, bp.ok);
    else builders_wait_item(done, bp.n - NBUF, spin, bp.ok);
    tc::fence_after();
    return bufs + (bp.n % NBUF) * BUF;
}
__device__ __forceinline__ void builders_end(uint64_t* ready, BPipe& bp)
{
    tc::fence_async_smem();
    tc::fence_before();
    mbar_arrive(&ready[bp.n % NBUF]);
    ++bp.n;
}
__device__ __forceinline__ void builders_drain(uint64_t* done, BPipe& bp, long long spin)
{
    builders_wait_item(done, bp.n - 1, spin, bp.ok);
    tc::fence_after();
}

// issuer: wait for the operands of item n, issue, commit; buffer b's descriptors are
// buffer 0's plus b * BUF / 16 in the address field (shared addresses stay below 2^18)
template <int R>
__device__ __forceinline__ bool issuer_item(uint64_t* ready, uint64_t* done, const BufDesc<R>& bd, int n, bool pair,
                                            uint32_t d0, uint32_t d1, long long spin)
{
    using S = Shape<R>;
    const int b = n % NBUF;
    const uint64_t o = (uint64_t)(b * (S::BUF >> 4));
    const bool ok = tc::mbar_wait(&ready[b], (uint32_t)((n / NBUF) & 1), spin);
    tc::fence_after();
    constexpr uint32_t id = tc::idesc_bf16(128, S::SLOT);
    if (pair) {
        issue_chain(d0, bd.ah + o, bd.al + o, bd.bh0 + o, bd.bl0 + o, S::KG, id);
        issue_chain(d1, bd.ah + o, bd.al + o, bd.bh1 + o, bd.bl1 + o, S::KG, id);
    } else {
        issue_chain(d0, bd.ah + o, bd.al + o, bd.bh0 + o, bd.bl0 + o, S::KP, id);
    }
    tc::commit(&done[b]);
    return ok;
}

// 8-byte copy that writes zeros instead when !valid (nothing is read then)
__device__ __forceinline__ void cp8z(void* dst, const void* src, bool valid)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory"); }

template <int R>
size_t front_tc_smem(const Geo& g, int NV)
{
    using S = Shape<R>;
    const size_t T = (size_t)1 << g.kH;
    size_t s = (size_t)NBUF * S::BUF +
               sizeof(float2) * ((size_t)g.kH * T * S::D2 + T * NV + T * R * R + (size_t)g.ra * T * NV) +
               sizeof(float) * ((size_t)NV * S::R4 + (size_t)g.kH * 2 * R * S::R4);
    return std::max<size_t>(s, 120 * 1024);  // one CTA per SM: the tile holds all 512 TMEM columns
}

template <int R>
size_t back_tc_smem(const Geo& g, int NU)
{
    using S = Shape<R>;
    const size_t T = (size_t)1 << g.kG;
    size_t s = (size_t)NBUF * S::BUF + sizeof(float2) * ((size_t)g.kG * T * S::D2 + T * NU + (size_t)g.ra * T * NU) +
               sizeof(float) * ((size_t)g.kG * 2 * R * S::R4 + (size_t)NU * S::R4);
    return std::max<size_t>(s, 120 * 1024);
}

// zero the B matrices of every operand buffer (their padding rows and K columns stay zero)
__device__ __forceinline__ void zero_B_regions(unsigned char* bufs, int BUF, int a_bytes, int b_bytes, int tid)
{
    for (int b = 0; b < NBUF; ++b) {
        uint4* p = reinterpret_cast<uint4*>(bufs + b * BUF + 2 * a_bytes);
        for (int i = tid; i < 4 * b_bytes / 16; i += kBuilders) p[i] = make_uint4(0, 0, 0, 0);
    }
}

// ------------------------------------------------------------------ front --
template <int R, int NV>
__global__ void __launch_bounds__(kTcThreads, 1) front_tc(TcArgs A)
{
    using S = Shape<R>;
    constexpr int R4 = S::R4;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_ready[NBUF], s_done[NBUF];
    const Geo& g = A.g;
    const int K = g.kH, T = 1 << K, ra = g.ra, mr = A.mr;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, qd = warp & 3, hw = (warp >> 2) & 1;
    const bool builder = warp < 8;
    const int row = 32 * qd + lane;
    const int slice = (int)(blockIdx.x % A.nslice);
    const int64_t tile = blockIdx.x / A.nslice;
    const int nP = 1 << g.l1;
    const int64_t p = tile & (nP - 1), c0 = tile >> g.l1;
    const int64_t nBh = (int64_t)1 << (g.L - g.h);
    const int64_t xi_base = c0 * T * NV;
    const int64_t N = g.N, P = g.P;

    unsigned char* bufs = smem;
    float2* EHs = reinterpret_cast<float2*>(smem + NBUF * S::BUF);  // [K][T][2R]
    float2* EVs = EHs + (size_t)K * T * S::D2;                      // [T*NV]
    float2* Ss = EVs + (size_t)T * NV;                              // [T][R*R] switch matrices
    float2* bks = Ss + (size_t)T * R * R;                           // [ra][T*NV] b_k on the tile's columns
    float* MvTs = reinterpret_cast<float*>(bks + (size_t)ra * T * NV); // [NV][R4]
    float* MHTs = MvTs + NV * R4;                                   // [K][2R][R4]

    if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) {
            tc::mbar_init(&s_ready[b], kBuilders);
            tc::mbar_init(&s_done[b], 1);
        }
    }
    stage_matrix(MvTs, A.MvT, NV, R, R4, tid);
    stage_matrix(MHTs, A.MHT, K * 2 * R, R, R4, tid);
    {
        const float2* ev = A.EV + p * N + xi_base;
        for (int e = tid; e < T * NV / 2; e += kTcThreads) cp16(EVs + 2 * e, ev + 2 * e);
        for (int k = 0; k < ra; ++k)
            for (int e = tid; e < T * NV / 2; e += kTcThreads) cp16(bks + k * T * NV + 2 * e, A.bk + k * N + xi_base + 2 * e);
        constexpr int RR2 = R * R / 2;
        for (int e = tid; e < T * RR2; e += kTcThreads) {
            const int lp = e / RR2, w = e - lp * RR2;
            cp16(Ss + lp * R * R + 2 * w, A.S + (((p << K) + lp) * nBh + c0) * R * R + 2 * w);
        }
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
    cp_commit();
    // F is staged per chunk of CS slots through the (still unused) operand buffers,
    // two chunks in flight: [CS * NV columns xi][mr right-hand sides]
    const int lmr = 31 - __clz(mr);
    const int slot_elems = NV * mr;
    int CS = T;
    while (CS > 2 && 2 * CS * slot_elems * (int)sizeof(float2) > NBUF * S::BUF) CS >>= 1;
    const int nch = T / CS;
    float2* Fst = reinterpret_cast<float2*>(bufs);
    auto issue_chunk = [&](int ch) {
        float2* dst = Fst + (ch & 1) * CS * slot_elems;
        const int64_t xi0 = xi_base + (int64_t)ch * CS * NV;
        for (int e = tid; e < CS * slot_elems; e += kBuilders) {
            const int xl = e >> lmr, c = e & (mr - 1);
            const int64_t col = (int64_t)slice * mr + c;
            const bool v = col < A.m;
            cp8z(dst + e, v ? A.F + (xi0 + xl) * A.m + col : A.F, v);
        }
        cp_commit();
    };
    if (builder) {
        issue_chunk(0);
        cp_wait<1>();
    } else {
        cp_wait<0>();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_tmem;
    const uint32_t tlane = tbase + ((uint32_t)(32 * qd) << 16);
    bool ok = true;

    if (!builder) {
        // ---------------- MMA issuer (one thread of warp 8)
        if (lane == 0) {
            BufDesc<R> bd;
            bd.init(bufs);
            int n = 0;
            for (int j = 1; j <= K; ++j)
                for (int grp = 0; grp < T / 2; ++grp) {
                    int s0, s1, lo0, lo1;
                    group_slots(K, j, grp, s0, s1, lo0, lo1);
                    ok = issuer_item<R>(s_ready, s_done, bd, n++, true, tbase + (uint32_t)(s0 * S::SLOT),
                                        tbase + (uint32_t)(s1 * S::SLOT), A.spin) && ok;
                }
            for (int lp = 0; lp < T; ++lp) {
                const int slot = (int)brev((unsigned)lp, K);
                ok = issuer_item<R>(s_ready, s_done, bd, n++, false, tbase + (uint32_t)(slot * S::SLOT), 0, A.spin) && ok;
            }
        }
    } else {
        // ---------------- builders: V (Eq. 1) into TMEM, F chunk by chunk
        {
            const int c = row / ra, k = row - c * ra;
            const float2* bkk = bks + k * T * NV;
            for (int ch = 0; ch < nch; ++ch) {
                if (ch + 1 < nch) {
                    issue_chunk(ch + 1);
                    cp_wait<1>();
                } else {
                    cp_wait<0>();
                }
                builders_sync();
                const float2* Fc = Fst + (ch & 1) * CS * slot_elems;
                for (int jj = hw; jj < CS; jj += 2) {
                    const int j = ch * CS + jj;
                    float v[S::D2];
#pragma unroll
                    for (int d = 0; d < S::D2; ++d) v[d] = 0.f;
#pragma unroll 4
                    for (int x = 0; x < NV; ++x) {
                        const float2 f = Fc[((jj * NV + x) << lmr) + c];
                        const float2 z = cmulf(EVs[j * NV + x], cmulf(bkk[j * NV + x], f));
                        const float* mv = MvTs + x * R4;
#pragma unroll
                        for (int t = 0; t < R; ++t) {
                            v[2 * t] = fmaf(mv[t], z.x, v[2 * t]);
                            v[2 * t + 1] = fmaf(mv[t], z.y, v[2 * t + 1]);
                        }
                    }
                    tc::st_dims<S::D2>(tlane + (uint32_t)(j * S::SLOT), v);
                }
                builders_sync();
            }
            tc::wait_st();
        }
        zero_B_regions(bufs, S::BUF, S::A_BYTES, S::B_BYTES, tid);
        tc::fence_before();
        builders_sync();
        tc::fence_after();

        BPipe bp;
        bp.n = 0;
        bp.ok = true;
        // ---- H levels (Eq. 2)
        for (int j = 1; j <= K; ++j) {
            const float* Mh = MHTs + (size_t)(j - 1) * 2 * R * R4;
            const float2* Pl = EHs + (size_t)(j - 1) * T * S::D2;
            for (int grp = 0; grp < T / 2; ++grp) {
                int s0, s1, lo0, lo1;
                group_slots(K, j, grp, s0, s1, lo0, lo1);
                unsigned char* buf = builders_begin(bufs, S::BUF, s_done, bp, grp == 0, A.spin);
                build_A_group<R>(buf, tlane, s0, s1, hw, row);
                build_B_group<R, 0>(buf, Mh, Pl + (size_t)lo0 * S::D2, Pl + (size_t)lo1 * S::D2, tid);
                builders_end(s_ready, bp);
            }
        }
        // ---- switch (step 4), one pair per item
        for (int lp = 0; lp < T; ++lp) {
            const int slot = (int)brev((unsigned)lp, K);
            unsigned char* buf = builders_begin(bufs, S::BUF, s_done, bp, lp == 0, A.spin);
            if (hw == 0) build_A_single<R>(buf, tlane, slot, row);
            build_B_switch<R>(buf, Ss + (size_t)lp * R * R, tid);
            builders_end(s_ready, bp);
        }
        builders_drain(s_done, bp, A.spin);
        ok = bp.ok;

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
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
    if (!ok) atomicExch(A.err, 3);
}

// ------------------------------------------------------------------- back --
template <int R, int NU>
__global__ void __launch_bounds__(kTcThreads, 1) back_tc(TcArgs A)
{
    using S = Shape<R>;
    constexpr int R4 = S::R4;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_ready[NBUF], s_done[NBUF];
    const Geo& g = A.g;
    const int K = g.kG, T = 1 << K, ra = g.ra, mr = A.mr;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, qd = warp & 3, hw = (warp >> 2) & 1;
    const bool builder = warp < 8;
    const int row = 32 * qd + lane;
    const int slice = (int)(blockIdx.x % A.nslice);
    const int64_t pp_x = blockIdx.x / A.nslice;  // x-node at level h
    const int nC = 1 << g.l1;
    const int64_t nBh = (int64_t)1 << (g.L - g.h);
    const int XN = T * NU;
    const int64_t N = g.N, P = g.P, x0g = pp_x * XN;

    unsigned char* bufs = smem;
    float2* FGs = reinterpret_cast<float2*>(smem + NBUF * S::BUF);  // [K][T][2R]
    float2* EUs = FGs + (size_t)K * T * S::D2;                      // [XN]
    float2* aks = EUs + XN;                                         // [ra][XN] a_k on the tile's rows
    float* MGTs = reinterpret_cast<float*>(aks + (size_t)ra * XN);  // [K][2][R][R4]
    float* MUs = MGTs + (size_t)K * 2 * R * R4;                     // [NU][R4]

    if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) {
            tc::mbar_init(&s_ready[b], kBuilders);
            tc::mbar_init(&s_done[b], 1);
        }
    }
    if (builder) zero_B_regions(bufs, S::BUF, S::A_BYTES, S::B_BYTES, tid);
    stage_matrix(MGTs, A.MGT, K * 2 * R, R, R4, tid);
    stage_matrix(MUs, A.MU, NU, R, R4, tid);
    for (int k = 0; k < ra; ++k)
        for (int e = tid; e < XN / 2; e += kTcThreads) cp16(aks + k * XN + 2 * e, A.ak + k * N + x0g + 2 * e);
    cp_commit_wait();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_tmem;
    const uint32_t tlane = tbase + ((uint32_t)(32 * qd) << 16);
    bool ok = true;

    if (!builder) {
        if (lane == 0) {
            BufDesc<R> bd;
            bd.init(bufs);
            int n = 0;
            for (int c0 = 0; c0 < nC; ++c0)
                for (int j = 1; j <= K; ++j)
                    for (int grp = 0; grp < T / 2; ++grp) {
                        int s0, s1, lo0, lo1;
                        group_slots(K, j, grp, s0, s1, lo0, lo1);
                        ok = issuer_item<R>(s_ready, s_done, bd, n++, true, tbase + (uint32_t)(s0 * S::SLOT),
                                            tbase + (uint32_t)(s1 * S::SLOT), A.spin) && ok;
                    }
        }
    } else {
        const int c = row / ra, k = row - c * ra;
        const int64_t cg = (int64_t)slice * mr + c;
        const bool valid = cg < A.m;
        const bool accum_old = A.beta != 0;
        const float2* akk = aks + k * XN;
        const float2* Win = A.W + (size_t)slice * P * 128 * R;
        BPipe bp;
        bp.n = 0;
        bp.ok = true;
        for (int c0 = 0; c0 < nC; ++c0) {
            // FG phases and EU of T_Omega node c0 (overlaps the W loads below)
            for (int jl = 1; jl <= K; ++jl) {
                const int64_t nBl = (int64_t)1 << (g.L - g.h - jl);
                const float2* fg = A.FG + (size_t)(jl - 1) * P * 2 * R;
                for (int e = tid; e < T * R; e += kBuilders) {
                    const int lp = e / R, w = e - lp * R;
                    const int64_t ap = (pp_x << jl) + (lp >> (K - jl));
                    const int64_t bq = ((int64_t)c0 << (K - jl)) + (lp & ((1 << (K - jl)) - 1));
                    cp16(FGs + ((size_t)(jl - 1) * T + lp) * 2 * R + 2 * w, fg + (ap * nBl + bq) * 2 * R + 2 * w);
                }
            }
            for (int e = tid; e < XN / 2; e += kBuilders) cp16(EUs + 2 * e, A.EU + (size_t)c0 * N + x0g + 2 * e);
            cp_commit();
            // switch-level pairs (pp_x, c0 T + j) -> TMEM slots j, two slots' loads in flight
            for (int j = hw; j < T; j += 4) {
                const bool two = j + 2 < T;
                const float4* src0 =
                    reinterpret_cast<const float4*>(Win + ((size_t)(pp_x * nBh + (int64_t)c0 * T + j) * 128 + row) * R);
                const float4* src1 = src0 + (two ? 2 * 128 * R / 2 : 0);
                float v0[S::D2], v1[S::D2];
#pragma unroll
                for (int i = 0; i < S::D2 / 4; ++i) {
                    const float4 a = __ldg(src0 + i);
                    v0[4 * i] = a.x; v0[4 * i + 1] = a.y; v0[4 * i + 2] = a.z; v0[4 * i + 3] = a.w;
                    const float4 b = __ldg(src1 + i);
                    v1[4 * i] = b.x; v1[4 * i + 1] = b.y; v1[4 * i + 2] = b.z; v1[4 * i + 3] = b.w;
                }
                tc::st_dims<S::D2>(tlane + (uint32_t)(j * S::SLOT), v0);
                if (two) tc::st_dims<S::D2>(tlane + (uint32_t)((j + 2) * S::SLOT), v1);
            }
            cp_wait<0>();
            tc::wait_st();
            tc::fence_before();
            builders_sync();
            tc::fence_after();

            // ---- G levels (Eq. 3)
            for (int j = 1; j <= K; ++j) {
                const float* Mg = MGTs + (size_t)(j - 1) * 2 * R * R4;
                const float2* Pl = FGs + (size_t)(j - 1) * T * S::D2;
                for (int grp = 0; grp < T / 2; ++grp) {
                    int s0, s1, lo0, lo1;
                    group_slots(K, j, grp, s0, s1, lo0, lo1);
                    unsigned char* buf = builders_begin(bufs, S::BUF, s_done, bp, grp == 0, A.spin);
                    build_A_group<R>(buf, tlane, s0, s1, hw, row);
                    build_B_group<R, 1>(buf, Mg, Pl + (size_t)lo0 * S::D2, Pl + (size_t)lo1 * S::D2, tid);
                    builders_end(s_ready, bp);
                }
            }
            builders_drain(s_done, bp, A.spin);

            // ---- U (Eq. bf3) of T_Omega node c0, summed over k, accumulated into this CTA's
            // rows of G; lane k of each column writes the rows i = k (mod r_alpha), all old
            // values loaded before any store
            const bool add_old = c0 > 0 || accum_old;
            for (int lp = hw; lp < T; lp += 2) {
                const int slot = (int)brev((unsigned)lp, K);
                float v[S::D2];
                tc::ld_dims<S::D2>(tlane + (uint32_t)(slot * S::SLOT), v);
                tc::wait_ld();
                float2 ctb[NU];
#pragma unroll
                for (int i = 0; i < NU; ++i) {
                    float2 w = make_float2(0.f, 0.f);
                    const float* mu = MUs + i * R4;
#pragma unroll
                    for (int s2 = 0; s2 < R; ++s2) {
                        w.x = fmaf(mu[s2], v[2 * s2], w.x);
                        w.y = fmaf(mu[s2], v[2 * s2 + 1], w.y);
                    }
                    float2 z = cmulf(cmulf(akk[lp * NU + i], EUs[lp * NU + i]), w);
                    for (int o = 1; o < ra; o <<= 1) {
                        z.x += __shfl_xor_sync(0xffffffffu, z.x, o);
                        z.y += __shfl_xor_sync(0xffffffffu, z.y, o);
                    }
                    ctb[i] = z;
                }
                if (valid) {
                    float2* gp = A.G + (x0g + lp * NU) * A.m + cg;
                    float2 old[NU];
#pragma unroll
                    for (int i = 0; i < NU; ++i)
                        old[i] = (add_old && (i & (ra - 1)) == k) ? gp[(int64_t)i * A.m] : make_float2(0.f, 0.f);
#pragma unroll
                    for (int i = 0; i < NU; ++i)
                        if ((i & (ra - 1)) == k) gp[(int64_t)i * A.m] = make_float2(ctb[i].x + old[i].x, ctb[i].y + old[i].y);
                }
            }
            tc::fence_before();
            builders_sync();
            tc::fence_after();
        }
        ok = bp.ok;
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
    if (!ok) atomicExch(A.err, 3);
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
