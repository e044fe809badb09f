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
//    2r x 2r block per output pair, built on the fly in shared memory from the
//    factored form (the real Lagrange matrix of the level times the pair's
//    phases) as its real embedding [[Re W, -Im W], [Im W, Re W]];
//  * the two output pairs of a group occupy adjacent slots (a "region"), so a
//    group is one MMA chain with N = 2 SLOT.  Two groups that read the same two
//    regions form a unit and write their outputs back over those regions (the
//    butterfly's radix-2 crossing), so the update stays in place: after level
//    j, logical slot s lives in region compress_{j-1}(s) (s with bit j-1
//    removed), half bit_{j-1}(s);
//  * operands are split x = hi + lo into BF16 (hi = bf16(x), lo = bf16(x - hi));
//    D = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 in TMEM by
//    tcgen05.mma (M = 128 rows, K = 16 per instruction), issued by one thread;
//  * 16 builder warps write operands into two double-buffered item buffers and
//    one issuer thread runs the MMAs; ready / done mbarriers hand items over.
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

constexpr int kBuilders = 512;                 // 16 builder warps
constexpr int kTcThreads = kBuilders + 32;     // + 1 MMA-issue warp
constexpr int NBUF = 2;                        // item buffers in flight

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
// 8-byte copy that writes zeros instead when !valid (nothing is read then)
__device__ __forceinline__ void cp8z(void* dst, const void* src, bool valid)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory"); }
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
    static constexpr int SLOT = D2 <= 16 ? 16 : 32;       // TMEM columns per pair
    static constexpr int NG = 2 * SLOT;                   // MMA N of a group: its two output pairs
    static constexpr int KS = (D2 + 7) / 8 * 8;           // K rows per input pair
    static constexpr int KG = 2 * KS;                     // K of a group MMA chain
    static constexpr int R4 = (R + 3) & ~3;
    static constexpr int SBO = (KG / 8) * 128;            // 8-row-group stride of A and B
    static constexpr int A_BYTES = 128 * KG * 2;          // one of A_hi / A_lo
    static constexpr int B_BYTES = NG * KG * 2;           // one of B_hi / B_lo
    static constexpr int GRP = 2 * A_BYTES + 2 * B_BYTES; // A_hi | A_lo | B_hi | B_lo of one group
    static constexpr int BUF = 2 * GRP;                   // one item: up to two groups
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
    return (row >> 3) * sbo + (k >> 3) * 128 + (row & 7) * 16;  // byte offset of the 8-value chunk of (row, k)
}

__device__ __forceinline__ void builders_sync() { asm volatile("bar.sync 1, 512;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::smem_u32(mbar)) : "memory");
}

// A of one group: this thread converts its row of one input pair (TMEM column
// tcol) into K columns [c KS, c KS + KS) of A_hi and A_lo (zero padded)
template <int R>
__device__ __forceinline__ void build_A(unsigned char* grp, uint32_t taddr, int c, int row)
{
    using S = Shape<R>;
    float v[S::KS];
#pragma unroll
    for (int d = S::D2; d < S::KS; ++d) v[d] = 0.f;
    tc::ld_dims<S::D2>(taddr, v);
    tc::wait_ld();
#pragma unroll
    for (int ch = 0; ch < S::KS / 8; ++ch) {
        uint4 h, l;
        tc::split2(v[8 * ch + 0], v[8 * ch + 1], h.x, l.x);
        tc::split2(v[8 * ch + 2], v[8 * ch + 3], h.y, l.y);
        tc::split2(v[8 * ch + 4], v[8 * ch + 5], h.z, l.z);
        tc::split2(v[8 * ch + 6], v[8 * ch + 7], h.w, l.w);
        const int off = opnd_off(row, c * S::KS + 8 * ch, S::SBO);
        *reinterpret_cast<uint4*>(grp + off) = h;
        *reinterpret_cast<uint4*>(grp + S::A_BYTES + off) = l;
    }
}

// One 16-byte chunk of B (hi and lo): B row n of the real embedding of four
// consecutive complex weights w[0..3] at K offset k0 (a multiple of 8).  Output
// component rho = 2t (real part of output t) holds (Re w, -Im w) per weight,
// rho = 2t + 1 (imaginary part) holds (Im w, Re w).
template <int R>
__device__ __forceinline__ void put_chunk(unsigned char* Bh, unsigned char* Bl, int n, int rho, int k0, const float2* w)
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
    const int off = opnd_off(n, k0, S::SBO);
    *reinterpret_cast<uint4*>(Bh + off) = h;
    *reinterpret_cast<uint4*>(Bl + off) = l;
}

// Items of the B of one group: (component rho, input pair c, chunk q, output pair s)
template <int R>
struct BItems {
    static constexpr int NQ = Shape<R>::KS / 8;
    static constexpr int N = Shape<R>::D2 * NQ * 4;
};

// B of a level group, item it of BItems: weights with s' >= r are the K padding.
// kind 0 (H, Eq. 2): W_s[t][(c, s')] = MH[t][c r + s'] * E_s[c][s'].
// kind 1 (G, Eq. 3): W_s[t][(c, s')] = FG_s[c][t] * MG_s[t][s'].
// kind 2 (switch):   W_s[t][(c, s')] = [c == s] S_s[t][s']  (two pairs, block diagonal).
template <int R, int KIND>
__device__ __forceinline__ void build_B_item(unsigned char* grp, int it, const float* Mt, const float2* P0,
                                             const float2* P1)
{
    using S = Shape<R>;
    constexpr int NQ = BItems<R>::NQ;
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
        w[e] = make_float2(0.f, 0.f);
        if (sp < R) {
            if (KIND == 0) {
                const float mv = Mt[(c * R + sp) * S::R4 + t];
                const float2 ph = Pp[c * R + sp];
                w[e] = make_float2(mv * ph.x, mv * ph.y);
            } else if (KIND == 1) {
                const float mv = Mt[(s * R + sp) * S::R4 + t];
                const float2 ph = Pp[c * R + t];
                w[e] = make_float2(mv * ph.x, mv * ph.y);
            } else if (c == s) {
                w[e] = Pp[t * R + sp];
            }
        }
    }
    unsigned char* Bh = grp + 2 * S::A_BYTES;
    put_chunk<R>(Bh, Bh + S::B_BYTES, s * S::SLOT + rho, rho, c * S::KS + 8 * q, w);
}

// ----------------------------------------------------------- schedule ----
// One pass over a tile of T = 2^K pairs: levels j = 1..K, then (front only) the
// switch as pass j = K + 1.  A pass has T / (2 UG) items ("units") of UG groups
// (UG = 2, or 1 when T = 2).  Physical slot of logical slot s after level j >= 1
// (and before level 1): 2 compress_{j-1}(s) + bit_{j-1}(s); level j >= 2 unit
// (hi, lo) reads regions R1 = (hi << (j-1)) | lo and R2 = R1 | 2^{j-2}; its
// group g takes half g of both and writes region g ? R2 : R1.
struct UnitGroup {
    int src0, src1;  // physical slots of input pairs c = 0, 1
    int dst;         // region written (physical slots 2 dst, 2 dst + 1)
    int p0, p1;      // output pairs' phase rows (levels) or logical pairs (switch)
};

__device__ __forceinline__ UnitGroup unit_group(int K, int j, int UG, int u, int g)
{
    UnitGroup G;
    if (j == 1 || j == K + 1) {
        const int rg = UG * u + g;
        G.src0 = 2 * rg;
        G.src1 = 2 * rg + 1;
        G.dst = rg;
        if (j == 1) {
            G.p0 = rg;
            G.p1 = (1 << (K - 1)) + rg;
        } else {
            G.p0 = (int)brev((unsigned)rg, K);
            G.p1 = G.p0 + 1;
        }
    } else {
        const int lo = u & ((1 << (j - 2)) - 1), hi = u >> (j - 2);
        const int R1 = (hi << (j - 1)) | lo, R2 = R1 | (1 << (j - 2));
        G.src0 = 2 * R1 + g;
        G.src1 = 2 * R2 + g;
        G.dst = g ? R2 : R1;
        const int a = (int)brev((unsigned)lo, j - 1) + g, half = 1 << (K - j);
        G.p0 = (2 * a) * half + hi;
        G.p1 = (2 * a + 1) * half + hi;
    }
    return G;
}

// unit of pass j that wrote region R
__device__ __forceinline__ int region_writer(int j, int UG, int R)
{
    if (j == 1) return R / UG;
    return ((R >> (j - 1)) << (j - 2)) | (R & ((1 << (j - 2)) - 1));
}

// latest unit of pass j - 1 whose output unit u of pass j reads (-1: none)
__device__ __forceinline__ int unit_dep(int K, int j, int UG, int u)
{
    if (j == 1) return -1;
    int dep = -1;
    for (int g = 0; g < UG; ++g) {
        const UnitGroup G = unit_group(K, j, UG, u, g);
        dep = max(dep, region_writer(j - 1, UG, G.src0 >> 1));
        dep = max(dep, region_writer(j - 1, UG, G.src1 >> 1));
    }
    return dep;
}

// physical slot of logical slot s after the last level K
__device__ __forceinline__ int phys_final(int K, int s)
{
    return 2 * (s & ((1 << (K - 1)) - 1)) + (s >> (K - 1));
}

// ----------------------------------------------------------- hand-over ---
// completion of item i (buffer i % NBUF, its (i / NBUF)-th use).  Callers wait
// only for i >= n - NBUF (n = item about to be built), so the barrier is at most
// one phase past the awaited one.
__device__ __forceinline__ bool wait_item(uint64_t* done, int i, long long spin)
{
    if (i < 0) return true;
    const bool ok = tc::mbar_wait(&done[i % NBUF], (uint32_t)((i / NBUF) & 1), spin);
    tc::fence_after();
    return ok;
}

// every builder thread makes its operand writes (and its TMEM reads) visible,
// then one lane per warp arrives: ready[] counts warps
__device__ __forceinline__ void publish(uint64_t* ready, int n)
{
    tc::fence_async_smem();
    tc::fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&ready[n % NBUF]);
}

template <int R>
struct BufDesc {
    uint64_t ah, al, bh, bl;  // group 0 of buffer 0; group g of buffer b adds (b BUF + g GRP) / 16
    __device__ void init(const unsigned char* buf)
    {
        using S = Shape<R>;
        ah = tc::desc(buf, 128, S::SBO);
        al = tc::desc(buf + S::A_BYTES, 128, S::SBO);
        bh = tc::desc(buf + 2 * S::A_BYTES, 128, S::SBO);
        bl = tc::desc(buf + 2 * S::A_BYTES + S::B_BYTES, 128, S::SBO);
    }
};

// D(d_tmem) = A_hi B_hi + A_hi B_lo + A_lo B_hi over K; a k-step adds 256 bytes (16 in the address field)
__device__ __forceinline__ void issue_chain(uint32_t d_tmem, uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl, int K,
                                            uint32_t idesc)
{
    const int nks = K / 16;
    for (int ks = 0; ks < nks; ++ks) tc::mma_bf16(d_tmem, ah + 16 * ks, bh + 16 * ks, idesc, ks > 0);
    for (int ks = 0; ks < nks; ++ks) tc::mma_bf16(d_tmem, ah + 16 * ks, bl + 16 * ks, idesc, 1);
    for (int ks = 0; ks < nks; ++ks) tc::mma_bf16(d_tmem, al + 16 * ks, bh + 16 * ks, idesc, 1);
}

// issuer: for every item of passes 1..npass (shared addresses stay below 2^18,
// so descriptor offsets add without carry)
template <int R>
__device__ __forceinline__ bool issue_passes(uint64_t* ready, uint64_t* done, const BufDesc<R>& bd, int& n, int K,
                                             int npass, int UG, uint32_t tbase, long long spin)
{
    using S = Shape<R>;
    constexpr uint32_t id = tc::idesc_bf16(128, S::NG);
    const int nunit = (1 << K) / (2 * UG);
    bool ok = true;
    for (int j = 1; j <= npass; ++j)
        for (int u = 0; u < nunit; ++u, ++n) {
            const int b = n % NBUF;
            ok = tc::mbar_wait(&ready[b], (uint32_t)((n / NBUF) & 1), spin) && ok;
            tc::fence_after();
            for (int g = 0; g < UG; ++g) {
                const UnitGroup G = unit_group(K, j, UG, u, g);
                const uint64_t o = (uint64_t)((b * S::BUF + g * S::GRP) >> 4);
                issue_chain(tbase + (uint32_t)(G.dst * S::NG), bd.ah + o, bd.al + o, bd.bh + o, bd.bl + o, S::KG, id);
            }
            tc::commit(&done[b]);
        }
    return ok;
}

// builders: operands of every item of passes 1..npass; KIND of levels 0 (H) / 1 (G),
// the switch pass (j = K + 1) uses the pairs' switch matrices Ss[lp][R * R]
template <int R, int KIND>
__device__ __forceinline__ bool build_passes(unsigned char* bufs, uint64_t* ready, uint64_t* done, int& n, int K,
                                             int npass, int UG, uint32_t tlane, const float* Mlev, const float2* Plev,
                                             const float2* Ss, int tid, int row, int role, long long spin)
{
    using S = Shape<R>;
    constexpr int R4 = S::R4;
    const int T = 1 << K, nunit = T / (2 * UG);
    const int ga = role >> 1, ca = role & 1;  // this warp's A work: group ga, input pair ca
    bool ok = true;
    const int n0 = n;
    for (int j = 1; j <= npass; ++j) {
        const bool sw = j == K + 1;
        const float* Mt = Mlev + (size_t)(j - 1) * 2 * R * R4;
        const float2* Pl = Plev + (size_t)(j - 1) * T * S::D2;
        for (int u = 0; u < nunit; ++u, ++n) {
            // the weights need only a free buffer: build them while the MMAs this
            // item's data depends on may still run
            ok = wait_item(done, n - NBUF, spin) && ok;
            unsigned char* buf = bufs + (n % NBUF) * S::BUF;
            for (int it = tid; it < UG * BItems<R>::N; it += kBuilders) {
                const int g = it >= BItems<R>::N;
                const UnitGroup G = unit_group(K, j, UG, u, g);
                unsigned char* grp = buf + g * S::GRP;
                if (sw)
                    build_B_item<R, 2>(grp, it - g * BItems<R>::N, nullptr, Ss + (size_t)G.p0 * R * R,
                                       Ss + (size_t)G.p1 * R * R);
                else
                    build_B_item<R, KIND>(grp, it - g * BItems<R>::N, Mt, Pl + (size_t)G.p0 * S::D2,
                                          Pl + (size_t)G.p1 * S::D2);
            }
            const int dep = unit_dep(K, j, UG, u);
            if (dep >= 0) ok = wait_item(done, max(n0 + (j - 2) * nunit + dep, n - NBUF), spin) && ok;
            if (ga < UG) {
                const UnitGroup G = unit_group(K, j, UG, u, ga);
                build_A<R>(buf + ga * S::GRP, tlane + (uint32_t)((ca ? G.src1 : G.src0) * S::SLOT), ca, row);
            }
            publish(ready, n);
        }
    }
    ok = wait_item(done, n - 1, spin) && ok;  // drain: one commit covers every earlier MMA
    return ok;
}

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

// zero the B matrices of every group of every item buffer (padding rows and K columns stay zero)
template <int R>
__device__ __forceinline__ void zero_B(unsigned char* bufs, int tid)
{
    using S = Shape<R>;
    constexpr int n16 = 2 * S::B_BYTES / 16;
    for (int i = tid; i < NBUF * 2 * n16; i += kBuilders) {
        const int gb = i / n16, e = i - gb * n16;
        reinterpret_cast<uint4*>(bufs + gb * S::GRP + 2 * S::A_BYTES)[e] = make_uint4(0, 0, 0, 0);
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
    const int K = g.kH, T = 1 << K, ra = g.ra, mr = A.mr, UG = T >= 4 ? 2 : 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, qd = warp & 3, role = (warp >> 2) & 3;
    const bool builder = warp < kBuilders / 32;
    const int row = 32 * qd + lane;
    const int slice = (int)(blockIdx.x % A.nslice);
    const int64_t tile = blockIdx.x / A.nslice;
    const int nP = 1 << g.l1;
    const int64_t p = tile & (nP - 1), c0 = tile >> g.l1;
    const int64_t nBh = (int64_t)1 << (g.L - g.h);
    const int64_t xi_base = c0 * T * NV;
    const int64_t N = g.N, P = g.P;

    unsigned char* bufs = smem;
    float2* EHs = reinterpret_cast<float2*>(smem + NBUF * S::BUF);    // [K][T][2R]
    float2* EVs = EHs + (size_t)K * T * S::D2;                        // [T*NV]
    float2* Ss = EVs + (size_t)T * NV;                                // [T][R*R] switch matrices
    float2* bks = Ss + (size_t)T * R * R;                             // [ra][T*NV] b_k on the tile's columns
    float* MvTs = reinterpret_cast<float*>(bks + (size_t)ra * T * NV); // [NV][R4]
    float* MHTs = MvTs + NV * R4;                                     // [K][2R][R4]

    if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
    if (tid == 0) {
        for (int b = 0; b < NBUF; ++b) {
            tc::mbar_init(&s_ready[b], kBuilders / 32);
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
    // F is staged per chunk of CS slots through the (still unused) item buffers,
    // two chunks in flight: [CS * NV columns xi][mr right-hand sides]
    const int lmr = 31 - __clz(mr);
    const int slot_elems = NV * mr;
    int CS = T;
    while (CS > 1 && 2 * CS * slot_elems * (int)sizeof(float2) > NBUF * S::BUF) CS >>= 1;
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
    int n = 0;

    if (!builder) {
        // ---------------- MMA issuer (one thread of the last warp): H levels, then the switch
        if (lane == 0) {
            BufDesc<R> bd;
            bd.init(bufs);
            ok = issue_passes<R>(s_ready, s_done, bd, n, K, K + 1, UG, tbase, A.spin);
        }
    } else {
        // ---------------- builders: V (Eq. 1) into TMEM slot j, F chunk by chunk
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
                for (int jj = role; jj < CS; jj += 4) {
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
        zero_B<R>(bufs, tid);
        tc::fence_before();
        builders_sync();
        tc::fence_after();

        // ---- H levels (Eq. 2) and the switch (step 4)
        ok = build_passes<R, 0>(bufs, s_ready, s_done, n, K, K + 1, UG, tlane, MHTs, EHs, Ss, tid, row, role, A.spin);

        // ---- write the switch-level coefficients: W[slice][q][row][R]
        float2* Wout = A.W + (size_t)slice * P * 128 * R;
        for (int lp = role; lp < T; lp += 4) {
            const int slot = phys_final(K, (int)brev((unsigned)lp, K));
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
    const int K = g.kG, T = 1 << K, ra = g.ra, mr = A.mr, UG = T >= 4 ? 2 : 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, qd = warp & 3, role = (warp >> 2) & 3;
    const bool builder = warp < kBuilders / 32;
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
            tc::mbar_init(&s_ready[b], kBuilders / 32);
            tc::mbar_init(&s_done[b], 1);
        }
    }
    if (builder) zero_B<R>(bufs, tid);
    stage_matrix(MGTs, A.MGT, K * 2 * R, R, R4, tid);
    stage_matrix(MUs, A.MU, NU, R, R4, tid);
    for (int k = 0; k < ra; ++k)
        for (int e = tid; e < XN / 2; e += kTcThreads) cp16(aks + k * XN + 2 * e, A.ak + k * N + x0g + 2 * e);
    cp_commit();
    cp_wait<0>();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = s_tmem;
    const uint32_t tlane = tbase + ((uint32_t)(32 * qd) << 16);
    bool ok = true;
    int n = 0;

    if (!builder) {
        if (lane == 0) {
            BufDesc<R> bd;
            bd.init(bufs);
            for (int c0 = 0; c0 < nC; ++c0) ok = issue_passes<R>(s_ready, s_done, bd, n, K, K, UG, tbase, A.spin) && ok;
        }
    } else {
        const int c = row / ra, k = row - c * ra;
        const int64_t cg = (int64_t)slice * mr + c;
        const bool valid = cg < A.m;
        const float2* akk = aks + k * XN;
        const float2* Win = A.W + (size_t)slice * P * 128 * R;
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
            // switch-level pairs (pp_x, c0 T + j) -> TMEM slot j, two slots' loads in flight
            for (int j = role; j < T; j += 8) {
                const bool two = j + 4 < T;
                const float4* src0 =
                    reinterpret_cast<const float4*>(Win + ((size_t)(pp_x * nBh + (int64_t)c0 * T + j) * 128 + row) * R);
                const float4* src1 = src0 + (two ? 4 * 128 * R / 2 : 0);
                float v0[S::D2], v1[S::D2];
#pragma unroll
                for (int i = 0; i < S::D2 / 4; ++i) {
                    const float4 a = __ldg(src0 + i);
                    v0[4 * i] = a.x; v0[4 * i + 1] = a.y; v0[4 * i + 2] = a.z; v0[4 * i + 3] = a.w;
                    const float4 b = __ldg(src1 + i);
                    v1[4 * i] = b.x; v1[4 * i + 1] = b.y; v1[4 * i + 2] = b.z; v1[4 * i + 3] = b.w;
                }
                tc::st_dims<S::D2>(tlane + (uint32_t)(j * S::SLOT), v0);
                if (two) tc::st_dims<S::D2>(tlane + (uint32_t)((j + 4) * S::SLOT), v1);
            }
            cp_wait<0>();
            tc::wait_st();
            tc::fence_before();
            builders_sync();
            tc::fence_after();

            // ---- G levels (Eq. 3), drained
            ok = build_passes<R, 1>(bufs, s_ready, s_done, n, K, K, UG, tlane, MGTs, FGs, nullptr, tid, row, role,
                                    A.spin) && ok;

            // ---- U (Eq. bf3) of T_Omega node c0, summed over k, accumulated into this CTA's
            // rows of G; lane k of each column writes the rows i = k (mod r_alpha); the old
            // values are loaded before the arithmetic that hides their latency
            const bool add_old = c0 > 0 || A.beta != 0;
            for (int lp = role; lp < T; lp += 4) {
                const int slot = phys_final(K, (int)brev((unsigned)lp, K));
                float v[S::D2];
                tc::ld_dims<S::D2>(tlane + (uint32_t)(slot * S::SLOT), v);
                tc::wait_ld();
                float2* gp = A.G + (x0g + lp * NU) * A.m + cg;
#pragma unroll
                for (int h2 = 0; h2 < NU; h2 += 8) {
                    float2 old[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        old[i] = (valid && add_old && ((h2 + i) & (ra - 1)) == k) ? gp[(int64_t)(h2 + i) * A.m]
                                                                                   : make_float2(0.f, 0.f);
                    float2 ctb[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float2 w = make_float2(0.f, 0.f);
                        const float* mu = MUs + (h2 + i) * R4;
#pragma unroll
                        for (int s2 = 0; s2 < R; ++s2) {
                            w.x = fmaf(mu[s2], v[2 * s2], w.x);
                            w.y = fmaf(mu[s2], v[2 * s2 + 1], w.y);
                        }
                        float2 z = cmulf(cmulf(akk[lp * NU + h2 + i], EUs[lp * NU + h2 + i]), w);
                        for (int o = 1; o < ra; o <<= 1) {
                            z.x += __shfl_xor_sync(0xffffffffu, z.x, o);
                            z.y += __shfl_xor_sync(0xffffffffu, z.y, o);
                        }
                        ctb[i] = z;
                    }
                    if (valid) {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (((h2 + i) & (ra - 1)) == k)
                                gp[(int64_t)(h2 + i) * A.m] = make_float2(ctb[i].x + old[i].x, ctb[i].y + old[i].y);
                    }
                }
            }
            tc::fence_before();
            builders_sync();
            tc::fence_after();
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
    if (!ok) atomicExch(A.err, 3);
}

template <int R, int NV>
cudaError_t launch_tc_rn(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws, int* err,
                         cudaStream_t st)
{
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

// leaf groups of V and U: 16 indices (the first level with more than r indices, r <= 12) or
// 32 (V and U one level higher, plans built with a larger l1)
template <int R>
cudaError_t launch_tc_r(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws, int* err,
                        cudaStream_t st)
{
    if (B.g.nv == 16) return launch_tc_rn<R, 16>(B, F, m, G, beta, ws, err, st);
    if (B.g.nv == 32) return launch_tc_rn<R, 32>(B, F, m, G, beta, ws, err, st);
    return cudaErrorNotSupported;
}

}  // namespace

bool tc_supported(const Geo& g, const char** why)
{
    const int r = g.r;
    if (r != 8 && r != 10 && r != 12) {
        if (why) *why = "split-BF16 kernels are built for r = 8, 10, 12";
        return false;
    }
    if (g.nv != 16 && g.nv != 32) {
        if (why) *why = "split-BF16 kernels need V and U leaf groups of 16 or 32 indices";
        return false;
    }
    if (g.ra != 1 && g.ra != 2 && g.ra != 4) {
        if (why) *why = "split-BF16 kernels need an amplitude rank of 1, 2 or 4";
        return false;
    }
    if (g.kH < 1 || g.kG < 1) {
        if (why) *why = "split-BF16 kernels need at least one H and one G level";
        return false;
    }
    const int slot = 2 * r <= 16 ? 16 : 32;
    const int T = 1 << (g.kH > g.kG ? g.kH : g.kG);
    if (T * slot > 512) {
        if (why) *why = "tile does not fit tensor memory (2^kH or 2^kG pairs x TMEM columns per pair > 512); use a "
                        "larger tolerance (r = 8) or V and U one level higher (bf_options.l1)";
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
