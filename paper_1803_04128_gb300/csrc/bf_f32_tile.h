// Tile bodies of the fused FP32 apply, shared by the kernels that read the
// phase tables (bf_kernels_f32.cu) and those that evaluate the phases
// themselves (bf_kernels_otf.cu).
//
// Fused FP32 apply of one sub-BF in two launches.
//
// Front pass (one CTA per tile x column slice): reads 2^kH consecutive
// xi-leaves of F, applies V (Eq. 1), all kH H levels (Eq. 2) and the switch
// (step 4 of Algorithm 4.1) with the coefficients held in shared memory, and
// writes the switch-level coefficients.  A front tile is fixed by an x-node p
// at level l1 and a chunk c0 of T_Omega nodes: its 2^kH pairs stay closed
// under the kH H levels because the pair (A, B) at level l only depends on
// (parent(A), children(B)) at level l-1 (Sec. 4).
//
// Back pass (one CTA per x-node p' at level h x column slice): loops over the
// 2^l1 chunks c0' of T_Omega nodes; for each, loads 2^kG switch-level pairs,
// applies the kG G levels (Eq. 3), and accumulates the U stage (Eq. bf3) of
// its 2^kG x-leaves in shared memory; finally multiplies by a_k and sums the
// amplitude terms (Eq. tg) into G.
//
// Inside a tile the levels run in place: after level j the coefficients of
// the logical pair [a: j bits][b: K-j bits] live in slot b * 2^j + rev_j(a),
// so every group of two pairs reads and writes the same two slots.
//
// Columns: a tile carries CT = r_alpha * mr live columns, col = k * mr + c
// (amplitude term k, right-hand side slice * mr + c), padded to CTp, a power
// of two, so that a thread's column is tid & (CTp - 1).  Global state between
// the passes: W[slice][q][t][CTp] (q = switch-level pair index).
//
// Every tile input (factor phases, Lagrange matrices, the F rows, b_k) is
// staged into shared memory with cp.async in one commit group before use.
#pragma once

#include "bf_device.h"
#include "bf_fused.h"

namespace bfi {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ void cfmaf(float2& acc, float2 a, float2 b)
{
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
// acc += w v for a real weight and a complex value as one packed two-lane FMA: the same two
// IEEE fused multiply-adds as two fmaf calls (bitwise the same), in one issue slot
__device__ __forceinline__ void rcfma(float2& acc, float w, float2 v)
{
    asm("{\n.reg .b64 wa, vb, ac;\nmov.b64 wa, {%2, %2};\nmov.b64 vb, {%3, %4};\nmov.b64 ac, {%0, %1};\n"
        "fma.rn.f32x2 ac, wa, vb, ac;\nmov.b64 {%0, %1}, ac;\n}"
        : "+f"(acc.x), "+f"(acc.y)
        : "f"(w), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ unsigned brev(unsigned v, int bits)
{
    return bits == 0 ? 0u : (__brev(v) >> (32 - bits));
}

// ---- cp.async (16- and 8-byte, the latter with zero fill) ----
__device__ __forceinline__ void cp16(void* dst, const void* src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp8(void* dst, const void* src, bool valid)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    int n = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most 0 / 1 of this thread's committed groups are still pending
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ---- phases evaluated in the kernel (Geo::otf; the layout is in OtfPhase) ----
// All phase arithmetic is mod 1 in units of 2^-32 turns (unsigned wrap-around),
// and all indices fit in 32 bits (Ng <= 2^30).  Every table entry is a signed
// sum of Phi at grid points in which, for the built-in kinds, the rho_i and
// xi^2 terms of a row or column that appears twice cancel, so each entry needs
// one integer residue and one product kappa |xi| (below, of kappa differences
// or |xi| differences, which wrap exactly mod 2^64).
struct OtfRow {
    unsigned R;            // round(frac(rho_i) 2^32)
    unsigned long long K;  // frac(kappa_i) 2^64
};
__device__ __forceinline__ OtfRow otf_row(const OtfPhase& o, int il)
{
    const uint4 w = __ldg(o.rows + (unsigned)(o.row0 + il));
    return OtfRow{w.z, ((unsigned long long)w.y << 32) | w.x};
}
__device__ __forceinline__ int otf_xi(const OtfPhase& o, int jl) { return o.col0 + jl - o.half; }
// K a 2^-64 mod 1 in 2^-32 turns, rounded, for |a| < 2^31: the low word of K
// times a (64-bit, plus the rounding half) and the high word times a (low 32
// bits); a negative a, taken as 2^32 + a, adds K_lo to the result, removed again.
__device__ __forceinline__ unsigned otf_kmul(unsigned long long K, int a)
{
    const unsigned ua = (unsigned)a, klo = (unsigned)K, khi = (unsigned)(K >> 32);
    const unsigned long long p = (unsigned long long)klo * ua + 0x80000000ull;
    const unsigned v = (unsigned)(p >> 32) + khi * ua;
    return a < 0 ? v - klo : v;
}
// (i xi mod Ng) / Ng, or 0 without the x xi term (linear in each argument)
__device__ __forceinline__ unsigned otf_ixi(const OtfPhase& o, int i, int xi)
{
    return o.sh1 >= 0 ? ((unsigned)i * (unsigned)xi) << o.sh1 : 0u;
}
// (xi^2 mod 4Ng) / (4Ng), or 0 without the xi^2 term
__device__ __forceinline__ unsigned otf_sq(const OtfPhase& o, int xi)
{
    return o.sh2 >= 0 ? ((unsigned)xi * (unsigned)xi) << o.sh2 : 0u;
}
// Phi(x_i, xi_j) mod 1 for block-local (i, j)
__device__ __forceinline__ unsigned otf_turns(const OtfPhase& o, int il, int jl)
{
    const OtfRow w = otf_row(o, il);
    const int xi = otf_xi(o, jl);
    return w.R + otf_ixi(o, o.row0 + il, xi) + otf_sq(o, xi) + otf_kmul(w.K, abs(xi));
}
// Phi(x_a, xi) - Phi(x_b, xi) (block-local rows a, b; column jl):
// rho_a - rho_b + (a - b) xi / Ng + (kappa_a - kappa_b) |xi|
__device__ __forceinline__ unsigned otf_rowdiff(const OtfPhase& o, int a, int b, int jl)
{
    const OtfRow wa = otf_row(o, a), wb = otf_row(o, b);
    const int xi = otf_xi(o, jl);
    return (wa.R - wb.R) + otf_ixi(o, a - b, xi) + otf_kmul(wa.K - wb.K, abs(xi));
}
// Phi(x_i, xi_c) - Phi(x_i, xi_d) (block-local row il; columns c, d):
// i (c - d) / Ng + kappa_i (|xi_c| - |xi_d|) + the xi^2 terms
__device__ __forceinline__ unsigned otf_coldiff(const OtfPhase& o, int il, int c, int d)
{
    const OtfRow w = otf_row(o, il);
    const int xc = otf_xi(o, c), xd = otf_xi(o, d);
    return otf_ixi(o, o.row0 + il, xc - xd) + otf_kmul(w.K, abs(xc) - abs(xd)) + (otf_sq(o, xc) - otf_sq(o, xd));
}
// e^{2 pi i t 2^-32}.  t is split into the nearest quarter turn q and a rest of
// at most 1/8 turn, theta in [-pi/4, pi/4]; cos and sin of theta are their Taylor
// series about 0 up to theta^10 and theta^9 (remainders below 1.2e-10 and 2e-9
// at |theta| = pi/4), then rotated by q quarter turns.
__device__ __forceinline__ float2 otf_exp(unsigned t)
{
    const unsigned q = (t + 0x20000000u) >> 30;
    const float th = (float)(int)(t - (q << 30)) * 1.46291807926715968e-9f;  // 2 pi 2^-32
    const float x2 = th * th;
    float sn = fmaf(x2, 2.75573192e-6f, -1.98412698e-4f);  // 1/9!, -1/7!
    sn = fmaf(x2, sn, 8.33333333e-3f);                     // 1/5!
    sn = fmaf(x2, sn, -1.66666667e-1f);                    // -1/3!
    sn = fmaf(x2 * th, sn, th);
    float cs = fmaf(x2, -2.75573192e-7f, 2.48015873e-5f);  // -1/10!, 1/8!
    cs = fmaf(x2, cs, -1.38888889e-3f);                    // -1/6!
    cs = fmaf(x2, cs, 4.16666667e-2f);                     // 1/4!
    cs = fmaf(x2, cs, -0.5f);
    cs = fmaf(x2, cs, 1.0f);
    float c = (q & 1) ? -sn : cs, s = (q & 1) ? cs : sn;
    if (q & 2) {
        c = -c;
        s = -s;
    }
    return make_float2(c, s);
}
__device__ __forceinline__ const int* otf_grid(const OtfPhase& o, int n)  // node of n = 2^e points
{
    return o.grids + (31 - __clz(n)) * 16;
}
__device__ __forceinline__ int centre_of(int start, int n) { return start + (n - 1) / 2; }

// real rows x cols matrix (row-major, global) -> shared rows padded to c4 floats, 8-byte copies
__device__ __forceinline__ void stage_matrix(float* dst, const float* src, int rows, int cols, int c4, int tid)
{
    const int half = cols / 2;
    for (int e = tid; e < rows * half; e += kThreads) {
        const int rr = e / half, cc = e - rr * half;
        cp8(dst + rr * c4 + 2 * cc, src + rr * cols + 2 * cc, true);
    }
}

// pair index of (a, b) of column slice sl in the workspace layout w
__device__ __forceinline__ int64_t w_pair(const WLayout& w, int64_t a, int64_t b, int sl)
{
    const int64_t d = a >> w.la, s = b >> w.lb;
    return d * w.sD + s * w.sS + sl * w.slice + ((a - (d << w.la)) << w.lb) + (b - (s << w.lb));
}

template <int R>
struct Pad4 {
    static constexpr int v = (R + 3) & ~3;
};

// H level (Eq. 2) on one (group, column): two inputs -> two outputs in place.
template <int R>
__device__ __forceinline__ void h_item(float2* x0, float2* x1, int CTp, const float2* E0, const float2* E1,
                                       const float* Mh)
{
    constexpr int R4 = Pad4<R>::v;
    float2 lam[2 * R];
#pragma unroll
    for (int s = 0; s < R; ++s) {
        lam[s] = x0[s * CTp];
        lam[R + s] = x1[s * CTp];
    }
    float2 o0[R], o1[R];
#pragma unroll
    for (int t = 0; t < R; ++t) o0[t] = o1[t] = make_float2(0.f, 0.f);
#pragma unroll
    for (int cs2 = 0; cs2 < R; ++cs2) {
        const float4 e0 = reinterpret_cast<const float4*>(E0)[cs2];
        const float4 e1 = reinterpret_cast<const float4*>(E1)[cs2];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            const int cs = 2 * cs2 + h2;
            const float2 u0 = cmulf(h2 ? make_float2(e0.z, e0.w) : make_float2(e0.x, e0.y), lam[cs]);
            const float2 u1 = cmulf(h2 ? make_float2(e1.z, e1.w) : make_float2(e1.x, e1.y), lam[cs]);
            const float4* mh = reinterpret_cast<const float4*>(Mh + cs * R4);
#pragma unroll
            for (int t4 = 0; t4 < R4 / 4; ++t4) {
                const float4 w = mh[t4];
                const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = 4 * t4 + q;
                    if (t < R) {
                        rcfma(o0[t], ww[q], u0);
                        rcfma(o1[t], ww[q], u1);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < R; ++t) {
        x0[t * CTp] = o0[t];
        x1[t * CTp] = o1[t];
    }
}

// G level (Eq. 3) on one (group, column): nu_pos = sum_c FG[pos][c] (MG[pos] nu_c).
template <int R>
__device__ __forceinline__ void g_item(float2* x0, float2* x1, int CTp, const float2* F0, const float2* F1,
                                       const float* Mg)
{
    constexpr int R4 = Pad4<R>::v;
    float2 nu0[R], nu1[R];
#pragma unroll
    for (int s = 0; s < R; ++s) {
        nu0[s] = x0[s * CTp];
        nu1[s] = x1[s * CTp];
    }
#pragma unroll
    for (int pos = 0; pos < 2; ++pos) {
        float2 w0[R], w1[R];
#pragma unroll
        for (int t = 0; t < R; ++t) w0[t] = w1[t] = make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < R; ++s) {
            const float4* mg = reinterpret_cast<const float4*>(Mg + (pos * R + s) * R4);
#pragma unroll
            for (int t4 = 0; t4 < R4 / 4; ++t4) {
                const float4 w = mg[t4];
                const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = 4 * t4 + q;
                    if (t < R) {
                        rcfma(w0[t], ww[q], nu0[s]);
                        rcfma(w1[t], ww[q], nu1[s]);
                    }
                }
            }
        }
        const float2* Fp = pos ? F1 : F0;  // [c][t]
        float2* xo = pos ? x1 : x0;
#pragma unroll
        for (int t2 = 0; t2 < R / 2; ++t2) {
            const float4 fa = reinterpret_cast<const float4*>(Fp)[t2];
            const float4 fb = reinterpret_cast<const float4*>(Fp + R)[t2];
            float2 o = cmulf(make_float2(fa.x, fa.y), w0[2 * t2]);
            cfmaf(o, make_float2(fb.x, fb.y), w1[2 * t2]);
            xo[(2 * t2) * CTp] = o;
            float2 o2 = cmulf(make_float2(fa.z, fa.w), w0[2 * t2 + 1]);
            cfmaf(o2, make_float2(fb.z, fb.w), w1[2 * t2 + 1]);
            xo[(2 * t2 + 1) * CTp] = o2;
        }
    }
}

// Switch blocks (step 4 of Algorithm 4.1) of the T = 2^K pairs (x-node (p << K) + lp at
// level h, T_Omega node c0 at level L-h), lp < T, evaluated into Ss [T][R][R]:
// entry (lp, t, s) = e(Phi(x_t, xi_s) - Phi(c_A, xi_s) - Phi(x_t, c_B)); one (lp, t) row per
// item, so the rows x_t and c_A are read once.
template <int R>
__device__ __forceinline__ void otf_switch_fill(const OtfPhase& ph, const Geo& g, int p, int K, int c0, float2* Ss,
                                                int tid)
{
    const int T = 1 << K, nah = (int)(g.N >> g.h), nbh = (int)(g.N >> (g.L - g.h));
    const int cB = centre_of(c0 * nbh, nbh);
    const int* gA = otf_grid(ph, nah);
    const int* gB = otf_grid(ph, nbh);
    for (int e = tid; e < T * R; e += kThreads) {
        const int lp = e / R, t = e - lp * R;
        const int a = (p << K) + lp, x = a * nah + __ldg(gA + t), ca = centre_of(a * nah, nah);
        const OtfRow wx = otf_row(ph, x), wa = otf_row(ph, ca);
        const unsigned base = (wx.R - wa.R) - otf_turns(ph, x, cB);
        const unsigned long long dK = wx.K - wa.K;
#pragma unroll
        for (int s = 0; s < R; ++s) {
            const int xi = otf_xi(ph, c0 * nbh + __ldg(gB + s));
            Ss[e * R + s] = otf_exp(base + otf_ixi(ph, x - ca, xi) + otf_kmul(dK, abs(xi)));
        }
    }
}

// Switch on one (pair, column): wo[t] = sum_s S[t][s] xs[s] (strides CTp); S row-major
// [R][R] in shared memory (FROM_SMEM) or global memory.
template <int R, bool FROM_SMEM>
__device__ __forceinline__ void switch_item(const float2* xs, int CTp, const float4* Sp, float2* wo)
{
    float2 mu[R];
#pragma unroll
    for (int s = 0; s < R; ++s) mu[s] = xs[s * CTp];
#pragma unroll
    for (int t = 0; t < R; ++t) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int s2 = 0; s2 < R / 2; ++s2) {
            const float4 sv = FROM_SMEM ? Sp[t * (R / 2) + s2] : __ldg(Sp + t * (R / 2) + s2);
            cfmaf(acc, make_float2(sv.x, sv.y), mu[2 * s2]);
            cfmaf(acc, make_float2(sv.z, sv.w), mu[2 * s2 + 1]);
        }
        wo[t * CTp] = acc;
    }
}

// ------------------------------------------------------------------ front --
// Shared memory: Mv^T [NV][R4] | MH^T [kH][2R][R4] | per tile u < tpc:
// X [T][R][CTp] | EH double buffer [2][T][2][R] | EV [T*NV] | F rows [T*NV][mr]
// | (OTF or s_smem, last pass only) switch blocks [T][R][R] | (bk_smem) b_k [ra][T*NV].
// The table switch blocks are copied with the last level's phases, so they arrive during
// the H levels; b_k comes with the F rows.
// A CTA applies tpc consecutive tiles (work indices work * tpc + u): with few
// columns per tile, several tiles share the CTA's threads and their loads are
// in flight together; each tile's arithmetic is the same for any tpc.  The
// phases of level j are staged (cp.async) while level j-1 is computed; b_k and
// the switch matrices are read through the read-only cache unless bk_smem /
// s_smem put them in shared memory (the single-operator apply, when they fit
// beside the tiles; the batched kernel keeps its slices wider).  With OTF the
// phase tables are not read: EV, each level's EH and the switch blocks are
// evaluated (otf_turns, otf_exp) into the same shared buffers.
template <int R, int NV, bool OTF = false>
__device__ __forceinline__ void front_tile(const FrontArgs& A, int64_t work, unsigned char* smem_raw)
{
    constexpr int R4 = Pad4<R>::v;
    const Geo& g = A.g;
    const int K = A.K, T = 1 << K, CTp = A.CTp, lct = A.lct, mr = A.mr, lmr = A.lmr, ra = g.ra, tpc = A.tpc;
    const int nP = 1 << g.l1;                        // x-nodes at level l1
    const int64_t nBh = (int64_t)1 << (g.L - g.h);   // T_Omega nodes at level L-h
    const int64_t N = g.N, P = g.P, m = A.m;
    const int L = g.L, l1 = g.l1;
    const bool sblk = A.last && (OTF || A.s_smem);  // switch blocks in shared memory
    const size_t tile_f2 = (size_t)T * R * CTp + (size_t)2 * T * 2 * R + (size_t)T * NV + (size_t)T * NV * mr +
                           (sblk ? (size_t)T * R * R : 0) + (A.bk_smem ? (size_t)ra * T * NV : 0);

    float* MvTs = reinterpret_cast<float*>(smem_raw);                      // [NV][R4]
    float* MHTs = MvTs + NV * R4;                                          // [K][2R][R4]
    float2* tiles = reinterpret_cast<float2*>(MHTs + (size_t)K * 2 * R * R4);
    auto Xof = [&](int u) { return tiles + (size_t)u * tile_f2; };                         // [T][R][CTp]
    auto EHof = [&](int u) { return Xof(u) + (size_t)T * R * CTp; };                       // [2][T][2][R]
    auto EVof = [&](int u) { return EHof(u) + (size_t)2 * T * 2 * R; };                    // [T*NV]
    auto Fof = [&](int u) { return EVof(u) + (size_t)T * NV; };                            // [T*NV][mr]
    auto Sof = [&](int u) { return Fof(u) + (size_t)T * NV * mr; };                        // [T][R][R] (sblk)
    auto BKof = [&](int u) { return Sof(u) + (sblk ? (size_t)T * R * R : 0); };           // [ra][T*NV] (bk_smem)
    // tile u: work index work * tpc + u -> (column slice, x-node p, T_Omega chunk c0)
    __shared__ int64_t s_p[16], s_c0[16];
    __shared__ int s_slice[16];
    const int tid = threadIdx.x;
    if (tid < tpc) {
        const int64_t idx = work * tpc + tid, tile = idx / A.nslice;
        s_slice[tid] = (int)(idx - tile * A.nslice);
        s_p[tid] = tile & (nP - 1);
        s_c0[tid] = A.c0_lo + (tile >> l1);
    }
    __syncthreads();
    auto slice_of = [&](int u) { return s_slice[u]; };
    auto p_of = [&](int u) { return s_p[u]; };
    auto c0_of = [&](int u) { return s_c0[u]; };

    const float2* EHg = A.EH;
    // switch blocks of the tiles (tables): pair (x-node (p << K) + lp, T_Omega node c0) at
    // q = ((p << K) + lp) * nBh + c0 of S [P][R][R], R*R/2 16-byte copies each
    auto stage_s = [&]() {
        for (int u = 0; u < tpc; ++u) {
            const int64_t p = p_of(u), c0 = c0_of(u);
            for (int e = tid; e < T * R * R / 2; e += kThreads) {
                const int lp = e / (R * R / 2), w = e - lp * (R * R / 2);
                cp16(Sof(u) + (size_t)lp * R * R + 2 * w, A.S + (((p << K) + lp) * nBh + c0) * R * R + 2 * w);
            }
        }
    };
    auto stage_eh = [&](int j) {  // phases of level l1 + j into buffer (j - 1) & 1 of every tile
        if constexpr (OTF) {  // EH entry (lp, c, s) = e(Phi(c_A, xi) - Phi(c_P, xi)), Eq. 2
            const int l = l1 + j, na = (int)(N >> l), nb = (int)(N >> (L - l));
            const int* gC = otf_grid(A.ph, nb / 2);
            for (int u = 0; u < tpc; ++u) {
                const int p = (int)p_of(u), c0 = (int)c0_of(u);
                float2* dst = EHof(u) + (size_t)((j - 1) & 1) * T * 2 * R;
                for (int e = tid; e < T * 2 * R; e += kThreads) {
                    const int lp = e / (2 * R), cs = e - lp * 2 * R, c = cs >= R, s = cs - c * R;
                    const int ap = (p << j) + (lp >> (K - j));
                    const int bp = (c0 << (K - j)) + (lp & ((1 << (K - j)) - 1));
                    const int xi = bp * nb + c * (nb / 2) + __ldg(gC + s);
                    const int cA = centre_of(ap * na, na), cP = centre_of((ap >> 1) * 2 * na, 2 * na);
                    dst[e] = otf_exp(otf_rowdiff(A.ph, cA, cP, xi));
                }
            }
            return;
        }
        const int64_t nBl = (int64_t)1 << (L - l1 - j);
        const float2* eh = EHg + (size_t)(j - 1) * P * 2 * R;
        for (int u = 0; u < tpc; ++u) {
            const int64_t p = p_of(u), c0 = c0_of(u);
            float2* dst = EHof(u) + (size_t)((j - 1) & 1) * T * 2 * R;
            for (int e = tid; e < T * R; e += kThreads) {  // R 16-byte chunks per pair
                const int lp = e / R, w = e - lp * R;
                const int64_t ap = (p << j) + (lp >> (K - j));
                const int64_t bp = (c0 << (K - j)) + (lp & ((1 << (K - j)) - 1));
                cp16(dst + (size_t)lp * 2 * R + 2 * w, eh + (ap * nBl + bp) * 2 * R + 2 * w);
            }
        }
        if (sblk && j == K) stage_s();
    };
    // group 0: matrices, EV, F rows, level-1 phases; group 1: level-2 phases
    stage_matrix(MvTs, A.MvT, NV, R, R4, tid);
    stage_matrix(MHTs, A.MHT, K * 2 * R, R, R4, tid);
    for (int u = 0; u < tpc; ++u) {
        const int64_t xi_base = c0_of(u) * T * NV;
        float2* EVs = EVof(u);
        if constexpr (OTF) {
            // EV entry xi = e(Phi(c_A, xi)), A = x-node p at level l1 (Eq. 1)
            const int na = (int)(N >> l1), cA = centre_of((int)p_of(u) * na, na), xb = (int)xi_base;
            for (int e = tid; e < T * NV; e += kThreads) EVs[e] = otf_exp(otf_turns(A.ph, cA, xb + e));
            if (A.last) otf_switch_fill<R>(A.ph, g, (int)p_of(u), K, (int)c0_of(u), Sof(u), tid);
        } else {
            const float2* ev = A.EV + p_of(u) * N + xi_base;
            for (int e = tid; e < T * NV / 2; e += kThreads) cp16(EVs + 2 * e, ev + 2 * e);
        }
        if (A.bk_smem)
            for (int e = tid; e < ra * T * NV / 2; e += kThreads) {
                const int k = e / (T * NV / 2), w = e - k * (T * NV / 2);
                cp16(BKof(u) + (size_t)k * T * NV + 2 * w, A.bk + (size_t)k * N + xi_base + 2 * w);
            }
        const int64_t cbase = (int64_t)slice_of(u) * mr;
        float2* Fs = Fof(u);
        for (int e = tid; e < T * NV * mr; e += kThreads) {
            const int row = e >> lmr, c = e & (mr - 1);
            const bool valid = cbase + c < m;
            cp8(Fs + e, A.F + (xi_base - A.xi_lo + row) * m + (valid ? cbase + c : 0), valid);
        }
    }
    if (K >= 1) stage_eh(1);
    if (!OTF && sblk && K == 0) stage_s();
    cp_commit();
    if (K >= 2) {
        stage_eh(2);
        cp_commit();
    }
    // padding columns of the tiles start (and stay) at zero
    for (int u = 0; u < tpc; ++u) {
        float2* X = Xof(u);
        for (int e = tid; e < T * R * CTp; e += kThreads)
            if ((e & (CTp - 1)) >= ra * mr) X[e] = make_float2(0.f, 0.f);
    }
    if (K >= 2) cp_wait1(); else cp_wait0();
    __syncthreads();

    // ---- V (Eq. 1): item (u, j, c) computes mu[j][.][k*mr + c] of tile u for every k
    // (with few items, one item per amplitude term k instead)
    const int nk = (ra > 1 && tpc * T * mr * 2 <= kThreads) ? ra : 1;
    for (int itk = tid; itk < tpc * T * mr * nk; itk += kThreads) {
        const int it = itk / nk, kk = itk - it * nk;
        const int c = it & (mr - 1), j = (it >> lmr) & (T - 1), u = it >> (lmr + K);
        const int64_t xi_base = c0_of(u) * T * NV;
        const float2* fs = Fof(u) + (size_t)j * NV * mr + c;
        const float2* EVs = EVof(u);
        float2 f[NV];
#pragma unroll
        for (int x = 0; x < NV; ++x) f[x] = fs[x * mr];
        for (int k = nk > 1 ? kk : 0; k < (nk > 1 ? kk + 1 : ra); ++k) {
            float2 acc[R];
#pragma unroll
            for (int t = 0; t < R; ++t) acc[t] = make_float2(0.f, 0.f);
            const float2* bk = A.bk_smem ? BKof(u) + (size_t)k * T * NV + j * NV : A.bk + (size_t)k * N + xi_base + j * NV;
#pragma unroll
            for (int x = 0; x < NV; ++x) {
                const float2 z = cmulf(EVs[j * NV + x], cmulf(A.bk_smem ? bk[x] : __ldg(bk + x), f[x]));
                const float4* mv = reinterpret_cast<const float4*>(MvTs + x * R4);
#pragma unroll
                for (int t4 = 0; t4 < R4 / 4; ++t4) {
                    const float4 w = mv[t4];
                    const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int t = 4 * t4 + q;
                        if (t < R) {
                            rcfma(acc[t], ww[q], z);
                        }
                    }
                }
            }
            float2* xo = Xof(u) + (size_t)j * R * CTp + k * mr + c;
#pragma unroll
            for (int t = 0; t < R; ++t) xo[t * CTp] = acc[t];
        }
    }
    __syncthreads();

    // ---- H levels (Eq. 2), in place; item (u, grp, col)
    for (int j = 1; j <= K; ++j) {
        if (j > 1) {
            if (j < K) cp_wait1(); else cp_wait0();
            __syncthreads();
        }
        const int kj = K - j, half = 1 << kj;
        const float* Mh = MHTs + (size_t)(j - 1) * 2 * R * R4;
        for (int it = tid; it < tpc * (T / 2) * CTp; it += kThreads) {
            const int col = it & (CTp - 1), grp = (it >> lct) & (T / 2 - 1), u = it >> (lct + K - 1);
            const int a = grp >> kj, bp = grp & (half - 1);
            const int base = (bp << j) + (int)brev((unsigned)a, j - 1);
            float2* x0 = Xof(u) + (size_t)base * R * CTp + col;
            float2* x1 = x0 + (size_t)(1 << (j - 1)) * R * CTp;
            const float2* Eh = EHof(u) + (size_t)((j - 1) & 1) * T * 2 * R;
            h_item<R>(x0, x1, CTp, Eh + (size_t)((2 * a) * half + bp) * 2 * R,
                      Eh + (size_t)((2 * a + 1) * half + bp) * 2 * R, Mh);
        }
        __syncthreads();
        if (j + 2 <= K) {
            stage_eh(j + 2);
            cp_commit();
        }
    }

    // ---- switch (step 4) and write-out of the switch-level coefficients; item (u, lp, col).
    // Without the switch (the H levels continue in a middle pass) the level-(l1 + K)
    // coefficients are written as they are.
    for (int it = tid; it < tpc * T * CTp; it += kThreads) {
        const int col = it & (CTp - 1), lp = (it >> lct) & (T - 1), u = it >> (lct + K);
        const int slot = (int)brev((unsigned)lp, K);
        const float2* xs = Xof(u) + (size_t)slot * R * CTp + col;
        if (A.last) {
            const int64_t q = ((p_of(u) << K) + lp) * nBh + c0_of(u);
            float2* wo = A.W + (size_t)w_pair(A.wl, (p_of(u) << K) + lp, c0_of(u), slice_of(u)) * R * CTp + col;
            if (sblk)
                switch_item<R, true>(xs, CTp, reinterpret_cast<const float4*>(Sof(u) + (size_t)lp * R * R), wo);
            else
                switch_item<R, false>(xs, CTp, reinterpret_cast<const float4*>(A.S + q * R * R), wo);
        } else {
            float2* wo = A.Wo + (size_t)w_pair(A.wlo, (p_of(u) << K) + lp, c0_of(u), slice_of(u)) * R * CTp + col;
#pragma unroll
            for (int s = 0; s < R; ++s) wo[s * CTp] = xs[s * CTp];
        }
    }
}

// ------------------------------------------------------------------- back --
// Shared memory: MG^T [kG][2][R][R4] | MU [NU][R4] | U accumulator [XN][mr] |
// per chunk u < tpc: X [T][R][CTp] | FG double buffer [2][T][2][R] | EU [XN].
// The 2^l1 chunks c0' of T_Omega nodes are taken tpc at a time: their loads and
// G levels run together, their U contributions are accumulated one chunk after
// the other in increasing c0' (the same order for any tpc).  With OTF, FG and
// EU are evaluated into their shared buffers instead of copied.
template <int R, int NU, bool OTF = false>
__device__ __forceinline__ void back_tile(const BackArgs& A, int64_t work, unsigned char* smem_raw)
{
    constexpr int R4 = Pad4<R>::v;
    const Geo& g = A.g;
    const int K = A.K, T = 1 << K, CTp = A.CTp, lct = A.lct, mr = A.mr, lmr = A.lmr, ra = g.ra, tpc = A.tpc;
    const int slice = (int)(work % A.nslice);
    const int64_t pp = A.pp_lo + work / A.nslice;  // x-node at level lb
    const int nC = 1 << g.l1;                      // chunks c0' (= T_Omega nodes at level l1)
    const int XN = T * NU;                         // output points of this CTA
    const int64_t N = g.N, P = g.P;
    const int L = g.L, h = A.lb;  // the pass starts at level lb (h unless the G levels are split)
    const int e0 = A.lb - g.h;    // index of level lb + 1 in the G matrix and phase stacks
    const size_t chunk_f2 = (size_t)T * R * CTp + (size_t)2 * T * 2 * R + XN;

    float* MGTs = reinterpret_cast<float*>(smem_raw);                 // [K][2][R][R4]
    float* MUs = MGTs + (size_t)K * 2 * R * R4;                       // [NU][R4]
    float2* acc = reinterpret_cast<float2*>(MUs + (size_t)NU * R4);   // [XN][mr]
    float2* chunks = acc + (size_t)XN * mr;
    auto Xof = [&](int u) { return chunks + (size_t)u * chunk_f2; };             // [T][R][CTp]
    auto FGof = [&](int u) { return Xof(u) + (size_t)T * R * CTp; };             // [2][T][2][R]
    auto EUof = [&](int u) { return FGof(u) + (size_t)2 * T * 2 * R; };          // [XN]

    const int tid = threadIdx.x;
    const int64_t x0g = pp * XN;
    const float2* FGg = A.FG;
    int c0b = 0;
    auto stage_fg = [&](int j) {  // phases of level h + j into buffer (j - 1) & 1 of every chunk
        if constexpr (OTF) {  // FG entry (lp, c, t) = e(Phi(x_t, c_C) - Phi(x_t, c_B)), Eq. 3
            const int l = h + j, na = (int)(N >> l), nb = (int)(N >> (L - l));
            const int* gA = otf_grid(A.ph, na);
            for (int u = 0; u < tpc; ++u) {
                float2* dst = FGof(u) + (size_t)((j - 1) & 1) * T * 2 * R;
                for (int e = tid; e < T * 2 * R; e += kThreads) {
                    const int lp = e / (2 * R), ct = e - lp * 2 * R, c = ct >= R, t = ct - c * R;
                    const int ap = ((int)pp << j) + (lp >> (K - j));
                    const int bp = ((c0b + u) << (K - j)) + (lp & ((1 << (K - j)) - 1));
                    const int x = ap * na + __ldg(gA + t);
                    const int cB = centre_of(bp * nb, nb), cC = centre_of(bp * nb + c * (nb / 2), nb / 2);
                    dst[e] = otf_exp(otf_coldiff(A.ph, x, cC, cB));
                }
            }
            return;
        }
        const int64_t nBl = (int64_t)1 << (L - h - j);
        const float2* fg = FGg + (size_t)(e0 + j - 1) * P * 2 * R;
        for (int u = 0; u < tpc; ++u) {
            float2* dst = FGof(u) + (size_t)((j - 1) & 1) * T * 2 * R;
            for (int e = tid; e < T * R; e += kThreads) {
                const int lp = e / R, w = e - lp * R;
                const int64_t ap = (pp << j) + (lp >> (K - j));
                const int64_t bp = ((int64_t)(c0b + u) << (K - j)) + (lp & ((1 << (K - j)) - 1));
                cp16(dst + (size_t)lp * 2 * R + 2 * w, fg + (ap * nBl + bp) * 2 * R + 2 * w);
            }
        }
    };
    stage_matrix(MGTs, A.MGT + (size_t)e0 * 2 * R * R, K * 2 * R, R, R4, tid);
    stage_matrix(MUs, A.MU, NU, R, R4, tid);
    for (int e = tid; e < XN * mr; e += kThreads) acc[e] = make_float2(0.f, 0.f);

    for (c0b = 0; c0b < nC; c0b += tpc) {
        __syncthreads();  // the previous chunks' U stage is done with X and EU
        for (int u = 0; u < tpc; ++u) {  // pairs (pp, c0 * T + j), j < T: one contiguous block of T*R*CTp
            const int c0 = c0b + u;
            const float2* src = A.W + (size_t)w_pair(A.wl, pp, (int64_t)c0 * T, slice) * R * CTp;
            float2* X = Xof(u);
            for (int e = tid; e < T * R * CTp / 2; e += kThreads) cp16(X + 2 * e, src + 2 * e);
            float2* EUs = EUof(u);
            if constexpr (OTF) {  // EU entry x = e(Phi(x, c_C)), C = T_Omega node c0 at level l1 (Eq. bf3)
                const int nc = (int)(N >> g.l1), cC = centre_of(c0 * nc, nc), xb = (int)x0g;
                for (int e = tid; e < XN; e += kThreads) EUs[e] = otf_exp(otf_turns(A.ph, xb + e, cC));
            } else {
                for (int e = tid; e < XN / 2; e += kThreads) cp16(EUs + 2 * e, A.EU + (size_t)c0 * N + x0g + 2 * e);
            }
        }
        if (K >= 1) stage_fg(1);
        cp_commit();
        if (K >= 2) {
            stage_fg(2);
            cp_commit();
        }
        if (K >= 2) cp_wait1(); else cp_wait0();
        __syncthreads();

        // ---- G levels (Eq. 3), in place; item (u, grp, col)
        for (int j = 1; j <= K; ++j) {
            if (j > 1) {
                if (j < K) cp_wait1(); else cp_wait0();
                __syncthreads();
            }
            const int kj = K - j, half = 1 << kj;
            const float* Mg = MGTs + (size_t)(j - 1) * 2 * R * R4;
            for (int it = tid; it < tpc * (T / 2) * CTp; it += kThreads) {
                const int col = it & (CTp - 1), grp = (it >> lct) & (T / 2 - 1), u = it >> (lct + K - 1);
                const int a = grp >> kj, bp = grp & (half - 1);
                const int base = (bp << j) + (int)brev((unsigned)a, j - 1);
                float2* x0 = Xof(u) + (size_t)base * R * CTp + col;
                float2* x1 = x0 + (size_t)(1 << (j - 1)) * R * CTp;
                const float2* Fg = FGof(u) + (size_t)((j - 1) & 1) * T * 2 * R;
                g_item<R>(x0, x1, CTp, Fg + (size_t)((2 * a) * half + bp) * 2 * R,
                          Fg + (size_t)((2 * a + 1) * half + bp) * 2 * R, Mg);
            }
            __syncthreads();
            if (j + 2 <= K) {
                stage_fg(j + 2);
                cp_commit();
            }
        }

        // ---- U (Eq. bf3) contributions of T_Omega nodes c0b .. c0b + tpc - 1, in that order;
        // each accumulator entry (lp, i, c) belongs to one thread.  Item (lp, c, part): part
        // of nis equal ranges of the NU points i (nis > 1 only when T * mr < kThreads)
        {
            int lnis = 0;
            while ((1 << lnis) < NU && ((T * mr) << (lnis + 1)) <= kThreads) ++lnis;
            const int nis = 1 << lnis, ni = NU >> lnis;
            const int c = tid & (mr - 1), part = (tid >> lmr) & (nis - 1);
            for (int lp = tid >> (lmr + lnis); lp < T; lp += kThreads >> (lmr + lnis)) {
                const int slot = (int)brev((unsigned)lp, K);
                float2* ap = acc + (size_t)lp * NU * mr + c;
                for (int u = 0; u < tpc; ++u) {
                    const float2* xs = Xof(u) + (size_t)slot * R * CTp + c;
                    const float2* EUs = EUof(u);
                    for (int k = 0; k < ra; ++k) {
                        float2 v[R];
#pragma unroll
                        for (int s = 0; s < R; ++s) v[s] = xs[s * CTp + k * mr];
                        const float2* ak = A.ak + (size_t)k * N + x0g + lp * NU;
#pragma unroll 4
                        for (int i = part * ni; i < (part + 1) * ni; ++i) {
                            float2 w = make_float2(0.f, 0.f);
                            const float4* mu = reinterpret_cast<const float4*>(MUs + i * R4);
#pragma unroll
                            for (int s4 = 0; s4 < R4 / 4; ++s4) {
                                const float4 m4 = mu[s4];
                                const float mm[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    const int s = 4 * s4 + q;
                                    if (s < R) {
                                        rcfma(w, mm[q], v[s]);
                                    }
                                }
                            }
                            float2 o = ap[i * mr];
                            cfmaf(o, cmulf(__ldg(ak + i), EUs[lp * NU + i]), w);
                            ap[i * mr] = o;
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    // ---- write G
    {
        const int c = tid & (mr - 1);
        const int64_t cg = (int64_t)slice * mr + c;
        if (cg < A.m) {
            for (int x = tid >> lmr; x < XN; x += kThreads >> lmr) {
                float2* gp = A.G + (x0g - A.x_lo + x) * A.m + cg;
                float2 v = acc[x * mr + c];
                if (A.beta) {
                    const float2 o = *gp;
                    v.x += o.x;
                    v.y += o.y;
                }
                *gp = v;
            }
        }
    }
}

// -------------------------------------------------------------------- mid --
// A middle pass of a split level range (MidArgs): K levels of H (GK = 0, Eq. 2) or
// G (GK = 1, Eq. 3) over tiles of T = 2^K pairs read from and written to HBM.
// Shared memory: M^T [K][2R][R4] | per tile u < tpc: X [T][R][CTp] | phase double
// buffer [2][T][2][R] | (OTF, last H pass) switch blocks [T][R][R].  The in-place slot
// order, the staging one level ahead and the level items are those of the front and
// back tiles, so each tile's arithmetic is the same as there.
template <int R, int GK, bool OTF = false>
__device__ __forceinline__ void mid_tile(const MidArgs& A, int64_t work, unsigned char* smem_raw)
{
    constexpr int R4 = Pad4<R>::v;
    const Geo& g = A.g;
    const int K = A.K, T = 1 << K, CTp = A.CTp, lct = A.lct, tpc = A.tpc, la = A.la, L = g.L;
    const int64_t N = g.N, P = g.P;
    const bool last = !GK && A.last;
    const size_t tile_f2 = (size_t)T * R * CTp + (size_t)2 * T * 2 * R + (OTF && last ? (size_t)T * R * R : 0);

    float* MTs = reinterpret_cast<float*>(smem_raw);                      // [K][2R][R4]
    float2* tiles = reinterpret_cast<float2*>(MTs + (size_t)K * 2 * R * R4);
    auto Xof = [&](int u) { return tiles + (size_t)u * tile_f2; };        // [T][R][CTp]
    auto Eof = [&](int u) { return Xof(u) + (size_t)T * R * CTp; };       // [2][T][2][R]
    auto Sof = [&](int u) { return Eof(u) + (size_t)2 * T * 2 * R; };     // [T][R][R]
    // tile u: work index work * tpc + u -> (column slice, x-node p at level la, chunk c)
    __shared__ int s_p[16], s_c[16], s_slice[16];
    const int tid = threadIdx.x;
    if (tid < tpc) {
        const int64_t idx = work * tpc + tid, tile = idx / A.nslice;
        s_slice[tid] = (int)(idx - tile * A.nslice);
        s_p[tid] = (int)(tile & ((1ll << la) - 1));
        s_c[tid] = (int)(tile >> la);
    }
    __syncthreads();

    auto stage = [&](int j) {  // phases of level la + j into buffer (j - 1) & 1 of every tile
        const int l = la + j;
        for (int u = 0; u < tpc; ++u) {
            const int p = s_p[u], c = s_c[u];
            float2* dst = Eof(u) + (size_t)((j - 1) & 1) * T * 2 * R;
            if constexpr (OTF) {
                const int na = (int)(N >> l), nb = (int)(N >> (L - l));
                const int* gr = otf_grid(A.ph, GK ? na : nb / 2);
                for (int e = tid; e < T * 2 * R; e += kThreads) {
                    const int lp = e / (2 * R), cs = e - lp * 2 * R, ch = cs >= R, s = cs - ch * R;
                    const int ap = (p << j) + (lp >> (K - j));
                    const int bp = (c << (K - j)) + (lp & ((1 << (K - j)) - 1));
                    if constexpr (GK) {  // FG entry (lp, ch, t) = e(Phi(x_t, c_C) - Phi(x_t, c_B))
                        const int x = ap * na + __ldg(gr + s);
                        const int cB = centre_of(bp * nb, nb), cC = centre_of(bp * nb + ch * (nb / 2), nb / 2);
                        dst[e] = otf_exp(otf_coldiff(A.ph, x, cC, cB));
                    } else {             // EH entry (lp, ch, s) = e(Phi(c_A, xi_s) - Phi(c_P, xi_s))
                        const int xi = bp * nb + ch * (nb / 2) + __ldg(gr + s);
                        const int cA = centre_of(ap * na, na), cP = centre_of((ap >> 1) * 2 * na, 2 * na);
                        dst[e] = otf_exp(otf_rowdiff(A.ph, cA, cP, xi));
                    }
                }
            } else {
                const int64_t nBl = (int64_t)1 << (L - l);
                const float2* tab = A.E + (size_t)(A.e0 + j - 1) * P * 2 * R;
                for (int e = tid; e < T * R; e += kThreads) {  // R 16-byte chunks per pair
                    const int lp = e / R, w = e - lp * R;
                    const int64_t ap = ((int64_t)p << j) + (lp >> (K - j));
                    const int64_t bp = ((int64_t)c << (K - j)) + (lp & ((1 << (K - j)) - 1));
                    cp16(dst + (size_t)lp * 2 * R + 2 * w, tab + (ap * nBl + bp) * 2 * R + 2 * w);
                }
            }
        }
    };
    // group 0: matrices, the tiles' pairs, level-1 phases; group 1: level-2 phases
    stage_matrix(MTs, A.MT + (size_t)A.e0 * 2 * R * R, K * 2 * R, R, R4, tid);
    for (int u = 0; u < tpc; ++u) {  // pairs (p, c T + i), i < T: one contiguous block of T*R*CTp
        const float2* src = A.Wi + (size_t)w_pair(A.wli, s_p[u], (int64_t)s_c[u] * T, s_slice[u]) * R * CTp;
        float2* X = Xof(u);
        for (int e = tid; e < T * R * CTp / 2; e += kThreads) cp16(X + 2 * e, src + 2 * e);
        if constexpr (OTF) {
            if (last) otf_switch_fill<R>(A.ph, g, s_p[u], K, s_c[u], Sof(u), tid);
        }
    }
    stage(1);
    cp_commit();
    if (K >= 2) {
        stage(2);
        cp_commit();
    }
    if (K >= 2) cp_wait1(); else cp_wait0();
    __syncthreads();

    for (int j = 1; j <= K; ++j) {
        if (j > 1) {
            if (j < K) cp_wait1(); else cp_wait0();
            __syncthreads();
        }
        const int kj = K - j, half = 1 << kj;
        const float* Mj = MTs + (size_t)(j - 1) * 2 * R * R4;
        for (int it = tid; it < tpc * (T / 2) * CTp; it += kThreads) {
            const int col = it & (CTp - 1), grp = (it >> lct) & (T / 2 - 1), u = it >> (lct + K - 1);
            const int a = grp >> kj, bp = grp & (half - 1);
            const int base = (bp << j) + (int)brev((unsigned)a, j - 1);
            float2* x0 = Xof(u) + (size_t)base * R * CTp + col;
            float2* x1 = x0 + (size_t)(1 << (j - 1)) * R * CTp;
            const float2* Eb = Eof(u) + (size_t)((j - 1) & 1) * T * 2 * R;
            const float2* E0 = Eb + (size_t)((2 * a) * half + bp) * 2 * R;
            const float2* E1 = Eb + (size_t)((2 * a + 1) * half + bp) * 2 * R;
            if constexpr (GK) g_item<R>(x0, x1, CTp, E0, E1, Mj);
            else h_item<R>(x0, x1, CTp, E0, E1, Mj);
        }
        __syncthreads();
        if (j + 2 <= K) {
            stage(j + 2);
            cp_commit();
        }
    }

    // ---- write-out at level la + K (after the switch if the pass reaches h); item (u, lp, col)
    for (int it = tid; it < tpc * T * CTp; it += kThreads) {
        const int col = it & (CTp - 1), lp = (it >> lct) & (T - 1), u = it >> (lct + K);
        const int slot = (int)brev((unsigned)lp, K);
        const float2* xs = Xof(u) + (size_t)slot * R * CTp + col;
        const int64_t a = ((int64_t)s_p[u] << K) + lp;
        float2* wo = A.Wo + (size_t)w_pair(A.wlo, a, s_c[u], s_slice[u]) * R * CTp + col;
        if (last) {
            if constexpr (OTF) {
                switch_item<R, true>(xs, CTp, reinterpret_cast<const float4*>(Sof(u) + (size_t)lp * R * R), wo);
            } else {
                const int64_t q = a * ((int64_t)1 << (L - g.h)) + s_c[u];
                switch_item<R, false>(xs, CTp, reinterpret_cast<const float4*>(A.S + q * R * R), wo);
            }
        } else {
#pragma unroll
            for (int s = 0; s < R; ++s) wo[s * CTp] = xs[s * CTp];
        }
    }
}

inline int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// shared memory of a front pass of K H levels (last: it reaches h and applies the switch;
// s_smem: with the table switch blocks in shared memory; bk_smem: with b_k)
inline size_t front_smem(const Geo& g, int K, bool last, int R, int NV, int CTp, int mr, int tpc,
                         bool s_smem = false, bool bk_smem = false)
{
    const size_t T = (size_t)1 << K, R4 = (R + 3) & ~3;
    return sizeof(float2) * (size_t)tpc *
               (T * R * CTp + 2 * T * 2 * R + T * NV + T * NV * mr + ((g.otf || s_smem) && last ? T * R * R : 0) +
                (bk_smem ? (size_t)(g.ra > 0 ? g.ra : 1) * T * NV : 0)) +
           sizeof(float) * ((size_t)NV * R4 + (size_t)K * 2 * R * R4);
}

// shared memory of a back pass of K G levels
inline size_t back_smem(const Geo& g, int K, int R, int NU, int CTp, int mr, int tpc)
{
    const size_t T = (size_t)1 << K, R4 = (R + 3) & ~3;
    const size_t XN = T * NU;
    return sizeof(float2) * (XN * mr + (size_t)tpc * (T * R * CTp + 2 * T * 2 * R + XN)) +
           sizeof(float) * ((size_t)K * 2 * R * R4 + (size_t)NU * R4);
}

// shared memory of a middle pass of K levels (last: an H pass that reaches h)
inline size_t mid_smem(const Geo& g, int K, bool last, int R, int CTp, int tpc)
{
    const size_t T = (size_t)1 << K, R4 = (R + 3) & ~3;
    return sizeof(float2) * (size_t)tpc * (T * R * CTp + 2 * T * 2 * R + (g.otf && last ? T * R * R : 0)) +
           sizeof(float) * ((size_t)K * 2 * R * R4);
}

template <int R>
constexpr int nv_of() { return (R < 8) ? 8 : (R < 16 ? 16 : 32); }

}  // namespace
}  // namespace bfi
