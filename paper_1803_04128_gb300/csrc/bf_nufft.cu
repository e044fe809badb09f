// NUFFT evaluation of Eq. (tg3), Sec. 3, for phases that are rank 1 on each
// half of the columns (the split at xi = 0 of Eq. FIOwq2, Sec. 5).
//
// For the built-in phases whose row terms have no xi^2 part (DFT, FIO,
// FIO_PW, ONES), Phi(x_i, xi) = t_i^h xi + rho_i on the half h of the columns
// (h = 0: xi >= 0, t = xxi x_i + kappa_i; h = 1: xi < 0, t = xxi x_i - kappa_i).
// Algorithm 6's lifting with r = 1 then removes the whole phase of each half,
// and with the amplitude split alpha ~ sum_k a_k(x) b_k(xi) (Algorithm 1),
//     g_i = sum_h sum_k a_k(x_i) e^{2 pi i rho_i} sum_{xi in h} e^{2 pi i t_i^h xi} b_k(xi) f(xi),
// i.e. 2 r_alpha one-dimensional NUFFTs with uniform modes and non-uniform
// targets per right-hand side.
//
// Each NUFFT is Gaussian gridding (phi(d) = exp(-d^2 / (4 tau)), 1-periodic),
// with M = N/2 modes shifted to jt in [-M/2, M/2) (xi = jt + s_h, s_h = +-M/2)
// and an oversampled grid of n = 2M = N points:
//   1. u_jt = b_k(xi) f(xi) / phihat(jt)                      (deconvolution)
//   2. hgrid_p = sum_jt u_jt e^{2 pi i p jt / n}               (inverse FFT, n points)
//   3. g_i += a_k(x_i) e^{2 pi i (t_i s_h + rho_i)} (1/n) sum_{|p - n t_i| <= msp} phi(t_i - p/n) hgrid_p.
// tau = msp / (12 pi M^2) balances the truncation of phi against the
// trapezoid rule's aliasing; both fall like exp(-2 pi msp / 3).
//
// Device work (three launches, all columns and both halves at once):
//   nufft_pass1: deconvolution fused into the first step of a four-step FFT
//                (n = n1 n2): for each j1, an n2-point DFT over j2 of the
//                inputs j = j1 + n1 j2, times the twiddle e^{2 pi i p2 j1 / n},
//                written to T[h][p2][j1][col];
//   nufft_pass2: for each p2, an n1-point DFT over j1, written to
//                H[h][p = p2 + n2 p1][col];
//   nufft_interp: for each target row i and right-hand side c, the 2 msp
//                weights of both halves and all k, written to G[i][c].
// Columns are col = k m + c (amplitude term k, right-hand side c), innermost
// in every buffer, so that every global access is a contiguous row segment.
// Inside a pass, an S = SA SB point DFT of CBK columns runs in two register
// stages (SA- and SB-point radix-2 DFTs) with one exchange through shared
// memory: stage 1 reads global memory, stage 2 writes it.
//
// Host planning (FP64): the targets, the interpolation windows and weights,
// the deconvolution factors times b_k, the centring phases times a_k, the
// twiddles.  All are O(N) and built once per plan (bf_nufft_prepare).
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "bf_device.h"

namespace bfi {

struct NufftState {
    int device = 0;
    int64_t N = 0, M = 0, n = 0;
    int n1 = 0, n2 = 0, lg1 = 0, lg2 = 0;
    int msp = 0, ra = 0;
    double tau = 0;
    void* arena = nullptr;
    float2* bD = nullptr;  // [2][ra][M]   b_k(xi) / exp(-4 pi^2 jt^2 tau), jt = idx - M/2
    float2* pa = nullptr;  // [2][ra][N]   a_k(x_i) e^{2 pi i (t_i s_h + rho_i)}
    float* W = nullptr;    // [2][N][2 msp] exp(-d^2 / (4 tau)) / (n sqrt(4 pi tau))
    int* p0 = nullptr;     // [2][N]       first grid point of the window (0 <= p0 < n)
    float2* tw = nullptr;  // [n]          e^{2 pi i k / n}
    void* ws = nullptr;    // T | H, each [2][n][Mc] c64
    size_t ws_bytes = 0;
};

namespace {

__constant__ float2 c_w32[32];  // e^{2 pi i k / 32}

constexpr int kNuThreads = 256;
constexpr int kMaxMsp = 16;

constexpr int brev_c(int v, int bits)
{
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
    return r;
}
constexpr int log2_c(int v) { return v <= 1 ? 0 : 1 + log2_c(v / 2); }

__device__ __forceinline__ float2 nu_cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// (u + t, u - t) on packed two-lane adds: the same IEEE additions as the scalar forms
__device__ __forceinline__ void nu_bfly(float2 u, float2 t, float2& p, float2& q)
{
    asm("{\n.reg .b64 a, b, c, d;\nmov.b64 a, {%4, %5};\nmov.b64 b, {%6, %7};\n"
        "add.rn.f32x2 c, a, b;\nsub.rn.f32x2 d, a, b;\nmov.b64 {%0, %1}, c;\nmov.b64 {%2, %3}, d;\n}"
        : "=f"(p.x), "=f"(p.y), "=f"(q.x), "=f"(q.y)
        : "f"(u.x), "f"(u.y), "f"(t.x), "f"(t.y));
}

// One radix-2 stage of butterflies of span LEN (twiddles e^{2 pi i j / LEN}), then the next;
// a template recursion, so that every register index is a compile-time constant.
template <int R, int LEN>
struct DftStage {
    __device__ __forceinline__ static void run(float2 (&v)[R])
    {
#pragma unroll
        for (int s0 = 0; s0 < R; s0 += LEN) {
#pragma unroll
            for (int j = 0; j < LEN / 2; ++j) {
                const float2 u = v[s0 + j];
                float2 t = v[s0 + j + LEN / 2];
                constexpr int kq = 8;  // e^{2 pi i k / 32} is i^(k / 8) for k a multiple of 8: exact
                const int tw = j * (32 / LEN);
                if (tw == kq) t = make_float2(-t.y, t.x);
                else if (tw == 2 * kq) t = make_float2(-t.x, -t.y);
                else if (tw == 3 * kq) t = make_float2(t.y, -t.x);
                else if (tw != 0) t = nu_cmul(c_w32[tw], t);
                nu_bfly(u, t, v[s0 + j], v[s0 + j + LEN / 2]);
            }
        }
        DftStage<R, 2 * LEN>::run(v);
    }
};
template <int R>
struct DftStage<R, 2 * R> {
    __device__ __forceinline__ static void run(float2 (&)[R]) {}
};

// v <- DFT_R(v) with the + sign: v_k = sum_j v_j e^{2 pi i j k / R} (radix-2, decimation in
// time on the bit-reversed input), R <= 32.
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&v)[R])
{
    constexpr int LB = log2_c(R);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = brev_c(i, LB);
        if (j > i) {
            const float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
    DftStage<R, 2>::run(v);
}

struct PassArgs {
    const float2* F;   // pass 1: [N][m]
    const float2* bD;  // pass 1
    const float2* tw;  // [n]
    const float2* in;  // pass 2: T
    float2* out;       // pass 1: T, pass 2: H
    int64_t N, M, n, m, Mc;
    int n1, n2, lg1, lg2, cbk, nblk;
};

// One S = SA * SB point DFT (+ sign) of cbk columns of a (half, row index, column block)
// tile.  PASS 1: inputs are the deconvolved F entries j = j1 + n1 (b + SB a); outputs
// T[h][p2][j1][col] times e^{2 pi i p2 j1 / n}.  PASS 2: inputs T[h][p2][b + SB a][col];
// outputs H[h][p2 + n2 p1][col].  Stage 1 item (b, cc): SA inputs, DFT_SA over a, the inner
// twiddle e^{2 pi i b ka / S}, into X[b + SB ka][cc]; stage 2 item (ka, cc): DFT_SB over b,
// output index ka + SA kb.
// Pass 1's nonzero inputs: jt = j (j < n/2) or j - n lies in [-M/2, M/2) iff j2 < n2/4 or
// j2 >= 3 n2/4 (n1 divides M/2), i.e. iff a < SA/4 or a >= 3 SA/4: a compile-time set, so
// the zero inputs cost no load and fold out of the first butterflies.  The F row of input
// j is jt + s_h + N/2.  The twiddles e^{2 pi i x / S} and (pass 1) e^{2 pi i p2 j1 / n} of the
// tile are staged in shared memory from the e^{2 pi i k / n} table.
template <int SA, int SB, int PASS>
__global__ void __launch_bounds__(kNuThreads) nufft_pass(const PassArgs A)
{
    constexpr int S = SA * SB;
    extern __shared__ float2 X[];  // [S][cbk] | twS [S] | (pass 1) twJ [S]
    const int cbk = A.cbk;
    float2* twS = X + (size_t)S * cbk;
    float2* twJ = twS + S;
    const int blk = (int)blockIdx.x;
    const int cb = blk % A.nblk;
    const int rest = blk / A.nblk;
    const int rowsz = PASS == 1 ? A.n1 : A.n2;  // j1 (pass 1) or p2 (pass 2) per half
    const int ridx = rest % rowsz;
    const int h = rest / rowsz;
    const int col0 = cb * cbk;
    const int tid = threadIdx.x;
    const int n = (int)A.n;
    const int64_t Mc = A.Mc;
    for (int x = tid; x < S; x += kNuThreads) {
        twS[x] = __ldg(A.tw + x * (n / S));
        if (PASS == 1) twJ[x] = __ldg(A.tw + ((x * ridx) & (n - 1)));
    }
    __syncthreads();

    for (int it = tid; it < SB * cbk; it += kNuThreads) {
        const int cc = it % cbk, b = it / cbk;
        const int col = col0 + cc;
        float2 v[SA];
#pragma unroll
        for (int a = 0; a < SA; ++a) v[a] = make_float2(0.f, 0.f);
        if (col < Mc) {
            if constexpr (PASS == 1) {
                const int k = (int)(col / A.m);
                const int64_t c = col - (int64_t)k * A.m;
                const int N = (int)A.N, M = (int)A.M;
                const int rowoff = h == 0 ? 3 * (N / 4) : N / 4;        // s_h + N/2
                const float2* bDk = A.bD + ((int64_t)h * (Mc / A.m) + k) * M + M / 2;
#pragma unroll
                for (int a = 0; a < SA; ++a) {
                    if (a < SA / 4 || a >= 3 * (SA / 4)) {
                        const int jt = ridx + A.n1 * (b + SB * a) - (a >= 3 * (SA / 4) ? n : 0);
                        const float2 f = __ldg(A.F + (int64_t)(jt + rowoff) * A.m + c);
                        v[a] = nu_cmul(__ldg(bDk + jt), f);
                    }
                }
            } else {
                const float2* src = A.in + ((int64_t)(h * A.n2 + ridx) * A.n1 + b) * Mc + col;
#pragma unroll
                for (int a = 0; a < SA; ++a) v[a] = __ldg(src + (int64_t)(SB * a) * Mc);
            }
        }
        dft_reg<SA>(v);
#pragma unroll
        for (int ka = 0; ka < SA; ++ka)
            X[(b + SB * ka) * cbk + cc] = ka == 0 ? v[ka] : nu_cmul(twS[(b * ka) & (S - 1)], v[ka]);
    }
    __syncthreads();
    for (int it = tid; it < SA * cbk; it += kNuThreads) {
        const int cc = it % cbk, ka = it / cbk;
        const int col = col0 + cc;
        float2 v[SB];
#pragma unroll
        for (int b = 0; b < SB; ++b) v[b] = X[(b + SB * ka) * cbk + cc];
        dft_reg<SB>(v);
        if (col >= Mc) continue;
        if constexpr (PASS == 1) {
            // p2 = ka + SA kb, j1 = ridx: twiddle e^{2 pi i p2 j1 / n}
            float2* dst = A.out + ((int64_t)(h * A.n2 + ka) * A.n1 + ridx) * Mc + col;
#pragma unroll
            for (int kb = 0; kb < SB; ++kb)
                dst[(int64_t)(SA * kb) * A.n1 * Mc] = nu_cmul(twJ[ka + SA * kb], v[kb]);
        } else {
            float2* dst = A.out + ((int64_t)h * n + ridx + (int64_t)A.n2 * ka) * Mc + col;
#pragma unroll
            for (int kb = 0; kb < SB; ++kb) dst[(int64_t)A.n2 * (SA * kb) * Mc] = v[kb];
        }
    }
}

struct InterpArgs {
    const float2* H;   // [2][n][Mc]
    const float2* pa;  // [2][ra][N]
    const float* W;    // [2][N][2 msp]
    const int* p0;     // [2][N]
    float2* G;         // [N][m]
    int64_t N, n, m, Mc;
    int ra, msp;
};

// G[i][c] = sum_h sum_k pa[h][k][i] sum_q W[h][i][q] H[h][(p0 + q) mod n][k m + c].
// A CTA takes a tile of kTile consecutive targets and 32 consecutive right-hand sides c; warp
// w takes the run of kRun targets i0 + w kRun .. and the 32 c (lanes).  The rounds r = (h, k),
// h outer, each need the grid rows that the tile's windows cover for half h (span_T rows from
// p_lo), columns k m + c0 .. + 31.  kBuf rounds are in flight at once: their rows are copied
// with cp.async (zero-filled past m) into a ring of kBuf shared buffers, one commit group per
// round, so that the next rounds' copies overlap the current round's arithmetic.  In a round
// each warp walks the union of its own run's windows once: every row feeds all kRun targets
// through the warp's dense weight block Wd[p - p_run][t] (zero outside target t's window),
// built at the first round of each half.  Tiles whose rows exceed a buffer (targets far apart,
// e.g. at a jump of the phase) read each target's window from global memory instead.  Every
// output is the sum over the same weights and rows in increasing p, then k, then h, either way.
constexpr int kRun = 8;
constexpr int kTile = 64;                   // targets per CTA = kRun * 8 warps
constexpr int kSpanMax = 48;                // rows of one warp's union of windows
constexpr int kRowsMax = 112;               // rows of one buffer
constexpr int kBuf = 2;                     // rounds whose rows are in flight together
constexpr size_t kInterpSmem = (size_t)kBuf * kRowsMax * 32 * sizeof(float2) +
                               (size_t)(kNuThreads / 32) * kSpanMax * kRun * sizeof(float);
__device__ __forceinline__ void nu_cp8(void* dst, const void* src, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    const int nb = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(nb) : "memory");
}
__device__ __forceinline__ void nu_cp16(void* dst, const void* src, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    const int nb = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(nb) : "memory");
}
// acc += w * v for a real weight and a complex value: one packed two-lane FMA
__device__ __forceinline__ void nu_fma2(float2& acc, float w, float2 v)
{
    asm("{\n.reg .b64 wa, vb, ac;\nmov.b64 wa, {%2, %2};\nmov.b64 vb, {%3, %4};\nmov.b64 ac, {%0, %1};\n"
        "fma.rn.f32x2 ac, wa, vb, ac;\nmov.b64 {%0, %1}, ac;\n}"
        : "+f"(acc.x), "+f"(acc.y)
        : "f"(w), "f"(v.x), "f"(v.y));
}
__global__ void __launch_bounds__(kNuThreads, 3) nufft_interp(const InterpArgs A)
{
    extern __shared__ __align__(16) unsigned char nu_sm[];
    float2(*Hb)[32] = reinterpret_cast<float2(*)[32]>(nu_sm);  // kBuf buffers of kRowsMax rows
    float(*Wd)[kRun] = reinterpret_cast<float(*)[kRun]>(nu_sm + (size_t)kBuf * kRowsMax * 32 * sizeof(float2)) +
                       (size_t)(threadIdx.x >> 5) * kSpanMax;
    __shared__ int Rel_all[2][kNuThreads / 32][kRun];
    __shared__ int s_lo[2][kNuThreads / 32], s_hi[2][kNuThreads / 32];
    __shared__ int s_pT[2], s_tlo[2], s_spanT[2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ncb = (A.m + 31) / 32;
    const int64_t tile = blockIdx.x / ncb;
    const int64_t c0 = (blockIdx.x % ncb) * 32;
    const int64_t iT = tile * kTile, i0 = iT + wid * kRun;
    const int64_t c = c0 + lane;
    const bool live = c < A.m;
    const int w2 = 2 * A.msp;
    const int nmask = (int)(A.n - 1);
    // window starts of both halves relative to the tile's first target, as signed offsets mod n
    for (int h = 0; h < 2; ++h) {
        const int pT = __ldg(A.p0 + h * A.N + iT);
        int rel = 0;
        if (lane < kRun) {
            int d = (__ldg(A.p0 + h * A.N + i0 + lane) - pT) & nmask;
            if (d > (int)(A.n / 2)) d -= (int)A.n;
            rel = d;
        }
        int lo = lane < kRun ? rel : INT_MAX, hi = lane < kRun ? rel : INT_MIN;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane < kRun) Rel_all[h][wid][lane] = rel - lo;
        if (lane == 0) {
            s_lo[h][wid] = lo;
            s_hi[h][wid] = hi;
        }
        if (threadIdx.x == 0) s_pT[h] = pT;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int h = threadIdx.x;
        int tlo = INT_MAX, thi = INT_MIN;
        for (int w = 0; w < kNuThreads / 32; ++w) {
            tlo = min(tlo, s_lo[h][w]);
            thi = max(thi, s_hi[h][w]);
        }
        s_tlo[h] = tlo;
        s_spanT[h] = thi - tlo + w2;
    }
    __syncthreads();
    const int nr = 2 * A.ra;  // rounds
    // the copies of round r into buffer r % kBuf (none for an untiled half), one commit group
    auto issue = [&](int r) {
        if (r < nr) {
            const int h = r / A.ra, k = r - h * A.ra, spanT = s_spanT[h];
            if (spanT <= kRowsMax) {
                float2(*Hs)[32] = Hb + (r % kBuf) * kRowsMax;
                const float2* src = A.H + (int64_t)h * A.n * A.Mc + k * A.m + c0;
                const int pl = s_pT[h] + s_tlo[h];
                if ((A.m & 1) == 0) {  // even m: every (row, column pair) is 16-byte aligned
                    const int cc = 2 * (threadIdx.x & 15);
                    const bool ok = c0 + cc < A.m;
                    const float2* sc = src + (ok ? cc : 0);
                    for (int pp = threadIdx.x >> 4; pp < spanT; pp += kNuThreads / 16)
                        nu_cp16(&Hs[pp][cc], sc + (int64_t)((pl + pp) & nmask) * A.Mc, ok);
                } else {
                    for (int e = threadIdx.x; e < spanT * 32; e += kNuThreads) {
                        const int pp = e >> 5, cc = e & 31;
                        const bool ok = c0 + cc < A.m;
                        nu_cp8(&Hs[pp][cc], src + (int64_t)((pl + pp) & nmask) * A.Mc + (ok ? cc : 0), ok);
                    }
                }
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
#pragma unroll
    for (int r = 0; r < kBuf; ++r) issue(r);
    float2 g[kRun];
#pragma unroll
    for (int t = 0; t < kRun; ++t) g[t] = make_float2(0.f, 0.f);
    for (int r = 0; r < nr; ++r) {
        const int h = r / A.ra, k = r - h * A.ra;
        const bool tiled = s_spanT[h] <= kRowsMax;                     // CTA-uniform
        const int lo = s_lo[h][wid], span = s_hi[h][wid] - lo + w2;  // warp-uniform
        const int* Rel = Rel_all[h][wid];
        // groups committed: kBuf + r; round r's is complete once at most kBuf - 1 are pending
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kBuf - 1) : "memory");
        __syncthreads();
        if (k == 0 && tiled && span <= kSpanMax) {
            // the warp's weights for half h: Wd = 0, then each target's 2 msp weights
            // (contiguous in W for the run: one coalesced read) at rows Rel[t] .. of its span
            for (int e = lane; e < kSpanMax * kRun / 4; e += 32)
                reinterpret_cast<float4*>(&Wd[0][0])[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncwarp();
            {   // lane: target t = lane / 4, weights q = lane % 4, + 4, ...
                const int t = lane >> 2, rt = Rel[t];
                const float* Wr = A.W + (h * A.N + i0 + t) * w2;
                for (int q = lane & 3; q < w2; q += 4) Wd[rt + q][t] = __ldg(Wr + q);
            }
            __syncwarp();
        }
        float2 acc[kRun];
#pragma unroll
        for (int t = 0; t < kRun; ++t) acc[t] = make_float2(0.f, 0.f);
        if (tiled) {
            float2(*Hs)[32] = Hb + (r % kBuf) * kRowsMax;
            const int base = lo - s_tlo[h];
            if (live && span <= kSpanMax) {
                for (int pp = 0; pp < span; ++pp) {
                    const float2 hv = Hs[base + pp][lane];
                    const float4 wa = *reinterpret_cast<const float4*>(&Wd[pp][0]);
                    const float4 wb = *reinterpret_cast<const float4*>(&Wd[pp][4]);
                    const float ww[kRun] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                    for (int t = 0; t < kRun; ++t) nu_fma2(acc[t], ww[t], hv);
                }
            } else if (live) {  // the run's windows are far apart: each target on its own
#pragma unroll
                for (int t = 0; t < kRun; ++t) {
                    const int b0 = base + Rel[t];
                    for (int q = 0; q < w2; ++q) {
                        const float2 hv = Hs[b0 + q][lane];
                        const float w = __ldg(A.W + (h * A.N + i0 + t) * w2 + q);
                        acc[t].x = fmaf(w, hv.x, acc[t].x);
                        acc[t].y = fmaf(w, hv.y, acc[t].y);
                    }
                }
            }
        } else if (live) {
            const float2* Hh = A.H + (int64_t)h * A.n * A.Mc;
#pragma unroll
            for (int t = 0; t < kRun; ++t) {
                const int64_t i = i0 + t;
                const int p0 = __ldg(A.p0 + h * A.N + i);
                const float* w = A.W + (h * A.N + i) * w2;
                for (int q = 0; q < w2; ++q) {
                    const float wq = __ldg(w + q);
                    const float2 hv = __ldg(Hh + (int64_t)((p0 + q) & nmask) * A.Mc + k * A.m + c);
                    acc[t].x = fmaf(wq, hv.x, acc[t].x);
                    acc[t].y = fmaf(wq, hv.y, acc[t].y);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < kRun; ++t) {
            const float2 pk = __ldg(A.pa + ((int64_t)h * A.ra + k) * A.N + i0 + t);
            g[t].x = fmaf(pk.x, acc[t].x, fmaf(-pk.y, acc[t].y, g[t].x));
            g[t].y = fmaf(pk.x, acc[t].y, fmaf(pk.y, acc[t].x, g[t].y));
        }
        __syncthreads();  // buffer r % kBuf and the weights are free
        issue(r + kBuf);
    }
    if (live) {
#pragma unroll
        for (int t = 0; t < kRun; ++t) A.G[(i0 + t) * A.m + c] = g[t];
    }
}

// S = SA * SB with SA <= SB, both powers of two in [4, 32]
template <int PASS>
cudaError_t launch_pass(int S, const PassArgs& a, int64_t grid, size_t smem, cudaStream_t st)
{
    void* args[] = {(void*)&a};
    const void* fn = nullptr;
    switch (S) {
    case 16: fn = (const void*)nufft_pass<4, 4, PASS>; break;
    case 32: fn = (const void*)nufft_pass<4, 8, PASS>; break;
    case 64: fn = (const void*)nufft_pass<8, 8, PASS>; break;
    case 128: fn = (const void*)nufft_pass<8, 16, PASS>; break;
    case 256: fn = (const void*)nufft_pass<16, 16, PASS>; break;
    case 512: fn = (const void*)nufft_pass<16, 32, PASS>; break;
    case 1024: fn = (const void*)nufft_pass<32, 32, PASS>; break;
    default: return cudaErrorNotSupported;
    }
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kNuThreads), args, smem, st);
}

// columns per pass tile: a power of two, at most 64, at most 4096 / S (32 KB of shared
// memory, so that four 256-thread tiles share an SM), at most the column count rounded up
// to a power of two
int cbk_for(int S, int64_t Mc)
{
    int c = 1;
    while (c < 64 && (int64_t)c < Mc && c * 2 * S <= 4096) c *= 2;
    return c;
}

const double kTwoPiD = 6.283185307179586476925286766559;

}  // namespace

void nufft_free(bf_plan* p)
{
    NufftState* s = p->nufft;
    if (!s) return;
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(s->device);
    cudaFree(s->arena);
    cudaFree(s->ws);
    if (cur >= 0) cudaSetDevice(cur);
    delete s;
    p->nufft = nullptr;
}

}  // namespace bfi

using namespace bfi;

extern "C" bf_status bf_nufft_prepare(bf_plan* p, double eps, int* msp_out)
{
    if (!p || !(eps > 0.0 && eps < 1.0)) {
        set_error("bf_nufft_prepare: NULL plan or eps outside (0, 1)");
        return BF_ERR_ARG;
    }
    const int64_t N = p->N;
    if (N < 256 || N > ((int64_t)1 << 20)) {
        set_error("bf_nufft_prepare: N = %lld outside the NUFFT's range 256 .. 2^20", (long long)N);
        return BF_ERR_UNSUPPORTED;
    }
    double kap0, rho0;
    int xxi, sq;
    if (p->kern.indirect || !p->kern.row_terms(0, &kap0, &rho0, &xxi, &sq) || sq) {
        set_error("bf_nufft_prepare: the phase is not rank 1 on the column halves (built-in DFT, FIO, FIO_PW "
                  "and ONES phases only)");
        return BF_ERR_UNSUPPORTED;
    }
    // msp from eps: the error falls like exp(-2 pi msp / 3)
    int msp = (int)std::ceil(-std::log(eps) * 3.0 / kTwoPiD);
    msp = std::max(2, std::min(kMaxMsp, msp));
    nufft_free(p);
    // amplitude split on the whole window (Algorithm 1)
    std::vector<cd> a, b;
    int ra = 0;
    double sr = 0;
    bf_status st = amplitude_split(p->kern, p->opt, 0, 0, N, a, b, ra, sr);
    if (st != BF_OK) return st;
    NufftState* s = new NufftState;
    s->device = p->opt.device;
    s->N = N;
    s->M = N / 2;
    s->n = N;
    s->lg1 = 0;
    while (((int64_t)1 << s->lg1) < N) ++s->lg1;
    const int lgn = s->lg1;
    s->lg1 = (lgn + 1) / 2;
    s->lg2 = lgn - s->lg1;
    s->n1 = 1 << s->lg1;
    s->n2 = 1 << s->lg2;
    s->msp = msp;
    s->ra = ra;
    const int64_t M = s->M, n = s->n;
    const double tau = (double)msp / (2.0 * kTwoPiD * 3.0 * (double)M * (double)M);  // msp / (12 pi M^2)
    s->tau = tau;
    const int w2 = 2 * msp;
    std::vector<float2> bD((size_t)(2 * ra * M)), pa((size_t)(2 * ra * N)), tw((size_t)n);
    std::vector<float> W((size_t)(2 * N * w2));
    std::vector<int> p0((size_t)(2 * N));
    const double wnorm = 1.0 / ((double)n * std::sqrt(2.0 * kTwoPiD * tau));  // 1 / (n sqrt(4 pi tau))
#pragma omp parallel for schedule(static)
    for (int64_t idx = 0; idx < M; ++idx) {
        const int64_t jt = idx - M / 2;
        const double dec = std::exp(kTwoPiD * kTwoPiD * (double)jt * (double)jt * tau);  // 1/exp(-4 pi^2 jt^2 tau)
        for (int h = 0; h < 2; ++h) {
            const int64_t xi = jt + (h == 0 ? M / 2 : -(M / 2));
            const int64_t col = xi + N / 2;
            for (int k = 0; k < ra; ++k) {
                const cd v = b[(size_t)(k * N + col)] * dec;
                bD[(size_t)((h * ra + k) * M + idx)] = make_float2((float)v.real(), (float)v.imag());
            }
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double kap, rho;
        int xx, sq2;
        p->kern.row_terms(i, &kap, &rho, &xx, &sq2);
        const double x = (double)i / (double)N;
        for (int h = 0; h < 2; ++h) {
            double t = (xx ? x : 0.0) + (h == 0 ? kap : -kap);
            t -= std::floor(t);  // t mod 1 in [0, 1)
            const int64_t sh = h == 0 ? M / 2 : -(M / 2);
            // t s_h mod 1: the x xi part i s_h / N exactly in integers, the kappa part in FP64
            double ph = xx ? (double)((((i * sh) % N) + N) % N) / (double)N : 0.0;
            double kp = (h == 0 ? kap : -kap) * (double)sh;
            kp -= std::floor(kp);
            ph += kp + rho;
            ph -= std::floor(ph);
            const cd cent(std::cos(kTwoPiD * ph), std::sin(kTwoPiD * ph));
            for (int k = 0; k < ra; ++k) {
                const cd v = a[(size_t)(k * N + i)] * cent;
                pa[(size_t)((h * ra + k) * N + i)] = make_float2((float)v.real(), (float)v.imag());
            }
            const double nt = (double)n * t;
            const int64_t base = (int64_t)std::floor(nt);
            const int64_t first = base - msp + 1;
            p0[(size_t)(h * N + i)] = (int)(((first % n) + n) % n);
            for (int q = 0; q < w2; ++q) {
                const double d = t - (double)(first + q) / (double)n;
                W[(size_t)((h * N + i) * w2 + q)] = (float)(std::exp(-d * d / (4.0 * tau)) * wnorm);
            }
        }
    }
    for (int64_t k = 0; k < n; ++k) {
        const double ang = kTwoPiD * (double)k / (double)n;
        tw[(size_t)k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    float2 w32[32];
    for (int k = 0; k < 32; ++k)
        w32[k] = make_float2((float)std::cos(kTwoPiD * k / 32.0), (float)std::sin(kTwoPiD * k / 32.0));
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t o_bD = 0, o_pa = o_bD + al(bD.size() * 8), o_W = o_pa + al(pa.size() * 8),
                 o_p0 = o_W + al(W.size() * 4), o_tw = o_p0 + al(p0.size() * 4), total = o_tw + al(tw.size() * 8);
    int cur = -1;
    cudaGetDevice(&cur);
    if (cudaSetDevice(s->device) != cudaSuccess || cudaMalloc(&s->arena, total) != cudaSuccess) {
        set_error("bf_nufft_prepare: device allocation of %zu bytes failed", total);
        delete s;
        if (cur >= 0) cudaSetDevice(cur);
        return BF_ERR_NOMEM;
    }
    char* base = (char*)s->arena;
    s->bD = (float2*)(base + o_bD);
    s->pa = (float2*)(base + o_pa);
    s->W = (float*)(base + o_W);
    s->p0 = (int*)(base + o_p0);
    s->tw = (float2*)(base + o_tw);
    cudaError_t e = cudaMemcpy(s->bD, bD.data(), bD.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->pa, pa.data(), pa.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->W, W.data(), W.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->p0, p0.data(), p0.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w32, w32, sizeof(w32));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(nufft_interp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInterpSmem);
    if (cur >= 0) cudaSetDevice(cur);
    if (e != cudaSuccess) {
        set_error("bf_nufft_prepare: upload failed: %s", cudaGetErrorString(e));
        cudaFree(s->arena);
        delete s;
        return BF_ERR_CUDA;
    }
    p->nufft = s;
    if (msp_out) *msp_out = msp;
    return BF_OK;
}

namespace bfi {

size_t nufft_ws_bytes(const bf_plan* p, int64_t m)
{
    const NufftState* s = p->nufft;
    return s ? (size_t)4 * s->n * s->ra * m * sizeof(float2) : 0;
}

// The three launches of one NUFFT apply with a caller-owned workspace (T | H).
bf_status nufft_apply_ws(bf_plan* p, const void* F, int64_t m, void* G, void* stream, void* ws, size_t ws_bytes)
{
    NufftState* s = p->nufft;
    if (!s) {
        set_error("NUFFT apply: call bf_nufft_prepare first");
        return BF_ERR_STATE;
    }
    if (ws_bytes < nufft_ws_bytes(p, m)) {
        set_error("NUFFT apply: workspace of %zu bytes too small (%zu needed)", ws_bytes, nufft_ws_bytes(p, m));
        return BF_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t Mc = (int64_t)s->ra * m;
    float2* T = (float2*)ws;
    float2* H = T + 2 * s->n * Mc;
    PassArgs pa{};
    pa.F = (const float2*)F;
    pa.bD = s->bD;
    pa.tw = s->tw;
    pa.N = s->N;
    pa.M = s->M;
    pa.n = s->n;
    pa.m = m;
    pa.Mc = Mc;
    pa.n1 = s->n1;
    pa.n2 = s->n2;
    pa.lg1 = s->lg1;
    pa.lg2 = s->lg2;
    cudaError_t e = cudaSuccess;
    {   // pass 1: n2-point DFTs over j2 for every (half, j1, column block)
        PassArgs a1 = pa;
        a1.out = T;
        a1.cbk = cbk_for(s->n2, Mc);
        a1.nblk = (int)((Mc + a1.cbk - 1) / a1.cbk);
        ProfScope ps("nufft_pass1", st);
        e = launch_pass<1>(s->n2, a1, (int64_t)2 * s->n1 * a1.nblk, (size_t)s->n2 * (a1.cbk + 2) * sizeof(float2), st);
    }
    if (e == cudaSuccess) {   // pass 2: n1-point DFTs over j1 for every (half, p2, column block)
        PassArgs a2 = pa;
        a2.in = T;
        a2.out = H;
        a2.cbk = cbk_for(s->n1, Mc);
        a2.nblk = (int)((Mc + a2.cbk - 1) / a2.cbk);
        ProfScope ps("nufft_pass2", st);
        e = launch_pass<2>(s->n1, a2, (int64_t)2 * s->n2 * a2.nblk, (size_t)s->n1 * (a2.cbk + 2) * sizeof(float2), st);
    }
    if (e == cudaSuccess) {
        InterpArgs ia{H, s->pa, s->W, s->p0, (float2*)G, s->N, s->n, m, Mc, s->ra, s->msp};
        const int64_t ctas = (s->N / kTile) * ((m + 31) / 32);
        ProfScope ps("nufft_interp", st);
        nufft_interp<<<(unsigned)ctas, kNuThreads, kInterpSmem, st>>>(ia);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error("NUFFT apply: launch failed: %s", cudaGetErrorString(e));
        return BF_ERR_CUDA;
    }
    return BF_OK;
}

}  // namespace bfi

extern "C" bf_status bf_nufft_apply(bf_plan* p, const void* F, int64_t m, void* G, void* stream)
{
    if (!p || !F || !G || m < 1) {
        set_error("bf_nufft_apply: NULL plan/buffer or m < 1");
        return BF_ERR_ARG;
    }
    if (F == G) {
        set_error("bf_nufft_apply: G must not alias F");
        return BF_ERR_ARG;
    }
    NufftState* s = p->nufft;
    if (!s) {
        set_error("bf_nufft_apply: call bf_nufft_prepare first");
        return BF_ERR_STATE;
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    const size_t need = nufft_ws_bytes(p, m);
    bf_status rs = BF_OK;
    if (s->ws_bytes < need) {
        cudaFree(s->ws);
        s->ws = nullptr;
        s->ws_bytes = 0;
        if (cudaMalloc(&s->ws, need) != cudaSuccess) {
            set_error("bf_nufft_apply: workspace of %zu bytes", need);
            rs = BF_ERR_NOMEM;
        } else {
            s->ws_bytes = need;
        }
    }
    if (rs == BF_OK) rs = nufft_apply_ws(p, F, m, G, stream, s->ws, s->ws_bytes);
    if (cur >= 0 && cur != s->device) cudaSetDevice(cur);
    return rs;
}

extern "C" bf_status bf_nufft_info(const bf_plan* p, int* msp, int* r_alpha, int64_t* ws_bytes_per_rhs)
{
    if (!p || !p->nufft) {
        set_error("bf_nufft_info: no NUFFT state (bf_nufft_prepare)");
        return BF_ERR_STATE;
    }
    if (msp) *msp = p->nufft->msp;
    if (r_alpha) *r_alpha = p->nufft->ra;
    if (ws_bytes_per_rhs) *ws_bytes_per_rhs = (int64_t)4 * p->nufft->n * p->nufft->ra * (int64_t)sizeof(float2);
    return BF_OK;
}
