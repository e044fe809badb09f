// Fused FP32 apply of one sub-BF in two launches.
//
// Front pass (one CTA per tile x column slice): reads 2^kH consecutive
// xi-leaves of F, applies V (Eq. 1), all kH H levels (Eq. 2) and the switch
// (step 4 of Algorithm 4.1) with the coefficients held in shared memory, and
// writes the switch-level coefficients.  A front tile is fixed by an x-node p
// at level l1 and a chunk c0 of T_Omega nodes: its 2^kH pairs stay closed
// under the kH H levels because the pair (A, B) at level l only depends on
// (parent(A), children(B)) at level l-1 (Sec. 4, "C > B", "P is A's parent").
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
// Columns: a tile carries CT = r_alpha * mr columns, col = k * mr + c
// (amplitude term k, right-hand side slice * mr + c).  Global state between
// the passes: W[slice][q][t][CT] (q = switch-level pair index).
#include <cstdio>

#include "bf_device.h"

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
__device__ __forceinline__ unsigned brev(unsigned v, int bits)
{
    return bits == 0 ? 0u : (__brev(v) >> (32 - bits));
}

struct FrontArgs {
    Geo g;
    const float2* F;  // [N][m]
    int64_t m;
    int mr, CT, nslice;
    const float2* bk;  // [ra][N]
    const float* MvT;  // [nv][R]
    const float2* EV;  // [2^l1][N]
    const float* MHT;  // [kH][2R][R]
    const float2* EH;  // [kH][P][2][R]
    const float2* S;   // [P][R][R]
    float2* W;         // [nslice][P][R][CT]
};

struct BackArgs {
    Geo g;
    int64_t m;
    int mr, CT, nslice;
    const float2* W;
    const float* MGT;  // [kG][2][R][R]  (pos, s, t)
    const float2* FG;  // [kG][P][2][R]
    const float* MU;   // [nv][R]
    const float2* EU;  // [2^l1][N]
    const float2* ak;  // [ra][N]
    float2* G;         // [N][m]
    int beta;
};

// ------------------------------------------------------------------ front --
template <int R>
__global__ void __launch_bounds__(kThreads, 2) front_f32(FrontArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geo& g = A.g;
    const int K = g.kH, T = 1 << K, CT = A.CT, mr = A.mr, nv = g.nv;
    const int slice = blockIdx.x % A.nslice;
    const int64_t tile = blockIdx.x / A.nslice;
    const int nP = 1 << g.l1;                  // x-nodes at level l1
    const int64_t p = tile % nP, c0 = tile / nP;
    const int64_t nBh = (int64_t)1 << (g.L - g.h);  // T_Omega nodes at level L-h

    float2* X = reinterpret_cast<float2*>(smem_raw);             // [T][R][CT]
    float2* EHs = X + (size_t)T * R * CT;                         // [K][T][2][R]
    float2* Ss = EHs + (size_t)K * T * 2 * R;                     // [T][R][R]
    float2* EVs = Ss + (size_t)T * R * R;                         // [T*nv]
    float* MvTs = reinterpret_cast<float*>(EVs + (size_t)T * nv); // [nv][R]
    float* MHTs = MvTs + nv * R;                                  // [K][2R][R]

    const int tid = threadIdx.x;
    // ---- stage factors of this tile into shared memory
    for (int e = tid; e < nv * R; e += kThreads) MvTs[e] = A.MvT[e];
    for (int e = tid; e < K * 2 * R * R; e += kThreads) MHTs[e] = A.MHT[e];
    {
        const float2* ev = A.EV + p * g.N + c0 * T * nv;
        for (int e = tid; e < T * nv; e += kThreads) EVs[e] = ev[e];
    }
    for (int j = 1; j <= K; ++j) {
        const int l = g.l1 + j;
        const int64_t nBl = (int64_t)1 << (g.L - l);
        const float2* eh = A.EH + (size_t)(j - 1) * g.P * 2 * R;
        for (int e = tid; e < T * 2 * R; e += kThreads) {
            const int lp = e / (2 * R), w = e % (2 * R);
            const int64_t ap = (p << j) + (lp >> (K - j));
            const int64_t bp = (c0 << (K - j)) + (lp & ((1 << (K - j)) - 1));
            EHs[((size_t)(j - 1) * T + lp) * 2 * R + w] = eh[(ap * nBl + bp) * 2 * R + w];
        }
    }
    for (int e = tid; e < T * R * R; e += kThreads) {
        const int lp = e / (R * R), w = e % (R * R);
        const int64_t q = ((p << K) + lp) * nBh + c0;
        Ss[(size_t)lp * R * R + w] = A.S[q * R * R + w];
    }
    __syncthreads();

    // ---- V (Eq. 1): item (j, c) computes mu[j][.][k*mr + c] for every k
    for (int it = tid; it < T * mr; it += kThreads) {
        const int j = it / mr, c = it % mr;
        const int64_t cg = (int64_t)slice * mr + c;
        const bool valid = cg < A.m;
        const int64_t xi0 = (c0 * T + j) * nv;
        for (int k = 0; k < g.ra; ++k) {
            float2 acc[R];
#pragma unroll
            for (int t = 0; t < R; ++t) acc[t] = make_float2(0.f, 0.f);
            const float2* bk = A.bk + (size_t)k * g.N + xi0;
            for (int x = 0; x < nv; ++x) {
                float2 f = valid ? A.F[(xi0 + x) * A.m + cg] : make_float2(0.f, 0.f);
                float2 z = cmulf(EVs[j * nv + x], cmulf(__ldg(bk + x), f));
#pragma unroll
                for (int t4 = 0; t4 < R / 2; ++t4) {
                    // R is even: read pairs of weights
                    float2 w = reinterpret_cast<const float2*>(MvTs + x * R)[t4];
                    acc[2 * t4].x = fmaf(w.x, z.x, acc[2 * t4].x);
                    acc[2 * t4].y = fmaf(w.x, z.y, acc[2 * t4].y);
                    acc[2 * t4 + 1].x = fmaf(w.y, z.x, acc[2 * t4 + 1].x);
                    acc[2 * t4 + 1].y = fmaf(w.y, z.y, acc[2 * t4 + 1].y);
                }
            }
            float2* xo = X + (size_t)j * R * CT + k * mr + c;
#pragma unroll
            for (int t = 0; t < R; ++t) xo[t * CT] = acc[t];
        }
    }

    // ---- H levels (Eq. 2), in place
    for (int j = 1; j <= K; ++j) {
        __syncthreads();
        const int half = 1 << (K - j);  // b' range
        const float* Mh = MHTs + (size_t)(j - 1) * 2 * R * R;
        const float2* Eh = EHs + (size_t)(j - 1) * T * 2 * R;
        for (int it = tid; it < (T / 2) * CT; it += kThreads) {
            const int grp = it / CT, col = it % CT;
            const int a = grp / half, bp = grp % half;
            const int base = (bp << j) + (int)brev((unsigned)a, j - 1);
            float2* x0 = X + (size_t)base * R * CT + col;
            float2* x1 = X + (size_t)(base + (1 << (j - 1))) * R * CT + col;
            float2 lam[2 * R];
#pragma unroll
            for (int s = 0; s < R; ++s) {
                lam[s] = x0[s * CT];
                lam[R + s] = x1[s * CT];
            }
            const float2* E0 = Eh + (size_t)((2 * a) * half + bp) * 2 * R;
            const float2* E1 = Eh + (size_t)((2 * a + 1) * half + bp) * 2 * R;
            float2 o0[R], o1[R];
#pragma unroll
            for (int t = 0; t < R; ++t) o0[t] = o1[t] = make_float2(0.f, 0.f);
#pragma unroll
            for (int cs = 0; cs < 2 * R; ++cs) {
                const float2 u0 = cmulf(E0[cs], lam[cs]);
                const float2 u1 = cmulf(E1[cs], lam[cs]);
                const float2* mh = reinterpret_cast<const float2*>(Mh + cs * R);
#pragma unroll
                for (int t2 = 0; t2 < R / 2; ++t2) {
                    const float2 w = mh[t2];
                    o0[2 * t2].x = fmaf(w.x, u0.x, o0[2 * t2].x);
                    o0[2 * t2].y = fmaf(w.x, u0.y, o0[2 * t2].y);
                    o0[2 * t2 + 1].x = fmaf(w.y, u0.x, o0[2 * t2 + 1].x);
                    o0[2 * t2 + 1].y = fmaf(w.y, u0.y, o0[2 * t2 + 1].y);
                    o1[2 * t2].x = fmaf(w.x, u1.x, o1[2 * t2].x);
                    o1[2 * t2].y = fmaf(w.x, u1.y, o1[2 * t2].y);
                    o1[2 * t2 + 1].x = fmaf(w.y, u1.x, o1[2 * t2 + 1].x);
                    o1[2 * t2 + 1].y = fmaf(w.y, u1.y, o1[2 * t2 + 1].y);
                }
            }
#pragma unroll
            for (int t = 0; t < R; ++t) {
                x0[t * CT] = o0[t];
                x1[t * CT] = o1[t];
            }
        }
    }
    __syncthreads();

    // ---- switch (step 4) and write-out of the switch-level coefficients
    float2* Wout = A.W + (size_t)slice * g.P * R * CT;
    for (int it = tid; it < T * CT; it += kThreads) {
        const int lp = it / CT, col = it % CT;
        const int slot = (int)brev((unsigned)lp, K);
        const float2* xs = X + (size_t)slot * R * CT + col;
        float2 mu[R];
#pragma unroll
        for (int s = 0; s < R; ++s) mu[s] = xs[s * CT];
        const float2* Sp = Ss + (size_t)lp * R * R;
        const int64_t q = ((p << K) + lp) * nBh + c0;
        float2* wo = Wout + (size_t)q * R * CT + col;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int s = 0; s < R; ++s) cfmaf(acc, Sp[t * R + s], mu[s]);
            wo[t * CT] = acc;
        }
    }
}

// ------------------------------------------------------------------- back --
template <int R, int NU>
__global__ void __launch_bounds__(kThreads, 2) back_f32(BackArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geo& g = A.g;
    const int K = g.kG, T = 1 << K, CT = A.CT, mr = A.mr, nu = g.nv;
    const int slice = blockIdx.x % A.nslice;
    const int64_t pp = blockIdx.x / A.nslice;     // x-node at level h
    const int nC = 1 << g.l1;                      // chunks c0' (= T_Omega nodes at level l1)
    const int64_t nBh = (int64_t)1 << (g.L - g.h);
    const int XN = T * nu;                         // output points of this CTA

    float2* X = reinterpret_cast<float2*>(smem_raw);    // [T][R][CT]
    float2* FGs = X + (size_t)T * R * CT;                // [K][T][2][R]
    float2* EUs = FGs + (size_t)K * T * 2 * R;           // [XN]
    float2* acc = EUs + XN;                              // [XN][mr]
    float* MGTs = reinterpret_cast<float*>(acc + (size_t)XN * mr);  // [K][2][R][R]
    float* MUs = MGTs + (size_t)K * 2 * R * R;                       // [nu][R]

    const int tid = threadIdx.x;
    for (int e = tid; e < K * 2 * R * R; e += kThreads) MGTs[e] = A.MGT[e];
    for (int e = tid; e < nu * R; e += kThreads) MUs[e] = A.MU[e];
    for (int e = tid; e < XN * mr; e += kThreads) acc[e] = make_float2(0.f, 0.f);
    const float2* Win = A.W + (size_t)slice * g.P * R * CT;
    const int64_t x0g = pp * XN;

    for (int c0 = 0; c0 < nC; ++c0) {
        __syncthreads();
        {   // coefficients of pairs (pp, c0 * T + j), j < T: one contiguous block
            const float4* src = reinterpret_cast<const float4*>(Win + (size_t)(pp * nBh + (int64_t)c0 * T) * R * CT);
            float4* dst = reinterpret_cast<float4*>(X);
            const int n4 = T * R * CT / 2;
            for (int e = tid; e < n4; e += kThreads) dst[e] = src[e];
            if ((T * R * CT) & 1) {
                if (tid == 0) X[T * R * CT - 1] = Win[(size_t)(pp * nBh + (int64_t)c0 * T) * R * CT + T * R * CT - 1];
            }
        }
        for (int j = 1; j <= K; ++j) {
            const int l = g.h + j;
            const int64_t nBl = (int64_t)1 << (g.L - l);
            const float2* fg = A.FG + (size_t)(j - 1) * g.P * 2 * R;
            for (int e = tid; e < T * 2 * R; e += kThreads) {
                const int lp = e / (2 * R), w = e % (2 * R);
                const int64_t ap = (pp << j) + (lp >> (K - j));
                const int64_t bp = ((int64_t)c0 << (K - j)) + (lp & ((1 << (K - j)) - 1));
                FGs[((size_t)(j - 1) * T + lp) * 2 * R + w] = fg[(ap * nBl + bp) * 2 * R + w];
            }
        }
        for (int e = tid; e < XN; e += kThreads) EUs[e] = A.EU[(size_t)c0 * g.N + x0g + e];

        // ---- G levels (Eq. 3), in place
        for (int j = 1; j <= K; ++j) {
            __syncthreads();
            const int half = 1 << (K - j);
            const float* Mg = MGTs + (size_t)(j - 1) * 2 * R * R;
            const float2* Fg = FGs + (size_t)(j - 1) * T * 2 * R;
            for (int it = tid; it < (T / 2) * CT; it += kThreads) {
                const int grp = it / CT, col = it % CT;
                const int a = grp / half, bp = grp % half;
                const int base = (bp << j) + (int)brev((unsigned)a, j - 1);
                float2* x0 = X + (size_t)base * R * CT + col;
                float2* x1 = X + (size_t)(base + (1 << (j - 1))) * R * CT + col;
                float2 nu0[R], nu1[R];
#pragma unroll
                for (int s = 0; s < R; ++s) {
                    nu0[s] = x0[s * CT];
                    nu1[s] = x1[s * CT];
                }
#pragma unroll
                for (int pos = 0; pos < 2; ++pos) {
                    // w_c = MG[pos] nu_c, for both children c
                    float2 w0[R], w1[R];
#pragma unroll
                    for (int t = 0; t < R; ++t) w0[t] = w1[t] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int s = 0; s < R; ++s) {
                        const float2* mg = reinterpret_cast<const float2*>(Mg + (pos * R + s) * R);
#pragma unroll
                        for (int t2 = 0; t2 < R / 2; ++t2) {
                            const float2 w = mg[t2];
                            w0[2 * t2].x = fmaf(w.x, nu0[s].x, w0[2 * t2].x);
                            w0[2 * t2].y = fmaf(w.x, nu0[s].y, w0[2 * t2].y);
                            w0[2 * t2 + 1].x = fmaf(w.y, nu0[s].x, w0[2 * t2 + 1].x);
                            w0[2 * t2 + 1].y = fmaf(w.y, nu0[s].y, w0[2 * t2 + 1].y);
                            w1[2 * t2].x = fmaf(w.x, nu1[s].x, w1[2 * t2].x);
                            w1[2 * t2].y = fmaf(w.x, nu1[s].y, w1[2 * t2].y);
                            w1[2 * t2 + 1].x = fmaf(w.y, nu1[s].x, w1[2 * t2 + 1].x);
                            w1[2 * t2 + 1].y = fmaf(w.y, nu1[s].y, w1[2 * t2 + 1].y);
                        }
                    }
                    const float2* Fp = Fg + (size_t)((2 * a + pos) * half + bp) * 2 * R;  // [c][t]
                    float2* xo = pos ? x1 : x0;
#pragma unroll
                    for (int t = 0; t < R; ++t) {
                        float2 o = cmulf(Fp[t], w0[t]);
                        cfmaf(o, Fp[R + t], w1[t]);
                        xo[t * CT] = o;
                    }
                }
            }
        }
        __syncthreads();

        // ---- U (Eq. bf3) contribution of T_Omega node c0 to this CTA's points
        for (int it = tid; it < T * mr; it += kThreads) {
            const int lp = it / mr, c = it % mr;
            const int slot = (int)brev((unsigned)lp, K);
            const float2* xs = X + (size_t)slot * R * CT + c;
            float2 res[NU];
#pragma unroll
            for (int i = 0; i < NU; ++i) res[i] = make_float2(0.f, 0.f);
            for (int k = 0; k < g.ra; ++k) {
                float2 v[R];
#pragma unroll
                for (int s = 0; s < R; ++s) v[s] = xs[s * CT + k * mr];
#pragma unroll
                for (int i = 0; i < NU; ++i) {
                    if (i < nu) {
                        float2 w = make_float2(0.f, 0.f);
                        const float2* mu = reinterpret_cast<const float2*>(MUs + i * R);
#pragma unroll
                        for (int s2 = 0; s2 < R / 2; ++s2) {
                            const float2 m2 = mu[s2];
                            w.x = fmaf(m2.x, v[2 * s2].x, fmaf(m2.y, v[2 * s2 + 1].x, w.x));
                            w.y = fmaf(m2.x, v[2 * s2].y, fmaf(m2.y, v[2 * s2 + 1].y, w.y));
                        }
                        const int64_t xg = x0g + lp * nu + i;
                        cfmaf(res[i], cmulf(__ldg(A.ak + (size_t)k * g.N + xg), EUs[lp * nu + i]), w);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < NU; ++i)
                if (i < nu) {
                    float2* ap = acc + (size_t)(lp * nu + i) * mr + c;
                    ap->x += res[i].x;
                    ap->y += res[i].y;
                }
        }
    }
    __syncthreads();
    // ---- write G
    for (int it = tid; it < XN * mr; it += kThreads) {
        const int x = it / mr, c = it % mr;
        const int64_t cg = (int64_t)slice * mr + c;
        if (cg >= A.m) continue;
        float2* gp = A.G + (x0g + x) * A.m + cg;
        float2 v = acc[it];
        if (A.beta) {
            float2 o = *gp;
            v.x += o.x;
            v.y += o.y;
        }
        *gp = v;
    }
}

size_t front_smem(const Geo& g, int R, int CT)
{
    const int T = 1 << g.kH;
    return sizeof(float2) * ((size_t)T * R * CT + (size_t)g.kH * T * 2 * R + (size_t)T * R * R + (size_t)T * g.nv) +
           sizeof(float) * ((size_t)g.nv * R + (size_t)g.kH * 2 * R * R);
}

size_t back_smem(const Geo& g, int R, int CT, int mr)
{
    const int T = 1 << g.kG;
    const size_t XN = (size_t)T * g.nv;
    return sizeof(float2) * ((size_t)T * R * CT + (size_t)g.kG * T * 2 * R + XN + XN * mr) +
           sizeof(float) * ((size_t)g.kG * 2 * R * R + (size_t)g.nv * R);
}

template <int R, int NU>
cudaError_t launch_r(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws,
                     cudaStream_t st)
{
    const Geo& g = B.g;
    const FusedCfg cfg = fused_f32_config(g, m);
    FrontArgs fa;
    fa.g = g;
    fa.F = F;
    fa.m = m;
    fa.mr = cfg.mr;
    fa.CT = g.ra * cfg.mr;
    fa.nslice = cfg.nslice;
    fa.bk = B.f32.b;
    fa.MvT = B.f32.Mv;
    fa.EV = B.f32.EV;
    fa.MHT = B.f32.MH;
    fa.EH = B.f32.EH;
    fa.S = B.f32.S;
    fa.W = ws;
    const size_t sf = front_smem(g, R, fa.CT);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(front_f32<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(back_f32<R, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const int64_t ntile = ((int64_t)1 << g.l1) * ((int64_t)1 << (g.L - g.h));
    {
        ProfScope ps("front_f32", st);
        front_f32<R><<<(unsigned)(ntile * cfg.nslice), kThreads, sf, st>>>(fa);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    BackArgs ba;
    ba.g = g;
    ba.m = m;
    ba.mr = cfg.mr;
    ba.CT = fa.CT;
    ba.nslice = cfg.nslice;
    ba.W = ws;
    ba.MGT = B.f32.MG;
    ba.FG = B.f32.FG;
    ba.MU = B.f32.MU;
    ba.EU = B.f32.EU;
    ba.ak = B.f32.a;
    ba.G = G;
    ba.beta = beta;
    const size_t sb = back_smem(g, R, fa.CT, cfg.mr);
    const int64_t nback = ((int64_t)1 << g.h) * cfg.nslice;
    {
        ProfScope ps("back_f32", st);
        back_f32<R, NU><<<(unsigned)nback, kThreads, sb, st>>>(ba);
    }
    return cudaGetLastError();
}

}  // namespace

bool fused_f32_supported(int r) { return r == 6 || r == 8 || r == 10 || r == 12 || r == 14 || r == 16; }

FusedCfg fused_f32_config(const Geo& g, int64_t m)
{
    const int Tmax = 1 << (g.kG > g.kH ? g.kG : g.kH);
    const int ra = g.ra > 0 ? g.ra : 1;
    // about 256 (group, column) items per level, and a tile of at most 48 KB
    int mr = 512 / (Tmax * ra);
    const int cap = (int)(48 * 1024 / ((size_t)Tmax * g.r * ra * sizeof(float2)));
    if (mr > cap) mr = cap;
    if (mr > 64) mr = 64;
    if (mr < 1) mr = 1;
    if ((int64_t)mr > m) mr = (int)m;
    // keep mr a power of two so that CT = ra * mr packs warps evenly
    int p2 = 1;
    while (p2 * 2 <= mr) p2 *= 2;
    mr = p2;
    FusedCfg c;
    c.mr = mr;
    c.nslice = (int)((m + mr - 1) / mr);
    return c;
}

size_t fused_f32_ws_bytes(const Geo& g, int64_t m)
{
    const FusedCfg c = fused_f32_config(g, m);
    return (size_t)c.nslice * g.P * g.r * g.ra * c.mr * sizeof(float2);
}

cudaError_t launch_fused_f32(const DevBlock& B, const float2* F, int64_t m, float2* G, int beta, float2* ws,
                             cudaStream_t st)
{
    if (B.g.ra == 0) {
        if (!beta) return cudaMemsetAsync(G, 0, (size_t)B.g.N * m * sizeof(float2), st);
        return cudaSuccess;
    }
    if (B.g.nv > 2 * B.g.r) return cudaErrorNotSupported;
    switch (B.g.r) {
    case 6: return launch_r<6, 12>(B, F, m, G, beta, ws, st);
    case 8: return launch_r<8, 16>(B, F, m, G, beta, ws, st);
    case 10: return launch_r<10, 20>(B, F, m, G, beta, ws, st);
    case 12: return launch_r<12, 24>(B, F, m, G, beta, ws, st);
    case 14: return launch_r<14, 28>(B, F, m, G, beta, ws, st);
    case 16: return launch_r<16, 32>(B, F, m, G, beta, ws, st);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace bfi
