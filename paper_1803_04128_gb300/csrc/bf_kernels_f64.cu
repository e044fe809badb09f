// Plain FP64 apply: one launch per butterfly stage (V, each H level, switch,
// each G level, U), the coefficient state round-tripping through global
// memory.  One thread per output coefficient.  This is the unfused form the
// fused FP32 kernels are measured against.
//
// State layout of level l: X[q][t][col], q = a * 2^(L-l) + b, t < r,
// col = k * m + c (amplitude term k < r_alpha, right-hand side c < m).
#include "bf_device.h"

namespace bfi {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc)
{
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}

// V (Eq. 1 at level l1): mu[q][t][col] = sum_x Mv[t][x] EV[a][b nv + x] b_k[b nv + x] F[b nv + x][c]
__global__ void v_f64(Geo g, const double* Mv, const double2* EV, const double2* bk, const double2* F,
                      int64_t m, double2* out)
{
    const int64_t M = (int64_t)g.ra * m;
    const int64_t total = g.P * g.r * M;
    const int64_t nB = g.P >> g.l1;  // T_Omega nodes at level L - l1
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = idx % M;
        const int t = (int)((idx / M) % g.r);
        const int64_t q = idx / (M * g.r);
        const int64_t a = q / nB, b = q % nB;
        const int k = (int)(col / m);
        const int64_t c = col % m;
        double2 acc = make_double2(0, 0);
        for (int x = 0; x < g.nv; ++x) {
            const int64_t xi = b * g.nv + x;
            double2 y = cmul(bk[k * g.N + xi], F[xi * m + c]);
            double2 z = cmul(EV[a * g.N + xi], y);
            double w = Mv[t * g.nv + x];
            acc.x = fma(w, z.x, acc.x);
            acc.y = fma(w, z.y, acc.y);
        }
        out[idx] = acc;
    }
}

// H level l (Eq. 2): mu_l[q'][t] = sum_{c,s} MH[t][c r + s] EH[q'][c][s] mu_{l-1}[(a'>>1) 2^(L-l+1) + 2b' + c][s]
__global__ void h_f64(Geo g, int l, const double* MH, const double2* EH, const double2* in, int64_t M,
                      double2* out)
{
    const int r = g.r;
    const int64_t total = g.P * r * M;
    const int64_t nB = (int64_t)1 << (g.L - l);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = idx % M;
        const int t = (int)((idx / M) % r);
        const int64_t q = idx / (M * r);
        const int64_t a = q / nB, b = q % nB;
        const int64_t qin0 = (a >> 1) * (2 * nB) + 2 * b;
        double2 acc = make_double2(0, 0);
        for (int c = 0; c < 2; ++c)
            for (int s = 0; s < r; ++s) {
                double2 z = cmul(EH[(q * 2 + c) * r + s], in[((qin0 + c) * r + s) * M + col]);
                double w = MH[t * 2 * r + c * r + s];
                acc.x = fma(w, z.x, acc.x);
                acc.y = fma(w, z.y, acc.y);
            }
        out[idx] = acc;
    }
}

// switch (step 4): nu[q][t] = sum_s S[q][t][s] mu[q][s]
__global__ void s_f64(Geo g, const double2* S, const double2* in, int64_t M, double2* out)
{
    const int r = g.r;
    const int64_t total = g.P * r * M;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = idx % M;
        const int t = (int)((idx / M) % r);
        const int64_t q = idx / (M * r);
        double2 acc = make_double2(0, 0);
        for (int s = 0; s < r; ++s) acc = cfma(S[(q * r + t) * r + s], in[(q * r + s) * M + col], acc);
        out[idx] = acc;
    }
}

// G level l (Eq. 3): nu_l[q'][t] = sum_c FG[q'][c][t] sum_s MG[a' & 1][t][s] nu_{l-1}[(a'>>1) 2^(L-l+1) + 2b' + c][s]
__global__ void g_f64(Geo g, int l, const double* MG, const double2* FG, const double2* in, int64_t M,
                      double2* out)
{
    const int r = g.r;
    const int64_t total = g.P * r * M;
    const int64_t nB = (int64_t)1 << (g.L - l);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = idx % M;
        const int t = (int)((idx / M) % r);
        const int64_t q = idx / (M * r);
        const int64_t a = q / nB, b = q % nB;
        const int64_t qin0 = (a >> 1) * (2 * nB) + 2 * b;
        const double* Mp = MG + (a & 1) * r * r + t * r;
        double2 acc = make_double2(0, 0);
        for (int c = 0; c < 2; ++c) {
            double2 w = make_double2(0, 0);
            for (int s = 0; s < r; ++s) {
                double2 v = in[((qin0 + c) * r + s) * M + col];
                w.x = fma(Mp[s], v.x, w.x);
                w.y = fma(Mp[s], v.y, w.y);
            }
            acc = cfma(FG[(q * 2 + c) * r + t], w, acc);
        }
        out[idx] = acc;
    }
}

// U (Eq. bf3 at level L - l1) and the amplitude terms of Eq. (tg):
// G[x][c] = beta G[x][c] + sum_k a_k[x] sum_{b < 2^l1} EU[b][x] sum_s MU[x % nv][s] nu[(x / nv) 2^l1 + b][s][k m + c]
__global__ void u_f64(Geo g, const double* MU, const double2* EU, const double2* ak, const double2* in,
                      int64_t m, int beta, double2* G)
{
    const int r = g.r;
    const int64_t M = (int64_t)g.ra * m;
    const int64_t total = g.N * m;
    const int nC = 1 << g.l1;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = idx % m;
        const int64_t x = idx / m;
        const int64_t A = x / g.nv;
        const int i = (int)(x % g.nv);
        double2 res = beta ? G[idx] : make_double2(0, 0);
        for (int k = 0; k < g.ra; ++k) {
            double2 uk = make_double2(0, 0);
            for (int b = 0; b < nC; ++b) {
                const int64_t q = A * nC + b;
                double2 w = make_double2(0, 0);
                for (int s = 0; s < r; ++s) {
                    double2 v = in[(q * r + s) * M + k * m + c];
                    double mu = MU[i * r + s];
                    w.x = fma(mu, v.x, w.x);
                    w.y = fma(mu, v.y, w.y);
                }
                uk = cfma(EU[(int64_t)b * g.N + x], w, uk);
            }
            res = cfma(ak[k * g.N + x], uk, res);
        }
        G[idx] = res;
    }
}

inline int grid_for(int64_t total, int threads)
{
    int64_t b = (total + threads - 1) / threads;
    return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

}  // namespace

size_t plain_f64_ws_bytes(const Geo& g, int64_t m)
{
    return (size_t)g.P * g.r * g.ra * m * sizeof(double2);
}

cudaError_t launch_plain_f64(const DevBlock& B, const double2* F, int64_t m, double2* G, int beta,
                             double2* ws0, double2* ws1, cudaStream_t st)
{
    const Geo& g = B.g;
    const auto& f = B.f64;
    const int T = 256;
    const int64_t M = (int64_t)g.ra * m;
    const int64_t nst = g.P * g.r * M;
    if (g.ra == 0) {  // zero amplitude: G = beta G
        if (!beta) return cudaMemsetAsync(G, 0, (size_t)g.N * m * sizeof(double2), st);
        return cudaSuccess;
    }
    {
        ProfScope ps("v_f64", st);
        v_f64<<<grid_for(nst, T), T, 0, st>>>(g, f.Mv, f.EV, f.b, F, m, ws0);
    }
    double2 *cur = ws0, *nxt = ws1;
    for (int j = 0; j < g.kH; ++j) {
        const int l = g.l1 + 1 + j;
        {
        ProfScope ps("h_f64", st);
        h_f64<<<grid_for(nst, T), T, 0, st>>>(g, l, f.MH + (size_t)j * g.r * 2 * g.r,
                                                   f.EH + (size_t)j * g.P * 2 * g.r, cur, M, nxt);
    }
        std::swap(cur, nxt);
    }
    {
        ProfScope ps("s_f64", st);
        s_f64<<<grid_for(nst, T), T, 0, st>>>(g, f.S, cur, M, nxt);
    }
    std::swap(cur, nxt);
    for (int j = 0; j < g.kG; ++j) {
        const int l = g.h + 1 + j;
        {
        ProfScope ps("g_f64", st);
        g_f64<<<grid_for(nst, T), T, 0, st>>>(g, l, f.MG + (size_t)j * 2 * g.r * g.r,
                                                   f.FG + (size_t)j * g.P * 2 * g.r, cur, M, nxt);
    }
        std::swap(cur, nxt);
    }
    {
        ProfScope ps("u_f64", st);
        u_f64<<<grid_for(g.N * m, T), T, 0, st>>>(g, f.MU, f.EU, f.a, cur, m, beta, G);
    }
    return cudaGetLastError();
}

}  // namespace bfi
