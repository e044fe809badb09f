// Construction of the phase tables on the device (bf_factor_device).
//
// Every entry of the tables EV, EH, S, FG and EU is an explicit formula: a
// phase difference at grid points of the two trees (Sec. 4, Eqs. 1, 2, 3, bf3
// and the switch step of Algorithm 4.1), exponentiated.  The host builds the
// small parts (amplitude split, the real Lagrange matrices, the grids); these
// kernels fill the O(r N log N) phase tables straight into the FP64 and FP32
// arenas, one thread per entry, in FP64 with the x xi term reduced exactly in
// integers, as the host construction does.  Only the built-in phase kinds
// have a device form.
#include <vector>

#include "bf_device.h"
#include "bf_internal.h"

namespace bfi {
namespace {

struct Ph {
    int kind;
    double s;              // phase parameter of c(x)
    int64_t Ng, row0, col0;
    int lNg;               // log2 Ng (N is a power of two)
    const double* sx;      // sin(2 pi i / Ng) for every global row i
};

struct Grid {  // mock-Chebyshev indices relative to a node, r <= 16
    int64_t v[16];
};

__device__ __forceinline__ int64_t centre_d(int64_t start, int64_t n) { return start + (n - 1) / 2; }

// fractional phase Phi(x_i, xi_j) for block-local (i, j); the integer part is
// irrelevant after exponentiation.  Ng is a power of two, so the exact integer
// reductions mod Ng and mod 4 Ng are masks.
__device__ double phase_frac(const Ph& d, int64_t il, int64_t jl)
{
    const int64_t i = d.row0 + il, j = d.col0 + jl, Ng = d.Ng;
    const int64_t xi = j - Ng / 2;
    const double axi = (double)(xi < 0 ? -xi : xi);
    const double inv = 1.0 / (double)Ng;  // exact
    double t1 = 0.0, t2 = 0.0;
    switch (d.kind) {
    case BF_PHASE_DFT:
        t1 = (double)((i * xi) & (Ng - 1)) * inv;
        break;
    case BF_PHASE_FIO:
        t1 = (double)((i * xi) & (Ng - 1)) * inv;
        t2 = (2.0 + d.s * d.sx[i]) / 16.0 * axi;
        break;
    case BF_PHASE_FIO_PW: {
        t1 = (double)((i * xi) & (Ng - 1)) * inv;
        const double c = (2.0 + d.s * d.sx[i]) / 16.0;
        t2 = (2 * i < Ng) ? c * axi : -0.5 * c * axi;
        break;
    }
    case BF_PHASE_SEP:
        t2 = 0.3 * d.sx[i] + (double)((xi * xi) & (4 * Ng - 1)) * (0.25 * inv);
        break;
    default:  // BF_PHASE_ONES
        break;
    }
    t2 -= rint(t2);
    return t1 + t2;
}

__device__ __forceinline__ void put(double f, double2* o64, float2* o32, int64_t k)
{
    double s, c;
    sincospi(2.0 * f, &s, &c);
    o64[k] = make_double2(c, s);
    o32[k] = make_float2((float)c, (float)s);
}

__device__ __forceinline__ int64_t tid64() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }

__global__ void k_sinx(int64_t Ng, double* sx)
{
    const int64_t i = tid64();
    if (i < Ng) sx[i] = sinpi(2.0 * (double)i / (double)Ng);
}

// V (Eq. 1 at level l1): EV[a][j] = e(Phi(c_A, j)), A = a-th node at level l1
__global__ void k_ev(Ph d, int64_t nA, int64_t na, int lN, double2* o64, float2* o32)
{
    const int64_t k = tid64();
    if (k >= (nA << lN)) return;
    const int64_t a = k >> lN, j = k & ((1ll << lN) - 1);
    put(phase_frac(d, centre_d(a * na, na), j), o64, o32, k);
}

// H at level l (Eq. 2): EH[a][bb][c][s] = e(Phi(c_A, xi) - Phi(c_P, xi)), xi = bb nb + c nb/2 + gC[s];
// one thread per (pair, c), the r entries of s in a loop
__global__ void k_eh(Ph d, Grid gC, int r, int64_t nA, int64_t na, int lnBl, int64_t nb, double2* o64, float2* o32)
{
    const int64_t k = tid64();
    if (k >= (nA << lnBl) * 2) return;
    const int c = (int)(k & 1);
    const int64_t ab = k >> 1, a = ab >> lnBl, bb = ab & ((1ll << lnBl) - 1);
    const int64_t cA = centre_d(a * na, na), cP = centre_d((a >> 1) * 2 * na, 2 * na);
    for (int s = 0; s < r; ++s) {
        const int64_t xi = bb * nb + c * (nb / 2) + gC.v[s];
        put(phase_frac(d, cA, xi) - phase_frac(d, cP, xi), o64, o32, k * r + s);
    }
}

// switch at h: S[a][bb][t][s] = e(Phi(x, xi) - Phi(x, c_B) - Phi(c_A, xi)), x = a na + gA[t], xi = bb nb + gB[s];
// one thread per (pair, t); Phi(c_A, xi_s) for the r columns kept in registers
__global__ void k_s(Ph d, Grid gA, Grid gB, int r, int64_t nA, int64_t na, int lnBl, int64_t nb, double2* o64,
                    float2* o32)
{
    const int64_t k = tid64();
    if (k >= (nA << lnBl) * r) return;
    const int64_t ab = k / r;
    const int t = (int)(k - ab * r);
    const int64_t a = ab >> lnBl, bb = ab & ((1ll << lnBl) - 1);
    const int64_t x = a * na + gA.v[t];
    const int64_t cA = centre_d(a * na, na), cB = centre_d(bb * nb, nb);
    const double fxc = phase_frac(d, x, cB);
    for (int s = 0; s < r; ++s) {
        const int64_t xi = bb * nb + gB.v[s];
        put(phase_frac(d, x, xi) - fxc - phase_frac(d, cA, xi), o64, o32, k * r + s);
    }
}

// G at level l (Eq. 3): FG[a][bb][c][t] = e(Phi(x, c_C) - Phi(x, c_B)), x = a na + gA[t];
// one thread per (pair, c)
__global__ void k_fg(Ph d, Grid gA, int r, int64_t nA, int64_t na, int lnBl, int64_t nb, double2* o64, float2* o32)
{
    const int64_t k = tid64();
    if (k >= (nA << lnBl) * 2) return;
    const int c = (int)(k & 1);
    const int64_t ab = k >> 1, a = ab >> lnBl, bb = ab & ((1ll << lnBl) - 1);
    const int64_t cB = centre_d(bb * nb, nb), cC = centre_d(bb * nb + c * (nb / 2), nb / 2);
    for (int t = 0; t < r; ++t) {
        const int64_t x = a * na + gA.v[t];
        put(phase_frac(d, x, cC) - phase_frac(d, x, cB), o64, o32, k * r + t);
    }
}

// U (Eq. bf3 at level L-l1): EU[c][x] = e(Phi(x, c_C)), C = c-th node at level L-l1 of T_Omega
__global__ void k_eu(Ph d, int64_t nC, int64_t nc, int lN, double2* o64, float2* o32)
{
    const int64_t k = tid64();
    if (k >= (nC << lN)) return;
    const int64_t c = k >> lN, x = k & ((1ll << lN) - 1);
    put(phase_frac(d, x, centre_d(c * nc, nc)), o64, o32, k);
}

int log2i(int64_t v)
{
    int l = 0;
    while (((int64_t)1 << l) < v) ++l;
    return l;
}

Grid grid_of(int64_t n, int r)
{
    Grid g{};
    const std::vector<int64_t> v = grid_rel(n, r);
    for (size_t i = 0; i < v.size() && i < 16; ++i) g.v[i] = v[i];
    return g;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

bool construct_supported(int phase_kind)
{
    return phase_kind == BF_PHASE_DFT || phase_kind == BF_PHASE_FIO || phase_kind == BF_PHASE_FIO_PW ||
           phase_kind == BF_PHASE_ONES || phase_kind == BF_PHASE_SEP;
}

cudaError_t construct_tables(const BlockFactors& B, int phase_kind, double phase_param, int64_t n_global,
                             const DevFactors<double, double2>& f64, const DevFactors<float, float2>& f32,
                             cudaStream_t st)
{
    const int64_t N = B.N, P = B.P();
    const int r = B.r, L = B.L, h = B.h, l1 = B.l1, lN = log2i(N);
    double* sx = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&sx, (size_t)n_global * sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_sinx<<<blocks_for(n_global), 256, 0, st>>>(n_global, sx);
    const Ph d{phase_kind, phase_param, n_global, B.row0, B.col0, log2i(n_global), sx};
    {
        ProfScope ps("construct_ev", st);
        const int64_t nA = (int64_t)1 << l1, na = N >> l1;
        k_ev<<<blocks_for(nA * N), 256, 0, st>>>(d, nA, na, lN, f64.EV, f32.EV);
    }
    {
        ProfScope ps("construct_eh", st);
        int64_t off = 0;
        for (int l = l1 + 1; l <= h; ++l, off += P * 2 * r) {
            const int64_t nA = (int64_t)1 << l, na = N >> l, nb = N >> (L - l);
            k_eh<<<blocks_for(P * 2), 256, 0, st>>>(d, grid_of(nb / 2, r), r, nA, na, L - l, nb, f64.EH + off,
                                                    f32.EH + off);
        }
    }
    {
        ProfScope ps("construct_s", st);
        const int64_t nA = (int64_t)1 << h, na = N >> h, nb = N >> (L - h);
        k_s<<<blocks_for(P * r), 256, 0, st>>>(d, grid_of(na, r), grid_of(nb, r), r, nA, na, L - h, nb, f64.S, f32.S);
    }
    {
        ProfScope ps("construct_fg", st);
        int64_t off = 0;
        for (int l = h + 1; l <= L - l1; ++l, off += P * 2 * r) {
            const int64_t nA = (int64_t)1 << l, na = N >> l, nb = N >> (L - l);
            k_fg<<<blocks_for(P * 2), 256, 0, st>>>(d, grid_of(na, r), r, nA, na, L - l, nb, f64.FG + off,
                                                    f32.FG + off);
        }
    }
    {
        ProfScope ps("construct_eu", st);
        const int64_t nC = (int64_t)1 << l1, nc = N >> l1;
        k_eu<<<blocks_for(nC * N), 256, 0, st>>>(d, nC, nc, lN, f64.EU, f32.EU);
    }
    e = cudaGetLastError();
    cudaFreeAsync(sx, st);
    return e;
}

}  // namespace bfi
