// Host FP64 construction of the IBF-MAT factors (off the timed path).
//
//  * amplitude split alpha ~ sum_k a_k(x) b_k(xi) by Algorithm 1 (Sec. 2.1);
//  * the butterfly factors of Eq. (BFM), Sec. 4, from the interpolative
//    low-rank factors of Algorithm 2 arranged by Algorithm 4.1, stored in a
//    factored form: each level's transfer is
//        (diagonal of phases) x (real Lagrange matrix, shared by all pairs of
//        the level) x (diagonal of phases),
//    which is the same sparse factor the paper stores, with its O(r^2) dense
//    blocks written as products of their diagonal and real parts.
//
// Let mu^{AB}_t = e^{2 pi i Phi(c_A, xi^B_t)} lambda^{AB}_t on the xi side and
// nu^{AB}_t = e^{-2 pi i Phi(x^A_t, c_B)} lambda^{AB}_t on the x side.  Then
//   V (Eq. 1, level l1):   mu^{AB}   = Mv (e^{2 pi i Phi(c_A, .)} y|_B)
//   H (Eq. 2, l1 < l <= h): mu^{AB}  = MH_l [EH_{A,C1} mu^{PC1}; EH_{A,C2} mu^{PC2}],
//                           EH_{A,C,s} = e^{2 pi i (Phi(c_A, xi^C_s) - Phi(c_P, xi^C_s))}
//   switch (step 4, l = h): nu^{AB}_t = sum_s S_{ts} mu^{AB}_s,
//                           S_{ts} = e^{2 pi i (Phi(x^A_t, xi^B_s) - Phi(x^A_t, c_B) - Phi(c_A, xi^B_s))}
//   G (Eq. 3, h < l <= L-l1): nu^{AB} = sum_{C > B} FG_{A,C} (MG_{pos(A)} nu^{PC}),
//                           FG_{A,C,t} = e^{2 pi i (Phi(x^A_t, c_C) - Phi(x^A_t, c_B))}
//   U (Eq. bf3, l = L-l1):  u(x) = sum_{C} e^{2 pi i Phi(x, c_C)} (MU nu^{AC})(x)
// Levels whose nodes have <= r indices use every index as grid point; there
// Algorithm 4.1 only copies (xi side) or sums (x side) coefficients, and those
// levels are folded into V (first l1 levels) and U (last l1 levels).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <omp.h>

#include "bf_internal.h"

namespace bfi {

static const double kTwoPi = 6.283185307179586476925286766559;

static int64_t mod_pos(int64_t a, int64_t n)
{
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

static inline cd expi(double frac) { return cd(std::cos(kTwoPi * frac), std::sin(kTwoPi * frac)); }

double PhaseLR::value(int64_t i, int64_t j) const
{
    const int64_t il = i - row0, jl = j - col0;
    double v = 0.0;
    for (int k = 0; k < rank; ++k) {
        const cd a = p[(size_t)k * N + il], b = q[(size_t)k * N + jl];
        v += a.real() * b.real() - a.imag() * b.imag();
    }
    return v;
}

double KernelFn::phase_frac(int64_t i, int64_t j) const
{
    if (indirect) {
        double t = lr ? lr->value(i, j) : std::arg(entry(i, j)) / kTwoPi;
        t -= std::floor(t);
        return t - std::nearbyint(t);
    }
    return phase_frac_explicit(i, j);
}

cd KernelFn::amplitude(int64_t i, int64_t j) const
{
    return indirect ? cd(std::abs(entry(i, j))) : amplitude_explicit(i, j);
}

void KernelFn::entries_matvec(const int64_t* I, const int64_t* J, int64_t n, cd* out) const
{
    // serve the pairs from whole columns when they touch fewer distinct columns than
    // rows, else from whole rows; unit vectors go through the callback in blocks of nb
    const int64_t Ng = n_global;
    std::vector<int64_t> rows(I, I + n), cols(J, J + n);
    for (auto* v : {&rows, &cols}) {
        std::sort(v->begin(), v->end());
        v->erase(std::unique(v->begin(), v->end()), v->end());
    }
    const bool by_cols = cols.size() <= rows.size();
    const std::vector<int64_t>& keys = by_cols ? cols : rows;
    std::vector<int64_t> kidx((size_t)n);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t)
        kidx[(size_t)t] = std::lower_bound(keys.begin(), keys.end(), by_cols ? J[t] : I[t]) - keys.begin();
    const int64_t nk = (int64_t)keys.size();
    const int64_t nb = std::max<int64_t>(1, std::min<int64_t>(64, ((int64_t)1 << 23) / Ng));  // <= 128 MB per buffer
    std::vector<cd> X((size_t)(Ng * std::min(nb, nk))), Y(X.size());
    for (int64_t k0 = 0; k0 < nk; k0 += nb) {
        const int64_t w = std::min(nb, nk - k0);
        std::fill(X.begin(), X.begin() + Ng * w, cd(0));
        for (int64_t c = 0; c < w; ++c) X[(size_t)(keys[(size_t)(k0 + c)] * w + c)] = cd(1);
        d.matvec(reinterpret_cast<const double*>(X.data()), w, by_cols ? 0 : 1, d.user,
                 reinterpret_cast<double*>(Y.data()));
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < n; ++t) {
            const int64_t c = kidx[(size_t)t] - k0;
            if (c < 0 || c >= w) continue;
            out[t] = Y[(size_t)((by_cols ? I[t] : J[t]) * w + c)];   // (K e_j)[i] or (K^T e_i)[j]
        }
    }
}

void KernelFn::entries(const int64_t* I, const int64_t* J, int64_t n, cd* out) const
{
    if (bulk() && !d.entries) {
        entries_matvec(I, J, n, out);
        return;
    }
    if (bulk()) {
        constexpr int64_t kPiece = (int64_t)1 << 20;
        for (int64_t s = 0; s < n; s += kPiece)
            d.entries(I + s, J + s, std::min(kPiece, n - s), d.user, reinterpret_cast<double*>(out + s));
        return;
    }
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t) out[t] = entry(I[t], J[t]);
}

cd KernelFn::entry(int64_t i, int64_t j) const
{
    if (bulk()) {
        cd v;
        entries(&i, &j, 1, &v);
        return v;
    }
    if (d.phase_kind == BF_PHASE_ENTRIES) {
        double re = 0, im = 0;
        d.entry((double)i / (double)n_global, (double)(j - n_global / 2), d.user, &re, &im);
        return cd(re, im);
    }
    return amplitude_explicit(i, j) * expi(phase_frac_explicit(i, j));
}

double KernelFn::phase_frac_explicit(int64_t i, int64_t j) const
{
    const int64_t Ng = n_global;
    const int64_t xi = j - Ng / 2;
    const double x = (double)i / (double)Ng;
    const double axi = (double)(xi < 0 ? -xi : xi);
    const double s = d.phase_param;
    double t1 = 0.0, t2 = 0.0;
    switch (d.phase_kind) {
    case BF_PHASE_DFT:
        t1 = (double)mod_pos(i * xi, Ng) / (double)Ng;
        break;
    case BF_PHASE_FIO:
        t1 = (double)mod_pos(i * xi, Ng) / (double)Ng;
        t2 = (2.0 + s * std::sin(kTwoPi * x)) / 16.0 * axi;
        break;
    case BF_PHASE_FIO_PW: {
        t1 = (double)mod_pos(i * xi, Ng) / (double)Ng;
        const double c = (2.0 + s * std::sin(kTwoPi * x)) / 16.0;
        t2 = (2 * i < Ng) ? c * axi : -0.5 * c * axi;
        break;
    }
    case BF_PHASE_ONES:
        break;
    case BF_PHASE_SEP:
        t2 = 0.3 * std::sin(kTwoPi * x) + (double)mod_pos(xi * xi, 4 * Ng) / (double)(4 * Ng);
        break;
    default: {
        double v = d.phi(x, (double)xi, d.user);
        t2 = v - std::floor(v);
        break;
    }
    }
    t2 -= std::nearbyint(t2);
    return t1 + t2;
}

bool KernelFn::row_terms(int64_t i, double* kappa, double* rho, int* xxi, int* sq) const
{
    if (indirect) return false;
    const double x = (double)i / (double)n_global;
    const double s = d.phase_param;
    *kappa = *rho = 0.0;
    *xxi = *sq = 0;
    switch (d.phase_kind) {
    case BF_PHASE_DFT:
        *xxi = 1;
        return true;
    case BF_PHASE_FIO:
        *xxi = 1;
        *kappa = (2.0 + s * std::sin(kTwoPi * x)) / 16.0;
        return true;
    case BF_PHASE_FIO_PW: {
        *xxi = 1;
        const double c = (2.0 + s * std::sin(kTwoPi * x)) / 16.0;
        *kappa = (2 * i < n_global) ? c : -0.5 * c;
        return true;
    }
    case BF_PHASE_ONES:
        return true;
    case BF_PHASE_SEP:
        *sq = 1;
        *rho = 0.3 * std::sin(kTwoPi * x);
        return true;
    default:
        return false;
    }
}

cd KernelFn::amplitude_explicit(int64_t i, int64_t j) const
{
    const int64_t Ng = n_global;
    const double x = (double)i / (double)Ng;
    const double xi = (double)(j - Ng / 2);
    switch (d.amp_kind) {
    case BF_AMP_ONE:
        return 1.0;
    case BF_AMP_SMOOTH:
        return 1.0 + 0.25 * std::sin(kTwoPi * x) * std::cos(kTwoPi * xi / (double)Ng);
    default: {
        double re = 0, im = 0;
        d.alpha(x, xi, d.user, &re, &im);
        return cd(re, im);
    }
    }
}

// ---------------------------------------------------------------------------
std::vector<int64_t> grid_rel(int64_t n, int r)
{
    std::vector<int64_t> g;
    if (n <= r) {
        for (int64_t i = 0; i < n; ++i) g.push_back(i);
        return g;
    }
    // Eq. (gdA)/(gdB) read as Round(t + (n - r)(1/2 - z_t)), z_t = cos((t-1) pi/(r-1))/2,
    // Round = nearest with ties (within 1e-9) to the lower index.
    for (int t = 1; t <= r; ++t) {
        double z = 0.5 * std::cos((double)(t - 1) * M_PI / (double)(r - 1));
        double v = (double)t + (double)(n - r) * (0.5 - z);
        g.push_back((int64_t)std::ceil(v - 0.5 - 1e-9) - 1);
    }
    return g;
}

std::vector<double> lagrange(const std::vector<int64_t>& nodes, const std::vector<double>& pts)
{
    const size_t r = nodes.size(), n = pts.size();
    std::vector<double> M(r * n, 1.0);
    for (size_t t = 0; t < r; ++t)
        for (size_t k = 0; k < n; ++k) {
            double v = 1.0;
            for (size_t j = 0; j < r; ++j)
                if (j != t) v *= (pts[k] - (double)nodes[j]) / (double)(nodes[t] - nodes[j]);
            M[t * n + k] = v;
        }
    return M;
}

int choose_l1(int r, int n0)
{
    int l = 0;
    while ((int64_t)n0 << l <= r) ++l;
    return l;
}

size_t BlockFactors::host_bytes() const
{
    size_t s = (a.size() + b.size() + EV.size() + S.size() + EU.size()) * sizeof(cd) +
               (Mv.size() + MU.size()) * sizeof(double);
    for (auto& v : MH) s += v.size() * sizeof(double);
    for (auto& v : MG) s += v.size() * sizeof(double);
    for (auto& v : EH) s += v.size() * sizeof(cd);
    for (auto& v : FG) s += v.size() * sizeof(cd);
    return s;
}

// ---------------------------------------------------------------------------
namespace {
struct SplitMix {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

std::vector<int64_t> sample_union(SplitMix& rng, int64_t n, int64_t k, const std::vector<int64_t>& base)
{
    std::vector<int64_t> out(base);
    k = std::min(k, n);
    // Floyd's algorithm for k distinct indices
    std::vector<int64_t> pick;
    for (int64_t j = n - k; j < n; ++j) {
        int64_t t = (int64_t)(rng.next() % (uint64_t)(j + 1));
        if (std::find(pick.begin(), pick.end(), t) != pick.end()) t = j;
        pick.push_back(t);
    }
    out.insert(out.end(), pick.begin(), pick.end());
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    return out;
}
}  // namespace

// Algorithm 1 (Sec. 2.1) on an N x N matrix seen through entries(I, J) (the submatrix)
// and entries_adj(I, J) (its adjoint): a = U0 Sigma0 and b = V0^* as [rank][N], with the
// rank cut at the singular values above tol * sigma_1.  seed_state starts the sampler.
bf_status lowrank_sampled(const EntriesFn& entries, const EntriesFn& entries_adj, int64_t N, int r, int q,
                          double tol, uint64_t seed_state, std::vector<cd>& a, std::vector<cd>& b, int& rank,
                          double& sigma_ratio, const std::vector<int64_t>& fixed_rows,
                          const std::vector<int64_t>& fixed_cols)
{
    r = std::max(1, r);
    // sample sets always hold the important rows / columns and the fixed ones
    auto with = [](std::vector<int64_t> v, const std::vector<int64_t>& extra) {
        v.insert(v.end(), extra.begin(), extra.end());
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        return v;
    };
    const int64_t rq = (int64_t)r * std::max(1, q);
    SplitMix rng{seed_state};
    std::vector<int64_t> all((size_t)N);
    for (int64_t i = 0; i < N; ++i) all[(size_t)i] = i;
    std::vector<int64_t> pi_col, pi_row, piv;
    CMat Q;
    const double qr_tol = 1e-15;
    for (int sweep = 0; sweep < 2; ++sweep) {
        // rq random rows + important rows; pivoted QR of K(I, :) picks columns
        auto I = sample_union(rng, N, rq, with(pi_row, fixed_rows));
        int kr = pivoted_qr(entries(I, all), r, qr_tol, Q, piv);
        pi_col.assign(piv.begin(), piv.begin() + std::max(kr, 1));
        std::sort(pi_col.begin(), pi_col.end());
        // rq random columns + important columns; pivoted LQ of K(:, J) picks rows
        auto J = sample_union(rng, N, rq, with(pi_col, fixed_cols));
        kr = pivoted_qr(entries_adj(all, J), r, qr_tol, Q, piv);
        pi_row.assign(piv.begin(), piv.begin() + std::max(kr, 1));
        std::sort(pi_row.begin(), pi_row.end());
    }
    CMat Qc, Qr;
    int kc = pivoted_qr(entries(all, pi_col), r, qr_tol, Qc, piv);
    int kr = pivoted_qr(entries_adj(pi_row, all), r, qr_tol, Qr, piv);
    if (kc == 0 || kr == 0) {  // zero matrix
        rank = 0;
        a.clear();
        b.clear();
        sigma_ratio = 0;
        return BF_OK;
    }
    auto J = sample_union(rng, N, rq, with(pi_col, fixed_cols));
    auto I = sample_union(rng, N, rq, with(pi_row, fixed_rows));
    CMat QcI((int64_t)I.size(), kc), QrJ(kr, (int64_t)J.size());
    for (size_t ii = 0; ii < I.size(); ++ii)
        for (int64_t c = 0; c < kc; ++c) QcI((int64_t)ii, c) = Qc(I[ii], c);
    for (size_t jj = 0; jj < J.size(); ++jj)
        for (int64_t c = 0; c < kr; ++c) QrJ(c, (int64_t)jj) = std::conj(Qr(J[jj], c));
    CMat M = matmul(matmul(pinv(QcI, 1e-14), entries(I, J)), pinv(QrJ, 1e-14));
    CMat UM, VM;
    std::vector<double> SM;
    jacobi_svd(M, UM, SM, VM);
    int keep = 0;
    while (keep < (int)SM.size() && SM[(size_t)keep] > tol * SM[0]) ++keep;
    sigma_ratio = keep < (int)SM.size() ? SM[(size_t)keep] / SM[0] : 0.0;
    rank = keep;
    CMat U0 = matmul(Qc, UM), V0 = matmul(Qr, VM);
    a.assign((size_t)(rank * N), cd(0));
    b.assign((size_t)(rank * N), cd(0));
    for (int kk = 0; kk < rank; ++kk)
        for (int64_t i = 0; i < N; ++i) {
            a[(size_t)(kk * N + i)] = U0(i, kk) * SM[(size_t)kk];
            b[(size_t)(kk * N + i)] = std::conj(V0(i, kk));
        }
    return BF_OK;
}

// Algorithm 1 on the amplitude window [row0, row0+N) x [col0, col0+N).
bf_status amplitude_split(const KernelFn& k, const bf_options& opt, int64_t row0, int64_t col0,
                          int64_t N, std::vector<cd>& a, std::vector<cd>& b, int& ra,
                          double& sigma_ratio)
{
    // indirect kernels: |K| on the whole block, fetched through KernelFn::entries
    auto block_abs = [&](const std::vector<int64_t>& I, const std::vector<int64_t>& J, bool adj) {
        const int64_t ni = (int64_t)I.size(), nj = (int64_t)J.size();
        std::vector<int64_t> ri((size_t)(ni * nj)), cj((size_t)(ni * nj));
#pragma omp parallel for schedule(static)
        for (int64_t jj = 0; jj < nj; ++jj)
            for (int64_t ii = 0; ii < ni; ++ii) {
                ri[(size_t)(jj * ni + ii)] = row0 + I[(size_t)ii];
                cj[(size_t)(jj * ni + ii)] = col0 + J[(size_t)jj];
            }
        std::vector<cd> kv((size_t)(ni * nj));
        k.entries(ri.data(), cj.data(), ni * nj, kv.data());
        CMat M(adj ? nj : ni, adj ? ni : nj);
#pragma omp parallel for schedule(static)
        for (int64_t jj = 0; jj < nj; ++jj)
            for (int64_t ii = 0; ii < ni; ++ii) {
                const double a = std::abs(kv[(size_t)(jj * ni + ii)]);
                if (adj) M(jj, ii) = a; else M(ii, jj) = a;
            }
        return M;
    };
    auto entries = [&](const std::vector<int64_t>& I, const std::vector<int64_t>& J) {
        if (k.indirect) return block_abs(I, J, false);
        CMat M((int64_t)I.size(), (int64_t)J.size());
#pragma omp parallel for schedule(static)
        for (int64_t jj = 0; jj < (int64_t)J.size(); ++jj)
            for (size_t ii = 0; ii < I.size(); ++ii)
                M((int64_t)ii, jj) = k.amplitude(row0 + I[ii], col0 + J[(size_t)jj]);
        return M;
    };
    // adjoint(entries(I, J)) built directly, in parallel over the rows I
    auto entries_adj = [&](const std::vector<int64_t>& I, const std::vector<int64_t>& J) {
        if (k.indirect) return block_abs(I, J, true);
        CMat M((int64_t)J.size(), (int64_t)I.size());
#pragma omp parallel for schedule(static)
        for (int64_t ii = 0; ii < (int64_t)I.size(); ++ii)
            for (size_t jj = 0; jj < J.size(); ++jj)
                M((int64_t)jj, ii) = std::conj(k.amplitude(row0 + I[(size_t)ii], col0 + J[jj]));
        return M;
    };
    return lowrank_sampled(entries, entries_adj, N, opt.amp_rank, opt.amp_oversample,
                           opt.amp_tol > 0 ? opt.amp_tol : 1e-13, opt.seed * 0x9E3779B97F4A7C15ull + 12345, a, b,
                           ra, sigma_ratio, {}, {});
}

// ---------------------------------------------------------------------------
bf_status factor_block(const KernelFn& k, const bf_options& opt, BlockFactors& B, bool tables)
{
    const int64_t N = B.N;
    const int r = B.r, n0 = B.n0;
    B.L = 0;
    while (((int64_t)n0 << B.L) < N) ++B.L;
    B.h = B.L / 2;
    B.l1 = std::max(choose_l1(r, n0), opt.l1);
    B.nv = n0 << B.l1;
    const int L = B.L, h = B.h, l1 = B.l1;
    if (h < l1) {
        set_error("N=%lld too small for r=%d, n0=%d (need floor(L/2) >= %d)", (long long)N, r, n0, l1);
        return BF_ERR_ARG;
    }
    const int64_t P = N / n0;
    auto F = [&](int64_t i, int64_t j) { return k.phase_frac(B.row0 + i, B.col0 + j); };

    const double t0 = omp_get_wtime();
    bf_status st = amplitude_split(k, opt, B.row0, B.col0, N, B.a, B.b, B.ra, B.amp_sigma_ratio);
    B.t_amp = omp_get_wtime() - t0;
    if (st != BF_OK) return st;

    // V at level l1 (Eq. 1 with the copy levels 1..l1-1 folded in)
    {
        const int64_t nv = B.nv, nA = (int64_t)1 << l1, na = N >> l1;
        auto gB = grid_rel(nv, r);
        std::vector<double> pts((size_t)nv);
        for (int64_t x = 0; x < nv; ++x) pts[(size_t)x] = (double)x;
        B.Mv = lagrange(gB, pts);
        if (tables) B.EV.assign((size_t)(nA * N), cd(0));
#pragma omp parallel for schedule(static) if (tables)
        for (int64_t a = 0; a < (tables ? nA : 0); ++a) {
            const int64_t cA = centre(a * na, na);
            for (int64_t j = 0; j < N; ++j) B.EV[(size_t)(a * N + j)] = expi(F(cA, j));
        }
    }
    // H levels (Eq. 2)
    B.MH.clear();
    B.EH.clear();
    for (int l = l1 + 1; l <= h; ++l) {
        const int64_t nA = (int64_t)1 << l, na = N >> l;
        const int64_t nBl = (int64_t)1 << (L - l), nb = N >> (L - l);
        auto gB = grid_rel(nb, r), gC = grid_rel(nb / 2, r);
        std::vector<double> pts;
        for (int c = 0; c < 2; ++c)
            for (int s = 0; s < r; ++s) pts.push_back((double)(gC[(size_t)s] + c * (nb / 2)));
        B.MH.push_back(lagrange(gB, pts));
        std::vector<cd> E(tables ? (size_t)(P * 2 * r) : 0);
#pragma omp parallel for schedule(static) if (tables)
        for (int64_t a = 0; a < (tables ? nA : 0); ++a) {
            const int64_t cA = centre(a * na, na), cP = centre((a >> 1) * 2 * na, 2 * na);
            for (int64_t bb = 0; bb < nBl; ++bb)
                for (int c = 0; c < 2; ++c)
                    for (int s = 0; s < r; ++s) {
                        const int64_t xi = bb * nb + c * (nb / 2) + gC[(size_t)s];
                        E[(size_t)((((a * nBl + bb) * 2 + c) * r) + s)] = expi(F(cA, xi) - F(cP, xi));
                    }
        }
        B.EH.push_back(std::move(E));
    }
    // switch at h
    {
        const int64_t nA = (int64_t)1 << h, na = N >> h;
        const int64_t nBl = (int64_t)1 << (L - h), nb = N >> (L - h);
        auto gA = grid_rel(na, r), gB = grid_rel(nb, r);
        if (tables) B.S.assign((size_t)(P * r * r), cd(0));
#pragma omp parallel for schedule(static) if (tables)
        for (int64_t a = 0; a < (tables ? nA : 0); ++a) {
            const int64_t cA = centre(a * na, na);
            for (int64_t bb = 0; bb < nBl; ++bb) {
                const int64_t cB = centre(bb * nb, nb);
                for (int t = 0; t < r; ++t) {
                    const int64_t x = a * na + gA[(size_t)t];
                    const double fxc = F(x, cB);
                    for (int s = 0; s < r; ++s) {
                        const int64_t xi = bb * nb + gB[(size_t)s];
                        B.S[(size_t)((((a * nBl + bb) * r) + t) * r + s)] = expi(F(x, xi) - fxc - F(cA, xi));
                    }
                }
            }
        }
    }
    // G levels (Eq. 3)
    B.MG.clear();
    B.FG.clear();
    for (int l = h + 1; l <= L - l1; ++l) {
        const int64_t nA = (int64_t)1 << l, na = N >> l;
        const int64_t nBl = (int64_t)1 << (L - l), nb = N >> (L - l);
        auto gA = grid_rel(na, r), gP = grid_rel(2 * na, r);
        std::vector<double> MG((size_t)(2 * r * r));
        for (int pos = 0; pos < 2; ++pos) {
            std::vector<double> pts;
            for (int t = 0; t < r; ++t) pts.push_back((double)(gA[(size_t)t] + pos * na));
            auto Lg = lagrange(gP, pts);  // [s][t]
            for (int t = 0; t < r; ++t)
                for (int s = 0; s < r; ++s) MG[(size_t)((pos * r + t) * r + s)] = Lg[(size_t)(s * r + t)];
        }
        B.MG.push_back(std::move(MG));
        std::vector<cd> E(tables ? (size_t)(P * 2 * r) : 0);
#pragma omp parallel for schedule(static) if (tables)
        for (int64_t a = 0; a < (tables ? nA : 0); ++a)
            for (int64_t bb = 0; bb < nBl; ++bb) {
                const int64_t cB = centre(bb * nb, nb);
                for (int c = 0; c < 2; ++c) {
                    const int64_t cC = centre(bb * nb + c * (nb / 2), nb / 2);
                    for (int t = 0; t < r; ++t) {
                        const int64_t x = a * na + gA[(size_t)t];
                        E[(size_t)((((a * nBl + bb) * 2 + c) * r) + t)] = expi(F(x, cC) - F(x, cB));
                    }
                }
            }
        B.FG.push_back(std::move(E));
    }
    // U at level L-l1 (Eq. bf3 with the summing levels L-l1+1..L folded in)
    {
        const int64_t nu = B.nv, nC = (int64_t)1 << l1, nc = N >> l1;
        auto gA = grid_rel(nu, r);
        std::vector<double> pts((size_t)nu);
        for (int64_t x = 0; x < nu; ++x) pts[(size_t)x] = (double)x;
        auto Lg = lagrange(gA, pts);  // [s][x]
        B.MU.assign((size_t)(nu * r), 0.0);
        for (int64_t x = 0; x < nu; ++x)
            for (int s = 0; s < r; ++s) B.MU[(size_t)(x * r + s)] = Lg[(size_t)(s * nu + x)];
        if (tables) B.EU.assign((size_t)(nC * N), cd(0));
#pragma omp parallel for schedule(static) if (tables)
        for (int64_t c = 0; c < (tables ? nC : 0); ++c) {
            const int64_t cC = centre(c * nc, nc);
            for (int64_t x = 0; x < N; ++x) B.EU[(size_t)(c * N + x)] = expi(F(x, cC));
        }
    }
    return BF_OK;
}

}  // namespace bfi
