// Indirect access (Scenario 1 of Table sc, Sec. 2.2): the amplitude and phase of K
// recovered from its entries alone, off the timed path.
//
//  * unwrap: Algorithm 3.  A vector v is rebuilt from u = v mod 1: the first entry
//    is u itself, the second the one nearest the first, the third keeps the first
//    difference, every later one makes the third difference smallest; a second
//    difference above tau starts a new smooth piece.
//  * PsiSampler: Algorithm 4 on one sub-BF window.  The discontinuities of one
//    column and one row cut the window into blocks.  In each block the first row
//    is unwrapped.  Then the first three columns are unwrapped along x: the first
//    from the first row's value, the next two through their differences with the
//    column before, so the three stay continuous along every row.  Every row
//    continues from its values in those three columns, and every column from its
//    values in the block's first three rows.  So any row or column of one Psi,
//    with e^{2 pi i Psi} = K / |K|, can be rebuilt on demand, and rows and
//    columns agree where they cross.
//  * recover_phase: Algorithm 5.  Algorithm 1 (lowrank_sampled) runs on Psi
//    through the sampler and gives Psi ~ Re sum_k p_k(x) q_k(xi).
// The amplitude is Algorithm 1 on |K| (amplitude_split with KernelFn::indirect).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include <omp.h>

#include "bf_internal.h"

namespace bfi {

namespace {

const double kTwoPi = 6.283185307179586476925286766559;

struct Mix64 {  // splitmix64 (Steele, Lea, Flood 2014)
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

// One sub-BF window [row0, row0 + N) x [col0, col0 + N) of Psi, Algorithm 4.
class PsiSampler {
  public:
    PsiSampler(const KernelFn& k, int64_t row0, int64_t col0, int64_t N, int64_t cfirst, int64_t rfirst,
               double tau, double tau_block)
        : k_(k), row0_(row0), col0_(col0), N_(N), tb_(tau_block)
    {
        std::vector<double> u((size_t)N), v((size_t)N);
        // discontinuities along one column (row cuts) and one row (column cuts)
        turns_col(cfirst, 0, N, u.data());
        unwrap(u.data(), N, tau, nullptr, 0, v.data(), &rb_);
        turns_row(rfirst, 0, N, u.data());
        unwrap(u.data(), N, tau, nullptr, 0, v.data(), &cb_);
        rb_.push_back(N);
        cb_.push_back(N);
        const int nbr = (int)rb_.size() - 1, nbc = (int)cb_.size() - 1;
        // a phase with more pieces than this is not piecewise smooth at this sampling
        if (nbr > kMaxPieces || nbc > kMaxPieces) return;
        colseed_.assign((size_t)(nbr * nbc), {});
        rowseed_.assign((size_t)(nbr * nbc), {});
        for (int bi = 0; bi < nbr; ++bi)
            for (int bj = 0; bj < nbc; ++bj) {
                const int64_t r0 = rb_[(size_t)bi], r1 = rb_[(size_t)bi + 1];
                const int64_t c0 = cb_[(size_t)bj], c1 = cb_[(size_t)bj + 1];
                const int64_t nr = r1 - r0, ncb = c1 - c0;
                // the block's first row
                std::vector<double> ur((size_t)ncb), first((size_t)ncb);
                turns_row(r0, c0, ncb, ur.data());
                unwrap(ur.data(), ncb, tb_, nullptr, 0, first.data(), nullptr);
                // its first three columns along x
                const int nc = (int)std::min<int64_t>(3, ncb);
                std::vector<double>& cs = colseed_[(size_t)(bi * nbc + bj)];
                cs.assign((size_t)(nc * nr), 0.0);
                std::vector<double> uc((size_t)(nc * nr)), dt((size_t)nr), w((size_t)nr);
                for (int t = 0; t < nc; ++t) turns_col(c0 + t, r0, nr, uc.data() + (size_t)t * nr);
                unwrap(uc.data(), nr, tb_, &first[0], 1, cs.data(), nullptr);
                for (int t = 1; t < nc; ++t) {
                    for (int64_t i = 0; i < nr; ++i) {
                        double d = uc[(size_t)(t * nr + i)] - uc[(size_t)((t - 1) * nr + i)];
                        dt[(size_t)i] = d - std::floor(d);
                    }
                    const double d0 = first[(size_t)t] - first[(size_t)t - 1];
                    unwrap(dt.data(), nr, tb_, &d0, 1, w.data(), nullptr);
                    for (int64_t i = 0; i < nr; ++i)
                        cs[(size_t)(t * nr + i)] = cs[(size_t)((t - 1) * nr + i)] + w[(size_t)i];
                }
                // its first three rows, from those columns
                const int nrr = (int)std::min<int64_t>(3, nr);
                std::vector<double>& rs = rowseed_[(size_t)(bi * nbc + bj)];
                rs.assign((size_t)(nrr * ncb), 0.0);
                for (int t = 0; t < nrr; ++t) {
                    turns_row(r0 + t, c0, ncb, ur.data());
                    row_block(r0 + t, bi, bj, ur.data(), rs.data() + (size_t)t * ncb);
                }
            }
    }

    static constexpr int kMaxPieces = 64;
    // the first and last two local indices of every row piece (rows) and column piece (cols)
    void edge_indices(std::vector<int64_t>& rows, std::vector<int64_t>& cols) const
    {
        auto edges = [&](const std::vector<int64_t>& e, std::vector<int64_t>& out) {
            for (size_t k = 0; k + 1 < e.size(); ++k)
                for (int64_t t : {e[k], e[k] + 1, e[k + 1] - 2, e[k + 1] - 1})
                    if (t >= e[k] && t < e[k + 1]) out.push_back(t);
            std::sort(out.begin(), out.end());
            out.erase(std::unique(out.begin(), out.end()), out.end());
        };
        edges(rb_, rows);
        edges(cb_, cols);
    }
    bool ok() const { return !colseed_.empty(); }
    int pieces_rows() const { return (int)rb_.size() - 1; }
    int pieces_cols() const { return (int)cb_.size() - 1; }

    // Phi mod 1 on local row i, columns c0 .. c0 + n (out: n values in [0, 1))
    void turns_row(int64_t i, int64_t c0, int64_t n, double* out) const
    {
        std::vector<int64_t> I((size_t)n, row0_ + i), J((size_t)n);
        for (int64_t t = 0; t < n; ++t) J[(size_t)t] = col0_ + c0 + t;
        fetch(I, J, out);
    }
    // Phi mod 1 on local column j, rows r0 .. r0 + n
    void turns_col(int64_t j, int64_t r0, int64_t n, double* out) const
    {
        std::vector<int64_t> I((size_t)n), J((size_t)n, col0_ + j);
        for (int64_t t = 0; t < n; ++t) I[(size_t)t] = row0_ + r0 + t;
        fetch(I, J, out);
    }
    // Phi mod 1 on the whole local row (by_row) or column idx, entry by entry from the
    // calling thread (sources that several threads may call at once: not a bulk callback)
    void turns_line(bool by_row, int64_t idx, double* out) const
    {
        for (int64_t t = 0; t < N_; ++t) {
            const cd v = by_row ? k_.entry(row0_ + idx, col0_ + t) : k_.entry(row0_ + t, col0_ + idx);
            const double a = std::arg(v) / kTwoPi;
            out[t] = a - std::floor(a);
        }
    }
    // Phi mod 1 on nv whole local rows (by_rows) or columns idx[0 .. nv), fetched in one
    // entries() call (out: [nv][N])
    void turns_lines(bool by_rows, const int64_t* idx, int64_t nv, double* out) const
    {
        std::vector<int64_t> I((size_t)(nv * N_)), J((size_t)(nv * N_));
#pragma omp parallel for collapse(2) schedule(static)
        for (int64_t v = 0; v < nv; ++v)
            for (int64_t t = 0; t < N_; ++t) {
                const size_t e = (size_t)(v * N_ + t);
                I[e] = row0_ + (by_rows ? idx[v] : t);
                J[e] = col0_ + (by_rows ? t : idx[v]);
            }
        fetch(I, J, out);
    }

    // local row i (N values of Psi) from its observations u (N values of Phi mod 1)
    void row(int64_t i, const double* u, double* out) const
    {
        const int bi = block_of(rb_, i), nbc = (int)cb_.size() - 1;
        for (int bj = 0; bj < nbc; ++bj) {
            const int64_t c0 = cb_[(size_t)bj];
            row_block(i, bi, bj, u + c0, out + c0);
        }
    }

    // local column j (N values of Psi) from its observations u (N values of Phi mod 1)
    void col(int64_t j, const double* u, double* out) const
    {
        const int bj = block_of(cb_, j), nbr = (int)rb_.size() - 1, nbc = (int)cb_.size() - 1;
        const int64_t c0 = cb_[(size_t)bj], ncb = cb_[(size_t)bj + 1] - c0;
        const double* work = u;
        for (int bi = 0; bi < nbr; ++bi) {
            const int64_t r0 = rb_[(size_t)bi], nr = rb_[(size_t)bi + 1] - r0;
            const std::vector<double>& rs = rowseed_[(size_t)(bi * nbc + bj)];
            const int ns = (int)(rs.size() / (size_t)ncb);
            double seed[3];
            for (int t = 0; t < ns; ++t) seed[t] = rs[(size_t)t * ncb + (j - c0)];
            unwrap(work + r0, nr, tb_, seed, ns, out + r0, nullptr);
        }
    }

  private:
    // Phi mod 1 in [0, 1) at the global index pairs (I[t], J[t]), read off K / |K|
    void fetch(const std::vector<int64_t>& I, const std::vector<int64_t>& J, double* out) const
    {
        const int64_t n = (int64_t)I.size();
        std::vector<cd> kv((size_t)n);
        k_.entries(I.data(), J.data(), n, kv.data());
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < n; ++t) {
            const double a = std::arg(kv[(size_t)t]) / kTwoPi;
            out[t] = a - std::floor(a);
        }
    }
    static int block_of(const std::vector<int64_t>& edges, int64_t x)
    {
        return (int)(std::upper_bound(edges.begin(), edges.end(), x) - edges.begin()) - 1;
    }
    // row i on block (bi, bj): u = its observations on the block's columns
    void row_block(int64_t i, int bi, int bj, const double* u, double* out) const
    {
        const int nbc = (int)cb_.size() - 1;
        const int64_t r0 = rb_[(size_t)bi], nr = rb_[(size_t)bi + 1] - r0;
        const int64_t ncb = cb_[(size_t)bj + 1] - cb_[(size_t)bj];
        const std::vector<double>& cs = colseed_[(size_t)(bi * nbc + bj)];
        const int ns = (int)(cs.size() / (size_t)nr);
        double seed[3];
        for (int t = 0; t < ns; ++t) seed[t] = cs[(size_t)t * nr + (i - r0)];
        unwrap(u, ncb, tb_, seed, ns, out, nullptr);
    }

    const KernelFn& k_;
    int64_t row0_, col0_, N_;
    double tb_;
    std::vector<int64_t> rb_, cb_;                // block edges (last = N)
    std::vector<std::vector<double>> colseed_;    // per block: first three columns [t][rows]
    std::vector<std::vector<double>> rowseed_;    // per block: first three rows [t][cols]
};

// largest singular value of a small complex matrix: power iteration on A^* A from a
// fixed start, sigma = sqrt(|A^* A x|) for the unit iterate x
double norm2(const CMat& A)
{
    std::vector<cd> x((size_t)A.n), y((size_t)A.m);
    double nx = 0;
    for (int64_t j = 0; j < A.n; ++j) {
        x[(size_t)j] = cd(1.0 + 0.01 * (double)(j % 7), 0.003 * (double)(j % 5));
        nx += std::norm(x[(size_t)j]);
    }
    for (auto& t : x) t /= std::sqrt(nx);
    double s = 0.0;
    for (int it = 0; it < 200; ++it) {
        for (int64_t i = 0; i < A.m; ++i) {
            cd t = 0;
            for (int64_t j = 0; j < A.n; ++j) t += A(i, j) * x[(size_t)j];
            y[(size_t)i] = t;
        }
        double nz = 0;
        for (int64_t j = 0; j < A.n; ++j) {
            cd t = 0;
            for (int64_t i = 0; i < A.m; ++i) t += std::conj(A(i, j)) * y[(size_t)i];
            x[(size_t)j] = t;
            nz += std::norm(t);
        }
        nz = std::sqrt(nz);
        if (nz == 0.0) return 0.0;
        for (auto& t : x) t /= nz;
        const double s_new = std::sqrt(nz);
        if (it > 5 && std::fabs(s_new - s) <= 1e-12 * s_new) return s_new;
        s = s_new;
    }
    return s;
}

}  // namespace

// Algorithm 3.  Compiled without FMA contraction, so that the nearest-integer choices are
// the same on every host and as in an evaluation step by step.
__attribute__((optimize("fp-contract=off"))) void unwrap(const double* u, int64_t n, double tau, const double* seed,
                                                         int nseed, double* v, std::vector<int64_t>* starts)
{
    if (starts) {
        starts->clear();
        starts->push_back(0);
    }
    if (n <= 0) return;
    auto near = [&](double p, int64_t a) { return u[a] + std::nearbyint(p - u[a]); };
    v[0] = nseed >= 1 ? seed[0] : u[0];
    if (n > 1) v[1] = nseed >= 2 ? seed[1] : near(v[0], 1);
    if (n > 2) v[2] = nseed >= 3 ? seed[2] : near(2 * v[1] - v[0], 2);
    int64_t a = 3;
    while (a < n) {
        v[a] = near(3 * v[a - 1] - 3 * v[a - 2] + v[a - 3], a);
        if (std::fabs(v[a] + v[a - 2] - 2 * v[a - 1]) > tau) {
            // a discontinuity: a new piece starts at a
            if (starts) starts->push_back(a);
            const int64_t st = a;
            v[st] = near(v[st - 1], st);
            if (st + 1 < n) v[st + 1] = near(2 * v[st] - v[st - 1], st + 1);
            a = st + 2;
            continue;
        }
        ++a;
    }
}

bf_status recover_phase(const KernelFn& k, const bf_options& opt, int64_t row0, int64_t col0, int64_t N,
                        PhaseLR& lr)
{
    // the column and row whose discontinuities cut the window (Algorithm 4's first samples)
    Mix64 rng{opt.seed * 0x9E3779B97F4A7C15ull + 777};
    const int64_t cfirst = (int64_t)(rng.next() % (uint64_t)N), rfirst = (int64_t)(rng.next() % (uint64_t)N);
    const double tau = opt.tau > 0 ? opt.tau : 0.25;
    PsiSampler smp(k, row0, col0, N, cfirst, rfirst, tau, 1.0);
    if (!smp.ok()) {
        set_error("bf_factor: the phase seen through the entries has %d x %d smooth pieces (more than %d along "
                  "a row or column): not piecewise smooth at this grid",
                  smp.pieces_rows(), smp.pieces_cols(), PsiSampler::kMaxPieces);
        return BF_ERR_ACCURACY;
    }
    // Psi[I][:, J] from whole rows (or whole columns when there are fewer of them).  A bulk
    // entry callback sees one caller: the observations of up to kGroup vectors are fetched
    // at a time by one entries() call from this thread, then unwrapped in parallel.  Other
    // sources are evaluated by the thread that unwraps the vector, in one pass.
    const bool grouped = k.bulk();
    const int64_t kGroup = grouped ? 16 : std::numeric_limits<int64_t>::max();
    auto fill = [&](const std::vector<int64_t>& I, const std::vector<int64_t>& J, bool adj) {
        const int64_t ni = (int64_t)I.size(), nj = (int64_t)J.size();
        CMat M(adj ? nj : ni, adj ? ni : nj);
        const bool by_rows = ni <= nj;
        const int64_t nv = by_rows ? ni : nj;
        const int64_t gmax = std::min(kGroup, nv);
        const int nth = grouped ? 1 : omp_get_max_threads();
        // grouped: u, psi hold gmax vectors; otherwise one u and one psi vector per thread
        std::vector<double> u((size_t)((grouped ? gmax : nth) * N)), psi((size_t)((grouped ? gmax : nth) * N));
        for (int64_t g0 = 0; g0 < nv; g0 += gmax) {
            const int64_t ng = std::min(gmax, nv - g0);
            if (grouped) smp.turns_lines(by_rows, (by_rows ? I : J).data() + g0, ng, u.data());
#pragma omp parallel for schedule(dynamic, 1)
            for (int64_t t = 0; t < ng; ++t) {
                const int64_t v = g0 + t;
                const size_t slot = grouped ? (size_t)t : (size_t)omp_get_thread_num();
                double* buf = psi.data() + slot * N;
                double* uv = u.data() + slot * N;
                if (!grouped) smp.turns_line(by_rows, by_rows ? I[(size_t)v] : J[(size_t)v], uv);
                if (by_rows) {
                    smp.row(I[(size_t)v], uv, buf);
                    for (int64_t jj = 0; jj < nj; ++jj) {
                        const double x = buf[(size_t)J[(size_t)jj]];
                        if (adj) M(jj, v) = x; else M(v, jj) = x;
                    }
                } else {
                    smp.col(J[(size_t)v], uv, buf);
                    for (int64_t ii = 0; ii < ni; ++ii) {
                        const double x = buf[(size_t)I[(size_t)ii]];
                        if (adj) M(v, ii) = x; else M(ii, v) = x;
                    }
                }
            }
        }
        return M;
    };
    EntriesFn ent = [&](const std::vector<int64_t>& I, const std::vector<int64_t>& J) { return fill(I, J, false); };
    EntriesFn ent_adj = [&](const std::vector<int64_t>& I, const std::vector<int64_t>& J) { return fill(I, J, true); };
    double sig = 0;
    lr.row0 = row0;
    lr.col0 = col0;
    lr.N = N;
    // the first and last two rows and columns of every smooth piece join Algorithm 1's
    // samples: a phase is least smooth at the edges of its pieces (a kernel's turning
    // points, the window's corners), where random samples rarely fall
    std::vector<int64_t> fr, fc;
    smp.edge_indices(fr, fc);
    return lowrank_sampled(ent, ent_adj, N, opt.phase_rank > 0 ? opt.phase_rank : 20,
                           opt.phase_oversample > 0 ? opt.phase_oversample : 5,
                           opt.phase_tol > 0 ? opt.phase_tol : 1e-13, opt.seed * 0x9E3779B97F4A7C15ull + 4242, lr.p,
                           lr.q, lr.rank, sig, fr, fc);
}

// eps^K and eps^amp of Sec. 5 on 256 x 256 sampled entries of the window
void recovery_errors(const KernelFn& k, BlockFactors& B, uint64_t seed)
{
    const int64_t N = B.N, ns = std::min<int64_t>(N, 256);
    Mix64 rng{seed * 0x9E3779B97F4A7C15ull + 99};
    std::vector<int64_t> S;
    while ((int64_t)S.size() < ns) {
        const int64_t t = (int64_t)(rng.next() % (uint64_t)N);
        if (std::find(S.begin(), S.end(), t) == S.end()) S.push_back(t);
    }
    CMat dK(ns, ns), K(ns, ns), dA(ns, ns), A(ns, ns);
    std::vector<int64_t> ri((size_t)(ns * ns)), cj((size_t)(ns * ns));
    for (int64_t jj = 0; jj < ns; ++jj)
        for (int64_t ii = 0; ii < ns; ++ii) {
            ri[(size_t)(jj * ns + ii)] = B.row0 + S[(size_t)ii];
            cj[(size_t)(jj * ns + ii)] = B.col0 + S[(size_t)jj];
        }
    std::vector<cd> kvs((size_t)(ns * ns));
    k.entries(ri.data(), cj.data(), ns * ns, kvs.data());
#pragma omp parallel for schedule(static)
    for (int64_t jj = 0; jj < ns; ++jj)
        for (int64_t ii = 0; ii < ns; ++ii) {
            const int64_t i = B.row0 + S[(size_t)ii], j = B.col0 + S[(size_t)jj];
            const cd kv = kvs[(size_t)(jj * ns + ii)];
            cd amp = 0;
            for (int q = 0; q < B.ra; ++q)
                amp += B.a[(size_t)q * N + S[(size_t)ii]] * B.b[(size_t)q * N + S[(size_t)jj]];
            const double ph = kTwoPi * B.lr.value(i, j);
            K(ii, jj) = kv;
            dK(ii, jj) = kv - amp * cd(std::cos(ph), std::sin(ph));
            A(ii, jj) = std::abs(kv);
            dA(ii, jj) = std::abs(kv) - amp;
        }
    const double nk = norm2(K), na = norm2(A);
    B.recover_err_k = nk > 0 ? norm2(dK) / nk : 0.0;
    B.recover_err_amp = na > 0 ? norm2(dA) / na : 0.0;
}

// Algorithm 6 (Sec. 3) on one sub-BF of a plan factored from its entries: may
// r-dimensional NUFFTs after dimension lifting evaluate it?  The inputs are the plan's
// recovered factorizations, Psi = sum_k p_k(x) q_k(xi) (rank r1) and alpha = sum_k
// a_k(x) b_k(xi).  Steps: (1) the r-leading SVD of the phase factorization, taken exactly
// (QR of both N x r1 factors, SVD of the r1 x r1 core), is the lifting P Q^T; (2) r_eps q
// random columns of the residual kernel alpha e^{2 pi i (Psi - P Q^T)} go through QR
// with column pivoting; (3) n counts the pivots above eps times the first, y = 1 iff
// n < r_eps; (4) if y = 1, Algorithm 1 (rank parameter r_eps) factors the residual
// kernel and terms is its rank, the number of NUFFTs.
bf_status nufft_decide(const BlockFactors& B, const PhaseLR& lr, int r, int r_eps, int q, double eps,
                       uint64_t seed, int& y, int& n, int& terms)
{
    const int64_t N = B.N;
    const int r1 = lr.rank, ra = B.ra;
    // (1) U1 V1^T = Qa (Ra Rb^T) Qb^T, Ra = Qa^* U1, Rb = Qb^* V1; the core's SVD
    CMat U1(N, r1), V1(N, r1);
    for (int k = 0; k < r1; ++k)
        for (int64_t i = 0; i < N; ++i) {
            U1(i, k) = lr.p[(size_t)k * N + i].real();
            V1(i, k) = lr.q[(size_t)k * N + i].real();
        }
    CMat Qa, Qb, Uc, Vc;
    std::vector<int64_t> piv;
    std::vector<double> S;
    if (r1 > 0) {  // a zero phase (rank 0) has nothing to lift
        pivoted_qr(U1, r1, 0.0, Qa, piv);
        pivoted_qr(V1, r1, 0.0, Qb, piv);
        const CMat C = matmul(matmul(adjoint(Qa), U1), adjoint(matmul(adjoint(Qb), V1)));
        jacobi_svd(C, Uc, S, Vc);
    }
    const int kr = std::min<int>(r, (int)S.size());
    // lift(i, j) = sum_l P(i, l) Q(j, l), P = Qa Uc S, Q = conj(Qb Vc), first kr columns
    CMat P, Q;
    if (kr > 0) {
        P = matmul(Qa, Uc);
        Q = matmul(Qb, Vc);
    }
    std::vector<double> Pl((size_t)(kr * N)), Ql((size_t)(kr * N));
    for (int l = 0; l < kr; ++l)
        for (int64_t i = 0; i < N; ++i) {
            Pl[(size_t)l * N + i] = (P(i, l) * S[(size_t)l]).real();
            Ql[(size_t)l * N + i] = std::conj(Q(i, l)).real();
        }
    auto residual = [&](int64_t i, int64_t j) {
        cd amp = 0;
        for (int k = 0; k < ra; ++k) amp += B.a[(size_t)k * N + i] * B.b[(size_t)k * N + j];
        double ph = 0;
        for (int k = 0; k < r1; ++k) ph += lr.p[(size_t)k * N + i].real() * lr.q[(size_t)k * N + j].real();
        for (int l = 0; l < kr; ++l) ph -= Pl[(size_t)l * N + i] * Ql[(size_t)l * N + j];
        ph -= std::nearbyint(ph);
        return amp * cd(std::cos(kTwoPi * ph), std::sin(kTwoPi * ph));
    };
    // (2) r_eps q distinct random columns (Floyd's algorithm), in increasing order
    Mix64 rng{seed * 0x9E3779B97F4A7C15ull + 606};
    const int64_t nc = std::min<int64_t>(N, (int64_t)r_eps * q);
    std::vector<int64_t> J;
    for (int64_t t = N - nc; t < N; ++t) {
        int64_t c = (int64_t)(rng.next() % (uint64_t)(t + 1));
        if (std::find(J.begin(), J.end(), c) != J.end()) c = t;
        J.push_back(c);
    }
    std::sort(J.begin(), J.end());
    CMat M(N, nc);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nc; ++t)
        for (int64_t i = 0; i < N; ++i) M(i, t) = residual(i, J[(size_t)t]);
    // (3) numerical rank of the sampled columns: pivots above eps |R(1,1)|
    CMat Qm;
    n = pivoted_qr(std::move(M), (int)nc, eps, Qm, piv);
    y = n < r_eps ? 1 : 0;
    terms = 0;
    if (!y) return BF_OK;
    // (4) Algorithm 1 on the residual kernel
    EntriesFn ent = [&](const std::vector<int64_t>& I, const std::vector<int64_t>& Jc) {
        CMat R((int64_t)I.size(), (int64_t)Jc.size());
#pragma omp parallel for schedule(static)
        for (int64_t jj = 0; jj < (int64_t)Jc.size(); ++jj)
            for (size_t ii = 0; ii < I.size(); ++ii) R((int64_t)ii, jj) = residual(I[ii], Jc[(size_t)jj]);
        return R;
    };
    EntriesFn ent_adj = [&](const std::vector<int64_t>& I, const std::vector<int64_t>& Jc) {
        CMat R((int64_t)Jc.size(), (int64_t)I.size());
#pragma omp parallel for schedule(static)
        for (int64_t ii = 0; ii < (int64_t)I.size(); ++ii)
            for (size_t jj = 0; jj < Jc.size(); ++jj) R((int64_t)jj, ii) = std::conj(residual(I[(size_t)ii], Jc[jj]));
        return R;
    };
    std::vector<cd> ua, ub;
    double sig = 0;
    bf_status st = lowrank_sampled(ent, ent_adj, N, r_eps, q, eps, seed * 0x9E3779B97F4A7C15ull + 707, ua, ub,
                                   terms, sig, {}, {});
    return st;
}

}  // namespace bfi

extern "C" bf_status bf_nufft_decide(const bf_plan* plan, int block, int r, int r_eps, int q, double eps,
                                     uint64_t seed, int* y, int* n, int* terms)
{
    if (!plan || !y || !n || !terms || r < 1 || r_eps < 1 || q < 1 || !(eps > 0.0)) {
        bfi::set_error("bf_nufft_decide: bad argument (non-NULL plan and outputs, r, r_eps, q >= 1, eps > 0)");
        return BF_ERR_ARG;
    }
    if (!plan->factored || block < 0 || block >= (int)plan->blocks.size()) {
        bfi::set_error("bf_nufft_decide: plan not factored or bad block");
        return plan->factored ? BF_ERR_ARG : BF_ERR_STATE;
    }
    const bfi::BlockFactors& B = plan->blocks[(size_t)block];
    if (B.a.empty()) {
        bfi::set_error("bf_nufft_decide: host factors were released after upload");
        return BF_ERR_STATE;
    }
    try {
        if (B.lr.rank >= 1) return bfi::nufft_decide(B, B.lr, r, r_eps, q, eps, seed, *y, *n, *terms);
        // an explicit built-in phase: its factors in closed form (turns, not reduced mod 1)
        // on the window's rows x_i = i / N_g and columns xi_j = j - N_g / 2
        const bf_kernel_desc& d = plan->kern.d;
        const int64_t Nb = B.N, Ng = plan->kern.n_global;
        const double s = d.phase_param;
        std::vector<std::vector<double>> pr, qc;  // factor functions of x and of xi
        auto add = [&](auto fx, auto fxi) {
            std::vector<double> a((size_t)Nb), b((size_t)Nb);
            for (int64_t t = 0; t < Nb; ++t) {
                a[(size_t)t] = fx((double)(B.row0 + t) / (double)Ng);
                b[(size_t)t] = fxi((double)(B.col0 + t - Ng / 2));
            }
            pr.push_back(std::move(a));
            qc.push_back(std::move(b));
        };
        auto cx = [&](double x) { return (2.0 + s * std::sin(bfi::kTwoPi * x)) / 16.0; };
        switch (d.phase_kind) {
        case BF_PHASE_DFT: add([](double x) { return x; }, [](double xi) { return xi; }); break;
        case BF_PHASE_FIO:
            add([](double x) { return x; }, [](double xi) { return xi; });
            add(cx, [](double xi) { return std::fabs(xi); });
            break;
        case BF_PHASE_FIO_PW:
            add([](double x) { return x; }, [](double xi) { return xi; });
            add([&](double x) { return x < 0.5 ? cx(x) : -0.5 * cx(x); }, [](double xi) { return std::fabs(xi); });
            break;
        case BF_PHASE_ONES: break;
        case BF_PHASE_SEP:
            add([](double x) { return 0.3 * std::sin(bfi::kTwoPi * x); }, [](double) { return 1.0; });
            add([](double) { return 1.0; }, [&](double xi) { return xi * xi / (4.0 * (double)Ng); });
            break;
        default:
            bfi::set_error("bf_nufft_decide: a user phase has no factorization (factor the plan from its entries)");
            return BF_ERR_STATE;
        }
        bfi::PhaseLR lr;
        lr.row0 = B.row0;
        lr.col0 = B.col0;
        lr.N = Nb;
        lr.rank = (int)pr.size();
        for (int k = 0; k < lr.rank; ++k)
            for (int64_t t = 0; t < Nb; ++t) {
                lr.p.push_back(pr[(size_t)k][(size_t)t]);
                lr.q.push_back(0.0);
            }
        for (int k = 0; k < lr.rank; ++k)
            for (int64_t t = 0; t < Nb; ++t) lr.q[(size_t)k * Nb + t] = qc[(size_t)k][(size_t)t];
        return bfi::nufft_decide(B, lr, r, r_eps, q, eps, seed, *y, *n, *terms);
    } catch (const std::bad_alloc&) {
        bfi::set_error("bf_nufft_decide: out of host memory");
        return BF_ERR_NOMEM;
    }
}

extern "C" bf_status bf_unwrap(const double* u, int64_t n, double tau, const double* seed, int nseed, double* v,
                               int64_t* starts, int64_t cap, int64_t* nstarts)
{
    if (n < 0 || nseed < 0 || nseed > 3 || nseed > n || (!u && n > 0) || (!v && n > 0) || !nstarts ||
        (nseed > 0 && !seed) || (!starts && cap > 0)) {
        bfi::set_error("bf_unwrap: bad argument (n >= 0, 0 <= nseed <= min(3, n), non-NULL buffers)");
        return BF_ERR_ARG;
    }
    std::vector<int64_t> S;
    bfi::unwrap(u, n, tau, seed, nseed, v, &S);
    for (int64_t t = 0; t < (int64_t)S.size() && t < cap; ++t) starts[t] = S[(size_t)t];
    *nstarts = (int64_t)S.size();
    return BF_OK;
}
