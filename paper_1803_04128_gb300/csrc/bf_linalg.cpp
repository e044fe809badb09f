// Small dense complex linear algebra for the host construction (FP64):
// Householder QR with column pivoting (early stop at numerical rank),
// one-sided Jacobi SVD, pseudo-inverse.  Used by Algorithm 1 (Sec. 2.1).
#include <algorithm>
#include <cmath>
#include <limits>

#include "bf_internal.h"

namespace bfi {

CMat matmul(const CMat& A, const CMat& B)
{
    CMat C(A.m, B.n);
    for (int64_t j = 0; j < B.n; ++j)
        for (int64_t k = 0; k < A.n; ++k) {
            cd bkj = B(k, j);
            if (bkj == cd(0)) continue;
            for (int64_t i = 0; i < A.m; ++i) C(i, j) += A(i, k) * bkj;
        }
    return C;
}

CMat adjoint(const CMat& A)
{
    CMat T(A.n, A.m);
    // blocks of 256 rows of A (columns of T) in parallel, so both sides stay in cache
#pragma omp parallel for schedule(static) if (A.m * A.n > (1 << 20))
    for (int64_t i0 = 0; i0 < A.m; i0 += 256) {
        const int64_t i1 = std::min(A.m, i0 + 256);
        for (int64_t j = 0; j < A.n; ++j)
            for (int64_t i = i0; i < i1; ++i) T(j, i) = std::conj(A(i, j));
    }
    return T;
}

// Neumaier-compensated sum (real and imaginary parts apart): the rounding error of every
// addition is carried separately, so a sum over a column of up to N entries stays within
// a few units in the last place instead of an error growing with its length.  The QR
// below needs that to separate a rank from rounding noise (Algorithm 1 on a recovered
// phase whose entries reach ~N turns).
struct CSum {
    double s[2] = {0.0, 0.0}, c[2] = {0.0, 0.0};
    void add1(int k, double x)
    {
        const double t = s[k] + x;
        c[k] += std::fabs(s[k]) >= std::fabs(x) ? (s[k] - t) + x : (x - t) + s[k];
        s[k] = t;
    }
    void add(cd x)
    {
        add1(0, x.real());
        add1(1, x.imag());
    }
    cd value() const { return cd(s[0] + c[0], s[1] + c[1]); }
};

// sum over i in [i0, m) of conj(v[i - i0]) * X(i, j): in fixed chunks of rows whose
// partial sums are added in chunk order, so the result does not depend on the
// number of threads; long columns are split over threads
static cd col_dot(const std::vector<cd>& v, const CMat& X, int64_t j, int64_t i0, int64_t m)
{
    constexpr int64_t kChunk = 1 << 15;
    const int64_t len = m - i0, nch = (len + kChunk - 1) / kChunk;
    if (nch <= 1) {
        CSum d;
        for (int64_t i = i0; i < m; ++i) d.add(std::conj(v[(size_t)(i - i0)]) * X(i, j));
        return d.value();
    }
    std::vector<cd> part((size_t)nch);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nch; ++c) {
        CSum d;
        const int64_t e = std::min(m, i0 + (c + 1) * kChunk);
        for (int64_t i = i0 + c * kChunk; i < e; ++i) d.add(std::conj(v[(size_t)(i - i0)]) * X(i, j));
        part[(size_t)c] = d.value();
    }
    CSum d;
    for (auto& x : part) d.add(x);
    return d.value();
}

// X(i, j) -= v[i - i0] * s for i in [i0, m), rows split over threads when long
static void col_axpy(const std::vector<cd>& v, CMat& X, int64_t j, int64_t i0, int64_t m, cd s)
{
#pragma omp parallel for schedule(static) if (m - i0 > (1 << 15))
    for (int64_t i = i0; i < m; ++i) X(i, j) -= v[(size_t)(i - i0)] * s;
}

int pivoted_qr(CMat R, int kmax, double tol, CMat& Q, std::vector<int64_t>& piv)
{
    const int64_t m = R.m, n = R.n;  // R starts as the input matrix (moved in by callers with temporaries)
    piv.resize((size_t)n);
    // Column norms of the trailing block: nrm holds the downdated estimates, nrm_ex the
    // norm at the column's last exact evaluation.  Downdating (nrm^2 -= |R(k, j)|^2)
    // cancels catastrophically once the trailing norm is far below the exact one, so a
    // column whose estimate has lost about half of its digits is summed again (the
    // safeguard of Drmac and Bujanovic, ACM TOMS 35(2), 2008).  Without it, the pivots
    // of a matrix whose singular values span more than ~1e-8 are chosen from rounding
    // noise, and the rank test below stops early.
    std::vector<double> nrm((size_t)n), nrm_ex((size_t)n);
    const bool wide = n > 4096;  // many columns: split the column loops over threads
    auto tail_norm = [&](int64_t j, int64_t i0) {
        CSum s;
        for (int64_t i = i0; i < m; ++i) s.add1(0, std::norm(R(i, j)));
        return std::sqrt(s.value().real());
    };
    const double tol3z = std::sqrt(std::numeric_limits<double>::epsilon());
#pragma omp parallel for schedule(static) if (wide)
    for (int64_t j = 0; j < n; ++j) {
        piv[(size_t)j] = j;
        nrm[(size_t)j] = nrm_ex[(size_t)j] = tail_norm(j, 0);
    }
    const int64_t kcap = std::min<int64_t>({(int64_t)kmax, m, n});
    std::vector<std::vector<cd>> vs;
    double ref = -1;
    int64_t k = 0;
    for (; k < kcap; ++k) {
        int64_t p = k;
        for (int64_t j = k + 1; j < n; ++j)
            if (nrm[(size_t)j] > nrm[(size_t)p]) p = j;
        // recompute the winner's norm exactly
        const double pn = tail_norm(p, k);
        if (ref < 0) ref = pn;
        if (pn <= tol * ref || pn == 0.0) break;
        if (p != k) {
            for (int64_t i = 0; i < m; ++i) std::swap(R(i, k), R(i, p));
            std::swap(nrm[(size_t)k], nrm[(size_t)p]);
            std::swap(nrm_ex[(size_t)k], nrm_ex[(size_t)p]);
            std::swap(piv[(size_t)k], piv[(size_t)p]);
        }
        // Householder vector for R[k:, k]
        std::vector<cd> v((size_t)(m - k));
        for (int64_t i = k; i < m; ++i) v[(size_t)(i - k)] = R(i, k);
        cd x0 = v[0];
        double ax0 = std::abs(x0);
        cd ph = ax0 > 0 ? x0 / ax0 : cd(1);
        cd alpha = -ph * pn;
        v[0] -= alpha;
        CSum vs2;
        for (auto& e : v) vs2.add1(0, std::norm(e));
        double vn = std::sqrt(vs2.value().real());
        if (vn > 0)
            for (auto& e : v) e /= vn;
        // apply H = I - 2 v v^* to R[k:, k:]
        if (wide) {
#pragma omp parallel for schedule(static)
            for (int64_t j = k; j < n; ++j) {
                CSum ds;
                for (int64_t i = k; i < m; ++i) ds.add(std::conj(v[(size_t)(i - k)]) * R(i, j));
                const cd dot = 2.0 * ds.value();
                for (int64_t i = k; i < m; ++i) R(i, j) -= v[(size_t)(i - k)] * dot;
            }
        } else {
            for (int64_t j = k; j < n; ++j) col_axpy(v, R, j, k, m, 2.0 * col_dot(v, R, j, k, m));
        }
#pragma omp parallel for schedule(static) if (wide)
        for (int64_t j = k + 1; j < n; ++j) {
            const double nj = nrm[(size_t)j];
            if (nj == 0.0) continue;
            const double t = std::abs(R(k, j)) / nj;
            const double rest = std::max(0.0, (1.0 - t) * (1.0 + t));   // (trailing / current)^2
            const double q = nj / nrm_ex[(size_t)j];
            if (rest * q * q <= tol3z) {
                nrm[(size_t)j] = nrm_ex[(size_t)j] = tail_norm(j, k + 1);
            } else {
                nrm[(size_t)j] = nj * std::sqrt(rest);
            }
        }
        vs.push_back(std::move(v));
    }
    // Q = H_0 ... H_{k-1} [I_k; 0]
    Q = CMat(m, k);
    for (int64_t j = 0; j < k; ++j) Q(j, j) = 1;
    for (int64_t s2 = k - 1; s2 >= 0; --s2) {
        const auto& v = vs[(size_t)s2];
        for (int64_t j = 0; j < k; ++j) col_axpy(v, Q, j, s2, m, 2.0 * col_dot(v, Q, j, s2, m));
    }
    return (int)k;
}

void jacobi_svd(const CMat& A0, CMat& U, std::vector<double>& S, CMat& V)
{
    CMat A = A0;
    const int64_t m = A.m, n = A.n;
    V = CMat(n, n);
    for (int64_t j = 0; j < n; ++j) V(j, j) = 1;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0;
        for (int64_t p = 0; p < n; ++p)
            for (int64_t q = p + 1; q < n; ++q) {
                double al = 0, be = 0;
                cd ga = 0;
                for (int64_t i = 0; i < m; ++i) {
                    al += std::norm(A(i, p));
                    be += std::norm(A(i, q));
                    ga += std::conj(A(i, p)) * A(i, q);
                }
                double ag = std::abs(ga);
                if (ag == 0.0 || ag <= 1e-15 * std::sqrt(al * be)) continue;
                off = std::max(off, ag / std::sqrt(al * be));
                cd e = ga / ag;  // rotate column q by conj(e) so that the Gram entry is real
                double zeta = (be - al) / (2 * ag);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1 + zeta * zeta));
                double c = 1 / std::sqrt(1 + t * t), s = c * t;
                for (int64_t i = 0; i < m; ++i) {
                    cd ap = A(i, p), aq = A(i, q) * std::conj(e);
                    A(i, p) = c * ap - s * aq;
                    A(i, q) = s * ap + c * aq;
                }
                for (int64_t i = 0; i < n; ++i) {
                    cd vp = V(i, p), vq = V(i, q) * std::conj(e);
                    V(i, p) = c * vp - s * vq;
                    V(i, q) = s * vp + c * vq;
                }
            }
        if (off < 1e-15) break;
    }
    std::vector<double> s0((size_t)n);
    for (int64_t j = 0; j < n; ++j) {
        double t = 0;
        for (int64_t i = 0; i < m; ++i) t += std::norm(A(i, j));
        s0[(size_t)j] = std::sqrt(t);
    }
    std::vector<int64_t> ord((size_t)n);
    for (int64_t j = 0; j < n; ++j) ord[(size_t)j] = j;
    std::sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return s0[(size_t)x] > s0[(size_t)y]; });
    U = CMat(m, n);
    CMat V2(n, n);
    S.assign((size_t)n, 0.0);
    for (int64_t jj = 0; jj < n; ++jj) {
        int64_t j = ord[(size_t)jj];
        S[(size_t)jj] = s0[(size_t)j];
        for (int64_t i = 0; i < m; ++i) U(i, jj) = s0[(size_t)j] > 0 ? A(i, j) / s0[(size_t)j] : cd(0);
        for (int64_t i = 0; i < n; ++i) V2(i, jj) = V(i, j);
    }
    V = V2;
}

CMat pinv(const CMat& A, double rcond)
{
    // A = U S V^*  ->  A^+ = V S^+ U^*; work on the thinner orientation
    if (A.m < A.n) return adjoint(pinv(adjoint(A), rcond));
    CMat U, V;
    std::vector<double> S;
    jacobi_svd(A, U, S, V);
    CMat P(A.n, A.m);
    double smax = S.empty() ? 0 : S[0];
    for (size_t k = 0; k < S.size(); ++k) {
        if (S[k] <= rcond * smax || S[k] == 0.0) continue;
        double inv = 1.0 / S[k];
        for (int64_t j = 0; j < A.m; ++j) {
            cd u = std::conj(U(j, (int64_t)k)) * inv;
            for (int64_t i = 0; i < A.n; ++i) P(i, j) += V(i, (int64_t)k) * u;
        }
    }
    return P;
}

}  // namespace bfi
