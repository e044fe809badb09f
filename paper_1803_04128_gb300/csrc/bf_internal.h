// Internal types of the butterfly-factorisation library (host side).
#pragma once

#include <complex>
#include <functional>
#include <map>
#include <cstdint>
#include <string>
#include <vector>

#include "bf.h"

namespace bfi {

using cd = std::complex<double>;

void set_error(const char* fmt, ...);

// ---------------------------------------------------------------------------
// A phase recovered from kernel entries on one sub-BF window (Algorithm 5):
// Psi(row0 + i, col0 + j) = Re sum_k p[k][i] q[k][j], with e^{2 pi i Psi} = e^{2 pi i Phi}.
struct PhaseLR {
    int64_t row0 = 0, col0 = 0, N = 0;
    int rank = 0;
    std::vector<cd> p, q;  // [rank][N]
    double value(int64_t i, int64_t j) const;  // global indices
};

// The operator: entries of alpha and of e^{2 pi i Phi} at global grid indices.
struct KernelFn {
    bf_kernel_desc d{};
    int64_t n_global = 0;  // grid size of x_i = i/n_global, xi_j = j - n_global/2
    // Indirect access (Scenario 1): the construction sees K only through entry();
    // amplitude() is then |K| and phase_frac() the recovered phase lr (per sub-BF window).
    bool indirect = false;
    const PhaseLR* lr = nullptr;
    // Phi(x_i, xi_j) reduced mod 1 (exactly for the built-in kinds).
    double phase_frac(int64_t i, int64_t j) const;
    // For the built-in kinds, phase_frac(i, j) = xxi (i xi mod Ng) / Ng + kappa_i |xi| + rho_i
    // + sq (xi^2 mod 4 Ng) / (4 Ng) mod 1 (xi = j - Ng/2); false for user phases and
    // indirect plans.
    bool row_terms(int64_t i, double* kappa, double* rho, int* xxi, int* sq) const;
    cd amplitude(int64_t i, int64_t j) const;
    // K(x_i, xi_j): the entry callback (BF_PHASE_ENTRIES) or the explicit alpha e^{2 pi i Phi}
    cd entry(int64_t i, int64_t j) const;
    // K at n index pairs; a bulk callback is called from this thread in pieces of at most
    // 2^20 entries, other sources are evaluated in parallel
    void entries(const int64_t* I, const int64_t* J, int64_t n, cd* out) const;
    bool bulk() const { return d.phase_kind == BF_PHASE_ENTRIES && (d.entries || d.matvec); }
    // Scenario 2: the requested entries read off whole columns K e_j or rows K^T e_i
    void entries_matvec(const int64_t* I, const int64_t* J, int64_t n, cd* out) const;
    // the explicit definitions (kinds and callbacks of d), whatever indirect says
    double phase_frac_explicit(int64_t i, int64_t j) const;
    cd amplitude_explicit(int64_t i, int64_t j) const;
};

// ---------------------------------------------------------------------------
// Factors of one N x N sub-BF, FP64, in the layouts documented in bf.h
// (bf_plan_view).  Levels: V at l1, H at l1+1..h, switch M^h at h, G at
// h+1..L-l1, U at L-l1 (levels with nodes of <= r indices are exact copies in
// Algorithm 4.1 and are merged into V and U).
struct BlockFactors {
    int64_t N = 0, row0 = 0, col0 = 0;
    int r = 0, n0 = 1, L = 0, h = 0, l1 = 0, nv = 0;
    int ra = 0;
    std::vector<cd> a, b;                 // [ra][N]
    std::vector<double> Mv;               // [r][nv]
    std::vector<cd> EV;                   // [2^l1][N]
    std::vector<std::vector<double>> MH;  // per H level: [r][2r]
    std::vector<std::vector<cd>> EH;      // per H level: [P][2][r]
    std::vector<cd> S;                    // [P][r][r]
    std::vector<std::vector<double>> MG;  // per G level: [2][r][r]
    std::vector<std::vector<cd>> FG;      // per G level: [P][2][r]
    std::vector<double> MU;               // [nu][r]
    std::vector<cd> EU;                   // [2^l1][N]
    double amp_sigma_ratio = 0.0;
    double t_amp = 0.0;  // host seconds of the amplitude split
    // indirect plans: the recovered phase and the recovery's accuracy and time
    PhaseLR lr;
    double t_recover = 0.0, recover_err_k = 0.0, recover_err_amp = 0.0;
    int64_t P() const { return N / n0; }
    int nH() const { return h - l1; }
    int nG() const { return L - l1 - h; }
    size_t host_bytes() const;
};

struct DeviceState;  // defined in the CUDA translation units
struct NufftState;   // bf_nufft.cu

}  // namespace bfi

struct bf_plan {
    bfi::KernelFn kern;
    bf_options opt{};
    double eps = 0;
    int64_t N = 0;
    int r = 0, n0 = 1, L = 0, h = 0, l1 = 0;
    bool factored = false;
    bool user_kinds_lost = false;  // loaded from file with user callbacks
    bool otf = false;              // factored by bf_factor_otf (no phase tables; FP32 applies only)
    std::vector<bfi::BlockFactors> blocks;  // 1 or 4
    bfi::DeviceState* dev = nullptr;
    bfi::NufftState* nufft = nullptr;  // bf_nufft_prepare (Sec. 3, Eq. tg3)
    std::map<int64_t, int> tuned_mr;  // autotuned column-slice width per m (FP32 fused apply)
    int mr_hint(int64_t m) const
    {
        auto it = tuned_mr.find(m);
        return it == tuned_mr.end() ? 0 : it->second;
    }
};

namespace bfi {

// grids / interpolation (Sec. 2.1)
std::vector<int64_t> grid_rel(int64_t n, int r);
std::vector<double> lagrange(const std::vector<int64_t>& nodes, const std::vector<double>& pts);
inline int64_t centre(int64_t start, int64_t n) { return start + (n - 1) / 2; }
int choose_l1(int r, int n0);

// construction
// tables = false: geometry, amplitude split and the real matrices only (the
// phase tables are then built on the device, bf_factor_device)
bf_status factor_block(const KernelFn& k, const bf_options& opt, BlockFactors& B, bool tables = true);
bf_status amplitude_split(const KernelFn& k, const bf_options& opt, int64_t row0, int64_t col0,
                          int64_t N, std::vector<cd>& a, std::vector<cd>& b, int& ra,
                          double& sigma_ratio);

// small dense complex linear algebra (column-major)
struct CMat {
    int64_t m = 0, n = 0;
    std::vector<cd> v;
    CMat() = default;
    CMat(int64_t m_, int64_t n_) : m(m_), n(n_), v((size_t)(m_ * n_)) {}
    cd& operator()(int64_t i, int64_t j) { return v[(size_t)(i + j * m)]; }
    const cd& operator()(int64_t i, int64_t j) const { return v[(size_t)(i + j * m)]; }
};
// Householder QR with column pivoting, stopped after kmax steps or when the
// largest remaining column norm falls below tol * (first pivot norm).
// Returns the rank k; Q is m x k (orthonormal columns), piv the full pivot order.
int pivoted_qr(CMat A, int kmax, double tol, CMat& Q, std::vector<int64_t>& piv);
// One-sided Jacobi SVD of a small matrix: A = U diag(S) V^*.
void jacobi_svd(const CMat& A, CMat& U, std::vector<double>& S, CMat& V);
CMat pinv(const CMat& A, double rcond);
CMat matmul(const CMat& A, const CMat& B);
CMat adjoint(const CMat& A);

// Algorithm 1 (Sec. 2.1) on an N x N matrix seen through submatrices: entries(I, J) and
// its adjoint entries_adj(I, J) (then J x I); a = U0 Sigma0, b = V0^* as [rank][N]
using EntriesFn = std::function<CMat(const std::vector<int64_t>&, const std::vector<int64_t>&)>;
// fixed_rows / fixed_cols join every sample set (e.g. where the matrix is least smooth)
bf_status lowrank_sampled(const EntriesFn& entries, const EntriesFn& entries_adj, int64_t N, int r, int q,
                          double tol, uint64_t seed_state, std::vector<cd>& a, std::vector<cd>& b, int& rank,
                          double& sigma_ratio, const std::vector<int64_t>& fixed_rows,
                          const std::vector<int64_t>& fixed_cols);
// indirect access (bf_recover.cpp): Algorithm 3 on one vector, and the phase of one
// sub-BF window by Algorithms 3-5; recovery_errors fills eps^K and eps^amp of Sec. 5
void unwrap(const double* u, int64_t n, double tau, const double* seed, int nseed, double* v,
            std::vector<int64_t>* starts);
bf_status recover_phase(const KernelFn& k, const bf_options& opt, int64_t row0, int64_t col0, int64_t N,
                        PhaseLR& lr);
void recovery_errors(const KernelFn& k, BlockFactors& B, uint64_t seed);

// device side (bf_device.cu)
bf_status device_upload(bf_plan* p);
// device construction of the phase tables (bf_construct.cu, bf_device.cu)
bool construct_supported(int phase_kind);
bf_status device_construct(bf_plan* p);
// device residency without phase tables (bf_factor_otf): the FP32 kernels evaluate the phases
bf_status device_otf(bf_plan* p);
bf_status device_reserve(bf_plan* p, bf_precision prec, int64_t m, void* stream);
bf_status device_apply(bf_plan* p, bf_precision prec, const void* F, int64_t m, void* G,
                       void* stream);
bf_status device_apply_host(bf_plan* p, bf_precision prec, const void* F, int64_t m, void* G,
                            void* stream);
bf_status device_sync_status(bf_plan* p, void* stream);
// apply with a caller-owned workspace (ws_bytes >= device_ws_bytes(p, prec, m))
size_t device_ws_bytes(const bf_plan* p, bf_precision prec, int64_t m);
bf_status device_apply_ws(bf_plan* p, bf_precision prec, const void* F, int64_t m, void* G, void* stream, void* ws,
                          size_t ws_bytes);
void device_free(bf_plan* p);
void nufft_free(bf_plan* p);  // bf_nufft.cu
// NUFFT apply (Sec. 3, Eq. tg3) with a caller-owned workspace of >= nufft_ws_bytes(p, m)
size_t nufft_ws_bytes(const bf_plan* p, int64_t m);
bf_status nufft_apply_ws(bf_plan* p, const void* F, int64_t m, void* G, void* stream, void* ws, size_t ws_bytes);
void device_info(const bf_plan* p, bf_plan_info* info);

}  // namespace bfi
