/*
 * bf.h -- C ABI of the GB300 butterfly-factorisation (IBF-MAT) apply library.
 *
 * The library evaluates the discretised oscillatory integral transform
 *     g = K f,   K_ij = alpha(x_i, xi_j) exp(2 pi i Phi(x_i, xi_j)),
 * x_i = i/N, xi_j = j - N/2 (Sec. 5, Eq. 1D-FIO / 1D-xandxi, 0-based), for
 * many right-hand sides at once, as
 *     g = sum_k diag(a_k) BF(e^{2 pi i Phi}) diag(b_k) f          (Sec. 1, Eq. tg)
 * where alpha ~ sum_k a_k(x) b_k(xi) comes from Algorithm 1 (Sec. 2.1) and BF
 * is the butterfly factorisation of Eq. (BFM), Sec. 4,
 *     e^{2 pi i Phi} ~ U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^1)^* (V^0)^*,
 * built from the interpolative low-rank factors of Algorithm 2 by the
 * recursion of Algorithm 4.1 (Eqs. 1, 2, 3, bf3 and the switch step).
 *
 * Conventions for every entry point:
 *  - Return value: BF_OK or an error code; bf_last_error() then returns a
 *    thread-local message describing the last failure on the calling thread.
 *  - Pointers documented as "device" are CUDA device pointers on the plan's
 *    device; "host" pointers are ordinary (preferably page-locked) memory.
 *  - Complex data are interleaved (re, im): "c64" = 2 x float, "c128" =
 *    2 x double.  Right-hand-side blocks are row-major [N][m] with the m
 *    right-hand sides innermost (PyTorch's layout for a contiguous (N, m)).
 *  - The caller owns F and G; the plan owns its factors and workspace.
 *  - Calls on one plan are not thread-safe.  Applies of one plan share its
 *    workspace (and its cached FP64 graph), so the caller keeps them from
 *    overlapping on the GPU (one stream, or ordered streams); concurrent
 *    applies of one operator go through a bf_server, whose slots each have
 *    their own workspace.
 *  - No entry point calls exit(), abort() or traps on the device; GPU-side
 *    failures (a bounded wait that ran out) are reported as BF_ERR_TIMEOUT
 *    by bf_sync_status().
 */
#ifndef BF_H
#define BF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_plan bf_plan;

typedef enum {
    BF_OK = 0,
    BF_ERR_ARG = 1,         /* invalid argument (size, pointer, option)            */
    BF_ERR_NOMEM = 2,       /* host or device allocation failed / budget exceeded  */
    BF_ERR_CUDA = 3,        /* a CUDA runtime call failed                           */
    BF_ERR_STATE = 4,       /* call out of order (e.g. apply before factor)        */
    BF_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out                  */
    BF_ERR_ACCURACY = 6,    /* construction could not meet the tolerance           */
    BF_ERR_IO = 7,          /* plan file could not be read or written               */
    BF_ERR_UNSUPPORTED = 8  /* feature not built for these parameters              */
} bf_status;

/* Arithmetic of the apply. */
typedef enum {
    BF_PREC_F64 = 0,    /* plain form: one launch per butterfly stage, c128 data    */
    BF_PREC_F32 = 1,    /* fused two-pass persistent apply, c64 data (default)      */
    BF_PREC_BF16X3 = 2  /* c64 data; level products on tensor cores with hi/lo BF16 */
} bf_precision;

/* Built-in phase functions Phi(x, xi) (numbering shared with the test oracle). */
typedef enum {
    BF_PHASE_DFT = 0,     /* x xi                                                         */
    BF_PHASE_FIO = 1,     /* x xi + c(x)|xi|, c(x) = (2 + s sin 2 pi x)/16 (Sec. 5, 1D FIO) */
    BF_PHASE_FIO_PW = 2,  /* x xi + c|xi| for x < 1/2; x xi - c|xi|/2 for x >= 1/2      */
    BF_PHASE_ONES = 3,    /* 0                                                            */
    BF_PHASE_SEP = 4,     /* 0.3 sin(2 pi x) + xi^2/(4N)  (R(A,B) of Eq. RAB vanishes)    */
    BF_PHASE_USER = 100,  /* Phi given by the phi callback                               */
    BF_PHASE_ENTRIES = 101 /* K known only through its entries (the entry callback): the    *
                            * amplitude and the phase are recovered (bf_options.indirect)  */
} bf_phase_kind;

/* Built-in amplitudes alpha(x, xi). */
typedef enum {
    BF_AMP_ONE = 0,       /* 1                                                 */
    BF_AMP_SMOOTH = 1,    /* 1 + 0.25 sin(2 pi x) cos(2 pi xi / N)  (rank 2)   */
    BF_AMP_USER = 100     /* alpha given by the alpha callback (complex)       */
} bf_amp_kind;

/* User phase: returns Phi(x, xi) (real).  Only its value mod 1 matters. */
typedef double (*bf_phase_fn)(double x, double xi, void* user);
/* User amplitude: writes alpha(x, xi) = *re + i *im. */
typedef void (*bf_amp_fn)(double x, double xi, void* user, double* re, double* im);
/* Bulk kernel entries (indirect access): writes K at the n grid index pairs (i[k], j[k]),
 * 0 <= i, j < N, as out[2k] + i out[2k+1].  Called from one thread at a time, with n up to
 * 2^20. */
typedef void (*bf_entries_fn)(const int64_t* i, const int64_t* j, int64_t n, void* user, double* out);
/* Products with the kernel matrix (indirect access, Scenario 2 of Table sc): writes
 * Y = K X (transpose = 0) or Y = K^T X (transpose = 1, no conjugation) for m vectors.
 * X and Y are host arrays [N][m] of complex numbers (re, im interleaved; the right-hand
 * sides innermost, as F and G of bf_apply).  Called from one thread at a time; the
 * library applies it to unit vectors to read whole columns (K e_j) and rows (K^T e_i). */
typedef void (*bf_matvec_fn)(const double* X, int64_t m, int transpose, void* user, double* Y);

/* The operator: the N x N transform on the grid x_i = i/N, xi_j = j - N/2. */
typedef struct {
    int64_t N;            /* power of two                                       */
    int phase_kind;       /* bf_phase_kind                                      */
    double phase_param;   /* s of BF_PHASE_FIO / FIO_PW (1.0 if 0 is given)      */
    int amp_kind;         /* bf_amp_kind                                        */
    bf_phase_fn phi;      /* used when phase_kind == BF_PHASE_USER              */
    bf_amp_fn alpha;      /* used when amp_kind == BF_AMP_USER                  */
    void* user;           /* passed to the callbacks                            */
    bf_amp_fn entry;      /* used when phase_kind == BF_PHASE_ENTRIES: writes    *
                           * K(x, xi) = alpha e^{2 pi i Phi}, alpha > 0 assumed; *
                           * amp_kind is then ignored                            */
    bf_entries_fn entries;/* the same in bulk by grid indices; with             *
                           * BF_PHASE_ENTRIES it is used instead of entry when  *
                           * not NULL                                            */
    bf_matvec_fn matvec;  /* with BF_PHASE_ENTRIES and entries NULL: K known     *
                           * only through products with K and K^T (Scenario 2);  *
                           * used instead of entry when not NULL                 */
} bf_kernel_desc;

typedef struct {
    int r;                /* interpolation points per node (r_eps); 0: from eps           */
    int n0;               /* leaf size of both trees (power of two, default 1, Fig. 2)    */
    int split;            /* 1: one BF; 2: four N/2 x N/2 sub-BFs (rows and columns cut    *
                           *    at N/2, i.e. at x = 1/2 and xi = 0)                        */
    int amp_rank;         /* rank parameter r of Algorithm 1 (default 8)                   */
    int amp_oversample;   /* oversampling q of Algorithm 1 (default 3)                     */
    double amp_tol;       /* relative singular-value cut for r_alpha (default 1e-13)       */
    uint64_t seed;        /* sampling seed of Algorithm 1 (default 0)                      */
    int keep_host;        /* keep the FP64 host factors after upload (default 1)           */
    int device;           /* CUDA device of the plan (default 0)                           */
    /* Indirect access (Scenario 1 of Table sc, Sec. 2.2).  With indirect = 1 (implied by
     * BF_PHASE_ENTRIES) bf_factor sees K only through its entries: built-in kinds are
     * evaluated as a black box.  It recovers the amplitude by Algorithm 1 on |K| and a
     * low-rank phase Psi, e^{2 pi i Psi} = K/|K|, by Algorithms 3-5.  It then builds
     * the butterfly of Sec. 4 from those factors.  Such plans are factored on the host
     * only (bf_factor). */
    int indirect;         /* 0 (default) or 1                                                 */
    int phase_rank;       /* rank parameter of the phase's Algorithm 1 step (default 20)      */
    int phase_oversample; /* its oversampling q (default 5)                                   */
    double phase_tol;     /* relative singular-value cut of the recovered phase (default 1e-13) */
    double tau;           /* discontinuity threshold of Algorithm 3 on second differences of  *
                           * Phi in turns (default 0.25: pi/2 of the phase 2 pi Phi)           */
    int l1;               /* level of the V and U stages (Eq. 1 and Eq. bf3 evaluated on leaf    *
                           * groups of n0 2^l1 indices); 0 (default): the first level whose       *
                           * nodes hold more than r indices, where skipping the levels below is   *
                           * exact.  A larger l1 starts the recursion higher: fewer H and G levels *
                           * (smaller tiles, e.g. for the split-BF16 kernels' tensor memory), more *
                           * V and U work; it must not exceed floor(L/2)                          */
} bf_options;

typedef struct {
    int64_t N;
    int r, n0, L, h, l1;   /* levels: V at l1, H l1+1..h, switch at h, G h+1..L-l1, U at L-l1 */
    int r_alpha;           /* amplitude rank                                                */
    int split;             /* 1 or 2                                                        */
    int64_t host_bytes;    /* FP64 host factors                                             */
    int64_t dev_bytes_f64; /* device factors, c128                                          */
    int64_t dev_bytes_f32; /* device factors, c64 (also used by BF16X3)                     */
    int64_t dev_bytes_bf16;/* device hi/lo BF16 copies of the level matrices                */
    int uploaded;
    double amp_sigma_ratio;/* sigma_{r_alpha+1}/sigma_1 of the amplitude (0 if exact)        */
    /* indirect plans (0 otherwise), each the maximum over the sub-BFs: */
    int phase_rank;        /* rank of the recovered phase Psi                                */
    double t_recover_s;    /* host seconds recovering amplitude and phase (Algorithms 1, 3-5) */
    double recover_err_k;  /* eps^K of Sec. 5: 2-norm error of the kernel rebuilt from the    *
                            * recovered factors against K on 256 x 256 sampled entries,        *
                            * relative to K's                                                  */
    double recover_err_amp;/* eps^amp of Sec. 5, the same for the amplitude against |K|      */
} bf_plan_info;

/* Fill *opt with the defaults listed above. */
bf_status bf_default_options(bf_options* opt);

/* Algorithm 3 (Sec. 2.2) on the host: rebuilds v from u = v mod 1 (u in [0, 1), n
 * entries), with the first nseed (0..3) values of v given in seed.  The first value
 * is u[0]; the second is the one nearest the first; the third keeps the first
 * difference; every later one makes the third difference smallest.  A second
 * difference above tau (turns) starts a new piece there.  v is u plus integers.
 * starts receives the start index of every piece (starts[0] = 0), at most cap of
 * them; *nstarts is their total count.  Errors: BF_ERR_ARG (n < 0, nseed outside
 * 0..3 or above n, NULL u/v/nstarts, starts NULL with cap > 0). */
bf_status bf_unwrap(const double* u, int64_t n, double tau, const double* seed, int nseed, double* v,
                    int64_t* starts, int64_t cap, int64_t* nstarts);

/* Algorithm 6 (Sec. 3): may sub-BF `block` of a plan be evaluated by r-dimensional NUFFTs
 * after dimension lifting (Eq. tg3), or does it need the butterfly?  Inputs are low-rank
 * factorizations of the phase, Psi = sum_k p_k(x) q_k(xi) of rank r1, and of the amplitude,
 * alpha = sum_k a_k(x) b_k(xi) (views 0, 1).  For a plan factored from its entries the
 * phase factors are the recovered ones (views 11, 12; r1 = phase_rank).  For a built-in
 * phase they are its closed form in turns: DFT (x)(xi); FIO (x, c(x))(xi, |xi|); FIO_PW the
 * same with c(x) for x < 1/2 and -c(x)/2 above; SEP (0.3 sin 2 pi x, 1)(1, xi^2 / 4N); ONES
 * none.  Steps:
 *  1. the r-leading SVD of the phase factorization is the lifting P Q^T (taken exactly:
 *     QR of both N x r1 factors, then the SVD of the r1 x r1 core; r >= r1 lifts the
 *     whole phase);
 *  2. r_eps * q random columns (seeded) of the residual kernel alpha e^{2 pi i (Psi - P Q^T)}
 *     are factored by QR with column pivoting;
 *  3. *n = the number of pivots above eps times the first; *y = 1 iff *n < r_eps (the
 *     printed algorithm's "r q" columns and "n < r" are read with r_eps);
 *  4. if *y = 1, Algorithm 1 (rank parameter r_eps, oversampling q, tolerance eps)
 *     factors the residual kernel and *terms receives its rank, the number of NUFFTs of
 *     Eq. tg3; otherwise *terms = 0.
 * Host only, O(N (r1^2 + r_eps q (r1 + r_alpha))) work; no NUFFT is run.  Errors:
 * BF_ERR_ARG (NULL plan or outputs, r, r_eps or q below 1, eps <= 0, bad block),
 * BF_ERR_STATE (plan not factored, host factors released, or a user phase callback,
 * whose factorization is unknown), BF_ERR_NOMEM. */
bf_status bf_nufft_decide(const bf_plan* plan, int block, int r, int r_eps, int q, double eps,
                          uint64_t seed, int* y, int* n, int* terms);

/* NUFFT evaluation of the transform (Sec. 3, Eq. tg3), for phases that are
 * rank 1 on each half of the columns: the built-in DFT, FIO, FIO_PW and ONES
 * kinds (Phi = t_h(x) xi + rho(x) on xi >= 0 and on xi < 0, the split of the
 * wave-equation FIO at xi = 0, Eq. FIOwq2 of Sec. 5).  There Algorithm 6's
 * lifting with r = 1 removes each half's whole phase, and
 *     g_i = sum_h sum_k a_k(x_i) e^{2 pi i rho_i} sum_{xi in h} e^{2 pi i t_h(x_i) xi} b_k(xi) f(xi)
 * is 2 r_alpha one-dimensional NUFFTs (uniform modes, non-uniform targets) per
 * right-hand side, with the amplitude split alpha ~ sum_k a_k b_k of
 * Algorithm 1.  The paper names no NUFFT algorithm; this one is Gaussian
 * gridding on a grid twice as fine as the modes, with msp grid points on each
 * side of a target: its error falls like exp(-2 pi msp / 3), and msp is the
 * smallest with exp(-2 pi msp / 3) <= eps (2 <= msp <= 16).
 *
 * bf_nufft_prepare: host FP64 planning of the targets, interpolation weights,
 * deconvolution factors and twiddles, uploaded to the plan's device (O(N)
 * memory; the plan need not be factored for the butterfly).  Replaces an
 * earlier preparation.  *msp_out (nullable) receives msp.  Requirements: a
 * power-of-two N with 256 <= N <= 2^20, a built-in phase of the kinds above
 * (else BF_ERR_UNSUPPORTED), eps in (0, 1) (else BF_ERR_ARG).  Errors also
 * BF_ERR_NOMEM, BF_ERR_CUDA.
 *
 * bf_nufft_apply: G = K F for m right-hand sides in complex FP32, F and G
 * device [N][m] c64 as for bf_apply (G must not alias F), asynchronously on
 * `stream`: three kernels (the deconvolution fused into the first pass of a
 * four-step inverse FFT, the second pass, the interpolation).  Uses a
 * workspace of 4 N r_alpha m c64 numbers owned by the plan, grown with
 * cudaMalloc when m grows (so: not inside stream capture for a new m).  Each
 * column is computed on its own: a column's result is bitwise the same for
 * any m and any neighbouring columns.
 * Errors: BF_ERR_ARG, BF_ERR_STATE (no bf_nufft_prepare), BF_ERR_NOMEM,
 * BF_ERR_CUDA.
 *
 * bf_nufft_info: msp, r_alpha, and the workspace bytes per right-hand side of
 * a prepared plan (each pointer nullable); BF_ERR_STATE if not prepared. */
bf_status bf_nufft_prepare(bf_plan* plan, double eps, int* msp_out);
bf_status bf_nufft_apply(bf_plan* plan, const void* F, int64_t m, void* G, void* stream);
bf_status bf_nufft_info(const bf_plan* plan, int* msp, int* r_alpha, int64_t* ws_bytes_per_rhs);

/* Create a plan for the operator *desc to tolerance eps (the target relative
 * l2 error eps^b of Sec. 5).  With opt->r == 0 the interpolation rank is taken
 * from eps by the rule r = 4 + ceil(-log10 eps), measured for 1D-FIO-like
 * phases (Table 1D-FIO).  opt may be NULL.  No GPU work.  *out owns the plan.
 * Errors: BF_ERR_ARG (N not a power of two, N too small for this r and n0,
 * eps not in (0, 1), bad kinds/callbacks). */
bf_status bf_plan_create(const bf_kernel_desc* desc, double eps, const bf_options* opt,
                         bf_plan** out);

/* Build the factorisation on the host in FP64: the amplitude split by
 * Algorithm 1 and, for each sub-BF, the factors V^0, H^l, M^h, G^l, U^L of
 * Eq. (BFM) from Algorithms 2 and 4.1.  Idempotent.  No GPU work. */
bf_status bf_factor(bf_plan* plan);

/* Copy the factors to the plan's device in the layouts the kernels consume
 * (c128 for F64, c64 for F32, plus BF16 hi/lo level matrices).  Called by the
 * first bf_apply if not called before; call it before any stream capture.
 * Errors: BF_ERR_STATE (not factored), BF_ERR_NOMEM, BF_ERR_CUDA. */
bf_status bf_upload(bf_plan* plan);

/* Factor and upload in one step, with the O(r N log N) phase tables (Eqs. 1,
 * 2, 3, bf3 and the switch step of Algorithm 4.1) computed on the device in
 * FP64 (and their FP32 copies) instead of on the host; the amplitude split
 * (Algorithm 1) and the real Lagrange matrices are still built on the host.
 * Only the built-in phase kinds (not BF_PHASE_USER) have a device form.  The
 * host keeps no phase tables, so bf_plan_save and bf_plan_view of tables
 * return BF_ERR_STATE.  On an already factored plan this is bf_upload.
 * Errors: BF_ERR_ARG, BF_ERR_STATE, BF_ERR_UNSUPPORTED (user phase),
 * BF_ERR_NOMEM, BF_ERR_CUDA. */
bf_status bf_factor_device(bf_plan* plan);

/* Factor for the on-the-fly apply: no phase tables anywhere.  The host builds
 * the amplitude split (Algorithm 1) and the real Lagrange matrices; the device
 * keeps those, 16 bytes of phase coefficients per global grid row and the
 * interpolation grids, i.e. O(r_alpha N) memory instead of the O(r N log N)
 * tables.  The FP32 apply kernels then evaluate every phase factor they use
 * (Eqs. 1, 2, 3, bf3 and the switch step of Algorithm 4.1: e^{2 pi i Phi} at
 * grid points of the two trees) from Phi's closed form, with Phi mod 1 held
 * as an exact 32-bit fixed-point number of turns.  Only the built-in phase
 * kinds, N <= 2^30 and BF_PREC_F32 applies (bf_apply, bf_apply_host,
 * bf_apply_f32_noalloc, the sharded apply); F64 and BF16X3 applies, batches
 * and servers return BF_ERR_UNSUPPORTED, bf_plan_save and table views
 * BF_ERR_STATE.  On an already factored plan: BF_ERR_STATE.
 * Errors: BF_ERR_ARG, BF_ERR_STATE, BF_ERR_UNSUPPORTED, BF_ERR_NOMEM,
 * BF_ERR_CUDA. */
bf_status bf_factor_otf(bf_plan* plan);

/* Pre-allocate device workspace for applies of up to m_max right-hand sides at
 * precision prec (so that later bf_apply calls allocate nothing and can be
 * captured in a CUDA graph).  Errors: BF_ERR_NOMEM, BF_ERR_CUDA. */
bf_status bf_reserve(bf_plan* plan, bf_precision prec, int64_t m_max);

/* G = K F for m right-hand sides, asynchronously on `stream` (a cudaStream_t,
 * NULL = legacy default stream).  F, G: device, [N][m], c128 for BF_PREC_F64
 * and c64 otherwise; G must not alias F.  Uses the plan's workspace (grown
 * with cudaMalloc when m exceeds the reserved size -- not capture-safe).
 * Errors: BF_ERR_ARG (m < 1, NULL pointers), BF_ERR_STATE, BF_ERR_NOMEM,
 * BF_ERR_CUDA (launch failure), BF_ERR_UNSUPPORTED (no kernels for this r). */
bf_status bf_apply(bf_plan* plan, bf_precision prec, const void* F, int64_t m, void* G,
                   void* stream);

/* Allocation-free form of bf_apply for BF_PREC_F32 (the paper has no
 * counterpart: this is an integration aid).  For callers that may not
 * allocate device memory when they apply -- a server or host application that
 * owns all device memory through its own pool, or a latency-critical path
 * that must not enter the CUDA allocator -- it uses a fixed 32 MiB scratch
 * array compiled into the library instead of the plan's workspace; every GPU
 * that loads the library holds that array until exit.  Requirements: the
 * plan is uploaded (bf_upload); the switch-level workspace for this N and m
 * fits in 32 MiB (else BF_ERR_ARG, message gives the size); bf_profile timing
 * is off (else BF_ERR_STATE).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and caches it: make that
 * first call before any stream capture.  The cached address belongs to the
 * device's primary context as it was at that first call: after
 * cudaDeviceReset (or anything else that destroys and re-creates the primary
 * context) it is stale, so a process that resets a device must not call this
 * entry point on that device again.  Calls share the array, so calls
 * that overlap on the GPU race; nothing in it needs clearing between calls.
 * F, G, m, stream as for bf_apply (c64).  Allocates nothing. */
bf_status bf_apply_f32_noalloc(bf_plan* plan, const void* F, int64_t m, void* G, void* stream);

/* Same as bf_apply but F and G are HOST buffers (pinned memory lets the copies
 * run asynchronously): copies F to the device, applies, copies G back, and
 * synchronises `stream` before returning.  The result is bitwise that of
 * bf_apply.  An FP32 apply of a one-sub-BF plan (one front and one back pass)
 * copies in four row ranges on the plan's own copy stream, overlapped with the
 * kernels of the other ranges.  Those kernels alternate between `stream` and a
 * second stream of the plan that first waits for `stream`'s earlier work.  Other
 * applies copy F, apply on `stream`, then copy G.  The staging buffers belong
 * to the plan, so host applies of one plan must not overlap. */
bf_status bf_apply_host(bf_plan* plan, bf_precision prec, const void* F_host, int64_t m,
                        void* G_host, void* stream);

/* Result of device-side checks of earlier applies on `stream` (synchronises):
 * BF_OK or BF_ERR_TIMEOUT. */
bf_status bf_sync_status(bf_plan* plan, void* stream);

bf_status bf_plan_get_info(const bf_plan* plan, bf_plan_info* info);

/* Read-only view of an FP64 host factor array of sub-BF `block` (0 unless
 * split == 2, then block = 2*row_half + col_half).  what: 0 a (amplitude,
 * [r_alpha][N] c128), 1 b ([r_alpha][N] c128), 2 Mv ([r][nv] real), 3 EV
 * ([2^l1][N] c128), 4 MH (level, [r][2r] real), 5 EH (level, [P][2][r] c128),
 * 6 S ([P][r][r] c128), 7 MG (level, [2][r][r] real), 8 FG (level, [P][2][r]
 * c128), 9 MU ([nu][r] real), 10 EU ([2^l1][N] c128), 11 and 12 the factors
 * p and q of a phase recovered from entries (Algorithm 5: Psi(i, j) =
 * Re sum_k p[k][i] q[k][j] on the sub-BF window, local indices; [phase_rank][N]
 * c128; *count = 0 for explicit phases).  *data points into the plan (valid
 * until bf_destroy), *count = number of doubles.  Requires a factored plan with
 * host factors kept.  For tests and inspection. */
bf_status bf_plan_view(const bf_plan* plan, int block, int what, int level,
                       const double** data, int64_t* count);

/* Save / load a factored plan (versioned header + FP64 factors), so that a
 * restarted server skips bf_factor.  Callbacks are not saved: a loaded plan
 * with user kinds can be applied but not re-factored. */
bf_status bf_plan_save(const bf_plan* plan, const char* path);
bf_status bf_plan_load(const char* path, const bf_options* opt, bf_plan** out);

/* Release the plan and its host and device memory.  NULL-safe. */
void bf_destroy(bf_plan* plan);

/* The mock-Chebyshev index grid of Eq. (gdA)/(gdB) for a node of n indices:
 * writes min(n, r) increasing 0-based offsets to out, *count = their number. */
bf_status bf_grid_indices(int64_t n, int r, int64_t* out, int* count);

/* Thread-local description of the last error on this thread. */
const char* bf_last_error(void);

/* Library version string. */
const char* bf_version(void);

/* Kernel timing, for measurement: between bf_profile_begin() and
 * bf_profile_end() every kernel the library launches is bracketed by CUDA
 * events recorded on the stream it is launched on.  bf_profile_end()
 * synchronises those events and aggregates them per kernel name;
 * bf_profile_count()/bf_profile_get() then read the aggregate (name,
 * launches, total milliseconds).  Process-wide; not for use inside stream
 * capture. */
bf_status bf_profile_begin(void);
bf_status bf_profile_end(void);
int bf_profile_count(void);
bf_status bf_profile_get(int i, const char** name, int64_t* launches, double* total_ms);

/* Measurement aid (the paper has no counterpart): the FP32 FMA throughput of
 * `device` from a register-only loop of fused multiply-adds (8 independent
 * chains per thread, every SM filled), best of 5 timed launches after one
 * warm-up, in TFLOP/s (2 flops per FMA); *sm_count receives the device's SM
 * count.  It is the ceiling the FP32 apply kernels, which are bound by FMA
 * issue, are held to.  Synchronises the device; allocates 256 KB for the
 * duration of the call.  Errors: BF_ERR_ARG (NULL output), BF_ERR_CUDA. */
bf_status bf_fp32_peak(int device, int* sm_count, double* tflops);
/* The same for FP64 fused multiply-adds (the ceiling of the plain FP64 form's
 * stage kernels), in TFLOP/s.  Errors: BF_ERR_ARG, BF_ERR_CUDA. */
bf_status bf_fp64_peak(int device, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* BF_H */
