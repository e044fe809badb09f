// C ABI: plan life cycle, options, errors, inspection, save/load.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <omp.h>

#include "bf_internal.h"

namespace bfi {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

}  // namespace bfi

using namespace bfi;

extern "C" {

const char* bf_last_error(void) { return g_err; }

const char* bf_version(void) { return "bf-gb300 0.1 (sm_103a)"; }

bf_status bf_default_options(bf_options* opt)
{
    if (!opt) {
        set_error("bf_default_options: NULL");
        return BF_ERR_ARG;
    }
    std::memset(opt, 0, sizeof(*opt));
    opt->r = 0;
    opt->n0 = 1;
    opt->split = 1;
    opt->amp_rank = 8;
    opt->amp_oversample = 3;
    opt->amp_tol = 1e-13;
    opt->seed = 0;
    opt->keep_host = 1;
    opt->device = 0;
    opt->indirect = 0;
    opt->phase_rank = 20;
    opt->phase_oversample = 5;
    opt->phase_tol = 1e-13;
    opt->tau = 0.25;
    return BF_OK;
}

bf_status bf_grid_indices(int64_t n, int r, int64_t* out, int* count)
{
    if (n < 1 || r < 2 || !out || !count) {
        set_error("bf_grid_indices: need n >= 1, r >= 2 and non-NULL outputs");
        return BF_ERR_ARG;
    }
    auto g = grid_rel(n, r);
    for (size_t i = 0; i < g.size(); ++i) out[i] = g[i];
    *count = (int)g.size();
    return BF_OK;
}

bf_status bf_plan_create(const bf_kernel_desc* desc, double eps, const bf_options* opt, bf_plan** out)
{
    if (!desc || !out) {
        set_error("bf_plan_create: NULL argument");
        return BF_ERR_ARG;
    }
    *out = nullptr;
    bf_options o;
    if (opt) o = *opt; else bf_default_options(&o);
    if (o.n0 <= 0) o.n0 = 1;
    if (o.split <= 0) o.split = 1;
    if (o.amp_rank <= 0) o.amp_rank = 8;
    if (o.amp_oversample <= 0) o.amp_oversample = 3;
    if (o.phase_rank <= 0) o.phase_rank = 20;
    if (o.phase_oversample <= 0) o.phase_oversample = 5;
    if (!(o.phase_tol > 0)) o.phase_tol = 1e-13;
    if (!(o.tau > 0)) o.tau = 0.25;
    const int64_t N = desc->N;
    if (N < 4 || (N & (N - 1)) != 0) {
        set_error("bf_plan_create: N=%lld is not a power of two >= 4", (long long)N);
        return BF_ERR_ARG;
    }
    if ((o.n0 & (o.n0 - 1)) != 0) {
        set_error("bf_plan_create: n0=%d is not a power of two", o.n0);
        return BF_ERR_ARG;
    }
    if (o.split != 1 && o.split != 2) {
        set_error("bf_plan_create: split must be 1 or 2");
        return BF_ERR_ARG;
    }
    if (!(eps > 0 && eps < 1) && o.r == 0) {
        set_error("bf_plan_create: eps=%g not in (0, 1)", eps);
        return BF_ERR_ARG;
    }
    int pk = desc->phase_kind, ak = desc->amp_kind;
    const bool entries = pk == BF_PHASE_ENTRIES;
    if (!(pk >= 0 && pk <= 4) && !(pk == BF_PHASE_USER && desc->phi) && !(entries && (desc->entry || desc->entries || desc->matvec))) {
        set_error("bf_plan_create: bad phase_kind %d (or missing phi / entry / matvec callback)", pk);
        return BF_ERR_ARG;
    }
    if (!entries && !(ak == 0 || ak == 1) && !(ak == BF_AMP_USER && desc->alpha)) {
        set_error("bf_plan_create: bad amp_kind %d (or missing alpha callback)", ak);
        return BF_ERR_ARG;
    }
    int r = o.r;
    if (r == 0) r = 4 + (int)std::ceil(-std::log10(eps) - 1e-12);
    if (r < 4 || r > 16 || (r % 2) != 0) {
        // kernels are instantiated for even r in [4, 16]; round odd r up
        if (r % 2) ++r;
        if (r < 4 || r > 16) {
            set_error("bf_plan_create: r=%d outside the supported range [4, 16]", r);
            return BF_ERR_UNSUPPORTED;
        }
    }
    const int64_t Nb = N / o.split;
    int l1 = choose_l1(r, o.n0);
    if (o.l1 < 0 || (o.l1 > 0 && o.l1 < l1)) {
        set_error("bf_plan_create: l1=%d below the first level whose nodes hold more than r=%d indices (%d)", o.l1, r,
                  l1);
        return BF_ERR_ARG;
    }
    if (o.l1 > l1) l1 = o.l1;
    int L = 0;
    while (((int64_t)o.n0 << L) < Nb) ++L;
    if (((int64_t)o.n0 << L) != Nb || L / 2 < l1) {
        set_error("bf_plan_create: block size %lld too small for r=%d, n0=%d (need N/n0 >= 4^%d)",
                  (long long)Nb, r, o.n0, l1);
        return BF_ERR_ARG;
    }
    bf_plan* p = new (std::nothrow) bf_plan();
    if (!p) {
        set_error("bf_plan_create: out of host memory");
        return BF_ERR_NOMEM;
    }
    p->kern.d = *desc;
    if (p->kern.d.phase_param == 0.0) p->kern.d.phase_param = 1.0;
    p->kern.n_global = N;
    p->kern.indirect = entries || o.indirect != 0;
    p->opt = o;
    p->eps = eps;
    p->N = N;
    p->r = r;
    p->n0 = o.n0;
    p->L = L;
    p->h = L / 2;
    p->l1 = l1;
    *out = p;
    return BF_OK;
}

bf_status bf_factor(bf_plan* p)
{
    if (!p) {
        set_error("bf_factor: NULL plan");
        return BF_ERR_ARG;
    }
    if (p->factored) return BF_OK;
    if (p->user_kinds_lost) {
        set_error("bf_factor: plan was loaded without its callbacks");
        return BF_ERR_STATE;
    }
    const int sp = p->opt.split;
    const int64_t Nb = p->N / sp;
    try {
        p->blocks.assign((size_t)(sp * sp), BlockFactors());
        for (int rh = 0; rh < sp; ++rh)
            for (int ch = 0; ch < sp; ++ch) {
                BlockFactors& B = p->blocks[(size_t)(rh * sp + ch)];
                B.N = Nb;
                B.row0 = rh * Nb;
                B.col0 = ch * Nb;
                B.r = p->r;
                B.n0 = p->n0;
                // indirect access: the phase of this window recovered from entries first
                // (Algorithms 3-5); the amplitude split inside factor_block then runs on |K|
                bfi::KernelFn kb = p->kern;
                if (kb.indirect) {
                    const double t0 = omp_get_wtime();
                    bf_status rs = bfi::recover_phase(kb, p->opt, B.row0, B.col0, Nb, B.lr);
                    B.t_recover = omp_get_wtime() - t0;
                    if (rs != BF_OK) return rs;
                    kb.lr = &B.lr;
                }
                bf_status st = factor_block(kb, p->opt, B);
                if (st != BF_OK) return st;
                if (kb.indirect) {
                    B.t_recover += B.t_amp;
                    bfi::recovery_errors(kb, B, p->opt.seed);
                }
            }
    } catch (const std::bad_alloc&) {
        p->blocks.clear();
        set_error("bf_factor: out of host memory");
        return BF_ERR_NOMEM;
    }
    p->factored = true;
    return BF_OK;
}

namespace {

// Geometry, amplitude split and the real Lagrange matrices of every sub-BF,
// without the phase tables (the device builds or evaluates those).
bf_status factor_host_parts(bf_plan* p, const char* who)
{
    const int sp = p->opt.split;
    const int64_t Nb = p->N / sp;
    try {
        p->blocks.assign((size_t)(sp * sp), BlockFactors());
        for (int rh = 0; rh < sp; ++rh)
            for (int ch = 0; ch < sp; ++ch) {
                BlockFactors& B = p->blocks[(size_t)(rh * sp + ch)];
                B.N = Nb;
                B.row0 = rh * Nb;
                B.col0 = ch * Nb;
                B.r = p->r;
                B.n0 = p->n0;
                bf_status st = factor_block(p->kern, p->opt, B, false);
                if (st != BF_OK) {
                    p->blocks.clear();
                    return st;
                }
            }
    } catch (const std::bad_alloc&) {
        p->blocks.clear();
        set_error("%s: out of host memory", who);
        return BF_ERR_NOMEM;
    }
    return BF_OK;
}

}  // namespace

bf_status bf_factor_device(bf_plan* p)
{
    if (!p) {
        set_error("bf_factor_device: NULL plan");
        return BF_ERR_ARG;
    }
    if (p->factored) return bf_upload(p);
    if (p->user_kinds_lost) {
        set_error("bf_factor_device: plan was loaded without its callbacks");
        return BF_ERR_STATE;
    }
    if (!bfi::construct_supported(p->kern.d.phase_kind) || p->kern.indirect) {
        set_error("bf_factor_device: phase kind %d%s has no device form (use bf_factor)", p->kern.d.phase_kind,
                  p->kern.indirect ? " seen through its entries" : "");
        return BF_ERR_UNSUPPORTED;
    }
    const bf_status hs = factor_host_parts(p, "bf_factor_device");
    if (hs != BF_OK) return hs;
    bf_status st = bfi::device_construct(p);
    if (st != BF_OK) {
        p->blocks.clear();
        return st;
    }
    p->factored = true;
    return BF_OK;
}

bf_status bf_factor_otf(bf_plan* p)
{
    if (!p) {
        set_error("bf_factor_otf: NULL plan");
        return BF_ERR_ARG;
    }
    if (p->factored) {
        set_error("bf_factor_otf: plan already factored");
        return BF_ERR_STATE;
    }
    if (p->user_kinds_lost) {
        set_error("bf_factor_otf: plan was loaded without its callbacks");
        return BF_ERR_STATE;
    }
    if (!bfi::construct_supported(p->kern.d.phase_kind) || p->kern.indirect) {
        set_error("bf_factor_otf: phase kind %d%s has no closed form on the device", p->kern.d.phase_kind,
                  p->kern.indirect ? " seen through its entries" : "");
        return BF_ERR_UNSUPPORTED;
    }
    const bf_status hs = factor_host_parts(p, "bf_factor_otf");
    if (hs != BF_OK) return hs;
    bf_status st = bfi::device_otf(p);
    if (st != BF_OK) {
        p->blocks.clear();
        return st;
    }
    p->factored = true;
    p->otf = true;
    return BF_OK;
}

bf_status bf_upload(bf_plan* p)
{
    if (!p) {
        set_error("bf_upload: NULL plan");
        return BF_ERR_ARG;
    }
    if (!p->factored) {
        set_error("bf_upload: plan not factored");
        return BF_ERR_STATE;
    }
    return device_upload(p);
}

bf_status bf_reserve(bf_plan* p, bf_precision prec, int64_t m_max)
{
    if (!p || m_max < 1) {
        set_error("bf_reserve: NULL plan or m_max < 1");
        return BF_ERR_ARG;
    }
    bf_status st = bf_upload(p);
    if (st != BF_OK) return st;
    return device_reserve(p, prec, m_max, nullptr);
}

bf_status bf_apply(bf_plan* p, bf_precision prec, const void* F, int64_t m, void* G, void* stream)
{
    if (!p || !F || !G || m < 1) {
        set_error("bf_apply: NULL plan/buffer or m < 1");
        return BF_ERR_ARG;
    }
    if (F == G) {
        set_error("bf_apply: G must not alias F");
        return BF_ERR_ARG;
    }
    if (prec != BF_PREC_F64 && prec != BF_PREC_F32 && prec != BF_PREC_BF16X3) {
        set_error("bf_apply: bad precision %d", (int)prec);
        return BF_ERR_ARG;
    }
    bf_status st = bf_upload(p);
    if (st != BF_OK) return st;
    return device_apply(p, prec, F, m, G, stream);
}

bf_status bf_apply_host(bf_plan* p, bf_precision prec, const void* F, int64_t m, void* G, void* stream)
{
    if (!p || !F || !G || m < 1) {
        set_error("bf_apply_host: NULL plan/buffer or m < 1");
        return BF_ERR_ARG;
    }
    bf_status st = bf_upload(p);
    if (st != BF_OK) return st;
    return device_apply_host(p, prec, F, m, G, stream);
}

bf_status bf_sync_status(bf_plan* p, void* stream)
{
    if (!p) {
        set_error("bf_sync_status: NULL plan");
        return BF_ERR_ARG;
    }
    if (!p->dev) return BF_OK;
    return device_sync_status(p, stream);
}

bf_status bf_plan_get_info(const bf_plan* p, bf_plan_info* info)
{
    if (!p || !info) {
        set_error("bf_plan_get_info: NULL argument");
        return BF_ERR_ARG;
    }
    std::memset(info, 0, sizeof(*info));
    info->N = p->N;
    info->r = p->r;
    info->n0 = p->n0;
    info->L = p->L;
    info->h = p->h;
    info->l1 = p->l1;
    info->split = p->opt.split;
    if (p->factored && !p->blocks.empty()) {
        int ra = 0;
        double sr = 0;
        int64_t hb = 0;
        for (auto& B : p->blocks) {
            ra = std::max(ra, B.ra);
            sr = std::max(sr, B.amp_sigma_ratio);
            hb += (int64_t)B.host_bytes();
        }
        info->r_alpha = ra;
        info->amp_sigma_ratio = sr;
        info->host_bytes = hb;
        for (auto& B : p->blocks) {
            info->phase_rank = std::max(info->phase_rank, B.lr.rank);
            info->t_recover_s += B.t_recover;
            info->recover_err_k = std::max(info->recover_err_k, B.recover_err_k);
            info->recover_err_amp = std::max(info->recover_err_amp, B.recover_err_amp);
        }
    }
    device_info(p, info);
    return BF_OK;
}

bf_status bf_plan_view(const bf_plan* p, int block, int what, int level, const double** data, int64_t* count)
{
    if (!p || !data || !count) {
        set_error("bf_plan_view: NULL argument");
        return BF_ERR_ARG;
    }
    if (!p->factored || block < 0 || block >= (int)p->blocks.size()) {
        set_error("bf_plan_view: plan not factored (or host factors freed) or bad block");
        return BF_ERR_STATE;
    }
    const BlockFactors& B = p->blocks[(size_t)block];
    auto cv = [&](const std::vector<cd>& v) {
        *data = reinterpret_cast<const double*>(v.data());
        *count = (int64_t)v.size() * 2;
    };
    auto rv = [&](const std::vector<double>& v) {
        *data = v.data();
        *count = (int64_t)v.size();
    };
    const int iH = level - (B.l1 + 1), iG = level - (B.h + 1);
    switch (what) {
    case 0: cv(B.a); break;
    case 1: cv(B.b); break;
    case 2: rv(B.Mv); break;
    case 3: cv(B.EV); break;
    case 4:
    case 5:
        if (iH < 0 || iH >= (int)B.MH.size()) {
            set_error("bf_plan_view: H level %d outside [%d, %d]", level, B.l1 + 1, B.h);
            return BF_ERR_ARG;
        }
        if (what == 4) rv(B.MH[(size_t)iH]); else cv(B.EH[(size_t)iH]);
        break;
    case 6: cv(B.S); break;
    case 7:
    case 8:
        if (iG < 0 || iG >= (int)B.MG.size()) {
            set_error("bf_plan_view: G level %d outside [%d, %d]", level, B.h + 1, B.L - B.l1);
            return BF_ERR_ARG;
        }
        if (what == 7) rv(B.MG[(size_t)iG]); else cv(B.FG[(size_t)iG]);
        break;
    case 9: rv(B.MU); break;
    case 10: cv(B.EU); break;
    case 11: cv(B.lr.p); break;
    case 12: cv(B.lr.q); break;
    default:
        set_error("bf_plan_view: unknown array %d", what);
        return BF_ERR_ARG;
    }
    if (*count == 0 && what >= 2 && what <= 10) {
        set_error("bf_plan_view: host factors were released after upload");
        return BF_ERR_STATE;
    }
    return BF_OK;
}

void bf_destroy(bf_plan* p)
{
    if (!p) return;
    nufft_free(p);
    device_free(p);
    delete p;
}

}  // extern "C"
