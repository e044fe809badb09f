// Plan persistence: a versioned binary header plus the FP64 host factors, so
// that the factorisation (computed once per operator, Sec. 1 footnote on
// saving precomputation for later applications) survives a restart.
#include <cstdio>
#include <cstring>
#include <new>

#include "bf_internal.h"

using namespace bfi;

namespace {

const char kMagic[8] = {'B', 'F', 'G', 'B', '3', '0', '0', '\0'};
const uint32_t kVersion = 1;

struct Writer {
    FILE* f;
    bool ok = true;
    void raw(const void* p, size_t n) { ok = ok && fwrite(p, 1, n, f) == n; }
    template <typename T> void val(T v) { raw(&v, sizeof(T)); }
    template <typename T> void vec(const std::vector<T>& v)
    {
        val<uint64_t>(v.size());
        raw(v.data(), v.size() * sizeof(T));
    }
};
struct Reader {
    FILE* f;
    bool ok = true;
    void raw(void* p, size_t n) { ok = ok && fread(p, 1, n, f) == n; }
    template <typename T> T val()
    {
        T v{};
        raw(&v, sizeof(T));
        return v;
    }
    template <typename T> void vec(std::vector<T>& v)
    {
        uint64_t n = val<uint64_t>();
        if (!ok || n > ((uint64_t)1 << 40)) {
            ok = false;
            return;
        }
        v.resize((size_t)n);
        raw(v.data(), (size_t)n * sizeof(T));
    }
};

}  // namespace

extern "C" {

bf_status bf_plan_save(const bf_plan* p, const char* path)
{
    if (!p || !path) {
        set_error("bf_plan_save: NULL argument");
        return BF_ERR_ARG;
    }
    if (!p->factored) {
        set_error("bf_plan_save: plan not factored");
        return BF_ERR_STATE;
    }
    for (auto& B : p->blocks)
        if (B.S.empty()) {
            set_error("bf_plan_save: the host holds no phase tables (keep_host = 0, bf_factor_device or bf_factor_otf)");
            return BF_ERR_STATE;
        }
    FILE* f = fopen(path, "wb");
    if (!f) {
        set_error("bf_plan_save: cannot open %s", path);
        return BF_ERR_IO;
    }
    Writer w{f};
    w.raw(kMagic, 8);
    w.val<uint32_t>(kVersion);
    w.val<int64_t>(p->N);
    w.val<int32_t>(p->r);
    w.val<int32_t>(p->n0);
    w.val<int32_t>(p->opt.split);
    w.val<int32_t>(p->kern.d.phase_kind);
    w.val<double>(p->kern.d.phase_param);
    w.val<int32_t>(p->kern.d.amp_kind);
    w.val<double>(p->eps);
    w.val<uint32_t>((uint32_t)p->blocks.size());
    for (auto& B : p->blocks) {
        w.val<int64_t>(B.N);
        w.val<int64_t>(B.row0);
        w.val<int64_t>(B.col0);
        w.val<int32_t>(B.ra);
        w.val<double>(B.amp_sigma_ratio);
        w.vec(B.a); w.vec(B.b); w.vec(B.Mv); w.vec(B.EV);
        w.val<uint32_t>((uint32_t)B.MH.size());
        for (size_t i = 0; i < B.MH.size(); ++i) { w.vec(B.MH[i]); w.vec(B.EH[i]); }
        w.vec(B.S);
        w.val<uint32_t>((uint32_t)B.MG.size());
        for (size_t i = 0; i < B.MG.size(); ++i) { w.vec(B.MG[i]); w.vec(B.FG[i]); }
        w.vec(B.MU); w.vec(B.EU);
    }
    bool ok = w.ok;
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("bf_plan_save: write to %s failed", path);
        return BF_ERR_IO;
    }
    return BF_OK;
}

bf_status bf_plan_load(const char* path, const bf_options* opt, bf_plan** out)
{
    if (!path || !out) {
        set_error("bf_plan_load: NULL argument");
        return BF_ERR_ARG;
    }
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) {
        set_error("bf_plan_load: cannot open %s", path);
        return BF_ERR_IO;
    }
    Reader rd{f};
    char magic[8];
    rd.raw(magic, 8);
    if (!rd.ok || std::memcmp(magic, kMagic, 8) != 0 || rd.val<uint32_t>() != kVersion) {
        fclose(f);
        set_error("bf_plan_load: %s is not a plan file of this version", path);
        return BF_ERR_IO;
    }
    bf_plan* p = new (std::nothrow) bf_plan();
    if (!p) {
        fclose(f);
        set_error("bf_plan_load: out of host memory");
        return BF_ERR_NOMEM;
    }
    if (opt) p->opt = *opt; else bf_default_options(&p->opt);
    p->N = rd.val<int64_t>();
    p->r = rd.val<int32_t>();
    p->n0 = rd.val<int32_t>();
    p->opt.split = rd.val<int32_t>();
    p->opt.r = p->r;
    p->opt.n0 = p->n0;
    p->kern.d.N = p->N;
    p->kern.d.phase_kind = rd.val<int32_t>();
    p->kern.d.phase_param = rd.val<double>();
    p->kern.d.amp_kind = rd.val<int32_t>();
    p->kern.n_global = p->N;
    p->eps = rd.val<double>();
    p->user_kinds_lost = p->kern.d.phase_kind == BF_PHASE_USER || p->kern.d.amp_kind == BF_AMP_USER ||
                         p->kern.d.phase_kind == BF_PHASE_ENTRIES;
    uint32_t nb = rd.val<uint32_t>();
    try {
        if (!rd.ok || nb > 4) throw std::bad_alloc();
        p->blocks.resize(nb);
        for (auto& B : p->blocks) {
            B.N = rd.val<int64_t>();
            B.row0 = rd.val<int64_t>();
            B.col0 = rd.val<int64_t>();
            B.ra = rd.val<int32_t>();
            B.amp_sigma_ratio = rd.val<double>();
            B.r = p->r;
            B.n0 = p->n0;
            B.L = 0;
            while (((int64_t)B.n0 << B.L) < B.N) ++B.L;
            B.h = B.L / 2;
            rd.vec(B.a); rd.vec(B.b); rd.vec(B.Mv); rd.vec(B.EV);
            // the leaf group of V (n0 2^l1 indices) from Mv's size [r][nv]: the level of V and U
            B.nv = B.r > 0 ? (int)(B.Mv.size() / (size_t)B.r) : 0;
            B.l1 = 0;
            while (B.l1 < 31 && (B.n0 << B.l1) < B.nv) ++B.l1;
            if (B.nv != (B.n0 << B.l1) || B.l1 < choose_l1(B.r, B.n0) || B.l1 > B.h) rd.ok = false;
            uint32_t nh = rd.val<uint32_t>();
            if (!rd.ok || nh > 64) throw std::bad_alloc();
            B.MH.resize(nh); B.EH.resize(nh);
            for (uint32_t i = 0; i < nh; ++i) { rd.vec(B.MH[i]); rd.vec(B.EH[i]); }
            rd.vec(B.S);
            uint32_t ng = rd.val<uint32_t>();
            if (!rd.ok || ng > 64) throw std::bad_alloc();
            B.MG.resize(ng); B.FG.resize(ng);
            for (uint32_t i = 0; i < ng; ++i) { rd.vec(B.MG[i]); rd.vec(B.FG[i]); }
            rd.vec(B.MU); rd.vec(B.EU);
            if ((int)nh != B.nH() || (int)ng != B.nG()) rd.ok = false;
        }
    } catch (const std::bad_alloc&) {
        rd.ok = false;
    }
    fclose(f);
    if (!rd.ok) {
        delete p;
        set_error("bf_plan_load: %s is truncated or corrupt", path);
        return BF_ERR_IO;
    }
    p->L = p->blocks[0].L;
    p->h = p->blocks[0].h;
    p->l1 = p->blocks[0].l1;
    p->factored = true;
    *out = p;
    return BF_OK;
}

}  // extern "C"
