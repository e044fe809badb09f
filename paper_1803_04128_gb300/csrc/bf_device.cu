// Device residency of the factors, workspaces and apply dispatch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "bf_device.h"

namespace bfi {
namespace {

#define BF_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error("%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return e_ == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA;   \
        }                                                                          \
    } while (0)

// Byte-packed host image of an arena; pointers are recorded as offsets.
struct Packer {
    std::vector<unsigned char> buf;
    size_t add(const void* src, size_t n)
    {
        size_t off = (buf.size() + 255) & ~(size_t)255;
        buf.resize(off + n);
        if (n) std::memcpy(buf.data() + off, src, n);
        return off;
    }
};

template <typename T>
std::vector<T> real_as(const std::vector<double>& v)
{
    std::vector<T> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
    return o;
}
template <typename C>
std::vector<C> cplx_as(const std::vector<cd>& v)
{
    std::vector<C> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        o[i].x = (decltype(o[i].x))v[i].real();
        o[i].y = (decltype(o[i].y))v[i].imag();
    }
    return o;
}
template <typename C, typename V>
std::vector<C> cplx_concat(const std::vector<V>& vs)
{
    std::vector<C> o;
    for (auto& v : vs) {
        auto c = cplx_as<C>(v);
        o.insert(o.end(), c.begin(), c.end());
    }
    return o;
}
template <typename T>
size_t add_vec(Packer& pk, const std::vector<T>& v) { return pk.add(v.data(), v.size() * sizeof(T)); }

// transposes used by the fused kernels
std::vector<double> transpose(const std::vector<double>& M, int rows, int cols)
{
    std::vector<double> T((size_t)rows * cols);
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j) T[(size_t)j * rows + i] = M[(size_t)i * cols + j];
    return T;
}

struct Offs {
    size_t a, b, Mv, EV, MH, EH, S, MG, FG, MU, EU;
};

template <typename T, typename C>
Offs pack_block(Packer& pk, const BlockFactors& B, bool transposed)
{
    Offs o;
    const int r = B.r;
    o.a = add_vec(pk, cplx_as<C>(B.a));
    o.b = add_vec(pk, cplx_as<C>(B.b));
    o.Mv = add_vec(pk, real_as<T>(transposed ? transpose(B.Mv, r, B.nv) : B.Mv));
    o.EV = add_vec(pk, cplx_as<C>(B.EV));
    std::vector<double> mh;
    for (auto& M : B.MH) {
        auto t = transposed ? transpose(M, r, 2 * r) : M;
        mh.insert(mh.end(), t.begin(), t.end());
    }
    o.MH = add_vec(pk, real_as<T>(mh));
    o.EH = add_vec(pk, cplx_concat<C>(B.EH));
    o.S = add_vec(pk, cplx_as<C>(B.S));
    std::vector<double> mg;
    for (auto& M : B.MG) {
        // natural [pos][t][s]; transposed [pos][s][t]
        for (int pos = 0; pos < 2; ++pos) {
            std::vector<double> blk(M.begin() + (size_t)pos * r * r, M.begin() + (size_t)(pos + 1) * r * r);
            auto t = transposed ? transpose(blk, r, r) : blk;
            mg.insert(mg.end(), t.begin(), t.end());
        }
    }
    o.MG = add_vec(pk, real_as<T>(mg));
    o.FG = add_vec(pk, cplx_concat<C>(B.FG));
    o.MU = add_vec(pk, real_as<T>(B.MU));
    o.EU = add_vec(pk, cplx_as<C>(B.EU));
    return o;
}

template <typename T, typename C>
void bind(DevFactors<T, C>& f, unsigned char* base, const Offs& o)
{
    f.a = reinterpret_cast<C*>(base + o.a);
    f.b = reinterpret_cast<C*>(base + o.b);
    f.Mv = reinterpret_cast<T*>(base + o.Mv);
    f.EV = reinterpret_cast<C*>(base + o.EV);
    f.MH = reinterpret_cast<T*>(base + o.MH);
    f.EH = reinterpret_cast<C*>(base + o.EH);
    f.S = reinterpret_cast<C*>(base + o.S);
    f.MG = reinterpret_cast<T*>(base + o.MG);
    f.FG = reinterpret_cast<C*>(base + o.FG);
    f.MU = reinterpret_cast<T*>(base + o.MU);
    f.EU = reinterpret_cast<C*>(base + o.EU);
}

Geo geo_of(const BlockFactors& B)
{
    Geo g;
    g.N = B.N;
    g.P = B.P();
    g.r = B.r;
    g.n0 = B.n0;
    g.L = B.L;
    g.h = B.h;
    g.l1 = B.l1;
    g.nv = B.nv;
    g.kH = B.nH();
    g.kG = B.nG();
    g.ra = B.ra;
    return g;
}

bf_status ensure(void** p, size_t* have, size_t need)
{
    if (*have >= need && *p) return BF_OK;
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
        *have = 0;
    }
    BF_CUDA(cudaMalloc(p, need));
    *have = need;
    return BF_OK;
}

}  // namespace

namespace {

// Arena layout without a host image of the phase tables: small parts are kept
// for copying, tables only get their (aligned) place.
struct Layout {
    size_t size = 0;
    std::vector<std::pair<size_t, std::vector<unsigned char>>> parts;
    size_t add(const void* src, size_t n)
    {
        const size_t off = (size + 255) & ~(size_t)255;
        size = off + n;
        if (src && n)
            parts.emplace_back(off, std::vector<unsigned char>((const unsigned char*)src, (const unsigned char*)src + n));
        return off;
    }
    template <typename V>
    size_t addv(const V& v)
    {
        return add(v.data(), v.size() * sizeof(typename V::value_type));
    }
};

// tables = false: no place for the phase tables (their offsets are not used)
template <typename T, typename C>
Offs layout_block(Layout& lo, const BlockFactors& B, bool transposed, bool tables = true)
{
    Offs o;
    const int r = B.r;
    const int64_t N = B.N, P = tables ? B.P() : 0, ntab = tables ? (int64_t)1 << B.l1 : 0;
    o.a = lo.addv(cplx_as<C>(B.a));
    o.b = lo.addv(cplx_as<C>(B.b));
    o.Mv = lo.addv(real_as<T>(transposed ? transpose(B.Mv, r, B.nv) : B.Mv));
    o.EV = lo.add(nullptr, (size_t)(ntab * N) * sizeof(C));
    std::vector<double> mh;
    for (auto& M : B.MH) {
        auto t = transposed ? transpose(M, r, 2 * r) : M;
        mh.insert(mh.end(), t.begin(), t.end());
    }
    o.MH = lo.addv(real_as<T>(mh));
    o.EH = lo.add(nullptr, (size_t)(B.nH() * P * 2 * r) * sizeof(C));
    o.S = lo.add(nullptr, (size_t)(P * r * r) * sizeof(C));
    std::vector<double> mg;
    for (auto& M : B.MG)
        for (int pos = 0; pos < 2; ++pos) {
            std::vector<double> blk(M.begin() + (size_t)pos * r * r, M.begin() + (size_t)(pos + 1) * r * r);
            auto t = transposed ? transpose(blk, r, r) : blk;
            mg.insert(mg.end(), t.begin(), t.end());
        }
    o.MG = lo.addv(real_as<T>(mg));
    o.FG = lo.add(nullptr, (size_t)(B.nG() * P * 2 * r) * sizeof(C));
    o.MU = lo.addv(real_as<T>(B.MU));
    o.EU = lo.add(nullptr, (size_t)(ntab * N) * sizeof(C));
    return o;
}

}  // namespace

bf_status device_construct(bf_plan* p)
{
    if (p->dev) return BF_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        set_error("bf_factor_device: no CUDA device available");
        return BF_ERR_CUDA;
    }
    if (p->opt.device < 0 || p->opt.device >= ndev) {
        set_error("bf_factor_device: device %d not present (%d devices)", p->opt.device, ndev);
        return BF_ERR_ARG;
    }
    BF_CUDA(cudaSetDevice(p->opt.device));
    DeviceState* ds = new (std::nothrow) DeviceState();
    if (!ds) {
        set_error("bf_factor_device: out of host memory");
        return BF_ERR_NOMEM;
    }
    ds->device = p->opt.device;
    Layout l64, l32;
    std::vector<Offs> o64, o32;
    for (auto& B : p->blocks) {
        o64.push_back(layout_block<double, double2>(l64, B, false));
        o32.push_back(layout_block<float, float2>(l32, B, true));
    }
    auto fail = [&](bf_status st) {
        if (ds->arena64) cudaFree(ds->arena64);
        if (ds->arena32) cudaFree(ds->arena32);
        if (ds->err) cudaFree(ds->err);
        delete ds;
        return st;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&ds->arena64, l64.size)) != cudaSuccess || (e = cudaMalloc(&ds->arena32, l32.size)) != cudaSuccess ||
        (e = cudaMalloc((void**)&ds->err, sizeof(int))) != cudaSuccess || (e = cudaMemset(ds->err, 0, sizeof(int))) != cudaSuccess) {
        set_error("bf_factor_device: cudaMalloc: %s", cudaGetErrorString(e));
        return fail(e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA);
    }
    for (auto* lo : {&l64, &l32}) {
        unsigned char* base = (unsigned char*)(lo == &l64 ? ds->arena64 : ds->arena32);
        for (auto& pt : lo->parts)
            if ((e = cudaMemcpy(base + pt.first, pt.second.data(), pt.second.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess) {
                set_error("bf_factor_device: copy: %s", cudaGetErrorString(e));
                return fail(BF_ERR_CUDA);
            }
    }
    ds->bytes64 = l64.size;
    ds->bytes32 = l32.size;
    for (size_t i = 0; i < p->blocks.size(); ++i) {
        DevBlock db;
        db.g = geo_of(p->blocks[i]);
        db.row0 = p->blocks[i].row0;
        db.col0 = p->blocks[i].col0;
        bind(db.f64, (unsigned char*)ds->arena64, o64[i]);
        bind(db.f32, (unsigned char*)ds->arena32, o32[i]);
        e = construct_tables(p->blocks[i], p->kern.d.phase_kind, p->kern.d.phase_param, p->kern.n_global, db.f64,
                             db.f32, 0);
        if (e != cudaSuccess) {
            set_error("bf_factor_device: table kernels: %s", cudaGetErrorString(e));
            return fail(BF_ERR_CUDA);
        }
        ds->blocks.push_back(db);
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        set_error("bf_factor_device: %s", cudaGetErrorString(e));
        return fail(BF_ERR_CUDA);
    }
    p->dev = ds;
    return BF_OK;
}

namespace {

// frac(v) 2^64 mod 2^64 (exact while the lowest set bit of v is at least 2^-64)
uint64_t fixed64(double v)
{
    const double f = v - std::trunc(v);  // exact, |f| < 1
    const uint64_t m = (uint64_t)std::ldexp(std::fabs(f), 64);
    return f < 0 ? (uint64_t)0 - m : m;
}

}  // namespace

bf_status device_otf(bf_plan* p)
{
    if (p->dev) return BF_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        set_error("bf_factor_otf: no CUDA device available");
        return BF_ERR_CUDA;
    }
    if (p->opt.device < 0 || p->opt.device >= ndev) {
        set_error("bf_factor_otf: device %d not present (%d devices)", p->opt.device, ndev);
        return BF_ERR_ARG;
    }
    const int64_t Ng = p->kern.n_global;
    int lNg = 0;
    while (((int64_t)1 << lNg) < Ng) ++lNg;
    double kappa, rho;
    int xxi = 0, sq = 0;
    if (!p->kern.row_terms(0, &kappa, &rho, &xxi, &sq) || lNg < 1 || lNg > 30) {
        set_error("bf_factor_otf: phase kind %d / N=%lld has no on-the-fly form", p->kern.d.phase_kind,
                  (long long)Ng);
        return BF_ERR_UNSUPPORTED;
    }
    BF_CUDA(cudaSetDevice(p->opt.device));
    // per-row phase coefficients and the interpolation grids of every node size
    std::vector<uint4> rows;
    std::vector<int> grids;
    try {
        rows.resize((size_t)Ng);
        int lN = 0;  // log2 of the block size: node sizes 2^0 .. 2^lN
        while (!p->blocks.empty() && ((int64_t)1 << lN) < p->blocks[0].N) ++lN;
        grids.assign((size_t)(lN + 1) * 16, 0);
        for (int e = 0; e <= lN; ++e) {
            const std::vector<int64_t> gv = grid_rel((int64_t)1 << e, p->r);
            for (size_t t = 0; t < gv.size() && t < 16; ++t) grids[(size_t)e * 16 + t] = (int)gv[t];
        }
    } catch (const std::bad_alloc&) {
        set_error("bf_factor_otf: out of host memory");
        return BF_ERR_NOMEM;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < Ng; ++i) {
        double k, r;
        int a, b;
        p->kern.row_terms(i, &k, &r, &a, &b);
        const uint64_t K = fixed64(k);
        const uint32_t R = (uint32_t)((fixed64(r) + 0x80000000ull) >> 32);
        rows[(size_t)i] = make_uint4((unsigned)(K & 0xffffffffu), (unsigned)(K >> 32), R, 0u);
    }
    DeviceState* ds = new (std::nothrow) DeviceState();
    if (!ds) {
        set_error("bf_factor_otf: out of host memory");
        return BF_ERR_NOMEM;
    }
    ds->device = p->opt.device;
    ds->otf = true;
    Layout l32;
    std::vector<Offs> o32;
    for (auto& B : p->blocks) o32.push_back(layout_block<float, float2>(l32, B, true, false));
    const size_t rows_bytes = rows.size() * sizeof(uint4), grid_off = (rows_bytes + 255) & ~(size_t)255;
    auto fail = [&](bf_status st) {
        if (ds->arena32) cudaFree(ds->arena32);
        if (ds->otf_data) cudaFree(ds->otf_data);
        if (ds->err) cudaFree(ds->err);
        delete ds;
        return st;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&ds->arena32, l32.size)) != cudaSuccess ||
        (e = cudaMalloc(&ds->otf_data, grid_off + grids.size() * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void**)&ds->err, sizeof(int))) != cudaSuccess || (e = cudaMemset(ds->err, 0, sizeof(int))) != cudaSuccess) {
        set_error("bf_factor_otf: cudaMalloc: %s", cudaGetErrorString(e));
        return fail(e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA);
    }
    for (auto& pt : l32.parts)
        if ((e = cudaMemcpy((unsigned char*)ds->arena32 + pt.first, pt.second.data(), pt.second.size(),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            break;
    if (e == cudaSuccess) e = cudaMemcpy(ds->otf_data, rows.data(), rows_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy((unsigned char*)ds->otf_data + grid_off, grids.data(), grids.size() * sizeof(int),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_error("bf_factor_otf: copy: %s", cudaGetErrorString(e));
        return fail(BF_ERR_CUDA);
    }
    ds->bytes32 = l32.size + grid_off + grids.size() * sizeof(int);
    for (size_t i = 0; i < p->blocks.size(); ++i) {
        const BlockFactors& Bf = p->blocks[i];
        DevBlock db;
        db.g = geo_of(Bf);
        db.g.otf = 1;
        db.row0 = Bf.row0;
        db.col0 = Bf.col0;
        bind(db.f32, (unsigned char*)ds->arena32, o32[i]);
        db.f32.EV = db.f32.EH = db.f32.S = db.f32.FG = db.f32.EU = nullptr;
        db.ph.rows = (const uint4*)ds->otf_data;
        db.ph.grids = (const int*)((const unsigned char*)ds->otf_data + grid_off);
        db.ph.row0 = (int)Bf.row0;
        db.ph.col0 = (int)Bf.col0;
        db.ph.half = (int)(Ng / 2);
        int lN = 0;
        while (((int64_t)1 << lN) < Bf.N) ++lN;
        db.ph.lN = lN;
        db.ph.sh1 = xxi ? 32 - lNg : -1;
        db.ph.sh2 = sq ? 30 - lNg : -1;
        ds->blocks.push_back(db);
    }
    p->dev = ds;
    return BF_OK;
}

bf_status device_upload(bf_plan* p)
{
    if (p->dev) return BF_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        set_error("bf_upload: no CUDA device available");
        return BF_ERR_CUDA;
    }
    if (p->opt.device < 0 || p->opt.device >= ndev) {
        set_error("bf_upload: device %d not present (%d devices)", p->opt.device, ndev);
        return BF_ERR_ARG;
    }
    BF_CUDA(cudaSetDevice(p->opt.device));
    DeviceState* ds = new (std::nothrow) DeviceState();
    if (!ds) {
        set_error("bf_upload: out of host memory");
        return BF_ERR_NOMEM;
    }
    ds->device = p->opt.device;
    Packer pk64, pk32;
    std::vector<Offs> o64, o32;
    try {
        for (auto& B : p->blocks) {
            o64.push_back(pack_block<double, double2>(pk64, B, false));
            o32.push_back(pack_block<float, float2>(pk32, B, true));
        }
    } catch (const std::bad_alloc&) {
        delete ds;
        set_error("bf_upload: out of host memory while packing");
        return BF_ERR_NOMEM;
    }
    auto fail = [&](bf_status st) {
        if (ds->arena64) cudaFree(ds->arena64);
        if (ds->arena32) cudaFree(ds->arena32);
        if (ds->err) cudaFree(ds->err);
        delete ds;
        return st;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&ds->arena64, pk64.buf.size())) != cudaSuccess ||
        (e = cudaMalloc(&ds->arena32, pk32.buf.size())) != cudaSuccess ||
        (e = cudaMalloc((void**)&ds->err, sizeof(int))) != cudaSuccess) {
        set_error("bf_upload: cudaMalloc: %s", cudaGetErrorString(e));
        return fail(e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA);
    }
    if ((e = cudaMemcpy(ds->arena64, pk64.buf.data(), pk64.buf.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ds->arena32, pk32.buf.data(), pk32.buf.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(ds->err, 0, sizeof(int))) != cudaSuccess) {
        set_error("bf_upload: copy: %s", cudaGetErrorString(e));
        return fail(BF_ERR_CUDA);
    }
    ds->bytes64 = pk64.buf.size();
    ds->bytes32 = pk32.buf.size();
    for (size_t i = 0; i < p->blocks.size(); ++i) {
        DevBlock db;
        db.g = geo_of(p->blocks[i]);
        db.row0 = p->blocks[i].row0;
        db.col0 = p->blocks[i].col0;
        bind(db.f64, (unsigned char*)ds->arena64, o64[i]);
        bind(db.f32, (unsigned char*)ds->arena32, o32[i]);
        ds->blocks.push_back(db);
    }
    p->dev = ds;
    if (!p->opt.keep_host) {
        for (auto& B : p->blocks) {
            BlockFactors slim;
            slim.N = B.N; slim.row0 = B.row0; slim.col0 = B.col0; slim.r = B.r; slim.n0 = B.n0;
            slim.L = B.L; slim.h = B.h; slim.l1 = B.l1; slim.nv = B.nv; slim.ra = B.ra;
            slim.amp_sigma_ratio = B.amp_sigma_ratio;
            B = std::move(slim);
        }
    }
    return BF_OK;
}

bf_status device_reserve(bf_plan* p, bf_precision prec, int64_t m, void*)
{
    DeviceState* ds = p->dev;
    if (ds->otf && prec != BF_PREC_F32) {
        set_error("plan factored by bf_factor_otf: only BF_PREC_F32 applies (no phase tables)");
        return BF_ERR_UNSUPPORTED;
    }
    BF_CUDA(cudaSetDevice(ds->device));
    size_t need = 0;
    for (auto& B : ds->blocks) {
        if (prec == BF_PREC_F64) need = std::max(need, 2 * plain_f64_ws_bytes(B.g, m));
        else if (prec == BF_PREC_BF16X3) need = std::max(need, tc_ws_bytes(B.g, m));
        else need = std::max(need, fused_f32_ws_bytes(B.g, m, p->mr_hint(m)));
    }
    if (need == 0) need = 256;
    if (prec == BF_PREC_F64) return ensure(&ds->ws64, &ds->ws64_bytes, need);
    return ensure(&ds->ws32, &ds->ws32_bytes, need);
}

namespace {

// The plain FP64 form launches one kernel per stage; at small N the launches
// dominate, so the sequence is captured once per (F, G, m, workspace) into a
// CUDA graph and replayed.  Skipped (direct launches) while the caller's
// stream is itself being captured.
bf_status apply_f64(bf_plan* p, const void* F, int64_t m, void* G, cudaStream_t st)
{
    DeviceState* ds = p->dev;
    const int sp = p->opt.split;
    auto launch_all = [&](cudaStream_t s) {
        for (size_t i = 0; i < ds->blocks.size(); ++i) {
            const DevBlock& B = ds->blocks[i];
            const int beta = (sp == 2 && (i % 2) == 1) ? 1 : 0;  // second column half accumulates
            const size_t half = ds->ws64_bytes / 2 / sizeof(double2);
            cudaError_t e = launch_plain_f64(B, (const double2*)F + B.col0 * m, m, (double2*)G + B.row0 * m, beta,
                                             (double2*)ds->ws64, (double2*)ds->ws64 + half, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        const cudaError_t e = launch_all(st);
        if (e != cudaSuccess) {
            set_error("bf_apply: kernel launch failed: %s", cudaGetErrorString(e));
            return BF_ERR_CUDA;
        }
        return BF_OK;
    }
    const bool hit = ds->g64 && ds->g64_F == F && ds->g64_G == G && ds->g64_m == m && ds->g64_ws == ds->ws64;
    if (!hit) {
        if (ds->g64) {
            cudaGraphExecDestroy(ds->g64);
            ds->g64 = nullptr;
        }
        if (!ds->cap) BF_CUDA(cudaStreamCreateWithFlags(&ds->cap, cudaStreamNonBlocking));
        prof_suppress(true);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(ds->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t el = launch_all(ds->cap);
            e = cudaStreamEndCapture(ds->cap, &g);
            if (e == cudaSuccess) e = el;
        }
        prof_suppress(false);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ds->g64, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ds->g64 = nullptr;
            cudaGetLastError();
            const cudaError_t e2 = launch_all(st);  // fall back to direct launches
            if (e2 != cudaSuccess) {
                set_error("bf_apply: kernel launch failed: %s", cudaGetErrorString(e2));
                return BF_ERR_CUDA;
            }
            return BF_OK;
        }
        ds->g64_F = F;
        ds->g64_G = G;
        ds->g64_m = m;
        ds->g64_ws = ds->ws64;
    }
    ProfScope ps("plain_f64_graph", st);
    const cudaError_t e = cudaGraphLaunch(ds->g64, st);
    if (e != cudaSuccess) {
        set_error("bf_apply: graph launch failed: %s", cudaGetErrorString(e));
        return BF_ERR_CUDA;
    }
    return BF_OK;
}

}  // namespace

bf_status device_apply(bf_plan* p, bf_precision prec, const void* F, int64_t m, void* G, void* stream)
{
    DeviceState* ds = p->dev;
    cudaStream_t st = (cudaStream_t)stream;
    if (ds->otf && prec != BF_PREC_F32) {
        set_error("bf_apply: plan factored by bf_factor_otf: only BF_PREC_F32 applies (no phase tables)");
        return BF_ERR_UNSUPPORTED;
    }
    if (prec == BF_PREC_BF16X3) {
        for (auto& B : ds->blocks) {
            const char* why = "";
            if (!tc_supported(B.g, &why)) {
                set_error("bf_apply: BF_PREC_BF16X3: %s (r=%d, kH=%d, kG=%d)", why, B.g.r, B.g.kH, B.g.kG);
                return BF_ERR_UNSUPPORTED;
            }
        }
    }
    if (prec == BF_PREC_F32) {
        for (auto& B : ds->blocks)
            if (!fused_f32_supported(B.g.r) || B.g.nv > 2 * B.g.r) {
                set_error("bf_apply: no fused FP32 kernels for r=%d, nv=%d", B.g.r, B.g.nv);
                return BF_ERR_UNSUPPORTED;
            }
    }
    bf_status rs = device_reserve(p, prec, m, stream);
    if (rs != BF_OK) return rs;
    if (prec == BF_PREC_F64) return apply_f64(p, F, m, G, st);
    const int sp = p->opt.split;
    for (size_t i = 0; i < ds->blocks.size(); ++i) {
        const DevBlock& B = ds->blocks[i];
        const int beta = (sp == 2 && (i % 2) == 1) ? 1 : 0;  // second column half accumulates
        cudaError_t e;
        if (prec == BF_PREC_F64) {
            const double2* Fb = (const double2*)F + B.col0 * m;
            double2* Gb = (double2*)G + B.row0 * m;
            const size_t half = ds->ws64_bytes / 2 / sizeof(double2);
            e = launch_plain_f64(B, Fb, m, Gb, beta, (double2*)ds->ws64, (double2*)ds->ws64 + half, st);
        } else if (prec == BF_PREC_BF16X3) {
            e = launch_tc(B, (const float2*)F + B.col0 * m, m, (float2*)G + B.row0 * m, beta, (float2*)ds->ws32,
                          ds->err, st);
        } else {
            const float2* Fb = (const float2*)F + B.col0 * m;
            float2* Gb = (float2*)G + B.row0 * m;
            e = launch_fused_f32(B, Fb, m, Gb, beta, (float2*)ds->ws32, st, p->mr_hint(m));
        }
        if (e != cudaSuccess) {
            set_error("bf_apply: kernel launch failed: %s", cudaGetErrorString(e));
            return BF_ERR_CUDA;
        }
    }
    return BF_OK;
}

size_t device_ws_bytes(const bf_plan* p, bf_precision prec, int64_t m)
{
    size_t need = 0;
    for (auto& B : p->dev->blocks) {
        if (prec == BF_PREC_F64) need = std::max(need, 2 * plain_f64_ws_bytes(B.g, m));
        else if (prec == BF_PREC_BF16X3) need = std::max(need, tc_ws_bytes(B.g, m));
        else need = std::max(need, fused_f32_ws_bytes(B.g, m, p->mr_hint(m)));
    }
    return need == 0 ? 256 : need;
}

bf_status device_apply_ws(bf_plan* p, bf_precision prec, const void* F, int64_t m, void* G, void* stream, void* ws,
                          size_t ws_bytes)
{
    DeviceState* ds = p->dev;
    cudaStream_t st = (cudaStream_t)stream;
    if (ds->otf && prec != BF_PREC_F32) {
        set_error("plan factored by bf_factor_otf: only BF_PREC_F32 applies (no phase tables)");
        return BF_ERR_UNSUPPORTED;
    }
    if (prec == BF_PREC_BF16X3) {
        for (auto& B : ds->blocks) {
            const char* why = "";
            if (!tc_supported(B.g, &why)) {
                set_error("BF_PREC_BF16X3: %s", why);
                return BF_ERR_UNSUPPORTED;
            }
        }
    }
    if (ws_bytes < device_ws_bytes(p, prec, m)) {
        set_error("workspace of %zu bytes too small (%zu needed)", ws_bytes, device_ws_bytes(p, prec, m));
        return BF_ERR_ARG;
    }
    const int sp = p->opt.split;
    for (size_t i = 0; i < ds->blocks.size(); ++i) {
        const DevBlock& B = ds->blocks[i];
        const int beta = (sp == 2 && (i % 2) == 1) ? 1 : 0;
        cudaError_t e;
        if (prec == BF_PREC_F64) {
            const size_t half = ws_bytes / 2 / sizeof(double2);
            e = launch_plain_f64(B, (const double2*)F + B.col0 * m, m, (double2*)G + B.row0 * m, beta, (double2*)ws,
                                 (double2*)ws + half, st);
        } else if (prec == BF_PREC_BF16X3) {
            e = launch_tc(B, (const float2*)F + B.col0 * m, m, (float2*)G + B.row0 * m, beta, (float2*)ws, ds->err, st);
        } else {
            e = launch_fused_f32(B, (const float2*)F + B.col0 * m, m, (float2*)G + B.row0 * m, beta, (float2*)ws, st,
                                 p->mr_hint(m));
        }
        if (e != cudaSuccess) {
            set_error("kernel launch failed: %s", cudaGetErrorString(e));
            return BF_ERR_CUDA;
        }
    }
    return BF_OK;
}

// FP32 apply of a one-sub-BF plan from host buffers in kHostChunks row ranges: the F rows of
// range k are copied on ds->copy while the front runs on the ranges before it; the G rows of
// range k are copied back while the back runs on the ranges after it.  Consecutive ranges
// alternate between st and ds->comp2.  The kernels and their arithmetic are those of bf_apply.
static bf_status apply_host_pipelined(bf_plan* p, const void* F, int64_t m, void* G, cudaStream_t st,
                                      unsigned char* dF, unsigned char* dG)
{
    DeviceState* ds = p->dev;
    constexpr int nch = DeviceState::kHostChunks;
    if (!ds->copy) BF_CUDA(cudaStreamCreateWithFlags(&ds->copy, cudaStreamNonBlocking));
    if (!ds->comp2) BF_CUDA(cudaStreamCreateWithFlags(&ds->comp2, cudaStreamNonBlocking));
    for (auto& ev : ds->hev)
        if (!ev) BF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEvent_t* fready = ds->hev;
    cudaEvent_t* gdone = ds->hev + nch;
    cudaEvent_t ev_in = ds->hev[2 * nch], ev_out = ds->hev[2 * nch + 1];
    const cudaEvent_t* join = ds->hev + 2 * nch + 2;
    const size_t rows = (size_t)p->N / nch, bytes = rows * (size_t)m * sizeof(float2);
    // the copies start after the caller's earlier work on st (it may still use the staging buffers)
    BF_CUDA(cudaEventRecord(ev_in, st));
    BF_CUDA(cudaStreamWaitEvent(ds->copy, ev_in, 0));
    for (int k = 0; k < nch; ++k) {
        BF_CUDA(cudaMemcpyAsync(dF + k * bytes, (const unsigned char*)F + k * bytes, bytes, cudaMemcpyHostToDevice,
                                ds->copy));
        BF_CUDA(cudaEventRecord(fready[k], ds->copy));
    }
    bf_status rs = device_reserve(p, BF_PREC_F32, m, st);
    if (rs != BF_OK) return rs;
    const cudaError_t e = launch_fused_f32_chunked(ds->blocks[0], (const float2*)dF, m, (float2*)dG,
                                                   (float2*)ds->ws32, st, ds->comp2, p->mr_hint(m), nch, fready,
                                                   gdone, join);
    if (e != cudaSuccess) {
        set_error("bf_apply_host: kernel launch failed: %s", cudaGetErrorString(e));
        return BF_ERR_CUDA;
    }
    for (int k = 0; k < nch; ++k) {
        BF_CUDA(cudaStreamWaitEvent(ds->copy, gdone[k], 0));
        BF_CUDA(cudaMemcpyAsync((unsigned char*)G + k * bytes, dG + k * bytes, bytes, cudaMemcpyDeviceToHost,
                                ds->copy));
    }
    BF_CUDA(cudaEventRecord(ev_out, ds->copy));
    BF_CUDA(cudaStreamWaitEvent(st, ev_out, 0));
    BF_CUDA(cudaStreamSynchronize(st));
    return BF_OK;
}

bf_status device_apply_host(bf_plan* p, bf_precision prec, const void* F, int64_t m, void* G, void* stream)
{
    DeviceState* ds = p->dev;
    cudaStream_t st = (cudaStream_t)stream;
    BF_CUDA(cudaSetDevice(ds->device));
    const size_t elt = prec == BF_PREC_F64 ? sizeof(double2) : sizeof(float2);
    const size_t nb = (size_t)p->N * m * elt;
    bf_status s = ensure(&ds->stage, &ds->stage_bytes, 2 * nb);
    if (s != BF_OK) return s;
    unsigned char* dF = (unsigned char*)ds->stage;
    unsigned char* dG = dF + nb;
    if (prec == BF_PREC_F32 && ds->blocks.size() == 1 && fused_f32_supported(ds->blocks[0].g.r) &&
        ds->blocks[0].g.nv <= 2 * ds->blocks[0].g.r &&
        fused_f32_chunkable(ds->blocks[0], m, p->mr_hint(m), DeviceState::kHostChunks))
        return apply_host_pipelined(p, F, m, G, st, dF, dG);
    BF_CUDA(cudaMemcpyAsync(dF, F, nb, cudaMemcpyHostToDevice, st));
    s = device_apply(p, prec, dF, m, dG, stream);
    if (s != BF_OK) return s;
    BF_CUDA(cudaMemcpyAsync(G, dG, nb, cudaMemcpyDeviceToHost, st));
    BF_CUDA(cudaStreamSynchronize(st));
    return BF_OK;
}

bf_status device_sync_status(bf_plan* p, void* stream)
{
    DeviceState* ds = p->dev;
    BF_CUDA(cudaSetDevice(ds->device));
    BF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int h = 0;
    BF_CUDA(cudaMemcpy(&h, ds->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) {
        set_error("device-side wait ran out (code %d)", h);
        cudaMemset(ds->err, 0, sizeof(int));
        return BF_ERR_TIMEOUT;
    }
    return BF_OK;
}

void device_free(bf_plan* p)
{
    DeviceState* ds = p->dev;
    if (!ds) return;
    cudaSetDevice(ds->device);
    cudaFree(ds->arena64);
    cudaFree(ds->arena32);
    if (ds->g64) cudaGraphExecDestroy(ds->g64);
    if (ds->cap) cudaStreamDestroy(ds->cap);
    cudaFree(ds->ws64);
    cudaFree(ds->ws32);
    cudaFree(ds->stage);
    if (ds->copy) cudaStreamDestroy(ds->copy);
    if (ds->comp2) cudaStreamDestroy(ds->comp2);
    for (auto& ev : ds->hev)
        if (ev) cudaEventDestroy(ev);
    cudaFree(ds->otf_data);
    cudaFree(ds->err);
    delete ds;
    p->dev = nullptr;
}

void device_info(const bf_plan* p, bf_plan_info* info)
{
    if (!p->dev) return;
    info->uploaded = 1;
    info->dev_bytes_f64 = (int64_t)p->dev->bytes64;
    info->dev_bytes_f32 = (int64_t)p->dev->bytes32;
}

}  // namespace bfi
