// Middle passes of a split level range (mid_tile of bf_f32_tile.h) with the phases
// evaluated in the kernel (plans factored by bf_factor_otf).
#include "bf_f32_tile.h"

namespace bfi {
namespace {

template <int R, int GK>
__global__ void __launch_bounds__(kThreads, 2) mid_f32_otf(MidArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    mid_tile<R, GK, true>(A, blockIdx.x, smem_raw);
}

template <int R>
cudaError_t launch_mid_otf_r(const MidArgs& ma, size_t smem, int64_t nblocks, cudaStream_t st)
{
    auto kern = ma.gkind ? mid_f32_otf<R, 1> : mid_f32_otf<R, 0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ProfScope ps(ma.gkind ? "mid_g_f32_otf" : "mid_h_f32_otf", st);
    kern<<<(unsigned)nblocks, kThreads, smem, st>>>(ma);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mid_otf(int r, const MidArgs& ma, size_t smem, int64_t nblocks, cudaStream_t st)
{
    if (nblocks < 1) return cudaSuccess;
    switch (r) {
    case 6: return launch_mid_otf_r<6>(ma, smem, nblocks, st);
    case 8: return launch_mid_otf_r<8>(ma, smem, nblocks, st);
    case 10: return launch_mid_otf_r<10>(ma, smem, nblocks, st);
    case 12: return launch_mid_otf_r<12>(ma, smem, nblocks, st);
    case 14: return launch_mid_otf_r<14>(ma, smem, nblocks, st);
    case 16: return launch_mid_otf_r<16>(ma, smem, nblocks, st);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace bfi
