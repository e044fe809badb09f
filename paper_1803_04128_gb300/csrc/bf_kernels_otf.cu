// Fused FP32 apply with the phases evaluated inside the kernels (Geo::otf):
// the tile bodies of bf_f32_tile.h instantiated with OTF = true.  The device
// then holds only O(N) data per operator (amplitude split, per-row phase
// coefficients, the shared Lagrange matrices) instead of the O(r N log N)
// phase tables.
#include "bf_f32_tile.h"

namespace bfi {
namespace {

template <int R, int NV>
__global__ void __launch_bounds__(kThreads, 2) front_f32_otf(FrontArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    front_tile<R, NV, true>(A, blockIdx.x, smem_raw);
}

template <int R, int NU>
__global__ void __launch_bounds__(kThreads, 2) back_f32_otf(BackArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    back_tile<R, NU, true>(A, blockIdx.x, smem_raw);
}

template <int R>
cudaError_t launch_otf_r(const FrontArgs* fa, const BackArgs* ba, size_t smem, int64_t nblocks, cudaStream_t st)
{
    constexpr int NV = nv_of<R>();
    cudaError_t e;
    if (fa) {
        if ((e = cudaFuncSetAttribute(front_f32_otf<R, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        ProfScope ps("front_f32_otf", st);
        front_f32_otf<R, NV><<<(unsigned)nblocks, kThreads, smem, st>>>(*fa);
    } else {
        if ((e = cudaFuncSetAttribute(back_f32_otf<R, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        ProfScope ps("back_f32_otf", st);
        back_f32_otf<R, NV><<<(unsigned)nblocks, kThreads, smem, st>>>(*ba);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_part_otf(int r, const FrontArgs* fa, const BackArgs* ba, size_t smem, int64_t nblocks,
                            cudaStream_t st)
{
    if (nblocks < 1) return cudaSuccess;
    switch (r) {
    case 6: return launch_otf_r<6>(fa, ba, smem, nblocks, st);
    case 8: return launch_otf_r<8>(fa, ba, smem, nblocks, st);
    case 10: return launch_otf_r<10>(fa, ba, smem, nblocks, st);
    case 12: return launch_otf_r<12>(fa, ba, smem, nblocks, st);
    case 14: return launch_otf_r<14>(fa, ba, smem, nblocks, st);
    case 16: return launch_otf_r<16>(fa, ba, smem, nblocks, st);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace bfi
