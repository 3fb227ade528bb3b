// Instantiates the kernels of one precision; included once per precision
// translation unit with DBM_REAL, DBM_W and DBM_NSTAGE defined.
#include "dbm_launch.h"

namespace dbm {

namespace {
constexpr int kW = DBM_W;
constexpr int kNS = DBM_NSTAGE;
constexpr int kHalo = Halo<DBM_REAL>::value;
constexpr int kSmem = (int)(sizeof(DBM_REAL) * kNS * NARR * (kW + 2 * kHalo) + 8 * kNS);
}  // namespace

template <>
cudaError_t kernel_info<DBM_REAL>(KernelInfo *out)
{
    auto kern = step_kernel<DBM_REAL, kW, kNS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kW, kSmem);
    if (e != cudaSuccess) return e;
    out->W = kW;
    out->nstage = kNS;
    out->halo = kHalo;
    out->smem = kSmem;
    out->blocks_per_sm = nb;
    return cudaSuccess;
}

template <>
cudaError_t launch_step<DBM_REAL>(const StepArgs<DBM_REAL> &A, int grid, cudaStream_t s)
{
    step_kernel<DBM_REAL, kW, kNS><<<grid, kW, kSmem, s>>>(A);
    return cudaGetLastError();
}

template <>
cudaError_t batch_kernel_info<DBM_REAL>(KernelInfo *out)
{
    auto kern = batch_step_kernel<DBM_REAL, kW, kNS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kW, kSmem);
    if (e != cudaSuccess) return e;
    out->W = kW;
    out->nstage = kNS;
    out->halo = kHalo;
    out->smem = kSmem;
    out->blocks_per_sm = nb;
    return cudaSuccess;
}

template <>
cudaError_t launch_batch_step<DBM_REAL>(const BatchArgs<DBM_REAL> &B, int grid, cudaStream_t s)
{
    batch_step_kernel<DBM_REAL, kW, kNS><<<grid, kW, kSmem, s>>>(B);
    return cudaGetLastError();
}

template <>
cudaError_t launch_init<DBM_REAL>(const InitArgs<DBM_REAL> &A, cudaStream_t s)
{
    const long long n = (long long)A.nr * A.ntheta;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    init_kernel<DBM_REAL><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <>
cudaError_t launch_moments<DBM_REAL>(const MomArgs<DBM_REAL> &A, int grid, cudaStream_t s)
{
    moments_kernel<DBM_REAL><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace dbm
