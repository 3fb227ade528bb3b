// FP32 kernels: 128 radial sites per CTA, 6-deep row ring (111 KB shared).
#define DBM_REAL float
#define DBM_W 128
#define DBM_NSTAGE 6
#include "dbm_launch_impl.cuh"

namespace dbm {
cudaError_t launch_totals(const double *partials, int nblocks, double *totals, cudaStream_t s)
{
    totals_kernel<<<1, 256, 0, s>>>(partials, nblocks, totals);
    return cudaGetLastError();
}

cudaError_t launch_batch_advance(long long *T, int k, cudaStream_t s)
{
    batch_advance_kernel<<<1, 32, 0, s>>>(T, k);
    return cudaGetLastError();
}
}  // namespace dbm
