// FP32 kernels.  Variants (id, pipeline, radial sites per CTA, ring depth,
// re-read f from shared memory, min CTAs per SM):
//   1  v1  128  6  no   2   CTA-wide barrier per row (111 KB shared)
//   2  v2  128  6  no   2   producer warp + full/empty mbarriers (111 KB)
//   3  v2  128  4  yes  3   as 2 with a 4-deep ring (74 KB) and <= 136 registers
//   4  v3  128  6  no   2   as 2, rows loaded by tensor-map TMA (3 copies per row)
//   5  v3  128  4  yes  3   as 3, rows loaded by tensor-map TMA
#include "dbm.h"
#define DBM_REAL float
#define DBM_VARIANTS(X) X(1, 1, 128, 6, false, 2) X(2, 2, 128, 6, false, 2) X(3, 2, 128, 4, true, 3) \
    X(4, 3, 128, 6, false, 2) X(5, 3, 128, 4, true, 3)
#define DBM_DEFAULT_VARIANT 4
#define DBM_FALLBACK_VARIANT 2
#define DBM_BATCH_CONST_SLOTS DBM_BATCH_CONST_FP32  // batch constant table entries (160 B each)
#include "dbm_launch_impl.cuh"

namespace dbm {
cudaError_t launch_totals(const double *partials, int nblocks, double *totals, cudaStream_t s)
{
    totals_kernel<<<1, 256, 0, s>>>(partials, nblocks, totals);
    return cudaGetLastError();
}

cudaError_t launch_rcp_selftest(const float *x, float *approx, float *ieee, int n, cudaStream_t s)
{
    rcp_selftest_kernel<<<256, 256, 0, s>>>(x, approx, ieee, n);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int *status, int arrive, long long limit, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 64, 0, s>>>(status, arrive, limit);
    return cudaGetLastError();
}

cudaError_t launch_batch_advance(long long *T, int k, cudaStream_t s)
{
    batch_advance_kernel<<<1, 32, 0, s>>>(T, k);
    return cudaGetLastError();
}
}  // namespace dbm
