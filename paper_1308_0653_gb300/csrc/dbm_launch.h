// Host-side launch interface between the C-ABI runtime and the kernels of one
// precision (each precision is its own translation unit, built in parallel).
#pragma once

#include <cuda_runtime.h>

#include "dbm_device.cuh"

namespace dbm {

struct KernelInfo {
    int W;             // radial sites per CTA
    int threads;       // threads per CTA (W, plus a producer warp in v2)
    int nstage;        // row buffers in the shared-memory ring
    int halo;          // halo columns per side (16 bytes)
    int smem;          // dynamic shared memory per CTA (bytes)
    int blocks_per_sm; // resident CTAs per SM
    int version;       // 1: CTA-wide row barrier, 2: producer warp + full/empty barriers,
                       // 3: as 2 with rows loaded by tensor-map TMA
};

constexpr int MAX_VARIANTS = 8;

// Kernel variants of one precision are numbered 1..num_variants<real>().
template <typename real> int num_variants();
template <typename real> int default_variant();
// The default when tensor maps cannot be used (a variant with version < 3).
template <typename real> int fallback_variant();
template <typename real> cudaError_t kernel_info(int variant, KernelInfo *out);
template <typename real> cudaError_t launch_step(int variant, const StepArgs<real> &A, int grid, cudaStream_t s);
template <typename real> cudaError_t batch_kernel_info(int variant, KernelInfo *out);
template <typename real>
cudaError_t launch_batch_step(int variant, const BatchArgs<real> &B, int grid, cudaStream_t s);
cudaError_t launch_batch_advance(long long *T, int k, cudaStream_t s);
// Entries of the batch constant table of a precision, and a stream-ordered
// write of n entries from host memory (pinned for an asynchronous copy).
template <typename real> int batch_const_capacity();
template <typename real>
cudaError_t upload_batch_consts(int first, const StepConsts<real> *src, int n, cudaStream_t s);
template <typename real> cudaError_t launch_init(const InitArgs<real> &A, cudaStream_t s);
template <typename real> cudaError_t launch_moments(const MomArgs<real> &A, int grid, cudaStream_t s);
template <typename real> cudaError_t launch_noneq(const MomArgs<real> &A, int grid, cudaStream_t s);
cudaError_t launch_totals(const double *partials, int nblocks, double *totals, cudaStream_t s);
cudaError_t launch_rcp_selftest(const float *x, float *approx, float *ieee, int n, cudaStream_t s);
cudaError_t launch_wait_selftest(int *status, int arrive, long long limit, cudaStream_t s);

constexpr int MOMENT_BLOCKS = 1024;  // partial-sum slots of the totals reduction

// Record a failed CUDA call as this thread's last error (dbm_last_error) and
// return DBM_ECUDA (defined by the C-ABI runtime).
int record_cuda_failure(cudaError_t e, const char *what);

}  // namespace dbm
