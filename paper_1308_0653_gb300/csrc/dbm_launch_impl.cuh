// Instantiates the kernels of one precision; included once per precision
// translation unit with DBM_REAL and the variant list DBM_VARIANTS(X) defined,
// X(id, version, W, NSTAGE, REREAD, MIN_BLOCKS_PER_SM), DBM_DEFAULT_VARIANT and
// DBM_FALLBACK_VARIANT (the default when tensor maps are unavailable).
// version 1: CTA-wide row barrier; 2: producer warp, per-array bulk copies;
// 3: producer warp, tensor-map TMA tiles.
#include "dbm_launch.h"

namespace dbm {

// Per-slot constants of the batched launches of this precision: entries are
// handed out to batches in contiguous ranges by the runtime and written with
// stream-ordered copies when a batch commits its slot table.
__constant__ StepConsts<DBM_REAL> c_batch_consts[DBM_BATCH_CONST_SLOTS];

template <>
__device__ __forceinline__ const StepConsts<DBM_REAL> &batch_consts<DBM_REAL>(int i)
{
    return c_batch_consts[i];
}

template <> int batch_const_capacity<DBM_REAL>() { return DBM_BATCH_CONST_SLOTS; }

template <>
cudaError_t upload_batch_consts<DBM_REAL>(int first, const StepConsts<DBM_REAL> *src, int n, cudaStream_t s)
{
    if (first < 0 || n < 0 || first + n > DBM_BATCH_CONST_SLOTS) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    return cudaMemcpyToSymbolAsync(c_batch_consts, src, sizeof(StepConsts<DBM_REAL>) * (size_t)n,
                                   sizeof(StepConsts<DBM_REAL>) * (size_t)first, cudaMemcpyHostToDevice, s);
}

namespace {

template <int VER, int W, int NS, bool RR, int MB> struct Variant;

template <int W, int NS, bool RR, int MB>
struct Variant<1, W, NS, RR, MB> {
    static constexpr int kThreads = W;
    static constexpr int kSmem =
        (int)(sizeof(DBM_REAL) * NS * NARR * (W + 2 * Halo<DBM_REAL>::value) + 8 * NS);
    static void *single() { return (void *)step_kernel<DBM_REAL, W, NS>; }
    static void *batch() { return (void *)batch_step_kernel<DBM_REAL, W, NS>; }
    static cudaError_t run(const StepArgs<DBM_REAL> &A, int g, cudaStream_t s)
    {
        step_kernel<DBM_REAL, W, NS><<<g, kThreads, kSmem, s>>>(A);
        return cudaGetLastError();
    }
    static cudaError_t run_batch(const BatchArgs<DBM_REAL> &B, int g, cudaStream_t s)
    {
        batch_step_kernel<DBM_REAL, W, NS><<<g, kThreads, kSmem, s>>>(B);
        return cudaGetLastError();
    }
};

template <int W, int NS, bool RR, int MB, bool TM>
struct VariantV2 {
    static constexpr int kThreads = W + 32;
    static constexpr int kSmem = smem_bytes_v2<DBM_REAL, W, NS>();
    static void *single() { return (void *)step_kernel_v2<DBM_REAL, W, NS, RR, MB, TM>; }
    static void *batch() { return (void *)batch_step_kernel_v2<DBM_REAL, W, NS, RR, MB, TM>; }
    static cudaError_t run(const StepArgs<DBM_REAL> &A, int g, cudaStream_t s)
    {
        step_kernel_v2<DBM_REAL, W, NS, RR, MB, TM><<<g, kThreads, kSmem, s>>>(A);
        return cudaGetLastError();
    }
    static cudaError_t run_batch(const BatchArgs<DBM_REAL> &B, int g, cudaStream_t s)
    {
        batch_step_kernel_v2<DBM_REAL, W, NS, RR, MB, TM><<<g, kThreads, kSmem, s>>>(B);
        return cudaGetLastError();
    }
};

template <int W, int NS, bool RR, int MB>
struct Variant<2, W, NS, RR, MB> : VariantV2<W, NS, RR, MB, false> {};

template <int W, int NS, bool RR, int MB>
struct Variant<3, W, NS, RR, MB> : VariantV2<W, NS, RR, MB, true> {};

template <typename V>
cudaError_t info_of(void *fn, int ver, int W, int NS, KernelInfo *out)
{
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, V::kSmem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, V::kThreads, V::kSmem);
    if (e != cudaSuccess) return e;
    out->W = W;
    out->threads = V::kThreads;
    out->nstage = NS;
    out->halo = Halo<DBM_REAL>::value;
    out->smem = V::kSmem;
    out->blocks_per_sm = nb;
    out->version = ver;
    return cudaSuccess;
}

}  // namespace

template <> int num_variants<DBM_REAL>()
{
    int n = 0;
#define X(id, ver, W, NS, RR, MB) n = n > id ? n : id;
    DBM_VARIANTS(X)
#undef X
    return n;
}

template <> int default_variant<DBM_REAL>() { return DBM_DEFAULT_VARIANT; }
template <> int fallback_variant<DBM_REAL>() { return DBM_FALLBACK_VARIANT; }

template <>
cudaError_t kernel_info<DBM_REAL>(int variant, KernelInfo *out)
{
    switch (variant) {
#define X(id, ver, W, NS, RR, MB) \
    case id: return info_of<Variant<ver, W, NS, RR, MB>>(Variant<ver, W, NS, RR, MB>::single(), ver, W, NS, out);
        DBM_VARIANTS(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t batch_kernel_info<DBM_REAL>(int variant, KernelInfo *out)
{
    switch (variant) {
#define X(id, ver, W, NS, RR, MB) \
    case id: return info_of<Variant<ver, W, NS, RR, MB>>(Variant<ver, W, NS, RR, MB>::batch(), ver, W, NS, out);
        DBM_VARIANTS(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_step<DBM_REAL>(int variant, const StepArgs<DBM_REAL> &A, int grid, cudaStream_t s)
{
    switch (variant) {
#define X(id, ver, W, NS, RR, MB) \
    case id: return Variant<ver, W, NS, RR, MB>::run(A, grid, s);
        DBM_VARIANTS(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_batch_step<DBM_REAL>(int variant, const BatchArgs<DBM_REAL> &B, int grid, cudaStream_t s)
{
    switch (variant) {
#define X(id, ver, W, NS, RR, MB) \
    case id: return Variant<ver, W, NS, RR, MB>::run_batch(B, grid, s);
        DBM_VARIANTS(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_init<DBM_REAL>(const InitArgs<DBM_REAL> &A, cudaStream_t s)
{
    const long long n = (long long)A.nr * (A.m1 - A.m0);
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    if (n <= 0) return cudaSuccess;
    init_kernel<DBM_REAL><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <>
cudaError_t launch_moments<DBM_REAL>(const MomArgs<DBM_REAL> &A, int grid, cudaStream_t s)
{
    moments_kernel<DBM_REAL><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <>
cudaError_t launch_noneq<DBM_REAL>(const MomArgs<DBM_REAL> &A, int grid, cudaStream_t s)
{
    noneq_kernel<DBM_REAL><<<grid, 256, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace dbm
