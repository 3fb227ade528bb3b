// Conservation totals of a state with no memory allocation at all.
//
// dbm_moments reduces its totals through partial sums kept in the caller's
// device buffer.  Some callers cannot supply or allocate device memory for
// that: a component that only holds raw device pointers to a state another
// component owns (a checkpoint writer, a monitor on its own thread), or code
// running under a fixed device-memory budget whose allocator forbids new
// allocations once a run has started.  dbm_totals_noalloc serves them: the
// per-row partial sums live in a file-scope static device array of fixed
// size, so the call needs nothing beyond its input and output pointers.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "dbm.h"
#include "dbm_launch.h"

namespace {

// Scratch: 4 FP64 partial sums per theta row, for at most DBM_NOALLOC_MAX_ROWS
// rows (512 KB).  Every GPU that loads the library holds it until exit.
__device__ __align__(256) double g_row_partials[DBM_NOALLOC_MAX_ROWS * 4];

// Device address of g_row_partials, looked up once per device and context:
// the address belongs to the context the module was loaded into, so a new
// primary context (after cudaDeviceReset, say) gets a fresh lookup.
constexpr int kMaxDevices = 64;
struct Setup {
    unsigned long long ctx_id;  // 0: not set up
    double *partials;
};
std::mutex g_setup_mu;
Setup g_setup[kMaxDevices];

using CtxGetCurrent = CUresult (*)(CUcontext *);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long *);

// The current context's unique id (never reused within the process), from
// the driver entry points (the library does not link libcuda); 0 if unknown.
unsigned long long current_context_id()
{
    static CtxGetCurrent get_current = nullptr;
    static CtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetId>(p);
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

const double kPi = 3.14159265358979323846;

// One CTA per theta row: each site's sums rho, jx, jy, e2 = sum f |v|^2 from
// its 33 f (Sec. II.B, Cartesian components) -- in FP32 ring by ring as the
// step and dbm_moments compute them, or in FP64 -- weighted by r and summed
// in FP64 into the row's 4 partials {mass, px, py, energy}, times dr dtheta
// (energy rho T + rho u^2 / 2 = e2 / 2 for D = 2).  f: [33][ntheta][ld].
template <typename real>
__global__ void __launch_bounds__(256) row_totals_kernel(const real *f, int nr, int ntheta, long long ld,
                                                         double r_in, double dr, double dtheta,
                                                         dbm::RingSpeeds<real> vv, double *partials)
{
    const int m = blockIdx.x;
    const long long plane = ld * ntheta;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < nr; j += blockDim.x) {
        const real *fp = f + (long long)m * ld + j;
        real fv[dbm::NV];
#pragma unroll
        for (int q = 0; q < dbm::NV; ++q) fv[q] = fp[(long long)q * plane];
        real rho, jx, jy, e2;
        if constexpr (sizeof(real) == 4) {
            dbm::ring_moments<real>(fv, vv.v, vv.v2, rho, jx, jy, e2);
        } else {
            double cx[8], cy[8];
            dbm::cart_dirs(cx, cy);
            rho = fv[0];
            jx = jy = e2 = 0.0;
            for (int k = 0; k < 4; ++k)
                for (int i = 0; i < 8; ++i) {
                    const double fq = fv[1 + 8 * k + i];
                    rho += fq;
                    jx += fq * vv.v[k] * cx[i];
                    jy += fq * vv.v[k] * cy[i];
                    e2 += fq * vv.v2[k];
                }
        }
        const double r = r_in + (j + 0.5) * dr;
        acc[0] += (double)rho * r;
        acc[1] += (double)jx * r;
        acc[2] += (double)jy * r;
        acc[3] += (double)e2 * r;
    }
    __shared__ double red[4][256];
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) {
        const double wa = dr * dtheta * (threadIdx.x == 3 ? 0.5 : 1.0);
        partials[(long long)m * 4 + threadIdx.x] = red[threadIdx.x][0] * wa;
    }
}

// Sum the row partials in a fixed order (one CTA).
__global__ void __launch_bounds__(256) rows_sum_kernel(const double *partials, int nrows,
                                                       double *totals)
{
    __shared__ double red[4][256];
    for (int c = 0; c < 4; ++c) {
        double s = 0.0;
        for (int m = threadIdx.x; m < nrows; m += blockDim.x) s += partials[m * 4 + c];
        red[c][threadIdx.x] = s;
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) totals[threadIdx.x] = red[threadIdx.x][0];
}

template <typename real>
cudaError_t launch_rows(const dbm_params *p, const void *d_f, long long ld, double dr, double dth,
                        double *partials, cudaStream_t s)
{
    const real *f = static_cast<const real *>(d_f);
    int nr = p->nr, nth = p->ntheta;
    double r_in = p->r_in;
    dbm::RingSpeeds<real> vv;
    for (int k = 0; k < 4; ++k) {
        vv.v[k] = (real)p->v[k];
        vv.v2[k] = (real)(p->v[k] * p->v[k]);
    }
    void *args[] = {&f, &nr, &nth, &ld, &r_in, &dr, &dth, &vv, &partials};
    // the launch's own status (not a sticky error left by earlier work)
    return cudaLaunchKernel(reinterpret_cast<const void *>(&row_totals_kernel<real>), dim3(nth), dim3(256),
                            args, 0, s);
}

}  // namespace

extern "C" int dbm_totals_noalloc(const dbm_params *p, const void *d_f, int64_t ld, double *d_totals,
                                  void *stream)
{
    if (!p || !d_f || !d_totals) return DBM_EINVAL;
    if (p->nr < 1 || p->ntheta < 1 || (p->precision != DBM_FP32 && p->precision != DBM_FP64))
        return DBM_EINVAL;
    if (ld == 0) ld = p->nr;
    if (ld < p->nr) return DBM_EINVAL;
    if (!(p->r_in >= 0.0) || !(p->r_out > p->r_in) || !std::isfinite(p->r_out)) return DBM_EINVAL;
    if (p->ntheta > DBM_NOALLOC_MAX_ROWS) return DBM_ENOMEM;  // beyond the static scratch

    // Set-up, once per device and context, with that device current: the
    // device address of the static scratch (host code cannot use the
    // symbol's name as a device address).
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dbm::record_cuda_failure(e, "dbm_totals_noalloc: device query");
    if (dev < 0 || dev >= kMaxDevices) return DBM_EINVAL;
    double *partials = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        const unsigned long long id = current_context_id();
        if (id == 0 || g_setup[dev].ctx_id != id) {
            void *addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_row_partials);
            if (e != cudaSuccess)
                return dbm::record_cuda_failure(e, "dbm_totals_noalloc: address of the static scratch");
            // the lookup made the primary context current if it was not yet
            g_setup[dev].ctx_id = id != 0 ? id : current_context_id();
            g_setup[dev].partials = static_cast<double *>(addr);
        }
        partials = g_setup[dev].partials;
    }

    // Every row's partials are rewritten before they are read, so nothing in
    // the scratch has to be cleared between calls.
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double dr = (p->r_out - p->r_in) / p->nr;
    const double dth = (p->sector ? kPi / 4.0 : 2.0 * kPi) / p->ntheta;
    e = p->precision == DBM_FP64 ? launch_rows<double>(p, d_f, (long long)ld, dr, dth, partials, s)
                                 : launch_rows<float>(p, d_f, (long long)ld, dr, dth, partials, s);
    if (e != cudaSuccess) return dbm::record_cuda_failure(e, "dbm_totals_noalloc: row kernel launch");
    int nrows = p->ntheta;
    void *args[] = {&partials, &nrows, &d_totals};
    e = cudaLaunchKernel(reinterpret_cast<const void *>(&rows_sum_kernel), dim3(1), dim3(256), args, 0, s);
    if (e != cudaSuccess) return dbm::record_cuda_failure(e, "dbm_totals_noalloc: sum kernel launch");
    return DBM_OK;
}
