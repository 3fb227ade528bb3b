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
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "dbm.h"
#include "dbm_device.cuh"

namespace {

// Scratch: 4 FP64 partial sums per theta row, for at most DBM_NOALLOC_MAX_ROWS
// rows (512 KB).  Every GPU that loads the library holds it until exit.
__device__ __align__(256) double g_row_partials[DBM_NOALLOC_MAX_ROWS * 4];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_partials_ptr[kMaxDevices];  // device address of g_row_partials, per device
bool g_setup_done[kMaxDevices];

const double kPi = 3.14159265358979323846;

// One CTA per theta row: FP64 moments of every site of the row (Sec. II.B
// definitions, Cartesian components), weighted by the area element
// r dr dtheta, summed into the row's 4 partials {mass, px, py, energy}.
template <typename real>
__global__ void __launch_bounds__(256) row_totals_kernel(const real *f, int nr, int ntheta,
                                                         double r_in, double dr, double dtheta,
                                                         double v0, double v1, double v2, double v3,
                                                         double *partials)
{
    const int m = blockIdx.x;
    const long long plane = (long long)nr * ntheta;
    const double v[4] = {v0, v1, v2, v3};
    double cx[8], cy[8];
    dbm::cart_dirs(cx, cy);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < nr; j += blockDim.x) {
        const real *fp = f + (long long)m * nr + j;
        double rho = (double)fp[0], jx = 0.0, jy = 0.0, e2 = 0.0;
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < 8; ++i) {
                const double fq = (double)fp[(long long)(1 + 8 * k + i) * plane];
                rho += fq;
                jx += fq * v[k] * cx[i];
                jy += fq * v[k] * cy[i];
                e2 += fq * v[k] * v[k];
            }
        const double w = (r_in + (j + 0.5) * dr) * dr * dtheta;
        acc[0] += rho * w;
        acc[1] += jx * w;
        acc[2] += jy * w;
        acc[3] += 0.5 * e2 * w;  // rho T + rho u^2 / 2 = (1/2) sum f v^2 for D = 2
    }
    __shared__ double red[4][256];
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) partials[(long long)m * 4 + threadIdx.x] = red[threadIdx.x][0];
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

}  // namespace

extern "C" int dbm_totals_noalloc(const dbm_params *p, const void *d_f, double *d_totals,
                                  void *stream)
{
    if (!p || !d_f || !d_totals) return DBM_EINVAL;
    if (p->nr < 1 || p->ntheta < 1 || (p->precision != DBM_FP32 && p->precision != DBM_FP64))
        return DBM_EINVAL;
    if (!(p->r_in >= 0.0) || !(p->r_out > p->r_in) || !std::isfinite(p->r_out)) return DBM_EINVAL;
    if (p->ntheta > DBM_NOALLOC_MAX_ROWS) return DBM_ENOMEM;  // beyond the static scratch

    // Set-up, once per device, with that device current: the device address
    // of the static scratch (host code cannot use the symbol's name).
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DBM_ECUDA;
    double *partials = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_setup_done[dev]) {
            if (cudaGetSymbolAddress(reinterpret_cast<void **>(&g_partials_ptr[dev]), g_row_partials) !=
                cudaSuccess)
                return DBM_ECUDA;
            g_setup_done[dev] = true;
        }
        partials = g_partials_ptr[dev];
    }

    // Every row's partials are rewritten before they are read, so nothing in
    // the scratch has to be cleared between calls.
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double dr = (p->r_out - p->r_in) / p->nr;
    const double dth = (p->sector ? kPi / 4.0 : 2.0 * kPi) / p->ntheta;
    if (p->precision == DBM_FP64)
        row_totals_kernel<double><<<p->ntheta, 256, 0, s>>>(static_cast<const double *>(d_f), p->nr,
                                                           p->ntheta, p->r_in, dr, dth, p->v[0],
                                                           p->v[1], p->v[2], p->v[3], partials);
    else
        row_totals_kernel<float><<<p->ntheta, 256, 0, s>>>(static_cast<const float *>(d_f), p->nr,
                                                          p->ntheta, p->r_in, dr, dth, p->v[0],
                                                          p->v[1], p->v[2], p->v[3], partials);
    if (cudaGetLastError() != cudaSuccess) return DBM_ECUDA;
    rows_sum_kernel<<<1, 256, 0, s>>>(partials, p->ntheta, d_totals);
    if (cudaGetLastError() != cudaSuccess) return DBM_ECUDA;
    return DBM_OK;
}
