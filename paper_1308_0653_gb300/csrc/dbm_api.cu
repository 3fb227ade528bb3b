// C-ABI runtime of the polar-coordinate discrete-Boltzmann detonation update
// (declarations and contracts in include/dbm.h).  Host code only: it
// validates parameters, carves the caller's device buffer, builds the
// geometry tables, picks the launch configuration and enqueues kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "dbm.h"
#include "dbm_launch.h"

using namespace dbm;

namespace {

thread_local char g_last_error[256] = "";

int cuda_fail(cudaError_t e, const char *what)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
    return DBM_ECUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

const double PI = 3.14159265358979323846;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int padded_ld(int nr) { return (nr + 31) / 32 * 32; }

// Byte layout of the caller buffer (offsets from its start).
struct Layout {
    size_t elem, plane_bytes;
    size_t f[2], lam[2], rowtab, inv_r, status, partials, totals, total;
};

Layout layout_of(const dbm_params &p)
{
    Layout L;
    L.elem = p.precision == DBM_FP64 ? 8 : 4;
    const size_t ld = (size_t)padded_ld(p.nr);
    L.plane_bytes = ld * (size_t)p.ntheta * L.elem;
    size_t off = 0;
    for (int b = 0; b < 2; ++b) {
        L.f[b] = off;
        off = align256(off + NV * L.plane_bytes);
    }
    for (int b = 0; b < 2; ++b) {
        L.lam[b] = off;
        off = align256(off + L.plane_bytes);
    }
    L.rowtab = off;
    off = align256(off + (size_t)p.ntheta * 16 * L.elem);
    L.inv_r = off;
    off = align256(off + ld * L.elem);
    L.status = off;
    off = align256(off + 64);
    L.partials = off;
    off = align256(off + (size_t)MOMENT_BLOCKS * 4 * sizeof(double));
    L.totals = off;
    off = align256(off + 8 * sizeof(double));
    L.total = off;
    return L;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// F_k(T) = T (c0 + T (c1 + T (c2 + T c3))) for k = 1..4 (Sec. II.B weights,
// last term with a minus sign; cyclic subscripts k+l -> k+l-4).
void weight_coeffs(const double v[4], double Fc[4][4])
{
    for (int k = 0; k < 4; ++k) {
        const double xk = v[k] * v[k];
        const double a = v[(k + 1) % 4] * v[(k + 1) % 4];
        const double b = v[(k + 2) % 4] * v[(k + 2) % 4];
        const double c = v[(k + 3) % 4] * v[(k + 3) % 4];
        const double den = xk * (xk - a) * (xk - b) * (xk - c);
        Fc[k][0] = -0.25 * a * b * c / den;
        Fc[k][1] = (a * b + b * c + c * a) / den;
        Fc[k][2] = -6.0 * (a + b + c) / den;
        Fc[k][3] = 48.0 / den;
    }
}

// cos and sin of (i pi/4 - theta_m); with ntheta a multiple of 8 the angle is
// taken from the integer index (i ntheta/8 - m) mod ntheta, so the table is
// exactly invariant under the pi/4 rotation (m -> m + ntheta/8, i -> i + 1).
void row_angles(const dbm_params &p, int m, double c[8], double s[8])
{
    for (int i = 0; i < 8; ++i) {
        double ang;
        if (p.ntheta % 8 == 0) {
            long long q = ((long long)i * (p.ntheta / 8) - m) % p.ntheta;
            if (q < 0) q += p.ntheta;
            ang = 2.0 * PI * (double)q / p.ntheta;
        } else {
            ang = i * PI / 4.0 - m * (2.0 * PI / p.ntheta);
        }
        c[i] = std::cos(ang);
        s[i] = std::sin(ang);
    }
}

}  // namespace

struct dbm_s {
    dbm_params p;
    Layout L;
    unsigned char *buf;
    size_t bytes;
    int ld;
    long long plane;
    int cur;
    int64_t steps;
    KernelInfo ki;
    int grid, rows_per_item, items;
    StepArgs<float> a32[2];   // [0]: f0 -> f1, [1]: f1 -> f0
    StepArgs<double> a64[2];
    cudaGraphExec_t graph;    // GRAPH_STEPS steps starting from buffer 0
    int device;
};

namespace {

constexpr int GRAPH_STEPS = 32;

template <typename real>
void fill_step_args(dbm_t *h, StepArgs<real> (&a)[2])
{
    const dbm_params &p = h->p;
    const double dr = (p.r_out - p.r_in) / p.nr;
    const double dth = 2.0 * PI / p.ntheta;
    double Fc[4][4];
    weight_coeffs(p.v, Fc);
    for (int b = 0; b < 2; ++b) {
        StepArgs<real> &A = a[b];
        std::memset(&A, 0, sizeof(A));
        A.f_in = reinterpret_cast<const real *>(h->buf + h->L.f[b]);
        A.f_out = reinterpret_cast<real *>(h->buf + h->L.f[1 - b]);
        A.lam_in = reinterpret_cast<const real *>(h->buf + h->L.lam[b]);
        A.lam_out = reinterpret_cast<real *>(h->buf + h->L.lam[1 - b]);
        A.rowtab = reinterpret_cast<const real *>(h->buf + h->L.rowtab);
        A.inv_r = reinterpret_cast<const real *>(h->buf + h->L.inv_r);
        A.status = reinterpret_cast<int *>(h->buf + h->L.status);
        A.plane = h->plane;
        A.nr = p.nr;
        A.ntheta = p.ntheta;
        A.ld = h->ld;
        A.strips = (p.nr + h->ki.W - 1) / h->ki.W;
        A.rows_per_item = h->rows_per_item;
        A.segs = (p.ntheta + h->rows_per_item - 1) / h->rows_per_item;
        A.items = A.strips * A.segs;
        A.reaction_energy = p.reaction_energy;
        A.general_pow = (p.m == 1.0 && p.n == 1.0) ? 0 : 1;
        A.cr_scale = (real)(p.dt / dr);
        A.ct_scale = (real)(p.dt / dth);
        A.decay = (real)std::exp(-p.dt / p.tau);
        A.one_m_decay = (real)(-std::expm1(-p.dt / p.tau));
        A.dt = (real)p.dt;
        A.Q = (real)p.Q;
        A.omega1 = (real)p.omega1;
        A.omega2 = (real)p.omega2;
        A.m_exp = (real)p.m;
        A.n_exp = (real)p.n;
        A.T_th = (real)p.T_th;
        for (int k = 0; k < 4; ++k) {
            A.v[k] = (real)p.v[k];
            A.v2[k] = (real)(p.v[k] * p.v[k]);
            for (int c = 0; c < 4; ++c) A.Fc[k][c] = (real)Fc[k][c];
        }
    }
}

template <typename real>
int upload_tables(dbm_t *h)
{
    const dbm_params &p = h->p;
    const double dr = (p.r_out - p.r_in) / p.nr;
    real *tab = new (std::nothrow) real[(size_t)p.ntheta * 16];
    real *ir = new (std::nothrow) real[(size_t)h->ld];
    if (!tab || !ir) {
        delete[] tab;
        delete[] ir;
        return DBM_ENOMEM;
    }
    for (int m = 0; m < p.ntheta; ++m) {
        double c[8], s[8];
        row_angles(p, m, c, s);
        for (int i = 0; i < 8; ++i) {
            tab[(size_t)m * 16 + i] = (real)c[i];
            tab[(size_t)m * 16 + 8 + i] = (real)s[i];
        }
    }
    for (int j = 0; j < h->ld; ++j) ir[j] = (real)(1.0 / (p.r_in + (j + 0.5) * dr));
    cudaError_t e = cudaMemcpy(h->buf + h->L.rowtab, tab, sizeof(real) * (size_t)p.ntheta * 16,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->buf + h->L.inv_r, ir, sizeof(real) * (size_t)h->ld, cudaMemcpyHostToDevice);
    delete[] tab;
    delete[] ir;
    if (e != cudaSuccess) return cuda_fail(e, "upload geometry tables");
    return DBM_OK;
}

int launch_one(dbm_t *h, int b, cudaStream_t s)
{
    cudaError_t e = h->p.precision == DBM_FP64 ? launch_step<double>(h->a64[b], h->grid, s)
                                               : launch_step<float>(h->a32[b], h->grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    return DBM_OK;
}

int build_graph(dbm_t *h)
{
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = DBM_OK;
    if (e == cudaSuccess) {
        for (int s = 0; s < GRAPH_STEPS && rc == DBM_OK; ++s) rc = launch_one(h, s & 1, cs);
        e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess && rc == DBM_OK) e = cudaGraphInstantiate(&h->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc != DBM_OK) return rc;
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return cuda_fail(e, "step graph capture");
    }
    return DBM_OK;
}

}  // namespace

extern "C" {

const char *dbm_version(void) { return "dbm-gb300 1.0 (sm_103a)"; }

const char *dbm_strerror(int status)
{
    switch (status) {
    case DBM_OK: return "ok";
    case DBM_EINVAL: return "invalid argument";
    case DBM_ECFL: return "Courant condition violated (max |C_r| + |C_theta| > 1)";
    case DBM_ENOMEM: return "not enough memory";
    case DBM_EBUSY: return "queue full";
    case DBM_ENOTREADY: return "not ready";
    case DBM_ETIMEOUT: return "timed out";
    case DBM_ENONFINITE: return "non-finite moment";
    case DBM_ECUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case DBM_ECANCELLED: return "cancelled";
    case DBM_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
    }
}

const char *dbm_last_error(void) { return g_last_error; }

int dbm_params_default(dbm_params *p)
{
    if (!p) return DBM_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->nr = 64;
    p->ntheta = 64;
    p->precision = DBM_FP32;
    p->reaction_energy = DBM_R_EXPLICIT;
    p->r_bc_inner = DBM_BC_OUTFLOW;
    p->r_bc_outer = DBM_BC_OUTFLOW;
    p->r_in = 0.05;
    p->r_out = 1.05;
    p->dt = 1e-5;
    p->tau = 1e-3;
    p->Q = 1.0;
    p->m = 1.0;
    p->n = 1.0;
    p->T_th = 1.1;
    p->v[0] = 1.5;
    p->v[1] = 3.5;
    p->v[2] = 7.5;
    p->v[3] = 12.5;
    return DBM_OK;
}

int dbm_check(const dbm_params *p, double *cfl)
{
    if (!p) return DBM_EINVAL;
    if (p->nr < 1 || p->ntheta < 1) return DBM_EINVAL;
    if ((long long)p->nr * p->ntheta > (1LL << 40)) return DBM_EINVAL;
    if (p->precision != DBM_FP32 && p->precision != DBM_FP64) return DBM_EINVAL;
    if (p->reaction_energy != DBM_R_EXPLICIT && p->reaction_energy != DBM_R_CONSISTENT) return DBM_EINVAL;
    if (p->r_bc_inner != DBM_BC_OUTFLOW || p->r_bc_outer != DBM_BC_OUTFLOW) return DBM_EINVAL;
    if (p->rows_per_item < 0 || p->reserved != 0) return DBM_EINVAL;
    if (!finite_pos(p->r_in) || !std::isfinite(p->r_out) || p->r_out <= p->r_in) return DBM_EINVAL;
    if (!finite_pos(p->dt) || !(p->tau > 0.0)) return DBM_EINVAL;  // tau may be +inf-like large
    if (!std::isfinite(p->Q) || !std::isfinite(p->T_th)) return DBM_EINVAL;
    if (!(p->omega1 >= 0.0) || !(p->omega2 >= 0.0) || !std::isfinite(p->omega1) ||
        !std::isfinite(p->omega2))
        return DBM_EINVAL;
    if (!std::isfinite(p->m) || !std::isfinite(p->n)) return DBM_EINVAL;
    for (int k = 0; k < 4; ++k) {
        if (!finite_pos(p->v[k])) return DBM_EINVAL;
        for (int l = 0; l < k; ++l)
            if (p->v[k] == p->v[l]) return DBM_EINVAL;
    }
    // Courant numbers of Sec. II.C; |C_theta| is largest at the innermost radius.
    const double dr = (p->r_out - p->r_in) / p->nr;
    const double dth = 2.0 * PI / p->ntheta;
    const double r0 = p->r_in + 0.5 * dr;
    double vmax = 0.0;
    for (int k = 0; k < 4; ++k) vmax = std::max(vmax, p->v[k]);
    double worst = 0.0;
    for (int m = 0; m < p->ntheta; ++m) {
        double c[8], s[8];
        row_angles(*p, m, c, s);
        for (int i = 0; i < 8; ++i)
            worst = std::max(worst, vmax * (std::fabs(c[i]) * p->dt / dr + std::fabs(s[i]) * p->dt / (r0 * dth)));
        if (p->ntheta > 4096 && m == 4096) break;  // the pattern repeats at pi/4 resolution
    }
    if (cfl) *cfl = worst;
    if (worst > 1.0 + 1e-12) return DBM_ECFL;
    return DBM_OK;
}

size_t dbm_state_bytes(const dbm_params *p)
{
    if (!p) return 0;
    int rc = dbm_check(p, nullptr);
    if (rc != DBM_OK && rc != DBM_ECFL) return 0;
    return layout_of(*p).total;
}

int dbm_create(const dbm_params *p, void *dev_buf, size_t dev_bytes, dbm_t **out)
{
    if (!p || !dev_buf || !out) return DBM_EINVAL;
    *out = nullptr;
    int rc = dbm_check(p, nullptr);
    if (rc != DBM_OK) return rc;
    if (((uintptr_t)dev_buf & 255) != 0) return DBM_EINVAL;
    const Layout L = layout_of(*p);
    if (dev_bytes < L.total) return DBM_ENOMEM;

    dbm_t *h = new (std::nothrow) dbm_t;
    if (!h) return DBM_ENOMEM;
    std::memset(h, 0, sizeof(*h));
    h->p = *p;
    h->L = L;
    h->buf = static_cast<unsigned char *>(dev_buf);
    h->bytes = dev_bytes;
    h->ld = padded_ld(p->nr);
    h->plane = (long long)h->ld * p->ntheta;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess)
        e = p->precision == DBM_FP64 ? kernel_info<double>(&h->ki) : kernel_info<float>(&h->ki);
    int nsm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "dbm_create: device query");
    }
    if (h->ki.blocks_per_sm < 1) {
        delete h;
        snprintf(g_last_error, sizeof(g_last_error), "step kernel does not fit on an SM");
        return DBM_ECUDA;
    }
    // Launch shape: persistent CTAs, one per resident slot; theta rows per
    // item chosen so the items fill the slots in one wave.
    const int slots = nsm * h->ki.blocks_per_sm;
    const int strips = (p->nr + h->ki.W - 1) / h->ki.W;
    int L_rows = p->rows_per_item;
    if (L_rows == 0) {
        const long long need = ((long long)p->ntheta * strips + slots - 1) / slots;
        L_rows = (int)std::max(1LL, need);
    }
    L_rows = std::min(L_rows, p->ntheta);
    h->rows_per_item = L_rows;
    h->items = strips * ((p->ntheta + L_rows - 1) / L_rows);
    h->grid = std::min(h->items, slots);

    e = cudaMemset(dev_buf, 0, L.total);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "dbm_create: clear buffer");
    }
    rc = p->precision == DBM_FP64 ? upload_tables<double>(h) : upload_tables<float>(h);
    if (rc != DBM_OK) {
        delete h;
        return rc;
    }
    if (p->precision == DBM_FP64)
        fill_step_args<double>(h, h->a64);
    else
        fill_step_args<float>(h, h->a32);
    *out = h;
    return DBM_OK;
}

int dbm_destroy(dbm_t *h)
{
    if (!h) return DBM_EINVAL;
    if (h->graph) cudaGraphExecDestroy(h->graph);
    delete h;
    return DBM_OK;
}

static int launch_init_from(dbm_t *h, const double *d_fields, cudaStream_t s)
{
    double Fc[4][4];
    weight_coeffs(h->p.v, Fc);
    cudaError_t e;
    if (h->p.precision == DBM_FP64) {
        InitArgs<double> A;
        A.fields = d_fields;
        A.f = reinterpret_cast<double *>(h->buf + h->L.f[0]);
        A.lam = reinterpret_cast<double *>(h->buf + h->L.lam[0]);
        A.plane = h->plane;
        A.nr = h->p.nr;
        A.ntheta = h->p.ntheta;
        A.ld = h->ld;
        std::memcpy(A.v, h->p.v, sizeof(A.v));
        std::memcpy(A.Fc, Fc, sizeof(Fc));
        e = launch_init<double>(A, s);
    } else {
        InitArgs<float> A;
        A.fields = d_fields;
        A.f = reinterpret_cast<float *>(h->buf + h->L.f[0]);
        A.lam = reinterpret_cast<float *>(h->buf + h->L.lam[0]);
        A.plane = h->plane;
        A.nr = h->p.nr;
        A.ntheta = h->p.ntheta;
        A.ld = h->ld;
        std::memcpy(A.v, h->p.v, sizeof(A.v));
        std::memcpy(A.Fc, Fc, sizeof(Fc));
        e = launch_init<float>(A, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "init kernel launch");
    h->cur = 0;
    h->steps = 0;
    return DBM_OK;
}

int dbm_init_state(dbm_t *h, const double *rho, const double *ur, const double *uth,
                   const double *T, const double *lam, void *stream)
{
    if (!h || !rho || !ur || !uth || !T || !lam) return DBM_EINVAL;
    const size_t N = (size_t)h->p.nr * h->p.ntheta;
    for (size_t s = 0; s < N; ++s) {
        if (!finite_pos(rho[s]) || !finite_pos(T[s]) || !std::isfinite(ur[s]) ||
            !std::isfinite(uth[s]) || !std::isfinite(lam[s]))
            return DBM_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Stage the fields in the second f buffer (free before the first step).
    double *stage = reinterpret_cast<double *>(h->buf + h->L.f[1]);
    const double *src[5] = {rho, ur, uth, T, lam};
    for (int c = 0; c < 5; ++c)
        CK(cudaMemcpyAsync(stage + c * N, src[c], N * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // host arrays may be reused on return
    return launch_init_from(h, stage, s);
}

int dbm_init_state_device(dbm_t *h, const double *d_fields, void *stream)
{
    if (!h || !d_fields) return DBM_EINVAL;
    return launch_init_from(h, d_fields, static_cast<cudaStream_t>(stream));
}

int dbm_step(dbm_t *h, int64_t nsteps, void *stream)
{
    if (!h || nsteps < 0) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    while (nsteps > 0) {
        if (nsteps >= GRAPH_STEPS && h->cur == 0) {
            if (!h->graph) {
                int rc = build_graph(h);
                if (rc != DBM_OK) return rc;
            }
            CK(cudaGraphLaunch(h->graph, s));
            nsteps -= GRAPH_STEPS;
            h->steps += GRAPH_STEPS;
        } else {
            int rc = launch_one(h, h->cur, s);
            if (rc != DBM_OK) return rc;
            h->cur ^= 1;
            nsteps -= 1;
            h->steps += 1;
        }
    }
    return DBM_OK;
}

static int launch_moments_into(dbm_t *h, double *d_out, cudaStream_t s)
{
    const dbm_params &p = h->p;
    const long long N = (long long)p.nr * p.ntheta;
    int grid = (int)std::min<long long>((N + 255) / 256, MOMENT_BLOCKS);
    double *partials = reinterpret_cast<double *>(h->buf + h->L.partials);
    int *status = reinterpret_cast<int *>(h->buf + h->L.status);
    cudaError_t e;
    if (p.precision == DBM_FP64) {
        MomArgs<double> A;
        A.f = reinterpret_cast<const double *>(h->buf + h->L.f[h->cur]);
        A.lam = reinterpret_cast<const double *>(h->buf + h->L.lam[h->cur]);
        A.out = d_out;
        A.partials = partials;
        A.status = status;
        A.plane = h->plane;
        A.nr = p.nr;
        A.ntheta = p.ntheta;
        A.ld = h->ld;
        A.r_in = p.r_in;
        A.dr = (p.r_out - p.r_in) / p.nr;
        A.dtheta = 2.0 * PI / p.ntheta;
        std::memcpy(A.v, p.v, sizeof(A.v));
        e = launch_moments<double>(A, grid, s);
    } else {
        MomArgs<float> A;
        A.f = reinterpret_cast<const float *>(h->buf + h->L.f[h->cur]);
        A.lam = reinterpret_cast<const float *>(h->buf + h->L.lam[h->cur]);
        A.out = d_out;
        A.partials = partials;
        A.status = status;
        A.plane = h->plane;
        A.nr = p.nr;
        A.ntheta = p.ntheta;
        A.ld = h->ld;
        A.r_in = p.r_in;
        A.dr = (p.r_out - p.r_in) / p.nr;
        A.dtheta = 2.0 * PI / p.ntheta;
        std::memcpy(A.v, p.v, sizeof(A.v));
        e = launch_moments<float>(A, grid, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "moments kernel launch");
    e = launch_totals(partials, grid, reinterpret_cast<double *>(h->buf + h->L.totals), s);
    if (e != cudaSuccess) return cuda_fail(e, "totals kernel launch");
    return DBM_OK;
}

int dbm_moments_device(dbm_t *h, double *d_out, void *stream)
{
    if (!h || !d_out) return DBM_EINVAL;
    return launch_moments_into(h, d_out, static_cast<cudaStream_t>(stream));
}

int dbm_moments(dbm_t *h, double *rho, double *ur, double *uth, double *T, double *lam,
                double totals[4], void *stream)
{
    if (!h) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t N = (size_t)h->p.nr * h->p.ntheta;
    double *stage = reinterpret_cast<double *>(h->buf + h->L.f[1 - h->cur]);
    int rc = launch_moments_into(h, stage, s);
    if (rc != DBM_OK) return rc;
    double *dst[5] = {rho, ur, uth, T, lam};
    for (int c = 0; c < 5; ++c)
        if (dst[c])
            CK(cudaMemcpyAsync(dst[c], stage + c * N, N * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (totals)
        CK(cudaMemcpyAsync(totals, h->buf + h->L.totals, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    int status = 0;
    CK(cudaMemcpyAsync(&status, h->buf + h->L.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (status & ST_WAIT_TIMEOUT) return DBM_ETIMEOUT;
    if (status & ST_NONFINITE) {
        CK(cudaMemsetAsync(h->buf + h->L.status, 0, sizeof(int), s));
        CK(cudaStreamSynchronize(s));
        return DBM_ENONFINITE;
    }
    return DBM_OK;
}

int64_t dbm_steps_done(const dbm_t *h) { return h ? h->steps : -1; }

int dbm_status(dbm_t *h, void *stream)
{
    if (!h) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int status = 0;
    CK(cudaMemcpyAsync(&status, h->buf + h->L.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (status & ST_WAIT_TIMEOUT) return DBM_ETIMEOUT;
    return DBM_OK;
}

int dbm_export_state(dbm_t *h, void *f, void *lam, int64_t *steps, void *stream)
{
    if (!h || !f || !lam) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t e = h->L.elem, row = (size_t)h->p.nr * e, pitch = (size_t)h->ld * e;
    CK(cudaMemcpy2DAsync(f, row, h->buf + h->L.f[h->cur], pitch, row, (size_t)NV * h->p.ntheta,
                         cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpy2DAsync(lam, row, h->buf + h->L.lam[h->cur], pitch, row, (size_t)h->p.ntheta,
                         cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (steps) *steps = h->steps;
    return DBM_OK;
}

int dbm_import_state(dbm_t *h, const void *f, const void *lam, int64_t steps, void *stream)
{
    if (!h || !f || !lam || steps < 0) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t e = h->L.elem, row = (size_t)h->p.nr * e, pitch = (size_t)h->ld * e;
    CK(cudaMemcpy2DAsync(h->buf + h->L.f[0], pitch, f, row, row, (size_t)NV * h->p.ntheta,
                         cudaMemcpyHostToDevice, s));
    CK(cudaMemcpy2DAsync(h->buf + h->L.lam[0], pitch, lam, row, row, (size_t)h->p.ntheta,
                         cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    h->cur = 0;
    h->steps = steps;
    return DBM_OK;
}

int dbm_launch_info(const dbm_t *h, int *grid, int *threads, int *smem_bytes, int *rows_per_item,
                    int *items)
{
    if (!h) return DBM_EINVAL;
    if (grid) *grid = h->grid;
    if (threads) *threads = h->ki.W;
    if (smem_bytes) *smem_bytes = h->ki.smem;
    if (rows_per_item) *rows_per_item = h->rows_per_item;
    if (items) *items = h->items;
    return DBM_OK;
}

}  // extern "C"
