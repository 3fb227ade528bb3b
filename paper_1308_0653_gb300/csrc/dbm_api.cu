// C-ABI runtime of the polar-coordinate discrete-Boltzmann detonation update
// (declarations and contracts in include/dbm.h).  Host code only: it
// validates parameters, carves the caller's device buffer, builds the
// geometry tables, picks the launch configuration and enqueues kernels.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <queue>
#include <type_traits>
#include <vector>

#include "dbm.h"
#include "dbm_launch.h"

using namespace dbm;

namespace {
// NVTX range for profilers (header-only NVTX3: no cost without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

namespace {

thread_local char g_last_error[256] = "";

int cuda_fail(cudaError_t e, const char *what)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
    return DBM_ECUDA;
}

}  // namespace

namespace dbm {
int record_cuda_failure(cudaError_t e, const char *what) { return cuda_fail(e, what); }
}  // namespace dbm

namespace {

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
double theta_span(const dbm_params &p) { return p.sector ? PI / 4.0 : 2.0 * PI; }

void row_angles(const dbm_params &p, int m, double c[8], double s[8])
{
    // Directions i and i + 4 are opposite: their entries are exact negatives
    // of each other (the step shares |C_r|, |C_theta| between them).  With
    // 8 | ntheta on a full grid the entry depends on q = (i ntheta/8 - m) mod
    // ntheta alone (8-fold rotation equivariance, bit for bit), and the half
    // turn q + ntheta/2 is the negation of q.
    if (!p.sector && p.ntheta % 8 == 0) {
        const long long half = p.ntheta / 2;
        for (int i = 0; i < 8; ++i) {
            long long q = ((long long)i * (p.ntheta / 8) - m) % p.ntheta;
            if (q < 0) q += p.ntheta;
            const double sign = q < half ? 1.0 : -1.0;
            const double ang = 2.0 * PI * (double)(q < half ? q : q - half) / p.ntheta;
            c[i] = sign * std::cos(ang);
            s[i] = sign * std::sin(ang);
        }
        return;
    }
    for (int i = 0; i < 4; ++i) {
        const double ang = p.sector ? i * PI / 4.0 - m * (PI / 4.0 / p.ntheta)
                                    : i * PI / 4.0 - m * (2.0 * PI / p.ntheta);
        c[i] = std::cos(ang);
        s[i] = std::sin(ang);
        c[i + 4] = -c[i];
        s[i + 4] = -s[i];
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
    int variant;              // kernel variant (1..num_variants)
    int grid, rows_per_item, items;
    StepArgs<float> a32[2];   // [0]: f0 -> f1, [1]: f1 -> f0
    StepArgs<double> a64[2];
    cudaGraphExec_t graph;    // GRAPH_STEPS steps starting from buffer 0
    int device;
    bool tmap_ok;             // tensor maps encoded (tensor-TMA variants usable)
    cudaEvent_t done;         // recorded after the last work that touches the buffers
    int host_word[2];         // host side of small device-to-host status copies
    cudaStream_t aux;         // second stream of the chunked host-array calls
    cudaEvent_t chunk_ev[4], join_ev;
};

namespace {

constexpr int GRAPH_STEPS = 32;

// Second word of the status region: set by the init kernel when an initial
// field value is invalid (rho <= 0, T <= 0, not finite).
int *bad_input_word(dbm_t *h) { return reinterpret_cast<int *>(h->buf + h->L.status) + 1; }

int bad_input_fail()
{
    snprintf(g_last_error, sizeof(g_last_error),
             "initial fields: some rho <= 0, T <= 0 or non-finite value (state undefined until the next init)");
    return DBM_EINVAL;
}

// Record that work touching the handle's buffers was enqueued on `s`, so
// that dbm_destroy can wait for it.  Not while `s` is being captured into a
// graph (the work then runs when the caller launches the graph).
void note_work(dbm_t *h, cudaStream_t s)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    cudaEventRecord(h->done, s);
}

// cuTensorMapEncodeTiled from the driver, looked up once (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor maps of one parity's inputs: f as (nr, ntheta, 33) and lambda as
// (nr, ntheta) with row stride ld, box = one row of W + 2 halo columns (all
// 33 planes for f).  The row padding [nr, ld) lies outside the maps: a box
// that overhangs the last radial site is filled with zeros there instead of
// reading the padding from memory (no site reads beyond nr - 1).
template <typename real>
bool encode_maps(const dbm_t *h, StepArgs<real> &A)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt =
        sizeof(real) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const cuuint64_t e = sizeof(real);
    const cuuint32_t bx = (cuuint32_t)(h->ki.W + 2 * h->ki.halo);
    const cuuint64_t gdim3[3] = {(cuuint64_t)h->p.nr, (cuuint64_t)h->p.ntheta, (cuuint64_t)NV};
    const cuuint64_t gstr3[2] = {(cuuint64_t)h->ld * e, (cuuint64_t)h->ld * h->p.ntheta * e};
    const cuuint32_t box3[3] = {bx, 1, (cuuint32_t)NV};
    const cuuint32_t one3[3] = {1, 1, 1};
    if (enc(&A.tm_f, dt, 3, (void *)A.f_in, gdim3, gstr3, box3, one3, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t gdim2[2] = {(cuuint64_t)h->p.nr, (cuuint64_t)h->p.ntheta};
    const cuuint64_t gstr2[1] = {(cuuint64_t)h->ld * e};
    const cuuint32_t box2[2] = {bx, 1};
    return enc(&A.tm_lam, dt, 2, (void *)A.lam_in, gdim2, gstr2, box2, one3, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename real>
void fill_step_args(dbm_t *h, StepArgs<real> (&a)[2])
{
    const dbm_params &p = h->p;
    const double dr = (p.r_out - p.r_in) / p.nr;
    const double dth = theta_span(p) / p.ntheta;
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
        A.c.reaction_energy = p.reaction_energy;
        A.c.general_pow = (p.m == 1.0 && p.n == 1.0) ? 0 : 1;
        A.c.sector = p.sector;
        A.c.centre = p.r_bc_inner == DBM_BC_CENTRE ? (p.sector ? 1 : 2) : 0;
        A.c.cr_scale = (real)(p.dt / dr);
        A.c.ct_scale = (real)(p.dt / dth);
        // 1 - E is taken from the rounded E (exact for E >= 1/2), so the two
        // weights of the BGK step sum to exactly 1 in `real`: independently
        // rounded they miss 1 by up to half an ulp, a relative mass error of
        // that size at every site and step with one sign, which is what
        // limits FP32 over long runs with small dt / tau
        A.c.decay = (real)std::exp(-p.dt / p.tau);
        A.c.one_m_decay = (real)1 - A.c.decay;
        A.c.dt = (real)p.dt;
        A.c.inv_dt = (real)(1.0 / p.dt);
        A.c.Q = (real)p.Q;
        A.c.omega1 = (real)p.omega1;
        A.c.omega2 = (real)p.omega2;
        A.c.m_exp = (real)p.m;
        A.c.n_exp = (real)p.n;
        A.c.T_th = (real)p.T_th;
        for (int k = 0; k < 4; ++k) {
            A.c.v[k] = (real)p.v[k];
            A.c.v2[k] = (real)(p.v[k] * p.v[k]);
            for (int c = 0; c < 4; ++c) A.c.Fc[k][c] = (real)Fc[k][c];
        }
    }
    h->tmap_ok = encode_maps(h, a[0]) && encode_maps(h, a[1]);
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
    cudaError_t e = h->p.precision == DBM_FP64 ? launch_step<double>(h->variant, h->a64[b], h->grid, s)
                                               : launch_step<float>(h->variant, h->a32[b], h->grid, s);
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

// Size classes of the autotuner: precision x ceil(log2 nr) x ceil(log2 ntheta).
std::mutex g_tune_mu;
std::map<long long, int> g_tuned;

long long size_class(const dbm_params &p)
{
    auto lg = [](int x) {
        int l = 0;
        while ((1LL << l) < x) ++l;
        return l;
    };
    return ((long long)p.precision << 16) | ((long long)lg(p.nr) << 8) | lg(p.ntheta);
}

int pick_variant(const dbm_params &p)
{
    if (p.variant > 0) return p.variant;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(size_class(p));
        if (it != g_tuned.end()) return it->second;
    }
    return p.precision == DBM_FP64 ? default_variant<double>() : default_variant<float>();
}

// Launch shape for a kernel variant: persistent CTAs, one per resident slot,
// and the rows per item above unless the parameters fix them.
int configure_launch(dbm_t *h, int variant)
{
    KernelInfo ki;
    cudaError_t e = h->p.precision == DBM_FP64 ? kernel_info<double>(variant, &ki)
                                               : kernel_info<float>(variant, &ki);
    if (e != cudaSuccess) return cuda_fail(e, "kernel variant query");
    if (ki.blocks_per_sm < 1) {
        snprintf(g_last_error, sizeof(g_last_error), "step kernel variant %d does not fit on an SM", variant);
        return DBM_ECUDA;
    }
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    const dbm_params &p = h->p;
    const int slots = nsm * ki.blocks_per_sm;
    int32_t L_rows = 0;
    int64_t n_items = 0;
    if (dbm_plan_items(p.nr, p.ntheta, ki.W, slots, p.rows_per_item, &L_rows, &n_items) != DBM_OK)
        return DBM_EINVAL;
    const KernelInfo old_ki = h->ki;
    h->ki = ki;
    if (p.precision == DBM_FP64)
        fill_step_args<double>(h, h->a64);
    else
        fill_step_args<float>(h, h->a32);
    if (ki.version == 3 && !h->tmap_ok) {  // tensor maps not encodable for this grid
        h->ki = old_ki;
        if (old_ki.W) {
            if (p.precision == DBM_FP64)
                fill_step_args<double>(h, h->a64);
            else
                fill_step_args<float>(h, h->a32);
        }
        snprintf(g_last_error, sizeof(g_last_error), "variant %d needs tensor maps, not available here", variant);
        return DBM_EINVAL;
    }
    h->variant = variant;
    h->rows_per_item = L_rows;
    h->items = (int)n_items;
    h->grid = std::min(h->items, slots);
    // the step arguments carry the launch shape too
    if (p.precision == DBM_FP64)
        fill_step_args<double>(h, h->a64);
    else
        fill_step_args<float>(h, h->a32);
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return DBM_OK;
}

}  // namespace

extern "C" {

const char *dbm_version(void) { return "dbm-gb300 1.0 (sm_103a)"; }

// Status bits of the device self-checks -> DBM_EDEVICE with a message.
static int device_check_status(int status)
{
    if (status & ST_SMEM_ALIGN) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "step kernel: dynamic shared memory not 128-byte aligned, step skipped");
        return DBM_EDEVICE;
    }
    if (status & ST_BOUNDS) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "step kernel (debug build): a copy or store out of bounds or misaligned was skipped");
        return DBM_EDEVICE;
    }
    return DBM_OK;
}

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
    case DBM_EDEVICE: return "device-side self-check failed";
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
    if (p->sector != 0 && p->sector != 1) return DBM_EINVAL;
    if (p->reserved != 0) return DBM_EINVAL;
    if (p->r_bc_outer != DBM_BC_OUTFLOW) return DBM_EINVAL;
    if (p->r_bc_inner == DBM_BC_CENTRE) {
        if (p->r_in != 0.0) return DBM_EINVAL;                 // the disc centre is at r = 0
        if (!p->sector && p->ntheta % 2 != 0) return DBM_EINVAL;  // full disc: row m + ntheta/2
    } else if (p->r_bc_inner != DBM_BC_OUTFLOW) {
        return DBM_EINVAL;
    }
    if (p->rows_per_item < 0 || p->variant < 0) return DBM_EINVAL;
    if (p->variant > (p->precision == DBM_FP64 ? num_variants<double>() : num_variants<float>()))
        return DBM_EINVAL;
    const bool disc = p->r_bc_inner == DBM_BC_CENTRE;
    if (!(disc ? p->r_in == 0.0 : finite_pos(p->r_in)) || !std::isfinite(p->r_out) ||
        p->r_out <= p->r_in)
        return DBM_EINVAL;
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
    const double dth = theta_span(*p) / p->ntheta;
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

int dbm_plan_items(int32_t nr, int32_t ntheta, int32_t width, int32_t slots, int32_t rows_requested,
                   int32_t *rows_per_item, int64_t *items)
{
    if (nr < 1 || ntheta < 1 || width < 1 || slots < 1 || rows_requested < 0) return DBM_EINVAL;
    const int64_t strips = ((int64_t)nr + width - 1) / width;
    int32_t L = ntheta;
    if (rows_requested > 0) {
        L = std::min(rows_requested, ntheta);
    } else {
        // every segment count per strip, each with its smallest rows per item
        int64_t best_cost = -1;
        for (int32_t segs = 1; segs <= ntheta; ++segs) {
            const int32_t rows = (ntheta + segs - 1) / segs;
            const int64_t n = strips * ((ntheta + rows - 1) / rows);
            const int64_t cost = (n + slots - 1) / slots * (rows + 2);
            if (best_cost < 0 || cost < best_cost) {
                L = rows;
                best_cost = cost;
            }
            if (rows == 1) break;
        }
    }
    if (rows_per_item) *rows_per_item = L;
    if (items) *items = strips * ((ntheta + L - 1) / L);
    return DBM_OK;
}

static void free_handle(dbm_t *h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->done) cudaEventDestroy(h->done);
    for (cudaEvent_t ev : h->chunk_ev)
        if (ev) cudaEventDestroy(ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    if (h->aux) cudaStreamDestroy(h->aux);
    delete h;
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
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming);
    for (cudaEvent_t &ev : h->chunk_ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_handle(h);
        return cuda_fail(e, "dbm_create: device query, events and streams");
    }
    const int v0 = pick_variant(*p);
    rc = configure_launch(h, v0);
    if (rc != DBM_OK && p->variant == 0) {  // chosen, not asked for: fall back to bulk copies
        const int fb = p->precision == DBM_FP64 ? fallback_variant<double>() : fallback_variant<float>();
        if (fb != v0) rc = configure_launch(h, fb);
    }
    if (rc != DBM_OK) {
        free_handle(h);
        return rc;
    }
    // cleared on the legacy stream, which the library's and the server's
    // non-blocking streams do not wait for: no device-wide synchronisation
    // (a server admits new simulations while a batched quantum runs)
    e = cudaMemset(dev_buf, 0, L.total);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
    if (e != cudaSuccess) {
        free_handle(h);
        return cuda_fail(e, "dbm_create: clear buffer");
    }
    rc = p->precision == DBM_FP64 ? upload_tables<double>(h) : upload_tables<float>(h);
    if (rc != DBM_OK) {
        free_handle(h);
        return rc;
    }
    *out = h;
    return DBM_OK;
}

int dbm_destroy(dbm_t *h)
{
    if (!h) return DBM_EINVAL;
    // the last work enqueued on the handle's buffers (its own calls, and
    // batched steps in which it was active) must finish before the caller
    // may reuse them
    const cudaError_t e = cudaEventSynchronize(h->done);
    free_handle(h);
    if (e != cudaSuccess) return cuda_fail(e, "dbm_destroy: wait for the handle's work");
    return DBM_OK;
}

}  // extern "C"

template <typename real>
static cudaError_t launch_init_as(dbm_t *h, const double *d_fields, cudaStream_t s, int m0, int m1)
{
    double Fc[4][4];
    weight_coeffs(h->p.v, Fc);
    InitArgs<real> A;
    std::memset(&A, 0, sizeof(A));
    A.fields = d_fields;
    A.f = reinterpret_cast<real *>(h->buf + h->L.f[0]);
    A.lam = reinterpret_cast<real *>(h->buf + h->L.lam[0]);
    A.rowtab = reinterpret_cast<const real *>(h->buf + h->L.rowtab);
    A.bad = bad_input_word(h);
    A.plane = h->plane;
    A.nr = h->p.nr;
    A.ntheta = h->p.ntheta;
    A.ld = h->ld;
    A.m0 = m0;
    A.m1 = m1;
    for (int k = 0; k < 4; ++k) {
        A.v[k] = (real)h->p.v[k];
        for (int c = 0; c < 4; ++c) A.Fc[k][c] = (real)Fc[k][c];
    }
    return launch_init<real>(A, s);
}

extern "C" {

// f = f^eq of the device fields into buffer 0 for theta rows [m0, m1); the
// kernel checks every value and sets the handle's bad-input word.
static int launch_init_rows(dbm_t *h, const double *d_fields, cudaStream_t s, int m0, int m1)
{
    const cudaError_t e = h->p.precision == DBM_FP64 ? launch_init_as<double>(h, d_fields, s, m0, m1)
                                                     : launch_init_as<float>(h, d_fields, s, m0, m1);
    if (e != cudaSuccess) return cuda_fail(e, "init kernel launch");
    return DBM_OK;
}

static int launch_init_from(dbm_t *h, const double *d_fields, cudaStream_t s)
{
    CK(cudaMemsetAsync(bad_input_word(h), 0, sizeof(int), s));
    const int rc = launch_init_rows(h, d_fields, s, 0, h->p.ntheta);
    if (rc != DBM_OK) return rc;
    h->cur = 0;
    h->steps = 0;
    return DBM_OK;
}

// Theta-row chunks of the host-array calls: their copies over the host link
// (about 200 GB/s) overlap the init or moments kernel of the neighbouring
// chunk, which runs on the handle's second stream.  Small grids are one chunk.
static int host_chunks(const dbm_t *h)
{
    const size_t bytes = (size_t)5 * h->p.nr * h->p.ntheta * sizeof(double);
    return (bytes >= ((size_t)32 << 20) && h->p.ntheta >= 16) ? 4 : 1;
}

int dbm_init_state(dbm_t *h, const double *rho, const double *ur, const double *uth,
                   const double *T, const double *lam, void *stream)
{
    if (!h || !rho || !ur || !uth || !T || !lam) return DBM_EINVAL;
    const size_t N = (size_t)h->p.nr * h->p.ntheta;
    const int nr = h->p.nr, nth = h->p.ntheta;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Stage the fields in the second f buffer (free before the first step);
    // the init kernel validates them on the GPU, and one synchronisation at
    // the end covers the copies (the host arrays may be reused on return)
    // and the validation result.  Chunk c's copies go on `stream`, its init
    // kernel on the second stream once they have landed, while chunk c + 1
    // is copied.
    double *stage = reinterpret_cast<double *>(h->buf + h->L.f[1]);
    const double *src[5] = {rho, ur, uth, T, lam};
    const int C = host_chunks(h);
    const int R = (nth + C - 1) / C;
    CK(cudaMemsetAsync(bad_input_word(h), 0, sizeof(int), s));
    for (int c = 0; c < C; ++c) {
        const int m0 = c * R, m1 = std::min(nth, m0 + R);
        if (m0 >= m1) break;
        const size_t off = (size_t)m0 * nr, cnt = (size_t)(m1 - m0) * nr;
        for (int f = 0; f < 5; ++f)
            CK(cudaMemcpyAsync(stage + f * N + off, src[f] + off, cnt * sizeof(double), cudaMemcpyHostToDevice, s));
        cudaStream_t ks = s;
        if (C > 1) {
            CK(cudaEventRecord(h->chunk_ev[c], s));
            CK(cudaStreamWaitEvent(h->aux, h->chunk_ev[c], 0));
            ks = h->aux;
        }
        const int rc = launch_init_rows(h, stage, ks, m0, m1);
        if (rc != DBM_OK) return rc;
    }
    if (C > 1) {
        CK(cudaEventRecord(h->join_ev, h->aux));
        CK(cudaStreamWaitEvent(s, h->join_ev, 0));
    }
    h->cur = 0;
    h->steps = 0;
    CK(cudaMemcpyAsync(&h->host_word[0], bad_input_word(h), sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    note_work(h, s);
    if (h->host_word[0] != 0) return bad_input_fail();
    return DBM_OK;
}

int dbm_init_state_device(dbm_t *h, const double *d_fields, void *stream)
{
    if (!h || !d_fields) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = launch_init_from(h, d_fields, s);
    if (rc == DBM_OK) note_work(h, s);
    return rc;
}

int dbm_step(dbm_t *h, int64_t nsteps, void *stream)
{
    if (!h || nsteps < 0) return DBM_EINVAL;
    NvtxRange range("dbm_step");
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
    note_work(h, s);
    return DBM_OK;
}

}  // extern "C"

template <typename real>
static cudaError_t launch_moments_as(dbm_t *h, double *d_out, double *partials, int grid, cudaStream_t s,
                                     int m0, int m1)
{
    const dbm_params &p = h->p;
    MomArgs<real> A;
    std::memset(&A, 0, sizeof(A));
    A.f = reinterpret_cast<const real *>(h->buf + h->L.f[h->cur]);
    A.lam = reinterpret_cast<const real *>(h->buf + h->L.lam[h->cur]);
    A.out = d_out;
    A.partials = partials;
    A.status = reinterpret_cast<int *>(h->buf + h->L.status);
    A.rowtab = reinterpret_cast<const real *>(h->buf + h->L.rowtab);
    A.plane = h->plane;
    A.nr = p.nr;
    A.ntheta = p.ntheta;
    A.ld = h->ld;
    A.r_in = p.r_in;
    A.dr = (p.r_out - p.r_in) / p.nr;
    A.dtheta = theta_span(p) / p.ntheta;
    A.th_over_pi = theta_span(p) / PI / p.ntheta;
    std::memcpy(A.v, p.v, sizeof(A.v));
    for (int k = 0; k < 4; ++k) {
        A.vr[k] = (real)p.v[k];
        A.v2r[k] = (real)(p.v[k] * p.v[k]);
    }
    A.m0 = m0;
    A.m1 = m1;
    return launch_moments<real>(A, grid, s);
}

extern "C" {

// Moments of theta rows [m0, m1) into d_out, their per-block partial sums at
// partial slot *slot0 onwards (advanced past them), at most max_blocks blocks.
static int launch_moments_rows(dbm_t *h, double *d_out, cudaStream_t s, int m0, int m1, int max_blocks,
                               int *slot0)
{
    const long long n = (long long)h->p.nr * (m1 - m0);
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, max_blocks));
    double *partials = reinterpret_cast<double *>(h->buf + h->L.partials) + (size_t)*slot0 * 4;
    const cudaError_t e = h->p.precision == DBM_FP64 ? launch_moments_as<double>(h, d_out, partials, grid, s, m0, m1)
                                                     : launch_moments_as<float>(h, d_out, partials, grid, s, m0, m1);
    if (e != cudaSuccess) return cuda_fail(e, "moments kernel launch");
    *slot0 += grid;
    return DBM_OK;
}

static int launch_totals_of(dbm_t *h, int nblocks, cudaStream_t s)
{
    const cudaError_t e = launch_totals(reinterpret_cast<double *>(h->buf + h->L.partials), nblocks,
                                        reinterpret_cast<double *>(h->buf + h->L.totals), s);
    if (e != cudaSuccess) return cuda_fail(e, "totals kernel launch");
    return DBM_OK;
}

static int launch_moments_into(dbm_t *h, double *d_out, cudaStream_t s)
{
    int nblocks = 0;
    int rc = launch_moments_rows(h, d_out, s, 0, h->p.ntheta, MOMENT_BLOCKS, &nblocks);
    if (rc != DBM_OK) return rc;
    return launch_totals_of(h, nblocks, s);
}

static int launch_noneq_into(dbm_t *h, double *d_out, cudaStream_t s)
{
    const dbm_params &p = h->p;
    const long long N = (long long)p.nr * p.ntheta;
    const int grid = (int)std::min<long long>((N + 255) / 256, 4096);
    cudaError_t e;
    if (p.precision == DBM_FP64) {
        MomArgs<double> A;
        std::memset(&A, 0, sizeof(A));
        A.f = reinterpret_cast<const double *>(h->buf + h->L.f[h->cur]);
        A.out = d_out;
        A.plane = h->plane;
        A.nr = p.nr;
        A.ntheta = p.ntheta;
        A.ld = h->ld;
        A.th_over_pi = theta_span(p) / PI / p.ntheta;
        std::memcpy(A.v, p.v, sizeof(A.v));
        A.m0 = 0;
        A.m1 = p.ntheta;
        e = launch_noneq<double>(A, grid, s);
    } else {
        MomArgs<float> A;
        std::memset(&A, 0, sizeof(A));
        A.f = reinterpret_cast<const float *>(h->buf + h->L.f[h->cur]);
        A.out = d_out;
        A.plane = h->plane;
        A.nr = p.nr;
        A.ntheta = p.ntheta;
        A.ld = h->ld;
        A.th_over_pi = theta_span(p) / PI / p.ntheta;
        std::memcpy(A.v, p.v, sizeof(A.v));
        A.m0 = 0;
        A.m1 = p.ntheta;
        e = launch_noneq<float>(A, grid, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "noneq kernel launch");
    return DBM_OK;
}

int dbm_noneq_device(dbm_t *h, double *d_out, void *stream)
{
    if (!h || !d_out) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = launch_noneq_into(h, d_out, s);
    if (rc == DBM_OK) note_work(h, s);
    return rc;
}

int dbm_noneq(dbm_t *h, double *out, void *stream)
{
    if (!h || !out) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t N = (size_t)h->p.nr * h->p.ntheta;
    // staging: the free f buffer holds 33 planes >= 12 doubles per site
    double *stage = reinterpret_cast<double *>(h->buf + h->L.f[1 - h->cur]);
    int rc = launch_noneq_into(h, stage, s);
    if (rc != DBM_OK) return rc;
    CK(cudaMemcpyAsync(out, stage, 12 * N * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return DBM_OK;
}

int dbm_moments_device(dbm_t *h, double *d_out, void *stream)
{
    if (!h || !d_out) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rc = launch_moments_into(h, d_out, s);
    if (rc == DBM_OK) note_work(h, s);
    return rc;
}

int dbm_moments(dbm_t *h, double *rho, double *ur, double *uth, double *T, double *lam,
                double totals[4], void *stream)
{
    if (!h) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t N = (size_t)h->p.nr * h->p.ntheta;
    const int nr = h->p.nr, nth = h->p.ntheta;
    double *stage = reinterpret_cast<double *>(h->buf + h->L.f[1 - h->cur]);
    double *dst[5] = {rho, ur, uth, T, lam};
    // Chunk c's moments kernel on `stream`; its copies to the host arrays on
    // the second stream once it is done, while chunk c + 1 is computed.
    const int C = host_chunks(h);
    const int R = (nth + C - 1) / C;
    int nblocks = 0;
    for (int c = 0; c < C; ++c) {
        const int m0 = c * R, m1 = std::min(nth, m0 + R);
        if (m0 >= m1) break;
        int rc = launch_moments_rows(h, stage, s, m0, m1, MOMENT_BLOCKS / C, &nblocks);
        if (rc != DBM_OK) return rc;
        cudaStream_t cs = s;
        if (C > 1) {
            CK(cudaEventRecord(h->chunk_ev[c], s));
            CK(cudaStreamWaitEvent(h->aux, h->chunk_ev[c], 0));
            cs = h->aux;
        }
        const size_t off = (size_t)m0 * nr, cnt = (size_t)(m1 - m0) * nr;
        for (int f = 0; f < 5; ++f)
            if (dst[f])
                CK(cudaMemcpyAsync(dst[f] + off, stage + f * N + off, cnt * sizeof(double), cudaMemcpyDeviceToHost, cs));
    }
    int rc = launch_totals_of(h, nblocks, s);
    if (rc != DBM_OK) return rc;
    if (totals)
        CK(cudaMemcpyAsync(totals, h->buf + h->L.totals, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->host_word, h->buf + h->L.status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (C > 1) {
        CK(cudaEventRecord(h->join_ev, h->aux));
        CK(cudaStreamWaitEvent(s, h->join_ev, 0));
    }
    CK(cudaStreamSynchronize(s));
    const int status = h->host_word[0];
    if (status & ST_WAIT_TIMEOUT) return DBM_ETIMEOUT;
    if (device_check_status(status) != DBM_OK) return DBM_EDEVICE;
    if (h->host_word[1] != 0) return bad_input_fail();
    if (status & ST_NONFINITE) {
        CK(cudaMemsetAsync(h->buf + h->L.status, 0, sizeof(int), s));
        CK(cudaStreamSynchronize(s));
        return DBM_ENONFINITE;
    }
    return DBM_OK;
}

int64_t dbm_steps_done(const dbm_t *h) { return h ? h->steps : -1; }

int dbm_state_device(const dbm_t *h, const void **d_f, const void **d_lam, int64_t *ld)
{
    if (!h) return DBM_EINVAL;
    if (d_f) *d_f = h->buf + h->L.f[h->cur];
    if (d_lam) *d_lam = h->buf + h->L.lam[h->cur];
    if (ld) *ld = h->ld;
    return DBM_OK;
}

int dbm_status(dbm_t *h, void *stream)
{
    if (!h) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaMemcpyAsync(h->host_word, h->buf + h->L.status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int status = h->host_word[0];
    if (status & ST_WAIT_TIMEOUT) return DBM_ETIMEOUT;
    const int rc = device_check_status(status);
    if (rc != DBM_OK) return rc;
    if (h->host_word[1] != 0) return bad_input_fail();
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
                    int *items, int *variant)
{
    if (!h) return DBM_EINVAL;
    if (grid) *grid = h->grid;
    if (variant) *variant = h->variant;
    if (threads) *threads = h->ki.threads;
    if (smem_bytes) *smem_bytes = h->ki.smem;
    if (rows_per_item) *rows_per_item = h->rows_per_item;
    if (items) *items = h->items;
    return DBM_OK;
}

int dbm_selftest_rcp(const float *d_x, float *d_approx, float *d_ieee, int n, void *stream)
{
    if (!d_x || !d_approx || !d_ieee || n < 0) return DBM_EINVAL;
    cudaError_t e = launch_rcp_selftest(d_x, d_approx, d_ieee, n, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rcp self-test launch");
    return DBM_OK;
}

int dbm_selftest_wait(int *d_status, int arrive, int64_t limit_cycles, void *stream)
{
    if (!d_status || limit_cycles < 1 || limit_cycles > kWaitLimitCycles) return DBM_EINVAL;
    cudaError_t e = launch_wait_selftest(d_status, arrive ? 1 : 0, (long long)limit_cycles,
                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test launch");
    return DBM_OK;
}

int dbm_num_variants(int precision)
{
    if (precision == DBM_FP32) return num_variants<float>();
    if (precision == DBM_FP64) return num_variants<double>();
    return 0;
}

int dbm_set_variant(dbm_t *h, int variant)
{
    if (!h || variant < 1 || variant > dbm_num_variants(h->p.precision)) return DBM_EINVAL;
    return configure_launch(h, variant);
}

int dbm_autotune(dbm_t *h, int steps, void *stream, int *best, float *ms_per_step)
{
    if (!h || steps < 1) return DBM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nv = dbm_num_variants(h->p.precision);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int bestv = 0;
    float bestms = 0.f;
    int rc = DBM_OK;
    for (int v = 1; v <= nv && rc == DBM_OK; ++v) {
        if (configure_launch(h, v) != DBM_OK) {  // not available for this grid
            if (ms_per_step) ms_per_step[v - 1] = 0.f;
            continue;
        }
        // two untimed steps, then `steps` timed single launches
        for (int k = 0; k < 2 && rc == DBM_OK; ++k) {
            rc = launch_one(h, h->cur, s);
            h->cur ^= 1;
            h->steps += 1;
        }
        if (rc != DBM_OK) break;
        cudaEventRecord(e0, s);
        for (int k = 0; k < steps && rc == DBM_OK; ++k) {
            rc = launch_one(h, h->cur, s);
            h->cur ^= 1;
            h->steps += 1;
        }
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= steps;
        if (ms_per_step) ms_per_step[v - 1] = ms;
        if (bestv == 0 || ms < bestms) {
            bestv = v;
            bestms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != DBM_OK) return rc;
    rc = configure_launch(h, bestv);
    if (rc != DBM_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[size_class(h->p)] = bestv;
    }
    if (best) *best = bestv;
    return DBM_OK;
}

}  // extern "C"

// ===========================================================================
// Batches: many uneven instances advanced by one persistent launch per step.
// ===========================================================================
struct dbm_batch_s {
    int precision;
    int max_slots;
    long long max_items;
    int rows_per_item;
    unsigned char *buf;
    size_t bytes;
    size_t off_slots, off_items, off_nitems, off_T, total;
    size_t slot_bytes;
    std::vector<dbm_t *> inst;
    std::vector<long long> start, end;
    std::vector<int> par0;
    unsigned char *stage;     // pinned host staging of the slot and item tables
    cudaEvent_t stage_ev;
    cudaEvent_t done;         // recorded after the last batched steps enqueued
    int cbase;                // first entry of the batch constant table held (-1: none)
    int device;
    unsigned char *cstage;    // pinned host staging of the slots' constants
    bool stage_pending;
    long long T;              // host mirror of the device step counter
    int n_items;
    bool dirty;
    KernelInfo ki;
    int variant;
    int forced_variant;       // 0: the precision's default (set by dbm_batch_autotune)
    int grid;
    int nsm;
    cudaGraphExec_t graph;    // GRAPH_STEPS batch steps + counter advance
};

namespace {

void note_batch_work(dbm_batch_t *b, cudaStream_t s)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    cudaEventRecord(b->done, s);
}

struct BatchLayout {
    size_t slot_bytes, slots, items, nitems, T, total;
};

// Theta rows per work item of one attached simulation: the batch's setting,
// or with rows_per_item = -1 scaled to the simulation's size (16 up to 512
// rows, 32 up to 1024, else 64): long items carry fewer halo rows per row
// computed, short ones balance better.
int batch_rows(const dbm_batch_t *b, const dbm_params &p)
{
    if (b->rows_per_item > 0) return b->rows_per_item;
    int L = 16;
    while (L < 64 && L * 32 < p.ntheta) L *= 2;
    return L;
}

BatchLayout batch_layout(int max_slots, long long max_items, int precision)
{
    BatchLayout L;
    L.slot_bytes = precision == DBM_FP64 ? sizeof(BatchSlot<double>) : sizeof(BatchSlot<float>);
    size_t off = 0;
    L.slots = off;
    off = align256(off + (size_t)max_slots * L.slot_bytes);
    L.items = off;
    off = align256(off + (size_t)max_items * sizeof(int4));
    L.nitems = off;
    off = align256(off + sizeof(int));
    L.T = off;
    off = align256(off + sizeof(long long));
    L.total = off;
    return L;
}

// Entries of the batch constant tables (one per precision), per device:
// each batch holds a contiguous range of max_slots entries.
std::mutex g_const_mu;
std::map<std::pair<int, int>, std::vector<char>> g_const_used;  // (device, precision) -> used flags

int const_alloc(int device, int precision, int n)
{
    std::lock_guard<std::mutex> lock(g_const_mu);
    const int cap = precision == DBM_FP64 ? batch_const_capacity<double>() : batch_const_capacity<float>();
    std::vector<char> &used = g_const_used[{device, precision}];
    used.resize(cap, 0);
    for (int first = 0; first + n <= cap; ++first) {
        int k = 0;
        while (k < n && !used[first + k]) ++k;
        if (k == n) {
            std::fill(used.begin() + first, used.begin() + first + n, 1);
            return first;
        }
        first += k;
    }
    return -1;
}

void const_free(int device, int precision, int first, int n)
{
    std::lock_guard<std::mutex> lock(g_const_mu);
    std::vector<char> &used = g_const_used[{device, precision}];
    for (int k = first; k < first + n && k < (int)used.size(); ++k) used[k] = 0;
}

template <typename real>
void fill_slot(dbm_batch_t *b, int s, unsigned char *dst)
{
    BatchSlot<real> sl;
    std::memset(&sl, 0, sizeof(sl));
    sl.cidx = b->cbase + s;
    StepConsts<real> *cst = reinterpret_cast<StepConsts<real> *>(b->cstage) + s;
    std::memset(cst, 0, sizeof(*cst));
    if (b->inst[s]) {
        const StepArgs<real> *a;
        if constexpr (std::is_same<real, double>::value)
            a = b->inst[s]->a64;
        else
            a = b->inst[s]->a32;
        sl.args[0] = a[0];
        sl.args[1] = a[1];
        *cst = a[0].c;
        sl.start = b->start[s];
        sl.end = b->end[s];
        sl.par0 = b->par0[s];
    } else {
        sl.start = 0;
        sl.end = 0;  // never active
    }
    std::memcpy(dst, &sl, sizeof(sl));
}

// Static load balance of the batch's work items over the persistent CTAs.
// CTA c runs items c, c + grid, c + 2 grid, ...  Items differ in cost: a strip
// that overhangs its instance's last radial site has idle lanes, and the
// ragged last run of rows is short.  Longest-processing-time-first: items in
// decreasing estimated cost (ties keep the interleaved order), each to the
// least loaded CTA; then laid out so CTA c finds its k-th item at k grid + c,
// padding with empty items (slot -1).  Cost estimate of an item of L rows and
// a active lanes of W: (L + 2) (0.3 + 0.7 a / W): every row moves through the
// CTA's pipeline, and the update time grows with the active lanes.  Returns
// the items in launch order; keeps the interleaved order if the padded table
// would exceed max_items.
struct PlanItem {
    int32_t slot, j0, mb, me;  // simulation, first radial site, theta rows [mb, me)
};
static_assert(sizeof(PlanItem) == sizeof(int4), "a plan item is one int4 of the device item table");

std::vector<PlanItem> balance_items(const std::vector<PlanItem> &items, int grid, int W, const int32_t *nr,
                                    long long max_items)
{
    const long long n = (long long)items.size();
    if (n <= grid || grid < 1) return items;
    std::vector<double> cost(n);
    for (long long i = 0; i < n; ++i) {
        const PlanItem &e = items[i];
        const int active = std::min(W, nr[e.slot] - e.j0);
        cost[i] = (double)(e.me - e.mb + 2) * (0.3 + 0.7 * (double)active / W);
    }
    std::vector<long long> order(n);
    for (long long i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](long long a, long long c) { return cost[a] > cost[c]; });
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int c = 0; c < grid; ++c) heap.push({0.0, c});
    std::vector<std::vector<PlanItem>> bins(grid);
    for (long long i : order) {
        Load l = heap.top();
        heap.pop();
        bins[l.second].push_back(items[i]);
        heap.push({l.first + cost[i], l.second});
    }
    size_t K = 0;
    for (const auto &bin : bins) K = std::max(K, bin.size());
    const long long total = (long long)K * grid;
    if (total > max_items) return items;
    std::vector<PlanItem> out((size_t)total);
    for (size_t k = 0; k < K; ++k)
        for (int c = 0; c < grid; ++c)
            out[k * grid + c] = k < bins[c].size() ? bins[c][k] : PlanItem{-1, 0, 0, 0};
    return out;
}

int batch_launch(dbm_batch_t *b, int s, cudaStream_t st)
{
    cudaError_t e;
    if (b->precision == DBM_FP64) {
        BatchArgs<double> B{reinterpret_cast<const BatchSlot<double> *>(b->buf + b->off_slots),
                            reinterpret_cast<const int4 *>(b->buf + b->off_items),
                            reinterpret_cast<const int *>(b->buf + b->off_nitems),
                            reinterpret_cast<const long long *>(b->buf + b->off_T), s};
        e = launch_batch_step<double>(b->variant, B, b->grid, st);
    } else {
        BatchArgs<float> B{reinterpret_cast<const BatchSlot<float> *>(b->buf + b->off_slots),
                           reinterpret_cast<const int4 *>(b->buf + b->off_items),
                           reinterpret_cast<const int *>(b->buf + b->off_nitems),
                           reinterpret_cast<const long long *>(b->buf + b->off_T), s};
        e = launch_batch_step<float>(b->variant, B, b->grid, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch step kernel launch");
    return DBM_OK;
}

int batch_advance(dbm_batch_t *b, int k, cudaStream_t st)
{
    cudaError_t e = launch_batch_advance(reinterpret_cast<long long *>(b->buf + b->off_T), k, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch advance launch");
    return DBM_OK;
}

int batch_build_graph(dbm_batch_t *b)
{
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = DBM_OK;
    if (e == cudaSuccess) {
        for (int s = 0; s < GRAPH_STEPS && rc == DBM_OK; ++s) rc = batch_launch(b, s, cs);
        if (rc == DBM_OK) rc = batch_advance(b, GRAPH_STEPS, cs);
        e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess && rc == DBM_OK) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc != DBM_OK) return rc;
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return cuda_fail(e, "batch graph capture");
    }
    return DBM_OK;
}

// Host bookkeeping of an attached instance after the clock moved t0 -> t1.
void batch_account(dbm_batch_t *b, int s, long long t0, long long t1)
{
    dbm_t *h = b->inst[s];
    if (!h) return;
    const long long a0 = std::min(std::max(t0, b->start[s]), b->end[s]);
    const long long a1 = std::min(std::max(t1, b->start[s]), b->end[s]);
    h->steps += a1 - a0;
    h->cur = (int)((b->par0[s] + (a1 - b->start[s])) & 1);
}

}  // namespace

extern "C" {

size_t dbm_batch_bytes(int max_slots, int64_t max_items, int precision)
{
    if (max_slots < 1 || max_items < 1 || (precision != DBM_FP32 && precision != DBM_FP64)) return 0;
    return batch_layout(max_slots, max_items, precision).total;
}

int dbm_batch_plan(int32_t nslots, const int32_t *nr, const int32_t *ntheta, const int32_t *rows_per_item,
                   int32_t width, int32_t grid, int64_t max_items, int32_t *items, int64_t *n_items)
{
    if (nslots < 0 || width < 1 || grid < 1 || max_items < 0 || !n_items ||
        (nslots > 0 && (!nr || !ntheta || !rows_per_item)))
        return DBM_EINVAL;
    *n_items = 0;
    std::vector<long long> strips(nslots, 0), count(nslots, 0);
    long long n = 0;
    for (int s = 0; s < nslots; ++s) {
        if (nr[s] == 0) continue;  // empty slot
        if (nr[s] < 0 || ntheta[s] < 1 || rows_per_item[s] < 1) return DBM_EINVAL;
        strips[s] = (nr[s] + width - 1) / width;
        count[s] = strips[s] * ((ntheta[s] + rows_per_item[s] - 1) / rows_per_item[s]);
        n += count[s];
    }
    if (n > max_items) return DBM_ENOMEM;
    // interleave the simulations' items so every CTA gets a share of each
    std::vector<PlanItem> list;
    list.reserve((size_t)n);
    std::vector<long long> cursor(nslots, 0);
    for (bool more = true; more;) {
        more = false;
        for (int s = 0; s < nslots; ++s) {
            if (cursor[s] >= count[s]) continue;
            const long long it = cursor[s]++;
            const int strip = (int)(it % strips[s]), seg = (int)(it / strips[s]);
            const int mb = seg * rows_per_item[s];
            list.push_back({s, strip * width, mb, std::min(mb + rows_per_item[s], ntheta[s])});
            more = true;
        }
    }
    const std::vector<PlanItem> out = balance_items(list, grid, width, nr, max_items);
    if (items && !out.empty()) std::memcpy(items, out.data(), out.size() * sizeof(PlanItem));
    *n_items = (int64_t)out.size();
    return DBM_OK;
}

int dbm_batch_create(int max_slots, int64_t max_items, int precision, int rows_per_item,
                     void *dev_buf, size_t dev_bytes, dbm_batch_t **out)
{
    if (!out || !dev_buf || max_slots < 1 || max_items < 1 || max_items > (1LL << 31) ||
        rows_per_item < -1 || (precision != DBM_FP32 && precision != DBM_FP64))
        return DBM_EINVAL;
    *out = nullptr;
    if (((uintptr_t)dev_buf & 255) != 0) return DBM_EINVAL;
    const BatchLayout L = batch_layout(max_slots, max_items, precision);
    if (dev_bytes < L.total) return DBM_ENOMEM;
    dbm_batch_t *b = new (std::nothrow) dbm_batch_t();
    if (!b) return DBM_ENOMEM;
    b->precision = precision;
    b->max_slots = max_slots;
    b->max_items = max_items;
    b->rows_per_item = rows_per_item != 0 ? rows_per_item : 16;
    b->buf = static_cast<unsigned char *>(dev_buf);
    b->bytes = dev_bytes;
    b->off_slots = L.slots;
    b->off_items = L.items;
    b->off_nitems = L.nitems;
    b->off_T = L.T;
    b->total = L.total;
    b->slot_bytes = L.slot_bytes;
    b->inst.assign(max_slots, nullptr);
    b->start.assign(max_slots, 0);
    b->end.assign(max_slots, 0);
    b->par0.assign(max_slots, 0);
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    b->variant = precision == DBM_FP64 ? default_variant<double>() : default_variant<float>();
    if (e == cudaSuccess)
        e = precision == DBM_FP64 ? batch_kernel_info<double>(b->variant, &b->ki)
                                  : batch_kernel_info<float>(b->variant, &b->ki);
    if (e == cudaSuccess) e = cudaHostAlloc(&b->stage, L.items + (size_t)max_items * sizeof(int4) + 256,
                                            cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&b->cstage, (size_t)max_slots * sizeof(StepConsts<double>),
                                            cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->stage_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(dev_buf, 0, L.total);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    b->device = dev;
    b->cbase = e == cudaSuccess ? const_alloc(dev, precision, max_slots) : -1;
    if (e != cudaSuccess || b->cbase < 0) {
        if (b->stage) cudaFreeHost(b->stage);
        if (b->cstage) cudaFreeHost(b->cstage);
        if (b->stage_ev) cudaEventDestroy(b->stage_ev);
        if (b->done) cudaEventDestroy(b->done);
        delete b;
        if (e == cudaSuccess) {
            snprintf(g_last_error, sizeof(g_last_error),
                     "dbm_batch_create: the batch constant table has no %d free entries on this device "
                     "(%d in all for this precision, shared by the live batches)", max_slots,
                     precision == DBM_FP64 ? batch_const_capacity<double>() : batch_const_capacity<float>());
            return DBM_ENOMEM;
        }
        return cuda_fail(e, "dbm_batch_create");
    }
    b->nsm = nsm;
    b->grid = nsm * std::max(1, b->ki.blocks_per_sm);
    b->dirty = true;
    *out = b;
    return DBM_OK;
}

int dbm_batch_destroy(dbm_batch_t *b)
{
    if (!b) return DBM_EINVAL;
    if (b->stage_pending) cudaEventSynchronize(b->stage_ev);
    cudaEventSynchronize(b->done);  // queued batched steps read the tables
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaEventDestroy(b->stage_ev);
    cudaEventDestroy(b->done);
    cudaFreeHost(b->stage);
    cudaFreeHost(b->cstage);
    const_free(b->device, b->precision, b->cbase, b->max_slots);
    delete b;
    return DBM_OK;
}

int dbm_batch_attach(dbm_batch_t *b, int slot, dbm_t *h, int64_t nsteps)
{
    if (!b || !h || slot < 0 || slot >= b->max_slots || nsteps < 0) return DBM_EINVAL;
    if (b->inst[slot]) return DBM_EBUSY;
    if (h->p.precision != b->precision) return DBM_EINVAL;
    for (int s = 0; s < b->max_slots; ++s)
        if (b->inst[s] == h) return DBM_EINVAL;
    b->inst[slot] = h;
    b->start[slot] = b->T;
    b->end[slot] = b->T + nsteps;
    b->par0[slot] = h->cur;
    b->dirty = true;
    return DBM_OK;
}

int dbm_batch_detach(dbm_batch_t *b, int slot)
{
    if (!b || slot < 0 || slot >= b->max_slots) return DBM_EINVAL;
    if (!b->inst[slot]) return DBM_ENOTFOUND;
    b->inst[slot] = nullptr;
    b->dirty = true;
    return DBM_OK;
}

int64_t dbm_batch_remaining(const dbm_batch_t *b, int slot)
{
    if (!b || slot < 0 || slot >= b->max_slots || !b->inst[slot]) return -1;
    return std::max(0LL, b->end[slot] - std::max(b->T, b->start[slot]));
}

int64_t dbm_batch_time(const dbm_batch_t *b) { return b ? b->T : -1; }

int dbm_batch_commit(dbm_batch_t *b, void *stream)
{
    if (!b) return DBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Kernel variant: the tensor-map default only if every attached instance
    // has its maps encoded with this kernel's tile width.
    {
        int v = b->forced_variant > 0 ? b->forced_variant
                : (b->precision == DBM_FP64 ? default_variant<double>() : default_variant<float>());
        KernelInfo ki;
        CK(b->precision == DBM_FP64 ? batch_kernel_info<double>(v, &ki) : batch_kernel_info<float>(v, &ki));
        bool maps_ok = true;
        for (int s = 0; s < b->max_slots; ++s)
            if (b->inst[s] && (!b->inst[s]->tmap_ok || b->inst[s]->ki.W != ki.W)) maps_ok = false;
        if (ki.version == 3 && !maps_ok) {
            v = b->precision == DBM_FP64 ? fallback_variant<double>() : fallback_variant<float>();
            CK(b->precision == DBM_FP64 ? batch_kernel_info<double>(v, &ki) : batch_kernel_info<float>(v, &ki));
        }
        if (v != b->variant) {
            if (b->graph) {  // captured with the other kernel
                CK(cudaStreamSynchronize(st));
                cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
            }
            b->variant = v;
            b->ki = ki;
            b->grid = b->nsm * std::max(1, ki.blocks_per_sm);
        }
    }
    // item table: W sites x rows_per_item rows of every attached instance
    long long n = 0;
    for (int s = 0; s < b->max_slots; ++s) {
        if (!b->inst[s]) continue;
        const dbm_params &p = b->inst[s]->p;
        const long long strips = (p.nr + b->ki.W - 1) / b->ki.W;
        const int L = batch_rows(b, p);
        const long long segs = (p.ntheta + L - 1) / L;
        n += strips * segs;
    }
    if (n > b->max_items) return DBM_ENOMEM;
    if (b->stage_pending) {
        CK(cudaEventSynchronize(b->stage_ev));
        b->stage_pending = false;
    }
    unsigned char *slots = b->stage;
    int4 *items = reinterpret_cast<int4 *>(b->stage + b->off_items);
    for (int s = 0; s < b->max_slots; ++s) {
        if (b->precision == DBM_FP64)
            fill_slot<double>(b, s, slots + (size_t)s * b->slot_bytes);
        else
            fill_slot<float>(b, s, slots + (size_t)s * b->slot_bytes);
    }
    std::vector<int32_t> nr(b->max_slots, 0), nth(b->max_slots, 0), rows(b->max_slots, 0);
    for (int s = 0; s < b->max_slots; ++s) {
        if (!b->inst[s]) continue;
        nr[s] = b->inst[s]->p.nr;
        nth[s] = b->inst[s]->p.ntheta;
        rows[s] = batch_rows(b, b->inst[s]->p);
    }
    int64_t planned = 0;
    const int rc = dbm_batch_plan(b->max_slots, nr.data(), nth.data(), rows.data(), b->ki.W, b->grid,
                                  b->max_items, reinterpret_cast<int32_t *>(items), &planned);
    if (rc != DBM_OK) return rc;
    n = planned;
    b->n_items = (int)n;
    std::memcpy(b->stage + b->off_nitems, &b->n_items, sizeof(int));
    CK(cudaMemcpyAsync(b->buf + b->off_slots, b->stage, (size_t)b->max_slots * b->slot_bytes,
                       cudaMemcpyHostToDevice, st));
    CK(b->precision == DBM_FP64
           ? upload_batch_consts<double>(b->cbase, reinterpret_cast<const StepConsts<double> *>(b->cstage),
                                         b->max_slots, st)
           : upload_batch_consts<float>(b->cbase, reinterpret_cast<const StepConsts<float> *>(b->cstage),
                                        b->max_slots, st));
    if (n > 0)
        CK(cudaMemcpyAsync(b->buf + b->off_items, b->stage + b->off_items, (size_t)n * sizeof(int4),
                           cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->buf + b->off_nitems, b->stage + b->off_nitems, sizeof(int),
                       cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(b->stage_ev, st));
    b->stage_pending = true;
    b->dirty = false;
    return DBM_OK;
}

int dbm_batch_step(dbm_batch_t *b, int64_t nsteps, void *stream)
{
    if (!b || nsteps < 0) return DBM_EINVAL;
    NvtxRange range("dbm_batch_step");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (b->dirty) {
        int rc = dbm_batch_commit(b, stream);
        if (rc != DBM_OK) return rc;
    }
    const long long t0 = b->T;
    while (nsteps > 0) {
        int rc;
        if (nsteps >= GRAPH_STEPS) {
            if (!b->graph) {
                rc = batch_build_graph(b);
                if (rc != DBM_OK) return rc;
            }
            CK(cudaGraphLaunch(b->graph, st));
            nsteps -= GRAPH_STEPS;
            b->T += GRAPH_STEPS;
        } else {
            const int k = (int)nsteps;
            for (int s = 0; s < k; ++s) {
                rc = batch_launch(b, s, st);
                if (rc != DBM_OK) return rc;
            }
            rc = batch_advance(b, k, st);
            if (rc != DBM_OK) return rc;
            nsteps = 0;
            b->T += k;
        }
    }
    for (int s = 0; s < b->max_slots; ++s) {
        // a simulation active in these steps: its dbm_destroy waits for them
        if (b->inst[s] && b->start[s] < b->T && b->end[s] > t0) note_work(b->inst[s], st);
        batch_account(b, s, t0, b->T);
    }
    note_batch_work(b, st);
    return DBM_OK;
}

int dbm_batch_autotune(dbm_batch_t *b, int steps, void *stream, int *variant, int *rows_per_item,
                       float *ms_per_step)
{
    if (!b || steps < 1) return DBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int vdef = b->precision == DBM_FP64 ? default_variant<double>() : default_variant<float>();
    const int vfb = b->precision == DBM_FP64 ? fallback_variant<double>() : fallback_variant<float>();
    const int vs[2] = {vdef, vfb};
    const int rows[4] = {16, 32, 64, -1};  // -1: scaled to each simulation's size
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int rc = DBM_OK, bestv = 0, bestr = 0;
    float bestms = 0.f;
    for (int c = 0; c < 8 && rc == DBM_OK; ++c) {
        const int v = vs[c / 4], r = rows[c % 4];
        if (ms_per_step) ms_per_step[c] = 0.f;
        if (c >= 4 && vfb == vdef) continue;
        b->forced_variant = v;
        b->rows_per_item = r;
        b->dirty = true;
        rc = dbm_batch_step(b, GRAPH_STEPS, stream);  // commit, graph capture, warm-up
        if (rc != DBM_OK) break;
        if (b->variant != v) continue;  // the tensor-map kernel is not usable for this batch
        float ms = 0.f;
        for (int rep = 0; rep < 2 && rc == DBM_OK; ++rep) {  // the better of two timings
            cudaEventRecord(e0, st);
            rc = dbm_batch_step(b, steps, stream);
            cudaEventRecord(e1, st);
            if (rc != DBM_OK) break;
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "batch autotune timing");
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            t /= steps;
            if (rep == 0 || t < ms) ms = t;
        }
        if (rc != DBM_OK) break;
        if (ms_per_step) ms_per_step[c] = ms;
        if (bestv == 0 || ms < bestms) {
            bestv = v;
            bestr = r;
            bestms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != DBM_OK) return rc;
    if (bestv == 0) return DBM_ECUDA;
    b->forced_variant = bestv;
    b->rows_per_item = bestr;
    b->dirty = true;
    rc = dbm_batch_commit(b, stream);
    if (rc != DBM_OK) return rc;
    if (variant) *variant = bestv;
    if (rows_per_item) *rows_per_item = bestr;
    return DBM_OK;
}

int dbm_batch_launch_info(const dbm_batch_t *b, int *grid, int *items, int *rows_per_item,
                          int *variant)
{
    if (!b) return DBM_EINVAL;
    if (variant) *variant = b->variant;
    if (grid) *grid = b->grid;
    if (items) *items = b->n_items;
    if (rows_per_item) *rows_per_item = b->rows_per_item;
    return DBM_OK;
}

}  // extern "C"
