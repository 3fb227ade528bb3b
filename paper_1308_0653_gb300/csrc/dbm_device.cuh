// Device code of the polar-coordinate discrete-Boltzmann detonation update
// (Lin, Xu, Zhang, Li, arXiv:1308.0653) for sm_103a.
//
// Data layout in HBM (one instance):
//   f[v][theta][ld]   33 planes, row length ld = nr rounded up to 32 elements,
//                     r contiguous (coalesced 128-byte rows)
//   lam[theta][ld]    reaction variable: lambda (FP64) or 1 - lambda (FP32,
//                     see LamStore)
//   rowtab[theta][16] cos(i pi/4 - theta_m), sin(i pi/4 - theta_m), i = 0..7
//   inv_r[ld]         1 / r_j at cell centres
//
// The fused step kernel is persistent: each CTA owns W consecutive radial
// sites (one per thread) of a run of theta rows ("work item") and marches down
// the rows.  A ring of NSTAGE shared-memory row buffers, each holding all 33
// f planes plus lambda for the strip and a 16-byte halo on both radial sides,
// is filled by TMA (tensor-map tiles, cp.async.bulk.tensor, in the default
// variant; per-array cp.async.bulk in the others), completion on an mbarrier
// per buffer.  Row m is computed from buffers m-1, m, m+1, so every f value
// is read from HBM once per step (plus the halo columns and two halo rows per
// item) and written once.  Variant v1 (march) uses one CTA-wide barrier per
// row; v2/v3 (march2) a producer warp and full/empty mbarriers.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; descriptors are encoded by the host runtime)
#include <cuda_runtime.h>
#include <stdint.h>

namespace dbm {

constexpr int NV = 33;    // D2V33 velocities (Sec. II.B)
constexpr int NARR = 34;  // 33 f planes + lambda

// Status bits written by kernels into the instance's status word.
constexpr int ST_WAIT_TIMEOUT = 1;   // an mbarrier wait gave up
constexpr int ST_NONFINITE = 2;      // a moment was NaN / inf (moments kernel)
constexpr int ST_SMEM_ALIGN = 4;     // dynamic shared memory not 128-byte aligned (step skipped)
constexpr int ST_BOUNDS = 8;         // DBM_DEBUG builds: a copy or store failed its bounds check

// DBM_DEBUG builds check every copy the producer issues (tensor coordinates on
// the 16-byte boundary TMA requires, rows inside the grid, bulk extents inside
// the row and 16-byte aligned) and every global store of the update, and skip
// a failing one with ST_BOUNDS set; a skipped copy ends the step through the
// abort path, like an expired wait.  Release builds compile the checks out.
#ifdef DBM_DEBUG
#define DBM_DEBUG_CHECK(cond, status_ptr) (dbm::debug_check((cond), (status_ptr)))
#else
#define DBM_DEBUG_CHECK(cond, status_ptr) (true)
#endif
__device__ __forceinline__ bool debug_check(bool ok, int *status)
{
    if (!ok) atomicOr(status, ST_BOUNDS);
    return ok;
}

template <typename real> struct Halo;
template <> struct Halo<float> { static constexpr int value = 4; };   // 16 bytes
template <> struct Halo<double> { static constexpr int value = 2; };  // 16 bytes

// Per-instance constants of the update (host-computed in double, rounded to
// real).  A single-instance launch reads them from its parameter block (the
// constant bank, as instruction operands); a batched launch reads them from
// a constant-memory table indexed by the item's slot.
template <typename real>
struct StepConsts {
    real cr_scale;        // dt / dr
    real ct_scale;        // dt / dtheta
    real decay;           // exp(-dt / tau)
    real one_m_decay;     // 1 - exp(-dt / tau)
    real dt, Q, omega1, omega2, m_exp, n_exp, T_th;
    real inv_dt;          // 1 / dt
    real v[4], v2[4];     // ring speeds and their squares
    real Fc[4][4];        // F_k(T) = T (Fc[k][0] + T (Fc[k][1] + T (Fc[k][2] + T Fc[k][3])))
    int reaction_energy;  // 0 explicit R, 1 consistent R
    int general_pow;      // 0: m = n = 1 (P^m = P), 1: pow()
    int sector;           // 1: pi/4 sector, theta wrap rotates velocities by one direction
    int centre;           // disc centre at r = 0: 1 in a sector (ghost j = -1 is j = 0 with
                          // i -> i+4), 2 on a full grid (ghost is j = 0 of row m + ntheta/2)
};

// Step arguments of one instance and one ping-pong parity.  The tensor maps
// describe this parity's input f as a 3-D tensor (ld, ntheta, 33) and lambda
// as 2-D (ld, ntheta), with a box of one row of W + 2 HALO columns; they are
// used by the tensor-TMA variants.
template <typename real>
struct StepArgs {
    CUtensorMap tm_f;     // 128 B, 64-byte aligned
    CUtensorMap tm_lam;
    const real *f_in;
    real *f_out;
    const real *lam_in;
    real *lam_out;
    const real *rowtab;   // [ntheta][16]
    const real *inv_r;    // [ld]
    int *status;          // sticky status word
    long long plane;      // ntheta * ld (elements between f planes)
    int nr, ntheta, ld;
    int strips;           // ceil(nr / W)
    int rows_per_item;    // theta rows per work item
    int segs;             // ceil(ntheta / rows_per_item)
    int items;            // strips * segs
    StepConsts<real> c;
};

// Constant-memory table of the batched launches' per-slot constants (one
// per precision translation unit, defined there).
template <typename real> __device__ const StepConsts<real> &batch_consts(int i);

// ---------------------------------------------------------------------------
// PTX helpers (mbarrier + TMA bulk copy)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// A tensor map read from global memory (the batch slot table, written by host
// copies) must be made visible to the tensor-map proxy before the first
// tensor copy that uses it.
__device__ __forceinline__ void fence_tensormap_acquire(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~2^31 SM cycles (about a second) and reports false.
constexpr long long kWaitLimitCycles = 1LL << 31;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long limit = kWaitLimitCycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Barrier over the first `nthreads` threads only (id 1; id 0 is __syncthreads).
__device__ __forceinline__ void named_bar_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Tensor TMA: tile of a 3-D / 2-D tensor map at coordinates (x, y[, z]),
// x innermost; out-of-range elements are filled with zeros.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

template <typename real> __device__ __forceinline__ real rcp_(real x) { return real(1) / x; }

template <typename real> __device__ __forceinline__ real expm1_(real x);
template <> __device__ __forceinline__ float expm1_<float>(float x) { return expm1f(x); }
template <> __device__ __forceinline__ double expm1_<double>(double x) { return expm1(x); }

template <typename real> __device__ __forceinline__ real pow_(real x, real y);
template <> __device__ __forceinline__ float pow_<float>(float x, float y) { return powf(x, y); }
template <> __device__ __forceinline__ double pow_<double>(double x, double y) { return pow(x, y); }

// ---------------------------------------------------------------------------
// Explicitly rounded arithmetic.  Every operation of the site update is an
// IEEE round-to-nearest intrinsic (no contraction, no reassociation), so the
// update is the same bit pattern in every kernel variant, in batched and
// single launches, and in graph replays.
// ---------------------------------------------------------------------------
template <typename real> struct Op;
template <> struct Op<float> {
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    // 1/x for normal, finite x of moderate size (densities, temperatures):
    // the hardware's approximate reciprocal refined by one Newton-Raphson
    // step for f(r) = 1/r - x, r1 = r0 + r0 (1 - x r0).  Branch-free; its
    // error against the correctly rounded reciprocal is checked on the GPU.
    static __device__ __forceinline__ float rcp(float x)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        const float e = __fmaf_rn(-x, r, 1.0f);
        return __fmaf_rn(r, e, r);
    }
};
template <> struct Op<double> {
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double rcp(double x) { return __ddiv_rn(1.0, x); }
};

// ---------------------------------------------------------------------------
// Unbiased rounding of the FP32 reaction variable.  Lambda grows by small
// amounts per step (1e-5 is typical), a few hundred float ulps, and rounding
// each new value to nearest drops the same fraction of an ulp step after step
// while that amount changes slowly: over 20 000 steps of the 2048^2 implosion
// that bias alone left lambda 1.7e-4 behind FP64.  The update is therefore
// summed exactly (TwoSum, Knuth) and rounded to one of the two floats around
// the exact value with probability given by the distance (stochastic
// rounding), which has no bias.  The uniform number comes from a hash of the
// site index and the site's previous value, so the result is a deterministic
// function of the state: identical in every kernel variant, batch and replay.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// 32-bit integer hash (C. Wellons' "lowbias32"): a bijection with full avalanche.
__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// s + e (|e| below a few ulps of s) rounded to a neighbouring float: towards
// the exact value's far neighbour with probability |residual| / ulp, u in [0, 1).
// Values outside (0, 1) are returned rounded to nearest (they are clamped next).
__device__ __forceinline__ float round_stochastic_unit(float s, float e, float u)
{
    const float y = __fadd_rn(s, e);
    if (!(y > 0.f && y < 1.f)) return y;
    const float r = __fadd_rn(__fsub_rn(s, y), e);  // s - y is exact (y is within an ulp of s)
    if (r == 0.f) return y;
    const float other = __int_as_float(__float_as_int(y) + (r > 0.f ? 1 : -1));
    const float gap = fabsf(__fsub_rn(other, y));     // one ulp, exact
    return fabsf(r) > __fmul_rn(u, gap) ? other : y;
}

// ---------------------------------------------------------------------------
// Stored reaction variable.  FP64 stores lambda itself.  FP32 stores the
// unburnt fraction y = 1 - lambda: as lambda -> 1 the reaction increments per
// step fall below half the spacing of floats just under 1 (6e-8) and would
// round away, so lambda would stall short of 1 while the heat release
// computed from (1 - lambda) went on; y keeps them with full relative
// precision.  Near lambda = 0 the spacing of y (6e-8) bounds the absolute
// error of a step instead, far below the reaction increments there.
// ---------------------------------------------------------------------------
template <typename real> struct LamStore {
    static constexpr bool complement = false;
    static __host__ __device__ __forceinline__ double to_lambda(double s) { return s; }
    static __host__ __device__ __forceinline__ double from_lambda(double l) { return l; }
};
template <> struct LamStore<float> {
    static constexpr bool complement = true;
    static __host__ __device__ __forceinline__ double to_lambda(double s) { return 1.0 - s; }
    static __host__ __device__ __forceinline__ double from_lambda(double l) { return 1.0 - l; }
};

// ---------------------------------------------------------------------------
// A site's moments from its 33 f (Sec. II.B), ring by ring in Cartesian
// components: rho = sum f, (jx, jy) = sum f v, e2 = sum f |v|^2.  Within a
// ring the 8 directions are summed pairwise and opposite directions are
// differenced first (exact for nearly equal values).  Shared by the step,
// the FP32 moments and the allocation-free totals, so all see the same values.
// ---------------------------------------------------------------------------
template <typename real>
struct RingSpeeds {
    real v[4], v2[4];  // ring speeds v_k and their squares
};

template <typename real>
__device__ __forceinline__ void ring_moments(const real (&f)[NV], const real (&v)[4], const real (&v2)[4],
                                             real &rho, real &jx, real &jy, real &e2)
{
    using O = Op<real>;
    const real H = real(0.70710678118654752440);  // cos(pi/4)
    rho = f[0];
    jx = real(0);
    jy = real(0);
    e2 = real(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const real *g = &f[1 + 8 * k];
        const real s0 = O::add(O::add(O::add(g[0], g[4]), O::add(g[2], g[6])),
                               O::add(O::add(g[1], g[5]), O::add(g[3], g[7])));
        const real a = O::sub(g[1], g[5]), b = O::sub(g[3], g[7]);
        const real sx = O::fma(H, O::sub(a, b), O::sub(g[0], g[4]));
        const real sy = O::fma(H, O::add(a, b), O::sub(g[2], g[6]));
        rho = O::add(rho, s0);
        jx = O::fma(v[k], sx, jx);
        jy = O::fma(v[k], sy, jy);
        e2 = O::fma(v2[k], s0, e2);
    }
}

// ---------------------------------------------------------------------------
// One site's update (Eq. LB_evolution_equation, Eq. Eqlambda), all 33
// velocities unrolled.  sp/sc/sn: shared-memory buffers of rows m-1, m, m+1;
// col = HALO + tx.  Velocity (k, i) has Cartesian direction i pi / 4, so its
// moments and equilibrium use the fixed direction cosines; its polar Courant
// numbers use the row's c_i = cos(i pi/4 - theta_m), s_i = sin(...).
// ---------------------------------------------------------------------------
template <typename real, int WP, bool REREAD = false, int LAMOFF = NV * WP, bool DIR_OUTER = false>
__device__ __forceinline__ void site_update(const StepArgs<real> &A, const StepConsts<real> &C,
                                            const real *__restrict__ sp,
                                            const real *__restrict__ sc,
                                            const real *__restrict__ sn, int col, int j, int m,
                                            real inv_r, const real (&cs)[8], const real (&sn8)[8])
{
    using O = Op<real>;
    const real H = real(0.70710678118654752440);  // cos(pi/4)
    const real one = real(1), half = real(0.5);
    // the site's stores stay inside its instance's planes
    if (!DBM_DEBUG_CHECK(j >= 0 && j < A.nr && A.nr <= A.ld && m >= 0 && m < A.ntheta, A.status)) return;

    // --- a1: load the site's 33 f and lambda -------------------------------
    real f[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) f[q] = sc[q * WP + col];
    constexpr bool kY = LamStore<real>::complement;
    const real lst = sc[LAMOFF + col];  // stored: lambda, or y = 1 - lambda
    const real lam = kY ? O::sub(one, lst) : lst;

    // --- a2: moments, ring by ring (Cartesian components) ------------------
    //     rho = sum f, rho u = sum f v, e2 = sum f v^2, T = (e2/rho - u^2)/2
    real rho, jx, jy, e2;
    ring_moments<real>(f, C.v, C.v2, rho, jx, jy, e2);
    const real inv_rho = O::rcp(rho);
    const real ux = O::mul(jx, inv_rho), uy = O::mul(jy, inv_rho);
    const real u2 = O::fma(ux, ux, O::mul(uy, uy));
    const real T = O::mul(half, O::sub(O::mul(e2, inv_rho), u2));
    const real inv_T = O::rcp(T);

    // --- a3: weights F_k(T), F_0 = 1 - 8 sum F_k ---------------------------
    real F[4];
    real Fsum = real(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        F[k] = O::mul(T, O::fma(T, O::fma(T, O::fma(T, C.Fc[k][3], C.Fc[k][2]), C.Fc[k][1]), C.Fc[k][0]));
        Fsum = O::add(Fsum, F[k]);
    }
    const real F0 = O::fma(real(-8), Fsum, one);

    // --- a4 coefficients: f^eq = rho F_k [A0 + A1 xi + A2 xi^2 + xi^3/6 + xi^4/24],
    //     xi = v.u / T ---------------------------------------------------------
    const real hh = O::mul(O::mul(half, u2), inv_T);
    const real A1 = O::sub(one, hh);
    const real A0 = O::fma(O::mul(half, hh), hh, A1);
    const real A2 = O::mul(half, A1);
    const real wx = O::mul(ux, inv_T), wy = O::mul(uy, inv_T);
    real w[8];
    w[0] = wx;
    w[2] = wy;
    w[1] = O::mul(H, O::add(wx, wy));
    w[3] = O::mul(H, O::sub(wy, wx));
    w[4] = -w[0];
    w[5] = -w[1];
    w[6] = -w[2];
    w[7] = -w[3];

    // --- a5: Cochran rate with ignition gate; exact lambda step (a9) -------
    const real P = O::mul(rho, T);
    real a = real(0), b = real(0);
    if (T > C.T_th) {
        if (C.general_pow) {
            a = O::mul(C.omega1, pow_(P, C.m_exp));
            b = O::mul(C.omega2, pow_(P, C.n_exp));
        } else {
            a = O::mul(C.omega1, P);
            b = O::mul(C.omega2, P);
        }
    }
    const real om = kY ? lst : O::sub(one, lam);  // 1 - lambda
    const real g = O::fma(b, lam, a);  // a + b lam
    real R = O::mul(om, g);
    const real sab = O::add(a, b);
    real dlam = real(0);
    if (sab > real(0)) {
        // lam+ - lam = (1-lam)(a+b lam)(E-1) / [(a+b) + (a+b lam)(E-1)], E = e^{(a+b)dt}
        const real em1 = expm1_(O::mul(sab, C.dt));
        dlam = O::mul(O::mul(O::mul(om, g), em1), O::rcp(O::fma(g, em1, sab)));
    }
    if (C.reaction_energy) R = O::mul(dlam, C.inv_dt);

    // --- a6+a7 coefficients: f_new = poly(xi) (beta_k - gamma_k xi) + ... ---
    //     M = f^eq ((v-u)^2 - 2T) / (2T^2) Q R with (v-u)^2 = v_k^2 + u^2 - 2 T xi
    const real dtQR = O::mul(C.dt, O::mul(C.Q, R));
    const real half_inv_T2 = O::mul(O::mul(half, inv_T), inv_T);
    const real gam = O::mul(dtQR, inv_T);
    const real u2m2T = O::fma(real(-2), T, u2);
    const real beta0 = O::mul(O::mul(rho, F0), O::fma(O::mul(dtQR, u2m2T), half_inv_T2, C.one_m_decay));

    // --- a8: per-direction Courant magnitudes and upwind neighbours --------
    const int to_prev = (int)(sp - sc), to_next = (int)(sn - sc);
    const bool wrap_prev = C.sector && m == 0;             // row -1 = last row, i -> i+1
    const bool wrap_next = C.sector && m == A.ntheta - 1;  // row ntheta = row 0, i -> i-1
    // direction i: |C_r| / v_k, |C_theta| / v_k, their sum, and the shared-memory
    // offsets of the upwind neighbours in r and theta (false: a debug check failed)
    auto geom = [&](int i, real &ar, real &at, real &sa, int &rn, int &tn) -> bool {
        ar = O::mul(fabs(cs[i]), C.cr_scale);
        at = O::mul(O::mul(fabs(sn8[i]), C.ct_scale), inv_r);
        sa = O::add(ar, at);
        int o = cs[i] >= real(0) ? -1 : 1;  // C_r >= 0: backward difference
        if (j == 0 && o < 0) {
            // inner ghost: zero-gradient; the disc centre in a sector (same
            // site, i -> i+4); on a full disc the site across the centre,
            // which fill_centre_ghost put in the halo column before col
            o = C.centre == 1 ? (((i + 4) & 7) - i) * WP : (C.centre == 2 ? -1 : 0);
        } else if (j == A.nr - 1 && o > 0) {
            o = 0;  // zero-gradient outer ghost
        }
        rn = col + o;
        if (sn8[i] >= real(0))  // C_theta >= 0: row m-1
            tn = col + to_prev + (wrap_prev ? (((i + 1) & 7) - i) * WP : 0);
        else
            tn = col + to_next + (wrap_next ? (((i + 7) & 7) - i) * WP : 0);
#ifdef DBM_DEBUG
        // velocity planes q = 1 + i .. 25 + i of direction i: neighbour
        // reads stay inside the 33 planes of their row buffer
        const int tr = tn - (sn8[i] >= real(0) ? to_prev : to_next);
        const bool ok = (1 + i) * WP + rn >= 0 && (25 + i) * WP + rn < NV * WP &&
                        (1 + i) * WP + tr >= 0 && (25 + i) * WP + tr < NV * WP;
        return DBM_DEBUG_CHECK(ok, A.status);
#else
        return true;
#endif
    };

    // --- a7 + a11: update all velocities and store ------------------------
    //     f_new = f^eq (1 - E + dt M/f^eq) + (E - |C_r| - |C_th|) f
    //             + |C_r| f(upwind r) + |C_th| f(upwind theta)
    //     with f^eq (1 - E + dt M / f^eq) = poly(xi) (beta_k - gamma_k xi) in ring k
    real *out = A.f_out + (long long)m * A.ld + j;
    out[0] = O::fma(A0, beta0, O::mul(C.decay, REREAD ? sc[col] : f[0]));
    if constexpr (sizeof(real) == 8 || !DIR_OUTER) {
        // Ring by ring with the geometry of all 8 directions held: the
        // single-instance kernels and FP64.
        real ar[8], at[8], sa[8];
        int rn[8], tn[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            // as geom(i, ...), written out: the compiler schedules this form better
            if (sizeof(real) == 8 && i >= 4) {
                // FP64: the trig table holds direction i + 4 as the exact
                // negation of direction i, so the magnitudes are the same bits
                ar[i] = ar[i - 4];
                at[i] = at[i - 4];
                sa[i] = sa[i - 4];
            } else {
                ar[i] = O::mul(fabs(cs[i]), C.cr_scale);
                at[i] = O::mul(O::mul(fabs(sn8[i]), C.ct_scale), inv_r);
                sa[i] = O::add(ar[i], at[i]);
            }
            int o = cs[i] >= real(0) ? -1 : 1;  // C_r >= 0: backward difference
            if (j == 0 && o < 0) {
                o = C.centre == 1 ? (((i + 4) & 7) - i) * WP : (C.centre == 2 ? -1 : 0);
            } else if (j == A.nr - 1 && o > 0) {
                o = 0;  // zero-gradient outer ghost
            }
            rn[i] = col + o;
            if (sn8[i] >= real(0))  // C_theta >= 0: row m-1
                tn[i] = col + to_prev + (wrap_prev ? (((i + 1) & 7) - i) * WP : 0);
            else
                tn[i] = col + to_next + (wrap_next ? (((i + 7) & 7) - i) * WP : 0);
#ifdef DBM_DEBUG
            {
                // velocity planes q = 1 + i .. 25 + i of direction i: neighbour
                // reads stay inside the 33 planes of their row buffer
                const int tr = tn[i] - (sn8[i] >= real(0) ? to_prev : to_next);
                const bool ok = (1 + i) * WP + rn[i] >= 0 && (25 + i) * WP + rn[i] < NV * WP &&
                                (1 + i) * WP + tr >= 0 && (25 + i) * WP + tr < NV * WP;
                if (!DBM_DEBUG_CHECK(ok, A.status)) return;
            }
#endif
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const real vk = C.v[k];
            const real rF = O::mul(rho, F[k]);
            const real beta = O::mul(rF, O::fma(O::mul(dtQR, O::add(C.v2[k], u2m2T)), half_inv_T2, C.one_m_decay));
            const real gamma = O::mul(rF, gam);
            // one velocity given its xi and the equilibrium polynomial at xi
            auto update_one = [&](int i, real xi, real poly) {
                const int q = 1 + 8 * k + i;
                real t = O::mul(poly, O::fma(-gamma, xi, beta));
                // REREAD: take f from shared memory again instead of holding all
                // 33 values in registers across the moment pass (fewer registers)
                const real fq = REREAD ? sc[q * WP + col] : f[q];
                t = O::fma(O::fma(-vk, sa[i], C.decay), fq, t);
                const real adv = O::fma(ar[i], sc[q * WP + rn[i]], O::mul(at[i], sc[q * WP + tn[i]]));
                t = O::fma(vk, adv, t);
                out[(long long)q * A.plane] = t;
            };
            if constexpr (sizeof(real) == 8) {
                // FP64 is bound by its arithmetic: opposite directions i and
                // i+4 have xi and -xi, so the polynomial splits into an even
                // part E and an odd part O evaluated once, poly(+-xi) = E +- O;
                // they also share |C_r| + |C_theta|, so the weight of the
                // site's own f, E - v_k (|C_r| + |C_theta|), is taken once
                auto update_pair_one = [&](int i, real xi, real poly, real keep) {
                    const int q = 1 + 8 * k + i;
                    real t = O::mul(poly, O::fma(-gamma, xi, beta));
                    const real fq = REREAD ? sc[q * WP + col] : f[q];
                    t = O::fma(keep, fq, t);
                    const real adv = O::fma(ar[i], sc[q * WP + rn[i]], O::mul(at[i], sc[q * WP + tn[i]]));
                    t = O::fma(vk, adv, t);
                    out[(long long)q * A.plane] = t;
                };
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const real xi = O::mul(vk, w[i]);
                    const real x2 = O::mul(xi, xi);
                    const real Ev = O::fma(x2, O::fma(x2, real(1.0 / 24.0), A2), A0);
                    const real Od = O::mul(xi, O::fma(x2, real(1.0 / 6.0), A1));
                    const real keep = O::fma(-vk, sa[i], C.decay);
                    update_pair_one(i, xi, O::add(Ev, Od), keep);
                    update_pair_one(i + 4, -xi, O::sub(Ev, Od), keep);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const real xi = O::mul(vk, w[i]);
                    update_one(i, xi, O::fma(xi, O::fma(xi, O::fma(xi, O::fma(xi, real(1.0 / 24.0), real(1.0 / 6.0)), A2), A1), A0));
                }
            }
        }
    } else {
        // FP32 with DIR_OUTER (batched launches, which hold each instance's
        // constants in registers): direction by direction, so that only one
        // direction's geometry is live at a time.  Each velocity's arithmetic
        // is the ring-by-ring one, operation for operation: same bits.
        real beta[4], gamma[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const real rF = O::mul(rho, F[k]);
            beta[k] = O::mul(rF, O::fma(O::mul(dtQR, O::add(C.v2[k], u2m2T)), half_inv_T2, C.one_m_decay));
            gamma[k] = O::mul(rF, gam);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            real ar, at, sa;
            int rn, tn;
            if (!geom(i, ar, at, sa, rn, tn)) return;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int q = 1 + 8 * k + i;
                const real vk = C.v[k];
                const real xi = O::mul(vk, w[i]);
                const real poly =
                    O::fma(xi, O::fma(xi, O::fma(xi, O::fma(xi, real(1.0 / 24.0), real(1.0 / 6.0)), A2), A1), A0);
                real t = O::mul(poly, O::fma(-gamma[k], xi, beta[k]));
                const real fq = REREAD ? sc[q * WP + col] : f[q];
                t = O::fma(O::fma(-vk, sa, C.decay), fq, t);
                const real adv = O::fma(ar, sc[q * WP + rn], O::mul(at, sc[q * WP + tn]));
                t = O::fma(vk, adv, t);
                out[(long long)q * A.plane] = t;
            }
        }
    }

    // --- a9 + a10: lambda = exact reaction step + upwind transport ---------
    const real cth = cs[0], sth = -sn8[0];  // cos(theta_m), sin(theta_m)
    const real ur = O::fma(ux, cth, O::mul(uy, sth));
    const real uth = O::fma(uy, cth, -O::mul(ux, sth));
    int orr = ur >= real(0) ? -1 : 1;
    if ((j == 0 && orr < 0 && C.centre != 2) || (j == A.nr - 1 && orr > 0)) orr = 0;
    // transport acts on the stored variable alike (y - y_nb = lambda_nb - lambda);
    // the reaction step adds dlam to lambda, so it is taken off y
    if (!DBM_DEBUG_CHECK(col + orr >= 0 && col + orr < WP, A.status)) return;
    const real lr = sc[LAMOFF + col + orr];
    const real lt = (uth >= real(0) ? sp : sn)[LAMOFF + col];
    const real tr = O::mul(O::mul(fabs(ur), C.cr_scale), O::sub(lst, lr));
    const real tt = O::mul(O::mul(O::mul(fabs(uth), C.ct_scale), inv_r), O::sub(lst, lt));
    real ln;
    if constexpr (sizeof(real) == 4) {
        // y - dlam - tr - tt summed exactly, then rounded without bias
        float sum, err, e2;
        two_sum_f(lst, -dlam, sum, err);
        two_sum_f(sum, -tr, sum, e2);
        err = __fadd_rn(err, e2);
        two_sum_f(sum, -tt, sum, e2);
        err = __fadd_rn(err, e2);
        const uint32_t site = (uint32_t)m * (uint32_t)A.ld + (uint32_t)j;
        const float u = (float)(hash32(site * 0x9e3779b9u ^ __float_as_uint(lst)) >> 8) * 0x1p-24f;
        ln = round_stochastic_unit(sum, err, u);
    } else {
        ln = kY ? O::sub(lst, dlam) : O::add(lst, dlam);
        ln = O::sub(ln, tr);
        ln = O::sub(ln, tt);
    }
    ln = fmin(fmax(ln, real(0)), real(1));
    A.lam_out[(long long)m * A.ld + j] = ln;
}

// ---------------------------------------------------------------------------
// Full disc (centre == 2, Sec. II.D with a full 2 pi grid): the inner ghost of
// radial site 0 in row m is site 0 of row m + ntheta/2, the point across the
// centre, with the same (Cartesian) velocity and the same lambda.  The thread
// of site 0 copies those 33 f and lambda from the step's input into the halo
// column HALO - 1 of its own row buffer, where its backward differences read
// them; no other thread reads that column of the row.  The caller fences the
// generic writes against the TMA copies that later refill the buffer.
// ---------------------------------------------------------------------------
template <typename real, int WP, int LAMOFF, int HALO>
__device__ __forceinline__ void fill_centre_ghost(const StepArgs<real> &A, real *sc, int m)
{
    const int half = A.ntheta / 2;
    const int mm = m + half < A.ntheta ? m + half : m + half - A.ntheta;
    const real *src = A.f_in + (long long)mm * A.ld;
    real g[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) g[q] = src[(long long)q * A.plane];
    const real lg = A.lam_in[(long long)mm * A.ld];
#pragma unroll
    for (int q = 0; q < NV; ++q) sc[q * WP + HALO - 1] = g[q];
    sc[LAMOFF + HALO - 1] = lg;
}

// ---------------------------------------------------------------------------
// Work lists.  A work item is W radial sites x a run of theta rows of one
// instance.  SingleWork decodes items of one instance arithmetically (its
// arguments live in kernel parameter space); BatchWork reads items of many
// uneven instances from a device table and decides on the device, from the
// global step counter T, which instances are active in this step.
// ---------------------------------------------------------------------------
template <typename real, int W>
struct SingleWork {
    static constexpr bool kCopyArgs = false;
    const StepArgs<real> *A;
    __device__ __forceinline__ int count() const { return A->items; }
    __device__ __forceinline__ bool item(int it, const StepArgs<real> *&a, int &j0, int &mb,
                                         int &me, int &cidx) const
    {
        a = A;
        cidx = -1;
        const int strip = it % A->strips;
        const int seg = it / A->strips;
        j0 = strip * W;
        mb = seg * A->rows_per_item;
        me = min(mb + A->rows_per_item, A->ntheta);
        return true;
    }
};

// One batch slot: the instance's step arguments for both ping-pong parities
// and the global steps [start, end) during which it advances.
template <typename real>
struct BatchSlot {
    StepArgs<real> args[2];  // [p]: reads buffer p, writes buffer 1 - p
    long long start, end;
    int par0;                // the instance's buffer index at global step start
    int cidx;                // the instance's entry in the batch constant table
};

template <typename real>
struct BatchArgs {
    const BatchSlot<real> *slots;
    const int4 *items;        // (slot, j0, mb, me)
    const int *n_items;       // device word: number of valid items
    const long long *T;       // device word: global step at the start of this replay
    int s;                    // step index within the replay
};

template <typename real, int W>
struct BatchWork {
    static constexpr bool kCopyArgs = true;
    const BatchSlot<real> *slots;
    const int4 *items;
    int n;
    long long T;
    __device__ __forceinline__ int count() const { return n; }
    __device__ __forceinline__ bool item(int it, const StepArgs<real> *&a, int &j0, int &mb,
                                         int &me, int &cidx) const
    {
        const int4 e = items[it];
        if (e.x < 0) return false;  // padding of the load-balanced table
        const BatchSlot<real> &sl = slots[e.x];
        if (T < sl.start || T >= sl.end) return false;
        a = &sl.args[(int)((T - sl.start + sl.par0) & 1)];
        cidx = sl.cidx;
        j0 = e.y;
        mb = e.z;
        me = e.w;
        return true;
    }
};

// ---------------------------------------------------------------------------
// The fused persistent step: march over this CTA's work items (items
// blockIdx.x, blockIdx.x + gridDim.x, ...), keeping the TMA row ring full
// across item boundaries.
// ---------------------------------------------------------------------------
template <typename real, int W, int NSTAGE, typename Work>
__device__ __forceinline__ void march(const Work &work, unsigned char *smem_raw,
                                      StepArgs<real> *sargs)
{
    constexpr int HALO = Halo<real>::value;
    constexpr int WP = W + 2 * HALO;
    constexpr int SLOT = NARR * WP;  // elements per row buffer
    static_assert(NSTAGE >= 3, "rows m-1, m, m+1 must be resident");

    real *sm = reinterpret_cast<real *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + sizeof(real) * NSTAGE * SLOT);
    __shared__ int abort_flag;

    const int tx = threadIdx.x;
    const int lane = tx & 31;
    const bool producer = tx < 32;  // warp 0 issues the copies
    const int nitems = work.count();

    if (tx == 0) {
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    // Total row loads of this CTA: rows mb-1 .. me of each active item.
    long long total_loads = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const StepArgs<real> *a;
        int j0, mb, me, cidx;
        if (work.item(it, a, j0, mb, me, cidx)) total_loads += (me - mb) + 2;
    }

    // Producer cursor (replicated in the lanes of warp 0).
    long long issued = 0;
    int p_item = blockIdx.x, p_row = 0;
    const StepArgs<real> *pa = nullptr;
    int pj0 = 0, pmb = 0, pme = 0, pcidx = 0;
    bool p_ok = false;

    auto issue_one = [&]() {
        while (!p_ok) {  // find the next active item
            p_ok = work.item(p_item, pa, pj0, pmb, pme, pcidx);
            if (!p_ok) p_item += gridDim.x;
        }
        int m = pmb - 1 + p_row;
        const int nth = pa->ntheta;
        m = m < 0 ? m + nth : (m >= nth ? m - nth : m);
        const int slot = (int)(issued % NSTAGE);
        const int jlo = max(pj0 - HALO, 0);
        const int jhi = min(pj0 + W + HALO, (pa->nr + HALO - 1) / HALO * HALO);  // row padding not read
        const uint32_t nbytes = (uint32_t)((jhi - jlo) * (int)sizeof(real));
        real *dst = sm + slot * SLOT + (jlo - (pj0 - HALO));
        if (lane == 0) mbar_arrive_expect_tx(&bars[slot], nbytes * NARR);
        __syncwarp();
        const long long roff = (long long)m * pa->ld + jlo;
        for (int a = lane; a < NARR; a += 32) {
            const real *src = (a < NV) ? pa->f_in + (long long)a * pa->plane + roff : pa->lam_in + roff;
            bulk_g2s(dst + a * WP, src, nbytes, &bars[slot]);
        }
        ++issued;
        if (++p_row == (pme - pmb) + 2) {
            p_row = 0;
            p_item += gridDim.x;
            p_ok = false;
        }
    };

    if (producer) {
        while (issued < NSTAGE && issued < total_loads) issue_one();
    }

    long long base = 0;  // sequence position of the current item's first load
    bool ok = true;
    for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        const StepArgs<real> *ga;
        int j0, mb, me, cidx;
        if (!work.item(it, ga, j0, mb, me, cidx)) continue;
        const StepArgs<real> *ap = ga;
        if constexpr (Work::kCopyArgs) {
            // per-instance constants into shared memory (read by every thread)
            const int nw = (int)(sizeof(StepArgs<real>) / sizeof(int));
            for (int q = tx; q < nw; q += blockDim.x)
                reinterpret_cast<int *>(sargs)[q] = reinterpret_cast<const int *>(ga)[q];
            __syncthreads();
            ap = sargs;
        }
        const StepArgs<real> &A = *ap;
        const StepConsts<real> &C = Work::kCopyArgs ? batch_consts<real>(cidx) : A.c;
        const int L = me - mb;
        const int j = j0 + tx;
        const bool active = j < A.nr;
        const real inv_r = A.inv_r[active ? j : 0];

        for (int c = 1; c <= L; ++c) {
            const long long P = base + c;
            // wait for rows at positions P-1, P, P+1
#pragma unroll
            for (int d = -1; d <= 1; ++d) {
                const long long Q = P + d;
                if (!mbar_wait_bounded(&bars[Q % NSTAGE], (uint32_t)((Q / NSTAGE) & 1))) {
                    atomicOr(A.status, ST_WAIT_TIMEOUT);
                    abort_flag = 1;
                }
            }
            const int m = mb + c - 1;
            if (active && !abort_flag) {
                real cs[8], sn8[8];
                const real *rt = A.rowtab + (long long)m * 16;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    cs[i] = rt[i];
                    sn8[i] = rt[8 + i];
                }
                const bool ghost = C.centre == 2 && j == 0;
                if (ghost) fill_centre_ghost<real, WP, NV * WP, HALO>(A, sm + (P % NSTAGE) * SLOT, m);
                site_update<real, WP>(A, C, sm + ((P - 1) % NSTAGE) * SLOT, sm + (P % NSTAGE) * SLOT,
                                      sm + ((P + 1) % NSTAGE) * SLOT, HALO + tx, j, m, inv_r, cs, sn8);
                if (ghost) fence_proxy_async_smem();
            }
            __syncthreads();
            if (abort_flag) {
                ok = false;
                break;
            }
            // positions before need_from are no longer read
            const long long need_from = (c < L) ? P : base + L + 2;
            if (producer) {
                fence_proxy_async_smem();
                while (issued < need_from + NSTAGE && issued < total_loads) issue_one();
            }
        }
        base += L + 2;
    }

    if (!ok && tx == 0) {
        // Drain: wait (bounded) for every copy still in flight before exiting.
        for (long long Q = base; Q < issued; ++Q)
            mbar_wait_bounded(&bars[Q % NSTAGE], (uint32_t)((Q / NSTAGE) & 1));
    }
}

template <typename real, int W, int NSTAGE>
__global__ void __launch_bounds__(W, 2) step_kernel(const __grid_constant__ StepArgs<real> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SingleWork<real, W> work{&A};
    march<real, W, NSTAGE>(work, smem_raw, nullptr);
}

template <typename real, int W, int NSTAGE>
__global__ void __launch_bounds__(W, 2) batch_step_kernel(const __grid_constant__ BatchArgs<real> B)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(16) StepArgs<real> sargs;
    BatchWork<real, W> work{B.slots, B.items, *B.n_items, *B.T + B.s};
    march<real, W, NSTAGE>(work, smem_raw, &sargs);
}

// Advance the batch's global step counter after a replay of k steps.
static __global__ void batch_advance_kernel(long long *T, int k)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *T += k;
}

// Row-buffer layout of the v2 pipeline (in elements of real).
template <typename real, int W>
struct V2Layout {
    static constexpr int wp = W + 2 * Halo<real>::value;
    static constexpr int a128 = 128 / (int)sizeof(real);
    static constexpr int lam = (NV * wp + a128 - 1) / a128 * a128;  // 128-byte aligned
    static constexpr int tab = lam + wp;                            // 16 trig values
    static constexpr int slot = (tab + 16 + a128 - 1) / a128 * a128;
};

// ---------------------------------------------------------------------------
// v2 pipeline: warp-specialised.  Warp W/32 is the producer: it issues the
// TMA bulk copies of each row (34 arrays + the row's 16 trig values) into a
// ring of NSTAGE buffers.  The W/32 consumer warps each update 32 sites of the
// row.  Per buffer, a "full" mbarrier (count 1 + transaction bytes) tells the
// consumers a row has landed, and an "empty" mbarrier (count = consumer warps)
// tells the producer every consumer warp is done with it.  There is no
// CTA-wide barrier per row, so warps drift within the ring instead of waiting
// for the slowest.  Positions are released after their last use: after
// centre P the buffer of P-1, and at an item's last centre also P and P+1.
// ---------------------------------------------------------------------------
template <typename real, int W, int NSTAGE, bool REREAD, bool TMAP, typename Work>
__device__ __forceinline__ void march2(const Work &work, unsigned char *smem_raw,
                                       StepArgs<real> *sargs2)
{
    constexpr int HALO = Halo<real>::value;
    constexpr int WP = W + 2 * HALO;
    constexpr int TAB = 16;
    constexpr int NCW = W / 32;            // consumer warps
    // Row buffer layout (elements): 33 f rows of WP, then lambda at the next
    // 128-byte boundary (tensor-TMA destinations must be 128-byte aligned),
    // then the 16 trig values; the buffer size is a multiple of 128 bytes.
    constexpr int LAMOFF = V2Layout<real, W>::lam;
    constexpr int RTOFF = V2Layout<real, W>::tab;
    constexpr int SLOT = V2Layout<real, W>::slot;
    static_assert(NSTAGE >= 3, "rows m-1, m, m+1 must be resident");
    static_assert((SLOT * sizeof(real)) % 128 == 0, "row buffers must be 128-byte aligned");
    static_assert((LAMOFF * sizeof(real)) % 128 == 0, "lambda tile must be 128-byte aligned");
    static_assert((RTOFF * sizeof(real)) % 16 == 0, "trig row must be 16-byte aligned");

    real *sm = reinterpret_cast<real *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + sizeof(real) * NSTAGE * SLOT);
    uint64_t *empty = full + NSTAGE;
    __shared__ int abort_flag;
    __shared__ int issued_total;

    const int tx = threadIdx.x;
    const int warp = tx >> 5, lane = tx & 31;
    const int nitems = work.count();

    if (tx == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        fence_mbar_init();
        abort_flag = 0;
        issued_total = 0;
    }
    __syncthreads();
    if ((smem_addr(smem_raw) & 127u) != 0u) {  // layout assumption broken: report, copy nothing
        if (tx == 0 && nitems > 0) {
            const StepArgs<real> *a;
            int j0, mb, me, cidx;
            for (int it = blockIdx.x; it < nitems; it += gridDim.x)
                if (work.item(it, a, j0, mb, me, cidx)) {
                    atomicOr(a->status, ST_SMEM_ALIGN);
                    break;
                }
        }
        return;
    }

    if (warp == NCW) {
        // ------------------------------ producer ------------------------------
        int total_loads = 0;  // ring positions of this CTA (32-bit: cheap slot arithmetic)
        for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
            const StepArgs<real> *a;
            int j0, mb, me, cidx;
            if (work.item(it, a, j0, mb, me, cidx)) total_loads += (me - mb) + 2;
        }
        int issued = 0;
        int p_item = blockIdx.x, p_row = 0;
        const StepArgs<real> *pa = nullptr;
        int pj0 = 0, pmb = 0, pme = 0, pcidx = 0;
        bool p_ok = false;
        while (issued < total_loads) {
            const int slot = issued % NSTAGE;
            while (!p_ok) {
                p_ok = work.item(p_item, pa, pj0, pmb, pme, pcidx);
                if (!p_ok) p_item += gridDim.x;
            }
            if (issued >= NSTAGE) {
                const uint32_t par = (uint32_t)((issued / NSTAGE - 1) & 1);
                if (!mbar_wait_bounded(&empty[slot], par)) {
                    if (lane == 0) atomicOr(pa->status, ST_WAIT_TIMEOUT);
                    abort_flag = 1;
                }
            }
            __syncwarp();
            if (*(volatile int *)&abort_flag) break;
            int m = pmb - 1 + p_row;
            const int nth = pa->ntheta;
            m = m < 0 ? m + nth : (m >= nth ? m - nth : m);
            real *buf = sm + slot * SLOT;
#ifdef DBM_DEBUG
            {
                // the row is in the grid; the strip starts inside the row; a tensor
                // box's first column is on a 16-byte boundary; bulk extents are
                // inside the padded row and multiples of 16 bytes
                const int jlo = max(pj0 - HALO, 0), jhi = min(pj0 + W + HALO, (pa->nr + HALO - 1) / HALO * HALO);
                bool ok = m >= 0 && m < nth && pj0 >= 0 && pj0 < pa->nr && pa->nr <= pa->ld;
                if (TMAP) ok = ok && ((pj0 - HALO) * (int)sizeof(real)) % 16 == 0;
                else ok = ok && jhi > jlo && ((jhi - jlo) * (int)sizeof(real)) % 16 == 0 &&
                          (((long long)m * pa->ld + jlo) * (long long)sizeof(real)) % 16 == 0;
                if (!ok) {  // uniform over the warp: every input is
                    if (lane == 0) {
                        atomicOr(pa->status, ST_BOUNDS);
                        abort_flag = 1;
                    }
                    break;
                }
            }
#endif
            if constexpr (TMAP) {
                // one 3-D tile (all 33 f planes of the strip's row), one 2-D tile
                // (lambda), one bulk copy (trig row); the box starts at the
                // halo column pj0 - HALO and out-of-range columns are zeros
                if (lane == 0) {
                    if (Work::kCopyArgs && p_row == 0) {  // maps of a batch slot, in global memory
                        fence_tensormap_acquire(&pa->tm_f);
                        fence_tensormap_acquire(&pa->tm_lam);
                    }
                    mbar_arrive_expect_tx(&full[slot], (uint32_t)(WP * NARR + TAB) * (uint32_t)sizeof(real));  // 33 + 1 rows + trig
                    fence_proxy_async_smem();
                    tma_load_3d(buf, &pa->tm_f, pj0 - HALO, m, 0, &full[slot]);
                    tma_load_2d(buf + LAMOFF, &pa->tm_lam, pj0 - HALO, m, &full[slot]);
                    bulk_g2s(buf + RTOFF, pa->rowtab + (long long)m * TAB, TAB * sizeof(real), &full[slot]);
                }
                __syncwarp();
            } else {
                const int jlo = max(pj0 - HALO, 0);
                const int jhi = min(pj0 + W + HALO, (pa->nr + HALO - 1) / HALO * HALO);  // row padding not read
                const uint32_t nbytes = (uint32_t)((jhi - jlo) * (int)sizeof(real));
                real *dst = buf + (jlo - (pj0 - HALO));
                if (lane == 0) mbar_arrive_expect_tx(&full[slot], nbytes * NARR + TAB * (uint32_t)sizeof(real));
                __syncwarp();
                fence_proxy_async_smem();
                const long long roff = (long long)m * pa->ld + jlo;
                for (int a = lane; a < NARR; a += 32) {
                    const real *src = (a < NV) ? pa->f_in + (long long)a * pa->plane + roff : pa->lam_in + roff;
                    bulk_g2s(a < NV ? dst + a * WP : dst + LAMOFF, src, nbytes, &full[slot]);
                }
                if (lane == 31) bulk_g2s(buf + RTOFF, pa->rowtab + (long long)m * TAB, TAB * sizeof(real), &full[slot]);
            }
            ++issued;
            if (++p_row == (pme - pmb) + 2) {
                p_row = 0;
                p_item += gridDim.x;
                p_ok = false;
            }
        }
        if (lane == 0) issued_total = issued;
    } else {
        // ------------------------------ consumers -----------------------------
        int base = 0;
        int parity = 0;
        bool ok = true;
        // One work item: rows [mb, me) of the strip starting at radial site j0.
        auto run_item = [&](const StepArgs<real> &A, const StepConsts<real> &C, int j0, int mb, int me) {
            const int L = me - mb;
            const int j = j0 + tx;
            const bool active = j < A.nr;
            const real inv_r = A.inv_r[active ? j : 0];
            for (int c = 1; c <= L; ++c) {
                const int P = base + c;
                for (int Q = (c == 1 ? P - 1 : P + 1); Q <= P + 1; ++Q) {
                    if (!mbar_wait_bounded(&full[Q % NSTAGE], (uint32_t)((Q / NSTAGE) & 1))) {
                        if (lane == 0) atomicOr(A.status, ST_WAIT_TIMEOUT);
                        abort_flag = 1;
                    }
                }
                if (*(volatile int *)&abort_flag) {
                    ok = false;
                    return;
                }
                const real *sc = sm + (P % NSTAGE) * SLOT;
                if (active) {
                    real cs[8], sn8[8];
                    const real *rt = sc + RTOFF;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        cs[i] = rt[i];
                        sn8[i] = rt[8 + i];
                    }
                    const bool ghost = C.centre == 2 && j == 0;
                    if (ghost)
                        fill_centre_ghost<real, WP, LAMOFF, HALO>(A, sm + (P % NSTAGE) * SLOT, mb + c - 1);
                    site_update<real, WP, REREAD, LAMOFF, Work::kCopyArgs>(A, C, sm + ((P - 1) % NSTAGE) * SLOT, sc,
                                                  sm + ((P + 1) % NSTAGE) * SLOT, HALO + tx, j,
                                                  mb + c - 1, inv_r, cs, sn8);
                    if (ghost) fence_proxy_async_smem();
                }
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&empty[(P - 1) % NSTAGE]);
                    if (c == L) {
                        mbar_arrive(&empty[P % NSTAGE]);
                        mbar_arrive(&empty[(P + 1) % NSTAGE]);
                    }
                }
            }
            base += L + 2;
        };
        for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
            const StepArgs<real> *ga;
            int j0, mb, me, cidx;
            if (!work.item(it, ga, j0, mb, me, cidx)) continue;
            if constexpr (Work::kCopyArgs) {
                // per-instance constants into shared memory, double-buffered:
                // the barrier of the previous item guarantees nobody still
                // reads the copy made two items ago
                StepArgs<real> *dst = sargs2 + parity;
                const int nw = (int)(sizeof(StepArgs<real>) / sizeof(int));
                for (int q = tx; q < nw; q += W)
                    reinterpret_cast<int *>(dst)[q] = reinterpret_cast<const int *>(ga)[q];
                named_bar_sync(1, W);
                parity ^= 1;
                // FP32: the item's pointers and sizes from there, and its
                // constants from the batch constant table, into registers for
                // the item (a single instance reads its constants from the
                // constant bank as instruction operands).  The table is
                // constant memory, so where registers run short the compiler
                // can load a constant again instead of spilling it.  FP64 is
                // bound by its arithmetic pipe and short of registers: it
                // reads them where they are.
                const StepConsts<real> &C = batch_consts<real>(cidx);
                if constexpr (sizeof(real) == 4) {
                    const StepArgs<real> Areg = *dst;
                    const StepConsts<real> Creg = C;
                    run_item(Areg, Creg, j0, mb, me);
                } else {
                    run_item(*dst, C, j0, mb, me);
                }
            } else {
                run_item(*ga, ga->c, j0, mb, me);
            }
        }
    }
    __syncthreads();
    if (abort_flag && tx == 0) {
        // Drain: wait (bounded) for the copies of the last NSTAGE positions.
        const int n = issued_total;
        for (int Q = (n > NSTAGE ? n - NSTAGE : 0); Q < n; ++Q)
            mbar_wait_bounded(&full[Q % NSTAGE], (uint32_t)((Q / NSTAGE) & 1));
    }
}

template <typename real, int W, int NSTAGE, bool REREAD, int MINB, bool TMAP>
__global__ void __launch_bounds__(W + 32, MINB) step_kernel_v2(const __grid_constant__ StepArgs<real> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SingleWork<real, W> work{&A};
    march2<real, W, NSTAGE, REREAD, TMAP>(work, smem_raw, nullptr);
}

template <typename real, int W, int NSTAGE, bool REREAD, int MINB, bool TMAP>
__global__ void __launch_bounds__(W + 32, MINB) batch_step_kernel_v2(const __grid_constant__ BatchArgs<real> B)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(64) StepArgs<real> sargs2[2];
    BatchWork<real, W> work{B.slots, B.items, *B.n_items, *B.T + B.s};
    march2<real, W, NSTAGE, REREAD, TMAP>(work, smem_raw, sargs2);
}

template <typename real, int W, int NSTAGE>
constexpr int smem_bytes_v2()
{
    return (int)(sizeof(real) * NSTAGE * V2Layout<real, W>::slot + 16 * NSTAGE);
}

// Self-test of the bounded wait every pipeline uses: one CTA waits on an
// mbarrier with `limit` cycles.  With arrive = 0 nothing ever arrives, the
// wait runs out and the kernel reports ST_WAIT_TIMEOUT in *status and returns
// (the context stays usable); with arrive = 1 warp 1 arrives and the wait
// succeeds.
static __global__ void wait_selftest_kernel(int *status, int arrive, long long limit)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 32) mbar_arrive(&bar);
    if (!mbar_wait_bounded(&bar, 0, limit) && (threadIdx.x & 31) == 0) atomicOr(status, ST_WAIT_TIMEOUT);
}

// Self-test of Op<float>::rcp against the correctly rounded division.
static __global__ void rcp_selftest_kernel(const float *x, float *approx, float *ieee, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        approx[i] = Op<float>::rcp(x[i]);
        ieee[i] = __fdiv_rn(1.0f, x[i]);
    }
}

// ---------------------------------------------------------------------------
// Initial state: f = f^eq(rho, u, T) (Eq. feq) of the initial fields, lambda
// stored.  fields: [5][ntheta][nr] doubles (rho, u_r, u_theta, T, lambda).
// f^eq is evaluated in the state's precision with the arithmetic of the
// step's own equilibrium (weights F_k by Horner, expansion coefficients from
// u^2 / T, xi = v_k (e_i . u) / T), from the fields rounded to `real` and the
// row's cos / sin of the geometry table; opposite directions share the even
// and odd parts of the expansion.  Every value is checked (rho > 0, T > 0,
// all finite): a block that finds a bad one sets *bad, which the host reports
// as DBM_EINVAL (the state is then undefined).
// ---------------------------------------------------------------------------
// Cartesian direction cosines of the 8 directions i pi / 4 (FP64 kernels).
__device__ __forceinline__ void cart_dirs(double (&cx)[8], double (&cy)[8])
{
    const double H = 0.70710678118654752440;
    const double c[8] = {1.0, H, 0.0, -H, -1.0, -H, 0.0, H};
    const double sn[8] = {0.0, H, 1.0, H, 0.0, -H, -1.0, -H};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        cx[i] = c[i];
        cy[i] = sn[i];
    }
}

template <typename real>
struct InitArgs {
    const double *fields;
    real *f;
    real *lam;
    const real *rowtab;  // [ntheta][16]: cos, sin of (i pi/4 - theta_m)
    int *bad;
    long long plane;
    int nr, ntheta, ld;
    int m0, m1;          // theta rows [m0, m1) of this launch
    real v[4];
    real Fc[4][4];
};

template <typename real>
__global__ void __launch_bounds__(256) init_kernel(const InitArgs<real> A)
{
    using O = Op<real>;
    const real H = real(0.70710678118654752440);
    const real one = real(1), half = real(0.5);
    const long long N = (long long)A.nr * A.ntheta;
    bool bad = false;
    for (long long s = (long long)A.m0 * A.nr + blockIdx.x * (long long)blockDim.x + threadIdx.x;
         s < (long long)A.m1 * A.nr; s += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(s / A.nr), j = (int)(s - (long long)m * A.nr);
        const double rho_d = A.fields[s], ur_d = A.fields[N + s], uth_d = A.fields[2 * N + s];
        const double T_d = A.fields[3 * N + s], lam_d = A.fields[4 * N + s];
        if (!(rho_d > 0.0) || !(T_d > 0.0) || !isfinite(rho_d) || !isfinite(T_d) || !isfinite(ur_d) ||
            !isfinite(uth_d) || !isfinite(lam_d)) {
            bad = true;
            continue;
        }
        const real rho = (real)rho_d, ur = (real)ur_d, uth = (real)uth_d, T = (real)T_d;
        const real cth = A.rowtab[(long long)m * 16], sth = -A.rowtab[(long long)m * 16 + 8];
        const real ux = O::fma(ur, cth, -O::mul(uth, sth));
        const real uy = O::fma(ur, sth, O::mul(uth, cth));
        const real u2 = O::fma(ux, ux, O::mul(uy, uy));
        const real inv_T = O::rcp(T);
        real F[4], Fsum = real(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            F[k] = O::mul(T, O::fma(T, O::fma(T, O::fma(T, A.Fc[k][3], A.Fc[k][2]), A.Fc[k][1]), A.Fc[k][0]));
            Fsum = O::add(Fsum, F[k]);
        }
        const real F0 = O::fma(real(-8), Fsum, one);
        const real hh = O::mul(O::mul(half, u2), inv_T);
        const real A1 = O::sub(one, hh);
        const real A0 = O::fma(O::mul(half, hh), hh, A1);
        const real A2 = O::mul(half, A1);
        const real wx = O::mul(ux, inv_T), wy = O::mul(uy, inv_T);
        const real w[4] = {wx, O::mul(H, O::add(wx, wy)), wy, O::mul(H, O::sub(wy, wx))};
        real *out = A.f + (long long)m * A.ld + j;
        out[0] = O::mul(O::mul(rho, F0), A0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const real rF = O::mul(rho, F[k]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const real xi = O::mul(A.v[k], w[i]);  // direction i + 4 has -xi
                const real x2 = O::mul(xi, xi);
                const real Ev = O::fma(x2, O::fma(x2, real(1.0 / 24.0), A2), A0);
                const real Od = O::mul(xi, O::fma(x2, real(1.0 / 6.0), A1));
                out[(long long)(1 + 8 * k + i) * A.plane] = O::mul(rF, O::add(Ev, Od));
                out[(long long)(5 + 8 * k + i) * A.plane] = O::mul(rF, O::sub(Ev, Od));
            }
        }
        A.lam[(long long)m * A.ld + j] = (real)LamStore<real>::from_lambda(lam_d);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(A.bad, 1);
}

// ---------------------------------------------------------------------------
// Moments (Sec. II.B) from f, plus per-block partial sums of the
// area-weighted totals {mass, momentum x, momentum y, energy}, summed in FP64
// across sites.  FP64 states: every site in FP64.  FP32 states: each site's
// rho, rho u and sum f v^2 in FP32, ring by ring exactly as the step computes
// them (ring_moments), u and T from those in FP32; the outputs are those
// values widened to double (the FP32 state itself carries ~6e-8 relative
// rounding per value, so FP64 per-site arithmetic would add no accuracy).
// out: [5][ntheta][nr] doubles; partials: [gridDim.x][4] (scratch).
// ---------------------------------------------------------------------------
template <typename real>
struct MomArgs {
    const real *f;
    const real *lam;
    double *out;
    double *partials;
    int *status;
    const real *rowtab;  // [ntheta][16] (FP32 moments)
    long long plane;
    int nr, ntheta, ld;
    double r_in, dr, dtheta;
    double th_over_pi;  // theta_m / pi per row
    double v[4];
    real vr[4], v2r[4];  // ring speeds and squares in real (FP32 moments)
    int m0, m1;          // theta rows [m0, m1) of this launch
};

template <typename real>
__global__ void __launch_bounds__(256) moments_kernel(const MomArgs<real> A)
{
    const long long N = (long long)A.nr * A.ntheta;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    if constexpr (sizeof(real) == 4) {
        using O = Op<float>;
        for (long long s = (long long)A.m0 * A.nr + blockIdx.x * (long long)blockDim.x + threadIdx.x;
             s < (long long)A.m1 * A.nr; s += (long long)gridDim.x * blockDim.x) {
            const int m = (int)(s / A.nr), j = (int)(s - (long long)m * A.nr);
            const float *fp = A.f + (long long)m * A.ld + j;
            float fv[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) fv[q] = fp[(long long)q * A.plane];
            float rho, jx, jy, e2;
            ring_moments<float>(fv, A.vr, A.v2r, rho, jx, jy, e2);
            const float inv_rho = O::rcp(rho);
            const float ux = O::mul(jx, inv_rho), uy = O::mul(jy, inv_rho);
            const float u2 = O::fma(ux, ux, O::mul(uy, uy));
            const float T = O::mul(0.5f, O::sub(O::mul(e2, inv_rho), u2));
            const float cth = A.rowtab[(long long)m * 16], sth = -A.rowtab[(long long)m * 16 + 8];
            const float ur = O::fma(ux, cth, O::mul(uy, sth));
            const float uth = O::fma(uy, cth, -O::mul(ux, sth));
            const double lam = LamStore<float>::to_lambda((double)A.lam[(long long)m * A.ld + j]);
            if (A.out) {
                A.out[s] = (double)rho;
                A.out[N + s] = (double)ur;
                A.out[2 * N + s] = (double)uth;
                A.out[3 * N + s] = (double)T;
                A.out[4 * N + s] = lam;
            }
            bad |= !isfinite(rho) || !isfinite(ur) || !isfinite(uth) || !isfinite(T) || !isfinite(lam);
            const double r = A.r_in + (j + 0.5) * A.dr;  // weight r dr dtheta: dr dtheta applied per block
            acc[0] += (double)rho * r;
            acc[1] += (double)jx * r;
            acc[2] += (double)jy * r;
            acc[3] += (double)e2 * r;  // rho T + rho u^2 / 2 = (1/2) sum f v^2 for D = 2
        }
        const double wa = A.dr * A.dtheta;
        acc[0] *= wa;
        acc[1] *= wa;
        acc[2] *= wa;
        acc[3] *= 0.5 * wa;
    } else {
        double cx[8], cy[8];
        cart_dirs(cx, cy);
        for (long long s = (long long)A.m0 * A.nr + blockIdx.x * (long long)blockDim.x + threadIdx.x;
             s < (long long)A.m1 * A.nr; s += (long long)gridDim.x * blockDim.x) {
            const int m = (int)(s / A.nr), j = (int)(s - (long long)m * A.nr);
            const real *fp = A.f + (long long)m * A.ld + j;
            double fv[NV];
            for (int q = 0; q < NV; ++q) fv[q] = (double)fp[(long long)q * A.plane];
            double rho = fv[0], jx = 0.0, jy = 0.0;
            for (int k = 0; k < 4; ++k)
                for (int i = 0; i < 8; ++i) {
                    const double fq = fv[1 + 8 * k + i];
                    rho += fq;
                    jx += fq * A.v[k] * cx[i];
                    jy += fq * A.v[k] * cy[i];
                }
            const double ux = jx / rho, uy = jy / rho;
            double e = 0.5 * fv[0] * (ux * ux + uy * uy);
            for (int k = 0; k < 4; ++k)
                for (int i = 0; i < 8; ++i) {
                    const double dx = A.v[k] * cx[i] - ux, dy = A.v[k] * cy[i] - uy;
                    e += 0.5 * fv[1 + 8 * k + i] * (dx * dx + dy * dy);
                }
            const double T = e / rho;
            double sth, cth;
            sincospi(A.th_over_pi * m, &sth, &cth);
            const double ur = ux * cth + uy * sth, uth = -ux * sth + uy * cth;
            const double lam = LamStore<real>::to_lambda((double)A.lam[(long long)m * A.ld + j]);
            if (A.out) {
                A.out[s] = rho;
                A.out[N + s] = ur;
                A.out[2 * N + s] = uth;
                A.out[3 * N + s] = T;
                A.out[4 * N + s] = lam;
            }
            bad |= !isfinite(rho) || !isfinite(ur) || !isfinite(uth) || !isfinite(T) || !isfinite(lam);
            const double w = (A.r_in + (j + 0.5) * A.dr) * A.dr * A.dtheta;
            acc[0] += rho * w;
            acc[1] += rho * ux * w;
            acc[2] += rho * uy * w;
            acc[3] += (rho * T + 0.5 * rho * (ux * ux + uy * uy)) * w;
        }
    }
    if (bad) atomicOr(A.status, ST_NONFINITE);
    // deterministic block reduction: warp shuffles, then warp 0 over the warps
    __shared__ double red[4][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[c][wid] = v;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double v = lane < nw ? red[c][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0 && A.partials) A.partials[blockIdx.x * 4 + c] = v;
        }
    }
}

// Non-equilibrium manifestations (Sec. II.E): Delta*_m = M*_m(f) - M*_m(f^eq)
// in FP64 from f.  The central moments of the discrete f^eq equal the
// Maxwellian's (M*_2 = rho T I, M*_3 = M*_{3,1} = 0, M*_{4,2} = 2 rho T^2 I for
// D = 2), so only f's moments are summed.  out: [12][ntheta][nr] doubles in the
// order rr, rth, thth | rrr, rrth, rthth, ththth | r, th | rr, rth, thth.
template <typename real>
__global__ void __launch_bounds__(256) noneq_kernel(const MomArgs<real> A)
{
    const long long N = (long long)A.nr * A.ntheta;
    double cx[8], cy[8];
    cart_dirs(cx, cy);
    for (long long s = (long long)A.m0 * A.nr + blockIdx.x * (long long)blockDim.x + threadIdx.x;
         s < (long long)A.m1 * A.nr; s += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(s / A.nr), j = (int)(s - (long long)m * A.nr);
        const real *fp = A.f + (long long)m * A.ld + j;
        double fv[NV];
        for (int q = 0; q < NV; ++q) fv[q] = (double)fp[(long long)q * A.plane];
        double rho = fv[0], jx = 0.0, jy = 0.0;
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < 8; ++i) {
                rho += fv[1 + 8 * k + i];
                jx += fv[1 + 8 * k + i] * A.v[k] * cx[i];
                jy += fv[1 + 8 * k + i] * A.v[k] * cy[i];
            }
        const double ux = jx / rho, uy = jy / rho;
        double sth, cth;
        sincospi(A.th_over_pi * m, &sth, &cth);
        double M[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int q = 0; q < NV; ++q) {
            const int k = q == 0 ? -1 : (q - 1) / 8, i = q == 0 ? 0 : (q - 1) % 8;
            const double vx = k < 0 ? 0.0 : A.v[k] * cx[i], vy = k < 0 ? 0.0 : A.v[k] * cy[i];
            const double dx = vx - ux, dy = vy - uy;
            const double a = dx * cth + dy * sth, b = -dx * sth + dy * cth;  // v* polar
            const double g = fv[q], s2 = a * a + b * b;
            M[0] += g * a * a;
            M[1] += g * a * b;
            M[2] += g * b * b;
            M[3] += g * a * a * a;
            M[4] += g * a * a * b;
            M[5] += g * a * b * b;
            M[6] += g * b * b * b;
            M[7] += 0.5 * g * s2 * a;
            M[8] += 0.5 * g * s2 * b;
            M[9] += 0.5 * g * s2 * a * a;
            M[10] += 0.5 * g * s2 * a * b;
            M[11] += 0.5 * g * s2 * b * b;
        }
        const double T = 0.5 * (M[0] + M[2]) / rho;  // f's own temperature
        M[0] -= rho * T;
        M[2] -= rho * T;
        M[9] -= 2.0 * rho * T * T;
        M[11] -= 2.0 * rho * T * T;
        for (int c = 0; c < 12; ++c) A.out[c * N + s] = M[c];
    }
}

// Sum the per-block partials in a fixed order (one block): totals[4].
static __global__ void __launch_bounds__(256) totals_kernel(const double *partials, int nblocks, double *totals)
{
    __shared__ double red[4][256];
    for (int c = 0; c < 4; ++c) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[b * 4 + c];
        red[c][threadIdx.x] = v;
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) totals[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace dbm
