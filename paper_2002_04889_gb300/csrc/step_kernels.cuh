// Step kernels of the finite-volume shallow-water solver (Giles et al., Sec. 2),
// templated on the arithmetic type.  Included by step_f32.cu and step_f64.cu;
// the FP64 file is compiled with --fmad=false so that every expression rounds
// as written.
//
// One SSP-RK(2,2) step (Sec. 2.3) is two persistent kernels plus a one-CTA
// epilogue:
//   stage 1:  R0 = L(w^n) for every cell (written to scratch) and the running
//             minimum of the CFL bound |K| / (3 max_f l_f a_f)
//   stage 2:  w1 = w^n + dt R0 (dry-fixed), recomputed where needed;
//             w^{n+1} = w^n / 2 + (w1 + dt L(w1)) / 2, dry-fixed
//   epilogue: t += dt, gauges, reset of the CFL minimum (util_kernels.cu)
//
// Each CTA owns a block of B consecutive (renumbered) cells and stages the
// block plus a two-ring halo in shared memory (ring 1: face neighbours of the
// block; ring 2: face neighbours of ring 1), with local indices precomputed on
// the host so that no phase chases an index through global memory:
//   A  load the state of block + ring-1 + ring-2 cells (smem sW: packed
//      (W, Hu, Hv, z) slots) and queue the block's owned faces (a face is owned
//      by the lower local index, a block cell facing the halo, or a wall)
//   B  reconstruct face values of block + ring-1 cells (smem sF: three packed
//      face slots per cell)
//   C  one thread per owned face computes the interface flux once and writes
//      both sides' terms into the two face slots it read
//   D  one thread per block cell gathers its three faces in local order,
//      forms the residual and updates the cell.
// A block whose cells and ring 1 are exactly dry has zero fluxes: B and C are
// skipped for it (dry land).
// No float atomics: the gather order is fixed, and the CFL minimum uses an
// integer atomicMin on the bits of a non-negative value (exact, order-free).
//
// Two arithmetic forms of the same scheme:
//  * FP64: the state is (H, Hu, Hv).  Two builds of the same code: the literal
//    one (FAST = false, step_f64.cu, no multiply-add contraction) evaluates every
//    formula as written, in the same order as any plain implementation of the
//    scheme; the fast one (FAST = true, step_f64_fast.cu, contraction allowed)
//    divides once where the literal form divides several times by the same value
//    (face velocities, the HLL star flux, the residual's 1/|K|) and finds the
//    limiter's smallest ratio by cross products with one division.
//  * FP32 ("deviation"): the state is (eta, Hu, Hv) with eta = H + z, and the
//    momentum flux through each face is carried relative to the hydrostatic
//    pressure g (eta_K - z_{K,f})^2 / 2 of the cell's own free surface over the
//    bed z_{K,f} under its face value.  Summed over a closed triangle these
//    references give exactly the centred bed-slope source of a cell standing on
//    its face beds (and zero for a cell on its flat cell bed), so the scheme is
//    unchanged; but the large terms g H^2 / 2 (1e8 in a 4000 m ocean) never
//    appear, only products of small differences (eta_f - eta_K, z* - z_K), so
//    still water stays still in FP32 and eta keeps full FP32 resolution.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "vg_internal.h"

namespace vg {

template <typename real>
struct KArgs {
    int64_t nc;
    int block, nblocks, max_halo, max_ring1, order;
    const real *geo;        // [GEO_ROWS][nc]
    const real *z;          // [nc]
    const real *zf;         // face beds: FP64 [3][nc]; FP32 [nc][2] z_f - z_K of faces 0, 1
    const int32_t *nbr;     // [3][nc]
    const uint16_t *nbrl;   // [3][nc]
    const int32_t *halo_ptr;  // [nblocks + 1]
    const int32_t *halo_n1;   // [nblocks] ring-1 count
    const int32_t *halo_ids;  // per block: ring 1 then ring 2
    const uint16_t *ring1_nbr;// [3 * ring cells] local neighbours of ring-1 cells
    const int32_t *fq_ptr;  // [nblocks + 1] into fq
    const uint16_t *fq;     // owned faces of each block: (local cell << 2) | face
    const real *w;          // w^n [3][nc]
    real *R0;               // [3][nc]
    real *wout;             // w^{n+1} [3][nc] (stage 2)
    uint8_t *mask2;         // optional: stage-2 dry-fix branch (0 none, 1 momentum cut, 2 emptied)
    real *fv_out;           // optional [3 vars][3 faces][nc]: face values of the block cells
    real *r1_out;           // optional [3][nc]: the stage-2 residual L(w1) (stage 2)
    uint8_t *rec_out;       // optional [nc]: 1 where the block cell reconstructed (FP64)
    DevScalars *sc;
    real g, half_g, hthr;
    double cfl, dt_fixed, dt_max, t_end;
    int cfl_min;            // stage 1: 1 adds the CFL bound to the step's minimum
};

__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ double vabs(double a) { return fabs(a); }
__device__ __forceinline__ float vsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double vsqrt(double a) { return sqrt(a); }

// Compare and select.  GB300 runs FP64 compares and min/max on its FP64 units,
// which issue two lane-operations per SM and cycle, while its integer units are
// idle in the FP64 kernels; so the FP64 forms below work on the IEEE bit patterns
// with integer instructions.  For the non-NaN values of the step they decide and
// select exactly as the FP64 instructions do (a zero result may carry the other
// sign, which no later operation of the step distinguishes).  The FP32 forms are
// the plain FP32 instructions.
//   gt_nn(x, y): x > y for y >= +0;  is_zero(x): x == 0;  is_neg(x): x < 0;
//   is_pos(x): x > 0;  smax / smin: max / min;  max0(x): max(0, x).
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ unsigned long long ubits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ long long okey(double x)   // order-preserving for every non-NaN x
{
    const long long b = dbits(x);
    return b < 0 ? b ^ 0x7fffffffffffffffLL : b;
}
__device__ __forceinline__ bool gt_nn(float x, float y) { return x > y; }
__device__ __forceinline__ bool gt_nn(double x, double y) { return dbits(x) > dbits(y); }
__device__ __forceinline__ bool is_zero(float x) { return x == 0.f; }
__device__ __forceinline__ bool is_zero(double x) { return (ubits(x) << 1) == 0; }
__device__ __forceinline__ bool is_neg(float x) { return x < 0.f; }
__device__ __forceinline__ bool is_neg(double x) { return dbits(x) < 0 && (ubits(x) << 1) != 0; }
__device__ __forceinline__ bool is_pos(float x) { return x > 0.f; }
__device__ __forceinline__ bool is_pos(double x) { return dbits(x) > 0; }
__device__ __forceinline__ float smax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double smax(double a, double b) { return okey(a) < okey(b) ? b : a; }
__device__ __forceinline__ float smin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double smin(double a, double b) { return okey(b) < okey(a) ? b : a; }
__device__ __forceinline__ float max0(float x) { return fmaxf(0.f, x); }
__device__ __forceinline__ double max0(double x) { return dbits(x) > 0 ? x : 0.0; }

template <typename real> __device__ __forceinline__ real real_inf();
template <> __device__ __forceinline__ float real_inf<float>() { return CUDART_INF_F; }
template <> __device__ __forceinline__ double real_inf<double>() { return CUDART_INF; }

// Order-preserving integer image of a non-negative real for atomicMin.
__device__ __forceinline__ unsigned long long min_bits(float v) { return (unsigned long long)__float_as_uint(v); }
__device__ __forceinline__ unsigned long long min_bits(double v) { return (unsigned long long)__double_as_longlong(v); }
template <typename real> __device__ __forceinline__ double decode_min(unsigned long long b);
template <> __device__ __forceinline__ double decode_min<float>(unsigned long long b) { return (double)__uint_as_float((unsigned int)b); }
template <> __device__ __forceinline__ double decode_min<double>(unsigned long long b) { return __longlong_as_double((long long)b); }

// Time step of the current step from the stage-1 CFL minimum (Sec. 2.3 CFL
// condition, read as dt = cfl * min_K |K| / (3 max_f l_f a_f)), then the
// dt_max and t_end clamps.
template <typename real>
__device__ __forceinline__ double step_dt(const DevScalars *sc, double cfl, double dt_fixed,
                                          double dt_max, double t_end)
{
    double dt;
    if (dt_fixed > 0.0) {
        dt = dt_fixed;
    } else {
        double mn = decode_min<real>(sc->dtmin_bits);
        dt = isinf(mn) ? (dt_max > 0.0 ? dt_max : 0.0) : cfl * mn;
    }
    if (dt_max > 0.0) dt = fmin(dt, dt_max);
    double t = sc->t;
    if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
    if (dt < 0.0) dt = 0.0;
    return dt;
}

// HLL flux in the face normal frame (Sec. 2.2) with the dry-bed speeds when one
// side is dry; each side is (H*, u_n, u_t).
template <typename real, bool FAST = false>
__device__ __forceinline__ void hll_normal(real g, real half_g, real HL, real unL, real utL,
                                           real HR, real unR, real utR, real F[3], real &amax)
{
    if (is_zero(HL) && is_zero(HR)) {
        F[0] = real(0); F[1] = real(0); F[2] = real(0);
        amax = real(0);
        return;
    }
    real cL = vsqrt(g * HL);
    real cR = vsqrt(g * HR);
    real sL, sR;
    if (is_zero(HL)) {
        sL = unR - real(2) * cR;
        sR = unR + cR;
    } else if (is_zero(HR)) {
        sL = unL - cL;
        sR = unL + real(2) * cL;
    } else {
        real us = real(0.5) * (unL + unR) + (cL - cR);
        real cs = real(0.5) * (cL + cR) - real(0.25) * (unR - unL);
        sL = smin(unL - cL, us - cs);
        sR = smax(us + cs, unR + cR);
    }
    real qL = HL * unL, qR = HR * unR;
    real FL0 = qL, FL1 = qL * unL + half_g * HL * HL, FL2 = qL * utL;
    real FR0 = qR, FR1 = qR * unR + half_g * HR * HR, FR2 = qR * utR;
    if (!is_neg(sL)) {
        F[0] = FL0; F[1] = FL1; F[2] = FL2;
    } else if (!is_neg(sR)) {
        real den = sR - sL;
        real sLR = sL * sR;
        if constexpr (FAST) {
            const real rd = real(1) / den;
            F[0] = ((sR * FL0 - sL * FR0) + sLR * (HR - HL)) * rd;
            F[1] = ((sR * FL1 - sL * FR1) + sLR * (qR - qL)) * rd;
            F[2] = ((sR * FL2 - sL * FR2) + sLR * (HR * utR - HL * utL)) * rd;
        } else {
            F[0] = ((sR * FL0 - sL * FR0) + sLR * (HR - HL)) / den;
            F[1] = ((sR * FL1 - sL * FR1) + sLR * (qR - qL)) / den;
            F[2] = ((sR * FL2 - sL * FR2) + sLR * (HR * utR - HL * utL)) / den;
        }
    } else {
        F[0] = FR0; F[1] = FR1; F[2] = FR2;
    }
    amax = smax(vabs(sL), vabs(sR));
}

// Flux through a face seen from its left cell: face velocities, hydrostatic
// interface depths z* = max(z_L, z_R), H*_s = max(0, H_{s,f} + z_s - z*) with z_s
// the bed under side s's face value (its face bed if it reconstructed), HLL,
// rotation back to (x, y), pressure corrections g (H_{s,f}^2 - H*_s^2) / 2.
// bnd: 0 interior; 1 wall, the ghost of Sec. 2.5 (u_n reversed, u_t kept, same
// depth); 2 open, the transmissive ghost (the face state itself); 3 absorbing,
// the characteristic ghost (u_n + 2c of the face state, u_n - 2c = -2 c_0 of the
// sea at rest with c_0 = sqrt(g max(0, -z)): depth c_g^2 / g, u_t kept).
template <typename real, bool FAST = false>
__device__ __forceinline__ void face_flux(real g, real half_g, real hthr,
                                          real HfL, real HufL, real HvfL, real zL,
                                          real HfR, real HufR, real HvfR, real zR,
                                          real nx, real ny, int bnd,
                                          real Phi[3], real &PL, real &PR, real &amax)
{
    real uL = real(0), vL = real(0);
    if (gt_nn(HfL, hthr)) {
        if constexpr (FAST) {
            const real r = real(1) / HfL;
            uL = HufL * r; vL = HvfL * r;
        } else {
            uL = HufL / HfL; vL = HvfL / HfL;
        }
    }
    real unL = uL * nx + vL * ny;
    real utL = -uL * ny + vL * nx;
    real HsL, HsR, unR, utR;
    if (bnd == 3) {
        // absorbing: the characteristic ghost of a sea at rest (eta = 0) beyond
        // the boundary, on the same bed (the oracle's order of operations)
        HsL = max0((HfL + zL) - zL);
        const real cL = vsqrt(g * HsL), c0 = vsqrt(g * max0(real(0) - zL));
        const real Rp = unL + real(2) * cL, Rm = real(0) - real(2) * c0;
        unR = real(0.5) * (Rp + Rm);
        const real cg = max0(real(0.25) * (Rp - Rm));
        HsR = cg * cg / g;
        utR = utL;
        HfR = HsR;
    } else if (bnd) {
        HsL = max0((HfL + zL) - zL);
        HsR = HsL;
        unR = bnd == 2 ? unL : -unL;
        utR = utL;
        HfR = HfL;
    } else {
        real uR = real(0), vR = real(0);
        if (gt_nn(HfR, hthr)) {
            if constexpr (FAST) {
                const real r = real(1) / HfR;
                uR = HufR * r; vR = HvfR * r;
            } else {
                uR = HufR / HfR; vR = HvfR / HfR;
            }
        }
        unR = uR * nx + vR * ny;
        utR = -uR * ny + vR * nx;
        real zs = smax(zL, zR);
        HsL = max0((HfL + zL) - zs);
        HsR = max0((HfR + zR) - zs);
    }
    real F[3];
    hll_normal<real, FAST>(g, half_g, HsL, unL, utL, HsR, unR, utR, F, amax);
    Phi[0] = F[0];
    Phi[1] = F[1] * nx - F[2] * ny;
    Phi[2] = F[1] * ny + F[2] * nx;
    PL = half_g * (HfL * HfL - HsL * HsL);
    PR = half_g * (HfR * HfR - HsR * HsR);
}

// Approximate reciprocal (PTX rcp.approx.ftz.f32, max error 1 ulp); rcp(0) = +inf.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Deviation form for FP32, literal form for FP64.
template <typename real> struct EtaForm { static constexpr bool value = false; };
template <> struct EtaForm<float> { static constexpr bool value = true; };

// FP32 cell geometry record, 16 floats (four 16-byte words, 64 bytes) per cell:
//   M00 M01 M02 M10 | M11 M12 area l0 | nx0 ny0 nx1 ny1 | nx2 ny2 l1 l2
// with M_fj = w_j . (x_f - x_K): the increments of the reconstruction are
// D_f = sum_j M_fj (q_j - q_K), the same quantity as grad q . (x_f - x_K) with the
// least-squares gradient grad q = sum_j w_j (q_j - q_K).  The face midpoints
// average to the centroid x_K, so D_2 = -(D_0 + D_1) and row 2 is not stored.
// (FP64 keeps the rows GEO_* and evaluates gradient then dot product, in the
// literal order.)
constexpr int G32 = 16;
constexpr int G32_AREA = 6;
__device__ __forceinline__ const float4 *g32(const float *geo, int k)
{
    return reinterpret_cast<const float4 *>(geo + (size_t)k * G32);
}
__device__ __forceinline__ float2 g32_normal(const float *geo, int k, int f)
{
    return *reinterpret_cast<const float2 *>(geo + (size_t)k * G32 + 8 + 2 * f);
}
__device__ __forceinline__ float g32_len(const float *geo, int k, int f)
{
    return geo[(size_t)k * G32 + (f == 0 ? 7 : 13 + f)];
}

// L1 prefetch (a hint: nothing waits for it and it holds no register).
__device__ __forceinline__ void prefetch_l1(const void *ptr)
{
    asm volatile("prefetch.global.L1 [%0];" :: "l"(ptr));
}

// Stored state of cell gid as seen by the stage (H or eta first, then Hu, Hv):
// stage 1 reads w^n; stage 2 forms w1 = w^n + dt R0 and applies the dry fix
// (negative depth emptied; at or below the threshold, momentum zeroed).
// Returns true if a negative depth was met.
template <typename real, int STAGE>
__device__ __forceinline__ bool stage_state(const KArgs<real> &a, int gid, real dt, real zc, real &W,
                                            real &Hu, real &Hv, real *wn = nullptr)
{
    constexpr bool ETA = EtaForm<real>::value;
    const int nc = (int)a.nc;
    W = a.w[gid];
    Hu = a.w[nc + gid];
    Hv = a.w[2 * nc + gid];
    if (wn) { wn[0] = W; wn[1] = Hu; wn[2] = Hv; }
    if (STAGE == 1) return false;
    W = W + dt * a.R0[gid];
    Hu = Hu + dt * a.R0[nc + gid];
    Hv = Hv + dt * a.R0[2 * nc + gid];
    real H = ETA ? W - zc : W;
    if (is_neg(H)) {
        W = ETA ? zc : real(0);
        Hu = real(0); Hv = real(0);
        return true;
    }
    if (!gt_nn(H, a.hthr)) { Hu = real(0); Hv = real(0); }
    return false;
}

// Deviation-form flux (FP32).  Inputs per side: face eta_f and momenta, the bed
// z under the face value (face bed or cell bed) and the cell's own eta; H below
// is eta - z of that side.  Same interface depths and HLL as face_flux, with
//   d* = H*_L - H*_R          (eta_fL - eta_fR when both sides are wet)
//   F1 - C_e for C_e = g H*_L H*_R / 2:  L: q_L u_nL + g H*_L d* / 2,
//                                        R: q_R u_nR - g H*_R d* / 2
// (HLL is affine in F with weights summing to one, so F* shifts by -C_e), and
// side terms Q_s = C_e + P_s - g H_s^2 / 2 that replace the pressure correction:
//   Q_L = g/2 [(eta_fL - eta_L)(H_fL + H_L) - H*_L d*],
//   Q_R = g/2 [(eta_fR - eta_R)(H_fR + H_R) + H*_R d*].
__device__ __forceinline__ void face_flux_dev(float g, float half_g, float hthr,
                                              float efL, float HufL, float HvfL, float zL, float eL,
                                              float efR, float HufR, float HvfR, float zR, float eR,
                                              float nx, float ny, int bnd,
                                              float Phi[3], float &QL, float &QR, float &amax)
{
    float HfL = efL - zL;
    float uL = 0.f, vL = 0.f;
    if (HfL > hthr) { const float r = rcp_approx(HfL); uL = HufL * r; vL = HvfL * r; }
    float unL = uL * nx + vL * ny;
    float utL = -uL * ny + vL * nx;
    float HsL, HsR, unR, utR, ds, HfR;
    if (bnd == 3) {
        // absorbing: the outgoing invariant u_n + 2c of the face state and the
        // incoming u_n - 2c of the sea at rest (eta = 0) beyond the boundary
        HsL = fmaxf(0.f, HfL);
        const float cL = sqrtf(g * HsL), c0 = sqrtf(g * fmaxf(0.f, -zL));
        const float Rp = unL + 2.f * cL, Rm = -2.f * c0;
        const float cg = fmaxf(0.f, 0.25f * (Rp - Rm));
        unR = 0.5f * (Rp + Rm);
        HsR = cg * cg / g;
        utR = utL;
        ds = HsL - HsR;
        HfR = HsR; efR = zL + HsR; eR = efR; zR = zL;
    } else if (bnd) {
        HsL = fmaxf(0.f, HfL);
        HsR = HsL;
        unR = bnd == 2 ? unL : -unL;
        utR = utL;
        ds = 0.f;
        HfR = HfL; efR = efL; eR = eL; zR = zL;
    } else {
        HfR = efR - zR;
        float uR = 0.f, vR = 0.f;
        if (HfR > hthr) { const float r = rcp_approx(HfR); uR = HufR * r; vR = HvfR * r; }
        unR = uR * nx + vR * ny;
        utR = -uR * ny + vR * nx;
        float zs = fmaxf(zL, zR);
        HsL = fmaxf(0.f, efL - zs);
        HsR = fmaxf(0.f, efR - zs);
        ds = (HsL > 0.f && HsR > 0.f) ? efL - efR : HsL - HsR;
    }
    float F[3];
    if (HsL == 0.f && HsR == 0.f) {
        F[0] = 0.f; F[1] = 0.f; F[2] = 0.f;
        amax = 0.f;
    } else {
        float cL = sqrtf(g * HsL), cR = sqrtf(g * HsR);
        float sL, sR;
        if (HsL == 0.f) {
            sL = unR - 2.f * cR;
            sR = unR + cR;
        } else if (HsR == 0.f) {
            sL = unL - cL;
            sR = unL + 2.f * cL;
        } else {
            float us = 0.5f * (unL + unR) + (cL - cR);
            float cs = 0.5f * (cL + cR) - 0.25f * (unR - unL);
            sL = fminf(unL - cL, us - cs);
            sR = fmaxf(us + cs, unR + cR);
        }
        float qL = HsL * unL, qR = HsR * unR;
        float FL0 = qL, FL1 = qL * unL + half_g * HsL * ds, FL2 = qL * utL;
        float FR0 = qR, FR1 = qR * unR - half_g * HsR * ds, FR2 = qR * utR;
        // HLL with the speeds clamped to a <= 0 <= b, which also gives F_L when
        // sL >= 0 and F_R when sR <= 0 (b - a > 0 unless both sides are dry)
        const float a = fminf(sL, 0.f), b = fmaxf(sR, 0.f);
        const float rden = rcp_approx(b - a), ab = a * b;
        F[0] = ((b * FL0 - a * FR0) - ab * ds) * rden;
        F[1] = ((b * FL1 - a * FR1) + ab * (qR - qL)) * rden;
        F[2] = ((b * FL2 - a * FR2) + ab * (HsR * utR - HsL * utL)) * rden;
        amax = fmaxf(fabsf(sL), fabsf(sR));
    }
    Phi[0] = F[0];
    Phi[1] = F[1] * nx - F[2] * ny;
    Phi[2] = F[1] * ny + F[2] * nx;
    float HL = eL - zL, HR = eR - zR;
    QL = half_g * ((efL - eL) * (HfL + HL) - HsL * ds);
    QR = half_g * ((efR - eR) * (HfR + HR) + HsR * ds);
}

// An exactly dry cell: no water and no momentum.
template <typename real>
__device__ __forceinline__ bool exactly_dry(real W, real Hu, real Hv, real zc)
{
    const real H = EtaForm<real>::value ? W - zc : W;
    return is_zero(H) && is_zero(Hu) && is_zero(Hv);
}

// Stored state of cell gid as seen by the stage, and its bed.
template <typename real, int STAGE>
__device__ __forceinline__ bool stage_cell(const KArgs<real> &a, int gid, real dt, real &W, real &Hu, real &Hv,
                                           real &zc, real *wn = nullptr)
{
    zc = a.z[gid];
    return stage_state<real, STAGE>(a, gid, dt, zc, W, Hu, Hv, wn);
}

// Four reals in shared memory, moved as one 16-byte (FP32) or two 16-byte
// (FP64) accesses.
__device__ __forceinline__ void ld4(const float *p, float &x, float &y, float &z, float &w)
{
    float4 v = *reinterpret_cast<const float4 *>(p);
    x = v.x; y = v.y; z = v.z; w = v.w;
}
__device__ __forceinline__ void st4(float *p, float x, float y, float z, float w)
{
    *reinterpret_cast<float4 *>(p) = make_float4(x, y, z, w);
}
__device__ __forceinline__ void ld4(const double *p, double &x, double &y, double &z, double &w)
{
    double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    x = a.x; y = a.y; z = b.x; w = b.y;
}
__device__ __forceinline__ void st4(double *p, double x, double y, double z, double w)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(x, y);
    reinterpret_cast<double2 *>(p)[1] = make_double2(z, w);
}

// SSP-RK(2,2) second stage (Sec. 2.3) of one cell: w^{n+1} = w^n / 2 + (w1 + dt R(w1)) / 2
// from w^n = x, w1 = (W1, Hu1, Hv1) and R(w1) = (RH, RHu, RHv), then the dry fix.
// Returns the fix's branch: 0 none, 1 momentum cut (depth at or below the
// threshold), 2 negative depth emptied.
template <typename real>
__device__ __forceinline__ uint8_t rk2_final(const real x[3], real W1, real Hu1, real Hv1, real RH, real RHu,
                                             real RHv, real dt, real z1, real hthr, real &W, real &Hu, real &Hv)
{
    constexpr bool ETA = EtaForm<real>::value;
    W = real(0.5) * x[0] + real(0.5) * (W1 + dt * RH);
    Hu = real(0.5) * x[1] + real(0.5) * (Hu1 + dt * RHu);
    Hv = real(0.5) * x[2] + real(0.5) * (Hv1 + dt * RHv);
    const real H = ETA ? W - z1 : W;
    if (is_neg(H)) {
        W = ETA ? z1 : real(0);
        Hu = real(0); Hv = real(0);
        return 2;
    }
    if (!gt_nn(H, hthr)) {
        Hu = real(0); Hv = real(0);
        return 1;
    }
    return 0;
}

// Phase D's end for block cell l (global gid), from the sums of its three face
// terms: R = -(aH, aHu, aHv) / |K|; stage 1 writes R0 and the CFL bound of
// am = max_f l_f a_f; stage 2 forms w^{n+1} = w^n / 2 + (w1 + dt R) / 2 with
// w^n = x, w1 from shared memory, and the dry fix.
template <typename real, int STAGE, bool FAST = false>
__device__ __forceinline__ void finish_cell(const KArgs<real> &a, int gid, const real *sWl, real aH, real aHu,
                                            real aHv, real am, const real x[3], real area, real dt, real &my_min,
                                            long long &my_neg, bool &bad)
{
    constexpr bool ETA = EtaForm<real>::value;
    const int nc = (int)a.nc;
    real RH, RHu, RHv;
    if constexpr (FAST) {
        const real ia = real(1) / area;
        RH = -aH * ia; RHu = -aHu * ia; RHv = -aHv * ia;
    } else {
        RH = -aH / area; RHu = -aHu / area; RHv = -aHv / area;
    }
    if (STAGE == 1) {
        a.R0[gid] = RH;
        a.R0[nc + gid] = RHu;
        a.R0[2 * nc + gid] = RHv;
        if (is_pos(am)) my_min = smin(my_min, area / (real(3) * am));
    } else {
        if (a.r1_out) {
            a.r1_out[gid] = RH;
            a.r1_out[nc + gid] = RHu;
            a.r1_out[2 * nc + gid] = RHv;
        }
        real W1, Hu1, Hv1, z1;
        ld4(sWl, W1, Hu1, Hv1, z1);
        real W, Hu, Hv;
        const uint8_t branch = rk2_final(x, W1, Hu1, Hv1, RH, RHu, RHv, dt, z1, a.hthr, W, Hu, Hv);
        if (branch == 2) my_neg++;
        if (a.mask2) a.mask2[gid] = branch;
        if (!isfinite(W) || !isfinite(Hu) || !isfinite(Hv)) bad = true;
        a.wout[gid] = W;
        a.wout[nc + gid] = Hu;
        a.wout[2 * nc + gid] = Hv;
    }
}

// Shared memory of one CTA: cell states [L] x 4, face slots [3][L1] x 4 (L1 =
// block + ring 1), with gids the global ids of block and ring-1 cells [L1],
// face codes and owned-face queue [3B] each, and for FP64 one byte per block and
// ring-1 cell: whether it reconstructed (phase D adds its bed-slope source).  Without gids phase B reads a
// ring-1 cell's global id again from the halo list: at 6 CTAs per SM every
// kilobyte of shared memory is a kilobyte less of L1.  The batched kernels keep
// the ids (their extra scenario state leaves no register for the reload).
template <typename real>
__host__ __device__ inline size_t stage_smem_bytes(int block, int max_halo, int max_ring1, bool gids = false)
{
    size_t L = (size_t)block + max_halo, L1 = (size_t)block + max_ring1;
    return sizeof(real) * 4 * (L + 3 * L1) + (gids ? sizeof(int32_t) * L1 : 0) + sizeof(uint16_t) * 6 * (size_t)block +
           (sizeof(real) == 8 ? L1 : 0) + 16;
}

// One block of cells for one scenario: phases A-D (see the top of this file).
// my_min collects the thread's stage-1 CFL bound, my_neg its negative-depth
// events, bad a non-finite result.  Every thread of the CTA must call it;
// qcount is the CTA's shared count of queued faces.
//
// The queue of owned faces is copied from the list built with the partition
// (LISTED) or formed in phase A from the face codes by a warp-aggregated
// append; the list is faster in the stage-2 kernels and the batched kernels,
// the append in the single-scenario stage-1 kernels.
// Either way every face of the block is queued once, and the result does not
// depend on the queue order (each face writes its own two slots).
//
// There is no barrier after phase D: a thread's phase D reads only its own
// cell's state slot and face slots, the next block's phase A writes state
// slots of its own cells, codes, the face queue and its count only, and face
// slots are next written in phase B, behind the barrier that ends phase A.
// Consecutive blocks use the two queue counters alternately (an append's
// counter is reset in phase D, which may come after other warps have started
// the next block).
//
// Shared layout: sW[l] = (W, Hu, Hv, z) of local cell l (W = eta for FP32, H
// for FP64); sF[f][l] = face values (W_f, Hu_f, Hv_f, z_f) of face f of cell l
// after phase B, z_f the bed the face value stands on, and after phase C the
// cell's own term (l_f Phi_0, l_f (Phi_1 + P n_x), l_f (Phi_2 + P n_y), l_f a_f).
// Stage 2's phase D reads w^n of its cell from global memory.
template <typename real, int STAGE, int DRY, bool LISTED, bool GIDS, bool FAST = false>
__device__ __forceinline__ void process_block(const KArgs<real> &a, const int b, const real dt,
                                              unsigned char *smem_raw, int &qcount, real &my_min,
                                              long long &my_neg, bool &bad)
{
    const int B = a.block;
    const int L = B + a.max_halo;
    const int L1 = B + a.max_ring1;
    const int nc = (int)a.nc;    // per-cell arrays hold < 2^31 entries (checked at upload)
    real *sW = reinterpret_cast<real *>(smem_raw);          // [L][4]
    real *sF = sW + 4 * L;                                   // [3][L1][4]
    int32_t *sGid = reinterpret_cast<int32_t *>(sF + 12 * L1);   // [L1] (GIDS)
    uint16_t *sCode = reinterpret_cast<uint16_t *>(GIDS ? sGid + L1 : sGid);   // [3][B]
    uint16_t *queue = sCode + 3 * B;                              // [3B]
    uint8_t *sRec = reinterpret_cast<uint8_t *>(queue + 3 * B);   // [L1]

    constexpr bool ETA = EtaForm<real>::value;
    const int tid = threadIdx.x;
    const real g = a.g, half_g = a.half_g, hthr = a.hthr;
    const real *geo = a.geo;

    const int c0 = b * B;
    const int ncell = min(B, nc - c0);
    const int h0 = a.halo_ptr[b];
    const int nh = a.halo_ptr[b + 1] - h0;
    const int n1 = a.halo_n1[b];

    // A: block + ring-1 + ring-2 states into shared memory, and the block's
    // owned faces (a boundary face, a face to the halo, or a face to a block
    // cell of higher local index: every face once) into the queue.  Thread
    // tid < B takes block cell tid.  The threads also note whether the block
    // and its ring 1 are exactly dry (dry land): then every face of the block
    // has zero interface depths on both sides, hence zero flux and zero
    // pressure terms, and phases B and C reduce to zero face terms.
    bool dry = true;
    {
        int gh = -1;
        if (tid < nh) gh = a.halo_ids[h0 + tid];
        if constexpr (LISTED) {
            const int q0 = a.fq_ptr[b], nq = a.fq_ptr[b + 1] - q0;
            for (int q = tid; q < nq; q += blockDim.x) queue[q] = a.fq[q0 + q];
            if (tid == 0) qcount = nq;
        }
        int owned = 0;
        if (tid < ncell) {
            const int gid = c0 + tid;
#pragma unroll
            for (int f = 0; f < 3; f++) {
                const uint16_t code = a.nbrl[f * nc + gid];
                sCode[f * B + tid] = code;
                if (!LISTED && (code >= NBR_ABSORB || (code >> 2) >= B || (int)(code >> 2) > tid)) owned |= 1 << f;
            }
            real W, Hu, Hv, zc;
            bool neg = stage_cell<real, STAGE>(a, gid, dt, W, Hu, Hv, zc);
            if constexpr (ETA) {
                // a wet cell may reconstruct: phase B reads its geometry record and
                // face beds right after the barrier below, so start bringing them
                // into L1 (a dry cell reads neither)
                if (W - zc > hthr) {
                    prefetch_l1(g32(geo, gid));
                    prefetch_l1(reinterpret_cast<const float2 *>(a.zf) + gid);
                }
            }
            if (neg) my_neg++;
            st4(sW + 4 * tid, W, Hu, Hv, zc);
            if constexpr (GIDS) sGid[tid] = gid;
            dry = exactly_dry(W, Hu, Hv, zc);
        }
        if (gh >= 0) {
            real W, Hu, Hv, zc;
            stage_cell<real, STAGE>(a, gh, dt, W, Hu, Hv, zc);
            if constexpr (ETA) {
                if (tid < n1 && W - zc > hthr) {     // a wet ring-1 cell: phase B reconstructs it too
                    prefetch_l1(g32(geo, gh));
                    prefetch_l1(reinterpret_cast<const float2 *>(a.zf) + gh);
                    prefetch_l1(a.ring1_nbr + 3 * (h0 + tid));
                }
            }
            st4(sW + 4 * (B + tid), W, Hu, Hv, zc);
            if (tid < n1) {
                if constexpr (GIDS) sGid[B + tid] = gh;
                dry = dry && exactly_dry(W, Hu, Hv, zc);
            }
        }
        for (int h = tid + blockDim.x; h < nh; h += blockDim.x) {
            const int gid = a.halo_ids[h0 + h];
            real W, Hu, Hv, zc;
            stage_cell<real, STAGE>(a, gid, dt, W, Hu, Hv, zc);
            st4(sW + 4 * (B + h), W, Hu, Hv, zc);
            if (h < n1) {
                if constexpr (GIDS) sGid[B + h] = gid;
                dry = dry && exactly_dry(W, Hu, Hv, zc);
            }
        }
        if constexpr (!LISTED) {
            // warp-aggregated queue append: n = popcount(owned) in 0..3
            const int n = __popc(owned);
            const unsigned lane = tid & 31;
            const unsigned lt = (1u << lane) - 1u;
            const unsigned b1 = __ballot_sync(0xffffffffu, n & 1), b2 = __ballot_sync(0xffffffffu, n & 2);
            const int total = __popc(b1) + 2 * __popc(b2);
            int base = 0;
            if (lane == 0 && total) base = atomicAdd(&qcount, total);
            base = __shfl_sync(0xffffffffu, base, 0);
            int pos = base + __popc(b1 & lt) + 2 * __popc(b2 & lt);
#pragma unroll
            for (int f = 0; f < 3; f++)
                if ((owned >> f) & 1) queue[pos++] = (uint16_t)((tid << 2) | f);
        }
    }
    // Dry land.  Mode 1 leaves the block here with a zero residual (phase D with
    // zero face terms; w^n from memory) and writes the adjoint's recordings as
    // the full phases would (a dry cell's face values are its own values); mode 2
    // has phase B write zero face terms for the block cells (and w^n for stage
    // 2) and phase C no faces, which costs a few instructions more but no
    // register spills where mode 1 would spill (runs with recordings take every
    // phase there).
    bool skip = false;
    if constexpr (DRY == 0)
        __syncthreads();
    else
        skip = __syncthreads_and(dry) && (DRY == 1 || (!a.fv_out && !a.mask2 && !a.r1_out && (ETA || !a.rec_out)));
    if (DRY == 1 && skip) {
        if (!LISTED && tid == 0) qcount = 0;
        if (tid < ncell) {
            const int gid = c0 + tid;
            if constexpr (!ETA)
                if (a.rec_out) a.rec_out[gid] = 0;
            if (a.fv_out) {
                real Wc, Huc, Hvc, zc;
                ld4(sW + 4 * tid, Wc, Huc, Hvc, zc);
#pragma unroll
                for (int f = 0; f < 3; f++) {
                    a.fv_out[(0 * 3 + f) * (size_t)nc + gid] = Wc;
                    a.fv_out[(1 * 3 + f) * (size_t)nc + gid] = Huc;
                    a.fv_out[(2 * 3 + f) * (size_t)nc + gid] = Hvc;
                }
            }
            real x[3] = {real(0), real(0), real(0)};
            if (STAGE == 2) { x[0] = a.w[gid]; x[1] = a.w[nc + gid]; x[2] = a.w[2 * nc + gid]; }
            // R = -0 / |K| = -0 for any area, so the area is not read
            finish_cell<real, STAGE, FAST>(a, gid, sW + 4 * tid, real(0), real(0), real(0), real(0), x, real(1), dt,
                                     my_min, my_neg, bad);
        }
        return;
    }
    const bool zero_terms = DRY == 2 && skip;

    // B: face values of block + ring-1 cells (Sec. 2.4, Eq. recon with the
    // Barth-Jespersen limiter); every neighbour is in shared memory
    for (int l = tid; l < (zero_terms ? ncell : B + n1); l += blockDim.x) {
        if (l < B && l >= ncell) continue;
        const int gid = GIDS ? sGid[l] : l < B ? c0 + l : a.halo_ids[h0 + (l - B)];
        if (zero_terms) {
#pragma unroll
            for (int f = 0; f < 3; f++) st4(sF + 4 * (f * L1 + l), real(0), real(0), real(0), real(0));
            if constexpr (!ETA) sRec[l] = 0;
            continue;
        }
        real WK, HuK, HvK, zK;
        ld4(sW + 4 * l, WK, HuK, HvK, zK);
        const real HK = ETA ? WK - zK : WK;
        real qK[3] = {ETA ? WK : HK + zK, HuK, HvK};
        real qn[3][3];
        bool recon = (a.order == 2) && gt_nn(HK, hthr);
#pragma unroll
        for (int f = 0; f < 3; f++) {
            uint16_t code;
            int nl;
            if (l < B) {
                code = sCode[f * B + l];
                nl = code >> 2;
            } else {
                code = a.ring1_nbr[3 * (h0 + (l - B)) + f];
                nl = code;
            }
            if (code < NBR_ABSORB) {
                real Wj, Huj, Hvj, zj;
                ld4(sW + 4 * nl, Wj, Huj, Hvj, zj);
                const real Hj = ETA ? Wj - zj : Wj;
                qn[f][0] = ETA ? Wj : Hj + zj;
                qn[f][1] = Huj;
                qn[f][2] = Hvj;
                if (!gt_nn(Hj, hthr)) recon = false;
            } else if (code != NBR_WALL) {
                // open or absorbing face: the cell's own values (zero gradient)
                qn[f][0] = qK[0];
                qn[f][1] = HuK;
                qn[f][2] = HvK;
            } else {
                real nxf, nyf;
                if constexpr (ETA) {
                    float2 nf = g32_normal(geo, gid, f);
                    nxf = nf.x; nyf = nf.y;
                } else {
                    nxf = geo[(GEO_NX + f) * nc + gid]; nyf = geo[(GEO_NY + f) * nc + gid];
                }
                real mn = HuK * nxf + HvK * nyf;
                qn[f][0] = qK[0];
                qn[f][1] = HuK - real(2) * mn * nxf;
                qn[f][2] = HvK - real(2) * mn * nyf;
            }
        }
        real Hf[3], Huf[3], Hvf[3];
        real zfK[3] = {zK, zK, zK};       // the bed under each face value
        if (recon) {
            real face[3][3];
            real Mf[2][3];          // FP32: rows 0 and 1 of M
            real fx[3], fy[3], wx[3], wy[3];
            if constexpr (ETA) {
                const float4 *r = g32(geo, gid);
                float4 a0 = r[0], a1 = r[1];
                Mf[0][0] = a0.x; Mf[0][1] = a0.y; Mf[0][2] = a0.z;
                Mf[1][0] = a0.w; Mf[1][1] = a1.x; Mf[1][2] = a1.y;
            } else {
#pragma unroll
                for (int f = 0; f < 3; f++) {
                    fx[f] = geo[(GEO_FX + f) * nc + gid];
                    fy[f] = geo[(GEO_FY + f) * nc + gid];
                    wx[f] = geo[(GEO_WX + f) * nc + gid];
                    wy[f] = geo[(GEO_WY + f) * nc + gid];
                }
            }
#pragma unroll
            for (int v = 0; v < 3; v++) {
                real d0 = qn[0][v] - qK[v], d1 = qn[1][v] - qK[v], d2 = qn[2][v] - qK[v];
                real D[3];
                if constexpr (ETA) {
                    D[0] = Mf[0][0] * d0 + Mf[0][1] * d1 + Mf[0][2] * d2;
                    D[1] = Mf[1][0] * d0 + Mf[1][1] * d1 + Mf[1][2] * d2;
                    D[2] = -(D[0] + D[1]);
                } else {
                    real gx = (wx[0] * d0 + wx[1] * d1) + wx[2] * d2;
                    real gy = (wy[0] * d0 + wy[1] * d1) + wy[2] * d2;
#pragma unroll
                    for (int f = 0; f < 3; f++) D[f] = gx * fx[f] + gy * fy[f];
                }
                real qmax = qK[v], qmin = qK[v];
#pragma unroll
                for (int f = 0; f < 3; f++) {
                    qmax = smax(qmax, qn[f][v]);
                    qmin = smin(qmin, qn[f][v]);
                }
                real alpha = real(1);
                if constexpr (ETA) {
                    // phi_f = |r_f| / |D_f| with r_f = qmax - q_K or q_K - qmin by the
                    // sign of D_f; D_f = 0 gives +inf or NaN, which fminf ignores
                    const float up = qmax - qK[v], dn = qK[v] - qmin;
#pragma unroll
                    for (int f = 0; f < 3; f++)
                        alpha = fminf(alpha, (D[f] > 0.f ? up : dn) * rcp_approx(fabsf(D[f])));
                } else if constexpr (FAST) {
                    // the smallest ratio |r_f| / |D_f| below 1 (r_f = q_max - q_K or
                    // q_K - q_min by the sign of D_f) found by cross products; one
                    // division, none when no face limits
                    const real up = qmax - qK[v], dn = qK[v] - qmin;
                    real num = real(1), den = real(1);
#pragma unroll
                    for (int f = 0; f < 3; f++) {
                        const real aD = vabs(D[f]);
                        const real r = is_pos(D[f]) ? up : dn;
                        if (gt_nn(num * aD, r * den)) { num = r; den = aD; }   // both products >= 0
                    }
                    if (num != den) alpha = num / den;
                } else {
#pragma unroll
                    for (int f = 0; f < 3; f++) {
                        real phi = real(1);
                        if (is_pos(D[f])) phi = smin(real(1), (qmax - qK[v]) / D[f]);
                        else if (is_neg(D[f])) phi = smin(real(1), (qmin - qK[v]) / D[f]);
                        alpha = smin(alpha, phi);
                    }
                }
#pragma unroll
                for (int f = 0; f < 3; f++) face[f][v] = qK[v] + alpha * D[f];
            }
            // the face values stand on the face beds z_f (the linear bed at the
            // face midpoints); the face depths must stay above the threshold
            if constexpr (ETA) {
                const float2 dz = reinterpret_cast<const float2 *>(a.zf)[gid];
                zfK[0] = zK + dz.x;
                zfK[1] = zK + dz.y;
                zfK[2] = zK - (dz.x + dz.y);
            } else {
#pragma unroll
                for (int f = 0; f < 3; f++) zfK[f] = a.zf[f * nc + gid];
            }
#pragma unroll
            for (int f = 0; f < 3; f++) {
                Hf[f] = face[f][0] - zfK[f];
                if (!gt_nn(Hf[f], hthr)) recon = false;
                if (ETA) Hf[f] = face[f][0];      // FP32 keeps eta_f
                Huf[f] = face[f][1];
                Hvf[f] = face[f][2];
            }
        }
        if (!recon) {
#pragma unroll
            for (int f = 0; f < 3; f++) { Hf[f] = ETA ? WK : HK; Huf[f] = HuK; Hvf[f] = HvK; zfK[f] = zK; }
        }
        if constexpr (!ETA) sRec[l] = recon ? 1 : 0;
        if constexpr (!ETA)              // (the adjoint, which reads it, is FP64 only)
            if (a.rec_out && l < B) a.rec_out[gid] = recon ? 1 : 0;
#pragma unroll
        for (int f = 0; f < 3; f++) st4(sF + 4 * (f * L1 + l), Hf[f], Huf[f], Hvf[f], zfK[f]);
        if (a.fv_out && l < B) {
#pragma unroll
            for (int f = 0; f < 3; f++) {
                a.fv_out[(0 * 3 + f) * (size_t)nc + gid] = Hf[f];
                a.fv_out[(1 * 3 + f) * (size_t)nc + gid] = Huf[f];
                a.fv_out[(2 * 3 + f) * (size_t)nc + gid] = Hvf[f];
            }
        }
    }
    __syncthreads();

    // C: owned faces, one flux each (Sec. 2.2).  The two face values a face
    // reads are used by no other face, so its thread overwrites them with the
    // two sides' terms l [Phi + P_s n_s] (the other side's flux and normal are
    // the exact negations, the face length the same).
    const int nq = zero_terms ? 0 : qcount;
    for (int q = tid; q < nq; q += blockDim.x) {
        const int item = queue[q];
        const int l = item >> 2, f = item & 3;
        const int gid = c0 + l;
        const uint16_t code = sCode[f * B + l];
        const bool wall = code >= NBR_ABSORB;         // wall, open or absorbing: no neighbour
        const int bnd = wall ? (code == NBR_WALL ? 1 : code == NBR_OPEN ? 2 : 3) : 0;
        const int nl = code >> 2, nf = code & 3;
        real *pL = sF + 4 * (f * L1 + l);
        real *pR = sF + 4 * (nf * L1 + nl);
        // zL, zR: the bed under each side's face value (its face bed where that
        // cell reconstructed, its cell bed otherwise), from the slots' 4th word
        real WfL, HufL, HvfL, zL, WL, HuK, HvK, zKL;
        ld4(pL, WfL, HufL, HvfL, zL);
        ld4(sW + 4 * l, WL, HuK, HvK, zKL);
        real WfR = real(0), HufR = real(0), HvfR = real(0), WR = real(0), zR = real(0);
        if (!wall) {
            real Huj, Hvj, zKR;
            ld4(pR, WfR, HufR, HvfR, zR);
            ld4(sW + 4 * nl, WR, Huj, Hvj, zKR);
        }
        real Phi[3], PL, PR, am, nx, ny, len;
        if constexpr (ETA) {
            float2 nv = g32_normal(geo, gid, f);
            nx = nv.x; ny = nv.y;
            len = g32_len(geo, gid, f);
            face_flux_dev(g, half_g, hthr, WfL, HufL, HvfL, zL, WL,
                          WfR, HufR, HvfR, zR, WR, nx, ny, bnd, Phi, PL, PR, am);
        } else {
            nx = geo[(GEO_NX + f) * nc + gid];
            ny = geo[(GEO_NY + f) * nc + gid];
            len = geo[(GEO_LEN + f) * nc + gid];
            face_flux<real, FAST>(g, half_g, hthr, WfL, HufL, HvfL, zL,
                            WfR, HufR, HvfR, zR, nx, ny, bnd, Phi, PL, PR, am);
        }
        const real t0 = len * Phi[0];
        const real la = len * am;
        st4(pL, t0, len * (Phi[1] + PL * nx), len * (Phi[2] + PL * ny), la);
        if (!wall) st4(pR, -t0, -(len * (Phi[1] + PR * nx)), -(len * (Phi[2] + PR * ny)), la);
    }
    __syncthreads();

    // D: residual R_K = -(1/|K|) sum_f l_f [Phi_f + (0, P_{K,f} n_f)], faces in local order
    if (!LISTED && tid == 0) qcount = 0;     // every thread read it before the barrier above
    if (tid < ncell) {
        const int l = tid;
        const int gid = c0 + l;
        real aH = real(0), aHu = real(0), aHv = real(0), am = real(0);
        real x[3];
        const real area = ETA ? geo[(size_t)gid * G32 + G32_AREA] : geo[GEO_AREA * nc + gid];
#pragma unroll
        for (int f = 0; f < 3; f++) {
            real t0, t1, t2;
            ld4(sF + 4 * (f * L1 + l), t0, t1, t2, x[f]);
            aH = aH + t0;
            aHu = aHu + t1;
            aHv = aHv + t2;
            if (STAGE == 1) am = smax(am, x[f]);
        }
        if constexpr (!ETA) {
            // centred bed-slope source of a cell standing on its face beds:
            // g sum_f l_f z_f (eta_K - z_f / 2) n_f, eta_K = H_K + z_K (the deviation
            // form carries it in its per-face terms)
            if (sRec[l]) {
                real HKs, Hus, Hvs, zKs;
                ld4(sW + 4 * l, HKs, Hus, Hvs, zKs);
                const real eK = HKs + zKs;
#pragma unroll
                for (int f = 0; f < 3; f++) {
                    const real zff = a.zf[f * nc + gid];
                    const real sf = g * (geo[(GEO_LEN + f) * nc + gid] * (zff * (eK - real(0.5) * zff)));
                    aHu = aHu + sf * geo[(GEO_NX + f) * nc + gid];
                    aHv = aHv + sf * geo[(GEO_NY + f) * nc + gid];
                }
            }
        }
        if (STAGE == 2) { x[0] = a.w[gid]; x[1] = a.w[nc + gid]; x[2] = a.w[2 * nc + gid]; }
        finish_cell<real, STAGE, FAST>(a, gid, sW + 4 * l, aH, aHu, aHv, am, x, area, dt, my_min, my_neg, bad);
    }
}

// Dry-land shortcut of the single-scenario kernels: leave the block early
// (mode 1) except in the FP32 stage-2 kernel, which at its 40-register budget
// spills with that second exit and takes mode 2.  The batched kernels use mode 2.
template <typename real, int STAGE> struct DryMode { static constexpr int value = 1; };
template <> struct DryMode<float, 2> { static constexpr int value = 2; };

// Resident CTAs per SM asked of the register allocator.  The FP32 kernels are
// latency-bound: 40 registers a thread (no spills in these kernels) and ~48 resident warps
// beat fewer warps with more registers (6 CTAs of 256 threads: 40 registers;
// 5: 48; unbounded: 63, 4 CTAs).  FP64 is left unbounded.
template <typename real, int MAXT> struct StageMinCtas { static constexpr int value = 1; };
template <> struct StageMinCtas<float, 256> { static constexpr int value = 6; };
template <> struct StageMinCtas<float, 384> { static constexpr int value = 4; };
template <> struct StageMinCtas<float, 512> { static constexpr int value = 3; };
// FP64 with one thread per cell: two CTAs per SM, so that one CTA's phases run
// while the other waits at a barrier (118-122 registers, no spills)
template <> struct StageMinCtas<double, 256> { static constexpr int value = 2; };
// The batched kernels' own budget (their extra scenario state needs the FP64
// registers of one CTA per SM).
template <typename real> struct BatchMinCtas { static constexpr int value = 1; };
template <> struct BatchMinCtas<float> { static constexpr int value = 6; };

template <typename real, int STAGE, int MAXT, bool FAST = false>
__global__ void __launch_bounds__(MAXT, StageMinCtas<real, MAXT>::value) stage_kernel(const KArgs<real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int qcount[2];
    __shared__ real red_min[32];
    __shared__ long long red_neg[32];
    const int tid = threadIdx.x;

    // a context that has reached t_end takes steps of dt = 0 that leave its state
    // as it is: stage 1 does nothing (the CFL minimum stays empty) and stage 2
    // copies w^n to the output buffer, bit for bit (computing w/2 + (w + 0 R)/2
    // would flush the smallest FP32 values to zero), as the batched kernels do
    if (a.t_end > 0.0 && a.sc->t >= a.t_end) {
        if (STAGE == 2) {
            const int64_t n3 = 3 * a.nc;
            for (int64_t i = blockIdx.x * (int64_t)blockDim.x + tid; i < n3; i += (int64_t)gridDim.x * blockDim.x)
                a.wout[i] = a.w[i];
        }
        return;
    }

    real dt = real(0);
    if (STAGE == 2) dt = (real)step_dt<real>(a.sc, a.cfl, a.dt_fixed, a.dt_max, a.t_end);

    real my_min = real_inf<real>();
    long long my_neg = 0;
    bool bad = false;
    if (tid < 2) qcount[tid] = 0;
    __syncthreads();

    int parity = 0;
    for (int b = blockIdx.x; b < a.nblocks; b += gridDim.x, parity ^= 1)
        process_block<real, STAGE, DryMode<real, STAGE>::value, STAGE == 2, false, FAST>(a, b, dt, smem_raw, qcount[parity],
                                                                                     my_min, my_neg, bad);

    // CTA-level reductions, then one atomic per CTA
    const int lane = tid & 31, warp = tid >> 5, nwarps = (blockDim.x + 31) >> 5;
    if (STAGE == 1) {
        for (int o = 16; o > 0; o >>= 1) my_min = vmin(my_min, __shfl_xor_sync(0xffffffffu, my_min, o));
        if (lane == 0) red_min[warp] = my_min;
    }
    for (int o = 16; o > 0; o >>= 1) my_neg += __shfl_xor_sync(0xffffffffu, my_neg, o);
    if (lane == 0) red_neg[warp] = my_neg;
    bad = __syncthreads_or(bad);
    if (tid == 0) {
        long long neg = 0;
        real mn = real_inf<real>();
        for (int w = 0; w < nwarps; w++) {
            neg += red_neg[w];
            if (STAGE == 1) mn = vmin(mn, red_min[w]);
        }
        if (STAGE == 1 && a.cfl_min && mn < real_inf<real>()) atomicMin(&a.sc->dtmin_bits, min_bits(mn));
        if (neg) atomicAdd((unsigned long long *)&a.sc->neg_count, (unsigned long long)neg);
        if (bad) atomicOr(&a.sc->flags, FLAG_NONFINITE_STATE);
    }
}

// ---------------------------------------------------------------------------
// Unfused SSP-RK(2,2) (Sec. 2.3; vg_params.rk_unfused): the two stage updates as
// kernels of their own, with w1 and R(w1) in global memory, to compare with the
// fused stage-2 kernel, which forms w1 = w^n + dt R0 as it loads a block and ends
// with the second update.  Update 1 writes w1 with the dry fix; the stage-1
// kernel, without its CFL bound, writes R(w1); update 2 writes w^{n+1}.  The
// arithmetic of each cell is the fused path's (stage_cell, rk2_final).
// 256 threads, grid-stride over the cells; one atomic per CTA for the counts.
template <typename real>
__device__ __forceinline__ void cta_counts(long long my_neg, bool bad, DevScalars *sc)
{
    __shared__ long long red[8];
    __shared__ int any_bad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) any_bad = 0;
    for (int o = 16; o > 0; o >>= 1) my_neg += __shfl_xor_sync(0xffffffffu, my_neg, o);
    if (lane == 0) red[warp] = my_neg;
    __syncthreads();
    if (bad) any_bad = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long n = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) n += red[w];
        if (n) atomicAdd((unsigned long long *)&sc->neg_count, (unsigned long long)n);
        if (any_bad) atomicOr(&sc->flags, FLAG_NONFINITE_STATE);
    }
}

template <typename real>
__global__ void __launch_bounds__(256) rk_update1_kernel(const KArgs<real> a, real *w1)
{
    if (a.t_end > 0.0 && a.sc->t >= a.t_end) return;     // finished: update 2 copies w^n
    const real dt = (real)step_dt<real>(a.sc, a.cfl, a.dt_fixed, a.dt_max, a.t_end);
    const int64_t nc = a.nc;
    long long my_neg = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
        const int gid = (int)i;
        real W, Hu, Hv, zc;
        if (stage_cell<real, 2>(a, gid, dt, W, Hu, Hv, zc)) my_neg++;
        w1[gid] = W;
        w1[nc + gid] = Hu;
        w1[2 * nc + gid] = Hv;
    }
    cta_counts<real>(my_neg, false, a.sc);
}

template <typename real>
__global__ void __launch_bounds__(256) rk_update2_kernel(const KArgs<real> a, const real *w1, const real *R1)
{
    const int64_t nc = a.nc;
    if (a.t_end > 0.0 && a.sc->t >= a.t_end) {           // as the fused kernel: w^n, bit for bit
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * nc; i += (int64_t)gridDim.x * blockDim.x)
            a.wout[i] = a.w[i];
        return;
    }
    const real dt = (real)step_dt<real>(a.sc, a.cfl, a.dt_fixed, a.dt_max, a.t_end);
    long long my_neg = 0;
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
        const int gid = (int)i;
        const real x[3] = {a.w[gid], a.w[nc + gid], a.w[2 * nc + gid]};
        real W, Hu, Hv;
        const uint8_t branch = rk2_final(x, w1[gid], w1[nc + gid], w1[2 * nc + gid], R1[gid], R1[nc + gid],
                                         R1[2 * nc + gid], dt, a.z[gid], a.hthr, W, Hu, Hv);
        if (branch == 2) my_neg++;
        if (!isfinite(W) || !isfinite(Hu) || !isfinite(Hv)) bad = true;
        a.wout[gid] = W;
        a.wout[nc + gid] = Hu;
        a.wout[2 * nc + gid] = Hv;
    }
    cta_counts<real>(my_neg, bad, a.sc);
}

// ---------------------------------------------------------------------------
// Batched ensembles: many scenarios on several meshes in one persistent launch
// per stage.  A work item is one block of one mesh; the CTA runs that block for
// every scenario of the mesh in turn, so the block's mesh data stays in L1/L2
// across scenarios.  Scenario e (meshes' scenarios numbered consecutively) has
// its own state slice, its own device scalars sc[e] and its own time step.
// ---------------------------------------------------------------------------

constexpr int kBatchMaxEntries = 512;

template <typename real>
struct BatchMesh {
    KArgs<real> a;         // mesh arrays; w, R0, wout, sc point at the mesh's first scenario
    int64_t stride;        // 3 * nc: distance between scenario slices
    int n_scen;            // scenarios of this mesh
    int first_item;        // first work item (block) of this mesh in the launch
    int first_entry;       // index of its first scenario among all scenarios
    int n_gauges;          // gauges of this mesh (0: none)
    const int32_t *gauge_cells;  // [n_gauges] internal cell ids
    double *ring_t;        // [n_scen][ring_cap] record times
    double *ring_eta;      // [n_scen][ring_cap][n_gauges] eta at the gauges
    int ring_cap, pad;
};

// Order-preserving integer image of a non-negative value, as 32 bits (FP32) or
// 64 bits (FP64), kept in shared memory per scenario.
template <typename real>
__device__ __forceinline__ unsigned long long warp_min_bits(real v)
{
    for (int o = 16; o > 0; o >>= 1) v = vmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return min_bits(v);
}

template <typename real, int STAGE, bool FAST = false>
__global__ void __launch_bounds__(256, (BatchMinCtas<real>::value)) batch_stage_kernel(const BatchMesh<real> *meshes, int n_mesh,
                                                          int n_items, int n_entries, DevScalars *sc_all)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int qcount[2];
    __shared__ unsigned long long s_min[kBatchMaxEntries];
    __shared__ real s_dt[kBatchMaxEntries];
    __shared__ unsigned char s_done[kBatchMaxEntries];
    __shared__ long long red_neg[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = (blockDim.x + 31) >> 5;
    const KArgs<real> &p0 = meshes[0].a;
    for (int e = tid; e < n_entries; e += blockDim.x) {
        s_min[e] = min_bits(real_inf<real>());
        s_dt[e] = STAGE == 2 ? (real)step_dt<real>(sc_all + e, p0.cfl, p0.dt_fixed, p0.dt_max, p0.t_end) : real(0);
        // a scenario that has reached t_end takes steps of dt = 0 that leave its
        // state as it is (as a single context's do): skip its work, copy its state
        s_done[e] = (p0.t_end > 0.0 && sc_all[e].t >= p0.t_end) ? 1 : 0;
    }
    if (tid < 2) qcount[tid] = 0;
    __syncthreads();
    long long my_neg = 0;
    int parity = 0;
    bool bad = false;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        int m = 0;
        while (m + 1 < n_mesh && item >= meshes[m + 1].first_item) m++;
        const BatchMesh<real> &bm = meshes[m];
        const int b = item - bm.first_item;
        for (int s = 0; s < bm.n_scen; s++) {
            if (s_done[bm.first_entry + s]) {
                if (STAGE == 2) {
                    // the state carries over to the other buffer of the pair
                    const int c = b * bm.a.block + tid, nc = (int)bm.a.nc;
                    if (tid < bm.a.block && c < nc) {
                        const real *wi = bm.a.w + s * bm.stride;
                        real *wo = bm.a.wout + s * bm.stride;
                        wo[c] = wi[c];
                        wo[nc + c] = wi[nc + c];
                        wo[2 * nc + c] = wi[2 * nc + c];
                    }
                }
                continue;
            }
            KArgs<real> a = bm.a;
            a.w += s * bm.stride;
            a.R0 += s * bm.stride;
            if (STAGE == 2) a.wout += s * bm.stride;
            a.sc += s;
            const int e = bm.first_entry + s;
            real mn = real_inf<real>();
            process_block<real, STAGE, 2, true, true, FAST>(a, b, s_dt[e], smem_raw, qcount[parity], mn, my_neg, bad);
            parity ^= 1;
            if (STAGE == 1) {
                unsigned long long bits = warp_min_bits<real>(mn);
                if (lane == 0 && bits != min_bits(real_inf<real>())) atomicMin(&s_min[e], bits);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) my_neg += __shfl_xor_sync(0xffffffffu, my_neg, o);
    if (lane == 0) red_neg[warp] = my_neg;
    bad = __syncthreads_or(bad);
    if (STAGE == 1)
        for (int e = tid; e < n_entries; e += blockDim.x)
            if (s_min[e] != min_bits(real_inf<real>())) atomicMin(&sc_all[e].dtmin_bits, s_min[e]);
    if (tid == 0) {
        long long neg = 0;
        for (int w = 0; w < nwarps; w++) neg += red_neg[w];
        if (neg) atomicAdd((unsigned long long *)&sc_all[n_entries].neg_count, (unsigned long long)neg);
        if (bad) atomicOr(&sc_all[n_entries].flags, FLAG_NONFINITE_STATE);
    }
}

// Gauge records of one batched step (after the epilogue): a scenario that
// advanced records eta at its mesh's gauges every gauge_every of its steps, in
// the circular ring at index n_rec mod ring_cap (the host drains often enough
// that no unread record is overwritten).  One CTA per mesh.
template <typename real>
__global__ void batch_gauge_kernel(const BatchMesh<real> *meshes, DevScalars *sc_all, int gauge_every)
{
    __shared__ int slot[kBatchMaxEntries];
    const BatchMesh<real> &bm = meshes[blockIdx.x];
    const int G = bm.n_gauges;
    if (G == 0) return;
    for (int s = threadIdx.x; s < bm.n_scen; s += blockDim.x) {
        const DevScalars *sc = sc_all + bm.first_entry + s;
        slot[s] = (sc->dt > 0.0 && sc->steps % gauge_every == 0) ? (int)(sc->n_rec % bm.ring_cap) : -1;
    }
    __syncthreads();
    const real *z = bm.a.z;
    for (int k = threadIdx.x; k < bm.n_scen * G; k += blockDim.x) {
        const int s = k / G, g = k - s * G;
        if (slot[s] < 0) continue;
        const real *w = bm.a.wout + s * bm.stride;
        const int32_t c = bm.gauge_cells[g];
        bm.ring_eta[((size_t)s * bm.ring_cap + slot[s]) * G + g] =
            EtaForm<real>::value ? (double)w[c] : (double)(w[c] + z[c]);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < bm.n_scen; s += blockDim.x) {
        if (slot[s] < 0) continue;
        DevScalars *sc = sc_all + bm.first_entry + s;
        bm.ring_t[(size_t)s * bm.ring_cap + slot[s]] = sc->t;
        sc->n_rec += 1;
    }
}

// Epilogue of one batched step: per scenario t += dt (dt = 0 once it reached
// t_end), and reset of its CFL minimum.
template <typename real>
__global__ void batch_post_kernel(int n_entries, DevScalars *sc_all, double cfl, double dt_fixed, double dt_max,
                                  double t_end)
{
    for (int e = threadIdx.x; e < n_entries; e += blockDim.x) {
        DevScalars *sc = sc_all + e;
        double dt = step_dt<real>(sc, cfl, dt_fixed, dt_max, t_end);
        sc->dt = dt;
        if (!isfinite(dt)) sc_all[n_entries].flags |= FLAG_NONFINITE_DT;
        if (dt > 0.0) {
            sc->t = sc->t + dt;
            sc->steps += 1;
        }
        sc->dtmin_bits = min_bits(real_inf<real>());
    }
}

template <typename real>
KArgs<real> make_args(const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out)
{
    KArgs<real> a;
    a.nc = d.nc;
    a.block = d.block;
    a.nblocks = d.nblocks;
    a.max_halo = d.max_halo;
    a.max_ring1 = d.max_ring1;
    a.order = p.order;
    a.geo = static_cast<const real *>(d.geo);
    a.z = static_cast<const real *>(d.z);
    a.zf = static_cast<const real *>(d.zf);
    a.nbr = d.nbr;
    a.nbrl = d.nbrl;
    a.halo_ptr = d.halo_ptr;
    a.halo_n1 = d.halo_n1;
    a.halo_ids = d.halo_ids;
    a.ring1_nbr = d.ring1_nbr;
    a.fq_ptr = d.fq_ptr;
    a.fq = d.fq;
    a.w = static_cast<const real *>(w_in);
    a.R0 = static_cast<real *>(d.R0);
    a.wout = static_cast<real *>(w_out);
    a.mask2 = d.mask2;
    a.fv_out = static_cast<real *>(d.fv_out);
    a.r1_out = static_cast<real *>(d.r1_out);
    a.rec_out = d.rec_out;
    a.sc = d.sc;
    a.g = (real)p.g;
    a.half_g = (real)(0.5 * p.g);
    a.hthr = (real)p.hthr;
    a.cfl = p.cfl;
    a.dt_fixed = p.dt_fixed;
    a.dt_max = p.dt_max;
    a.t_end = p.t_end;
    a.cfl_min = 1;
    return a;
}

// Kernel instance for a launch: the register budget follows the thread count
// (launch bounds 256 or 512).
template <typename real, bool FAST = false>
void *stage_kernel_ptr(int stage, int threads)
{
    if (threads <= 256)
        return stage == 1 ? (void *)stage_kernel<real, 1, 256, FAST> : (void *)stage_kernel<real, 2, 256, FAST>;
    if (threads <= 384)
        return stage == 1 ? (void *)stage_kernel<real, 1, 384, FAST> : (void *)stage_kernel<real, 2, 384, FAST>;
    return stage == 1 ? (void *)stage_kernel<real, 1, 512, FAST> : (void *)stage_kernel<real, 2, 512, FAST>;
}

// The dynamic shared memory limit is an attribute of the kernel function, shared
// by every context in the process: it is only ever raised, so that a context
// configured later with a smaller block never lowers it below what another
// context's launches need.
inline cudaError_t raise_smem_limit(const void *kern, size_t smem)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename real, bool FAST = false>
int stage_config(const DevPtrs &d, int stage, LaunchCfg &cfg)
{
    cfg.smem = stage_smem_bytes<real>(d.block, d.max_halo, d.max_ring1);
    const void *kern = stage_kernel_ptr<real, FAST>(stage, d.threads);
    cudaError_t e = raise_smem_limit(kern, cfg.smem);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, d.threads, cfg.smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long grid = (long long)sms * per_sm;
    if (grid > d.nblocks) grid = d.nblocks;
    cfg.grid = (int)(grid < 1 ? 1 : grid);
    return 0;
}

template <typename real, bool FAST = false>
int launch_stage_args(const KArgs<real> &a, int threads, int stage, const LaunchCfg &c, cudaStream_t s)
{
    const int t = threads;
    if (t <= 256) {
        if (stage == 1) stage_kernel<real, 1, 256, FAST><<<c.grid, t, c.smem, s>>>(a);
        else stage_kernel<real, 2, 256, FAST><<<c.grid, t, c.smem, s>>>(a);
    } else if (t <= 384) {
        if (stage == 1) stage_kernel<real, 1, 384, FAST><<<c.grid, t, c.smem, s>>>(a);
        else stage_kernel<real, 2, 384, FAST><<<c.grid, t, c.smem, s>>>(a);
    } else {
        if (stage == 1) stage_kernel<real, 1, 512, FAST><<<c.grid, t, c.smem, s>>>(a);
        else stage_kernel<real, 2, 512, FAST><<<c.grid, t, c.smem, s>>>(a);
    }
    return (int)cudaGetLastError();
}

// The unfused step's three launches after stage 1 (part 0: update 1; 1: the
// stage-1 kernel on w1 writing R(w1) to R1, without its CFL bound; 2: update 2).
// w1 and R1 are [3][nc] buffers of the context.
template <typename real, bool FAST = false>
int launch_rk_unfused(const DevPtrs &d, const StepParams &p, int part, const void *w_in, void *w_out, void *w1,
                      void *R1, const LaunchCfg &c1, void *stream)
{
    KArgs<real> a = make_args<real>(d, p, w_in, w_out);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (part == 1) {
        a.w = static_cast<const real *>(w1);
        a.R0 = static_cast<real *>(R1);
        a.wout = nullptr;
        a.cfl_min = 0;
        return launch_stage_args<real, FAST>(a, d.threads, 1, c1, s);
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (d.nc + 255) / 256, cap = 8LL * (sms > 0 ? sms : 1);
    const int grid = (int)(want < 1 ? 1 : want < cap ? want : cap);
    if (part == 0) rk_update1_kernel<real><<<grid, 256, 0, s>>>(a, static_cast<real *>(w1));
    else rk_update2_kernel<real><<<grid, 256, 0, s>>>(a, static_cast<const real *>(w1), static_cast<const real *>(R1));
    return (int)cudaGetLastError();
}

template <typename real, bool FAST = false>
int launch_stage(const DevPtrs &d, const StepParams &p, int stage, const void *w_in, void *w_out,
                 const LaunchCfg &c, void *stream)
{
    KArgs<real> a = make_args<real>(d, p, w_in, w_out);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d.threads <= 256) {
        if (stage == 1) stage_kernel<real, 1, 256, FAST><<<c.grid, d.threads, c.smem, s>>>(a);
        else stage_kernel<real, 2, 256, FAST><<<c.grid, d.threads, c.smem, s>>>(a);
    } else if (d.threads <= 384) {
        if (stage == 1) stage_kernel<real, 1, 384, FAST><<<c.grid, d.threads, c.smem, s>>>(a);
        else stage_kernel<real, 2, 384, FAST><<<c.grid, d.threads, c.smem, s>>>(a);
    } else {
        if (stage == 1) stage_kernel<real, 1, 512, FAST><<<c.grid, d.threads, c.smem, s>>>(a);
        else stage_kernel<real, 2, 512, FAST><<<c.grid, d.threads, c.smem, s>>>(a);
    }
    return (int)cudaGetLastError();
}

template <typename real, bool FAST = false>
int batch_config(int block, int max_halo, int max_ring1, int &grid, size_t &smem)
{
    smem = stage_smem_bytes<real>(block, max_halo, max_ring1, true);
    int best = 1 << 30;
    for (int stage = 1; stage <= 2; stage++) {
        auto kern = stage == 1 ? batch_stage_kernel<real, 1, FAST> : batch_stage_kernel<real, 2, FAST>;
        cudaError_t e = raise_smem_limit((const void *)kern, smem);
        if (e != cudaSuccess) return (int)e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
        if (e != cudaSuccess) return (int)e;
        best = per_sm < best ? per_sm : best;
    }
    if (best < 1) return (int)cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = sms * best;
    return 0;
}

template <typename real, bool FAST = false>
int launch_batch_step(const void *table, int n_mesh, int n_items, int n_entries, DevScalars *sc_all, int block,
                      int grid, size_t smem, const StepParams &p, bool gauges, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const BatchMesh<real> *t = static_cast<const BatchMesh<real> *>(table);
    batch_stage_kernel<real, 1, FAST><<<grid, block, smem, s>>>(t, n_mesh, n_items, n_entries, sc_all);
    batch_stage_kernel<real, 2, FAST><<<grid, block, smem, s>>>(t, n_mesh, n_items, n_entries, sc_all);
    batch_post_kernel<real><<<1, 256, 0, s>>>(n_entries, sc_all, p.cfl, p.dt_fixed, p.dt_max, p.t_end);
    if (gauges) batch_gauge_kernel<real><<<n_mesh, 256, 0, s>>>(t, sc_all, p.gauge_every);
    return (int)cudaGetLastError();
}

template <typename real>
void fill_batch_mesh(void *dst, const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out,
                     int n_scen, int first_item, int first_entry)
{
    BatchMesh<real> *bm = static_cast<BatchMesh<real> *>(dst);
    bm->a = make_args<real>(d, p, w_in, w_out);
    bm->stride = 3 * d.nc;
    bm->n_scen = n_scen;
    bm->first_item = first_item;
    bm->first_entry = first_entry;
    bm->n_gauges = d.n_gauges;
    bm->gauge_cells = d.gauge_cells;
    bm->ring_t = d.ring_t;
    bm->ring_eta = d.ring_eta;
    bm->ring_cap = d.ring_cap;
    bm->pad = 0;
}

}  // namespace vg
