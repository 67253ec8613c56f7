// Hand-written discrete adjoint of the FP64 step (reverse mode), built with
// --fmad=false like the FP64 forward kernels.
//
// The residual R = L(w; z) of Sec. 2 is reversed in four kernels, each thread
// owning what it writes (no atomics, fixed summation order):
//   adj_face_values   forward face values FV[3 vars][3 faces][nc] at w
//   adj_flux_vjp      per owned face: Phi-bar, P-bar from R-bar of both cells,
//                     reverse of the interface (hydrostatic depths, HLL with its
//                     branch and speed choices, velocities) -> FV-bar and the
//                     adjoint of the bed under each face value into the (cell,
//                     face) slots of both sides
//   adj_recon_vjp     per cell: reverse of the limited least-squares
//                     reconstruction and, for a cell standing on its face beds,
//                     of the centred bed-slope source -> the cell's own w-bar,
//                     cell-bed and face-bed adjoints, and what it sends to each
//                     face neighbour ((cell, face) slots)
//   adj_gather        per cell: own part + the slots its neighbours sent to it
// Branches are frozen where the forward run took them; min/max ties resolve to
// the first argument (the convention of the oracle's taping adjoint).
// Around them, elementwise kernels reverse the SSP-RK(2,2) stage updates, the
// dry fixes and the gauge functional.
#include <cuda_runtime.h>

#include "step_kernels.cuh"

namespace vg {

namespace {

// Exact IEEE comparisons of FP64 values on the integer units (for every
// non-NaN input), beside the sign and threshold tests of step_kernels.cuh:
// the reverse kernels record which argument of a min / max or which side of a
// test carried the value, so a tie between +0 and -0 must decide as FP64 does.
__device__ __forceinline__ bool lt_x(double a, double b)      // a < b
{
    return okey(a) < okey(b) && ((ubits(a) | ubits(b)) << 1) != 0;
}
__device__ __forceinline__ bool lt_pos(double x, double y)    // x < y for y > 0
{
    return dbits(x) < dbits(y);
}
__device__ __forceinline__ bool gt_abs(double a, double b)    // |a| > |b|
{
    return (dbits(a) & 0x7fffffffffffffffLL) > (dbits(b) & 0x7fffffffffffffffLL);
}

struct AdjMesh {
    int nc, order;
    const double *geo;       // [GEO_ROWS][nc]
    const double *z;         // [nc]
    const double *zf;        // [3][nc] face beds
    const uint8_t *rec;      // [nc] the stage's reconstruction flags (forward record)
    const int32_t *nbr;      // [3][nc]
    const uint16_t *nbrl;    // [3][nc]: low 2 bits = neighbour's face (not a wall)
    const int32_t *faces;    // every face once: (owning cell << 2) | face
    int nfaces;
    double g, half_g, hthr;
};

__device__ __forceinline__ double G(const AdjMesh &m, int row, int k) { return m.geo[row * m.nc + k]; }

// The bed under face value f of cell K: its face bed where K reconstructed,
// its cell bed otherwise.
__device__ __forceinline__ double bed_under(const AdjMesh &m, int K, int f)
{
    return m.rec[K] ? m.zf[f * m.nc + K] : m.z[K];
}

// Forward reconstruction of cell K (the same evaluation order as the forward
// kernels), keeping what the reverse needs.
struct ReconFwd {
    double qK[3], qn[3][3];
    bool wall[3];            // boundary face (wall, open or absorbing)
    bool open[3];            // open or absorbing face: the ghost is the cell itself
    bool recon;
    double D[3][3];          // [v][f]
    double alpha[3];
    int fa[3];               // face whose phi is the active limiter (-1: alpha = 1)
    int imax[3], imin[3];    // stencil index of q_max / q_min (-1 = the cell)
    double r[3];             // q_max - q_K or q_min - q_K of the active face
};

__device__ void recon_forward(const AdjMesh &m, const double *w, int K, ReconFwd &R, double Hf[3],
                              double Huf[3], double Hvf[3])
{
    const int nc = m.nc;
    const double *H = w, *Hu = w + nc, *Hv = w + 2 * (size_t)nc;
    double zK = m.z[K];
    double HK = H[K], HuK = Hu[K], HvK = Hv[K];
    R.qK[0] = HK + zK;
    R.qK[1] = HuK;
    R.qK[2] = HvK;
    bool recon = (m.order == 2) && (HK > m.hthr);
    for (int f = 0; f < 3; f++) {
        int j = m.nbr[f * nc + K];
        R.wall[f] = j < 0;
        R.open[f] = j == -2 || j == -3;
        if (j >= 0) {
            R.qn[f][0] = H[j] + m.z[j];
            R.qn[f][1] = Hu[j];
            R.qn[f][2] = Hv[j];
            if (!(H[j] > m.hthr)) recon = false;
        } else if (R.open[f]) {
            R.qn[f][0] = R.qK[0];
            R.qn[f][1] = HuK;
            R.qn[f][2] = HvK;
        } else {
            double nx = G(m, GEO_NX + f, K), ny = G(m, GEO_NY + f, K);
            double mn = HuK * nx + HvK * ny;
            R.qn[f][0] = R.qK[0];
            R.qn[f][1] = HuK - 2.0 * mn * nx;
            R.qn[f][2] = HvK - 2.0 * mn * ny;
        }
    }
    if (recon) {
        double face[3][3];
        for (int v = 0; v < 3; v++) {
            double d0 = R.qn[0][v] - R.qK[v], d1 = R.qn[1][v] - R.qK[v], d2 = R.qn[2][v] - R.qK[v];
            double gx = (G(m, GEO_WX, K) * d0 + G(m, GEO_WX + 1, K) * d1) + G(m, GEO_WX + 2, K) * d2;
            double gy = (G(m, GEO_WY, K) * d0 + G(m, GEO_WY + 1, K) * d1) + G(m, GEO_WY + 2, K) * d2;
            double qmax = R.qK[v], qmin = R.qK[v];
            int imax = -1, imin = -1;
            for (int f = 0; f < 3; f++) {
                if (lt_x(qmax, R.qn[f][v])) { qmax = R.qn[f][v]; imax = f; }
                if (lt_x(R.qn[f][v], qmin)) { qmin = R.qn[f][v]; imin = f; }
            }
            double alpha = 1.0;
            int fa = -1;
            double ra = 0.0;
            for (int f = 0; f < 3; f++) {
                double D = gx * G(m, GEO_FX + f, K) + gy * G(m, GEO_FY + f, K);
                R.D[v][f] = D;
                double phi = 1.0, rr = 0.0;
                bool lim = false;
                if (is_pos(D)) { rr = qmax - R.qK[v]; double t = rr / D; if (lt_pos(t, 1.0)) { phi = t; lim = true; } }
                else if (is_neg(D)) { rr = qmin - R.qK[v]; double t = rr / D; if (lt_pos(t, 1.0)) { phi = t; lim = true; } }
                if (lt_x(phi, alpha)) { alpha = phi; fa = lim ? f : -1; ra = rr; }
            }
            R.alpha[v] = alpha;
            R.fa[v] = fa;
            R.r[v] = ra;
            R.imax[v] = imax;
            R.imin[v] = imin;
            for (int f = 0; f < 3; f++) face[f][v] = R.qK[v] + alpha * R.D[v][f];
        }
        for (int f = 0; f < 3; f++) {
            Hf[f] = face[f][0] - m.zf[f * nc + K];
            if (!(Hf[f] > m.hthr)) recon = false;
            Huf[f] = face[f][1];
            Hvf[f] = face[f][2];
        }
    }
    R.recon = recon;
    if (!recon) {
        for (int f = 0; f < 3; f++) { Hf[f] = HK; Huf[f] = HuK; Hvf[f] = HvK; }
    }
}

// Face values are needed only where a face's flux adjoint can be nonzero, i.e.
// where the cell or a face neighbour has a nonzero residual adjoint; elsewhere
// the flux VJP skips the face (the VJP of zero is zero).
__device__ __forceinline__ bool rb_nonzero(const double *Rb, int nc, int k)
{
    return !is_zero(Rb[k]) || !is_zero(Rb[nc + k]) || !is_zero(Rb[2 * (size_t)nc + k]);
}

__global__ void adj_face_values_kernel(AdjMesh m, const double *w, const double *Rb, double *FV)
{
    const int nc = m.nc;
    for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < nc; K += gridDim.x * blockDim.x) {
        bool need = rb_nonzero(Rb, nc, K);
        for (int f = 0; f < 3 && !need; f++) {
            int j = m.nbr[f * nc + K];
            if (j >= 0) need = rb_nonzero(Rb, nc, j);
        }
        if (!need) continue;
        ReconFwd R;
        double Hf[3], Huf[3], Hvf[3];
        recon_forward(m, w, K, R, Hf, Huf, Hvf);
        for (int f = 0; f < 3; f++) {
            FV[(0 * 3 + f) * (size_t)nc + K] = Hf[f];
            FV[(1 * 3 + f) * (size_t)nc + K] = Huf[f];
            FV[(2 * 3 + f) * (size_t)nc + K] = Hvf[f];
        }
    }
}

// Reverse of the face flux seen from L (forward: face_flux / hll_normal).
// Inputs: the two face states, beds, normal, wall flag, and the adjoints of
// Phi[3], P_L, P_R and of the wave speed a = max(|s_L|, |s_R|) (amb: nonzero
// only for the face that sets the CFL time step); bnd, the kind of a boundary
// face: 1 wall, 2 open, 3 absorbing.  Outputs: adjoints of (H_f, Hu_f, Hv_f, z)
// on each side.  The absorbing ghost (characteristic ghost of a sea at rest at
// eta = 0 beyond the face) depends on the face state through the outgoing
// invariant u_n + 2c and on the bed under the face through c_0 = sqrt(g max(0, -z)).
__device__ void flux_vjp(const AdjMesh &m, double HfL, double HufL, double HvfL, double zL, double HfR,
                         double HufR, double HvfR, double zR, double nx, double ny, bool wall,
                         const double Pb[3], double PLb, double PRb, double bL[4], double bR[4],
                         double amb = 0.0, int bnd = 1)
{
    const double g = m.g, hg = m.half_g, hthr = m.hthr;
    for (int k = 0; k < 4; k++) { bL[k] = 0.0; bR[k] = 0.0; }
    // ---- forward
    double uL = 0.0, vL = 0.0;
    bool velL = gt_nn(HfL, hthr);
    if (velL) { uL = HufL / HfL; vL = HvfL / HfL; }
    double unL = uL * nx + vL * ny;
    double utL = -uL * ny + vL * nx;
    double HsL, HsR, unR, utR, uR = 0.0, vR = 0.0, zs = 0.0;
    bool velR = false, zR_max = false, actL, actR = false;
    double xL, xR = 0.0;
    double cgL = 0.0, c0 = 0.0, cg = 0.0;    // absorbing ghost: c of the face state, of the sea, of the ghost
    bool act0 = false, actg = false;
    if (wall && bnd == 3) {
        xL = (HfL + zL) - zL;
        actL = is_pos(xL);
        HsL = actL ? xL : 0.0;
        cgL = sqrt(g * HsL);
        const double x0 = 0.0 - zL;
        act0 = is_pos(x0);
        c0 = sqrt(g * (act0 ? x0 : 0.0));
        const double Rp = unL + 2.0 * cgL, Rm = 0.0 - 2.0 * c0;
        unR = 0.5 * (Rp + Rm);
        const double y = 0.25 * (Rp - Rm);
        actg = is_pos(y);
        cg = actg ? y : 0.0;
        HsR = cg * cg / g;
        utR = utL;
    } else if (wall) {
        xL = (HfL + zL) - zL;
        actL = is_pos(xL);
        HsL = actL ? xL : 0.0;
        HsR = HsL;
        unR = bnd == 2 ? unL : -unL;
        utR = utL;
    } else {
        velR = gt_nn(HfR, hthr);
        if (velR) { uR = HufR / HfR; vR = HvfR / HfR; }
        unR = uR * nx + vR * ny;
        utR = -uR * ny + vR * nx;
        zR_max = lt_x(zL, zR);
        zs = zR_max ? zR : zL;
        xL = (HfL + zL) - zs;
        xR = (HfR + zR) - zs;
        actL = is_pos(xL);
        actR = is_pos(xR);
        HsL = actL ? xL : 0.0;
        HsR = actR ? xR : 0.0;
    }
    // ---- reverse of the rotation and pressure terms
    double Fb0 = Pb[0];
    double Fb1 = Pb[1] * nx + Pb[2] * ny;
    double Fb2 = -Pb[1] * ny + Pb[2] * nx;
    double HfLb = PLb * hg * 2.0 * HfL, HsLb = -PLb * hg * 2.0 * HsL;
    double HfRb = 0.0, HsRb = 0.0;
    if (!wall) { HfRb = PRb * hg * 2.0 * HfR; HsRb = -PRb * hg * 2.0 * HsR; }
    double unLb = 0.0, utLb = 0.0, unRb = 0.0, utRb = 0.0;
    // ---- reverse of HLL
    if (!(is_zero(HsL) && is_zero(HsR))) {
        double cL = sqrt(g * HsL), cR = sqrt(g * HsR);
        double sL, sR, us = 0.0, cs = 0.0;
        int case_ = 0;    // 0 both wet, 1 L dry, 2 R dry
        bool sL_first = true, sR_first = true;
        if (is_zero(HsL)) {
            case_ = 1;
            sL = unR - 2.0 * cR;
            sR = unR + cR;
        } else if (is_zero(HsR)) {
            case_ = 2;
            sL = unL - cL;
            sR = unL + 2.0 * cL;
        } else {
            us = 0.5 * (unL + unR) + (cL - cR);
            cs = 0.5 * (cL + cR) - 0.25 * (unR - unL);
            double a1 = unL - cL, a2 = us - cs;
            sL_first = !lt_x(a2, a1);
            sL = sL_first ? a1 : a2;
            double b1 = us + cs, b2 = unR + cR;
            sR_first = !lt_x(b1, b2);
            sR = sR_first ? b1 : b2;
        }
        double qL = HsL * unL, qR = HsR * unR;
        double FL[3] = {qL, qL * unL + hg * HsL * HsL, qL * utL};
        double FR[3] = {qR, qR * unR + hg * HsR * HsR, qR * utR};
        double wL[3] = {HsL, qL, HsL * utL};
        double wR[3] = {HsR, qR, HsR * utR};
        double Fb[3] = {Fb0, Fb1, Fb2};
        double FLb[3] = {0, 0, 0}, FRb[3] = {0, 0, 0}, wLb[3] = {0, 0, 0}, wRb[3] = {0, 0, 0};
        double sLb = 0.0, sRb = 0.0;
        if (!is_neg(sL)) {
            for (int k = 0; k < 3; k++) FLb[k] = Fb[k];
        } else if (!is_neg(sR)) {
            double den = sR - sL, sLR = sL * sR, iden = 1.0 / den;
            double denb = 0.0, sLRb = 0.0;
            for (int k = 0; k < 3; k++) {
                double N = (sR * FL[k] - sL * FR[k]) + sLR * (wR[k] - wL[k]);
                double F = N * iden;
                double Nb = Fb[k] * iden;
                denb -= Fb[k] * F * iden;
                FLb[k] += Nb * sR;
                FRb[k] -= Nb * sL;
                sRb += Nb * FL[k];
                sLb -= Nb * FR[k];
                sLRb += Nb * (wR[k] - wL[k]);
                wRb[k] += Nb * sLR;
                wLb[k] -= Nb * sLR;
            }
            sLb += sLRb * sR;
            sRb += sLRb * sL;
            sRb += denb;
            sLb -= denb;
        } else {
            for (int k = 0; k < 3; k++) FRb[k] = Fb[k];
        }
        // physical fluxes and conserved variables -> (Hs, q, un, ut)
        double qLb = FLb[0] + FLb[1] * unL + FLb[2] * utL + wLb[1];
        unLb += FLb[1] * qL;
        HsLb += FLb[1] * 2.0 * hg * HsL + wLb[0] + wLb[2] * utL;
        utLb += FLb[2] * qL + wLb[2] * HsL;
        HsLb += qLb * unL;
        unLb += qLb * HsL;
        double qRb = FRb[0] + FRb[1] * unR + FRb[2] * utR + wRb[1];
        unRb += FRb[1] * qR;
        HsRb += FRb[1] * 2.0 * hg * HsR + wRb[0] + wRb[2] * utR;
        utRb += FRb[2] * qR + wRb[2] * HsR;
        HsRb += qRb * unR;
        unRb += qRb * HsR;
        // the wave speed a = max(|s_L|, |s_R|) (a tie takes |s_L|; |s| at s = 0 takes +s)
        if (!is_zero(amb)) {
            if (gt_abs(sR, sL)) sRb += is_neg(sR) ? -amb : amb;
            else sLb += is_neg(sL) ? -amb : amb;
        }
        // speeds
        double cLb = 0.0, cRb = 0.0;
        if (case_ == 1) {
            unRb += sLb + sRb;
            cRb += -2.0 * sLb + sRb;
        } else if (case_ == 2) {
            unLb += sLb + sRb;
            cLb += -sLb + 2.0 * sRb;
        } else {
            double usb = 0.0, csb = 0.0;
            if (sL_first) { unLb += sLb; cLb -= sLb; } else { usb += sLb; csb -= sLb; }
            if (sR_first) { usb += sRb; csb += sRb; } else { unRb += sRb; cRb += sRb; }
            unLb += 0.5 * usb;
            unRb += 0.5 * usb;
            cLb += usb;
            cRb -= usb;
            cLb += 0.5 * csb;
            cRb += 0.5 * csb;
            unRb -= 0.25 * csb;
            unLb += 0.25 * csb;
        }
        if (is_pos(cL)) HsLb += cLb * (0.5 / cL) * g;
        if (is_pos(cR)) HsRb += cRb * (0.5 / cR) * g;
    }
    // ---- reverse of the interface depths and velocities
    if (wall && bnd == 3) {
        // HsR = c_g^2 / g, c_g = max(0, (R+ - R-)/4), u_n,R = (R+ + R-)/2,
        // R+ = u_n,L + 2 c_L, R- = -2 c_0
        const double yb = actg ? HsRb * (2.0 * cg / g) : 0.0;
        const double Rpb = 0.5 * unRb + 0.25 * yb, Rmb = 0.5 * unRb - 0.25 * yb;
        unLb += Rpb;
        if (is_pos(cgL)) HsLb += (2.0 * Rpb) * (0.5 / cgL) * g;
        if (is_pos(c0) && act0) bL[3] -= (-2.0 * Rmb) * (0.5 / c0) * g;
        utLb += utRb;
        if (actL) { HfLb += HsLb; bL[3] += HsLb; bL[3] -= HsLb; }
    } else if (wall) {
        unLb += bnd == 2 ? unRb : -unRb;
        utLb += utRb;
        HsLb += HsRb;
        if (actL) { HfLb += HsLb; bL[3] += HsLb; bL[3] -= HsLb; }
    } else {
        double zsb = 0.0;
        if (actL) { HfLb += HsLb; bL[3] += HsLb; zsb -= HsLb; }
        if (actR) { HfRb += HsRb; bR[3] += HsRb; zsb -= HsRb; }
        if (zR_max) bR[3] += zsb; else bL[3] += zsb;
        double uRb = unRb * nx - utRb * ny, vRb = unRb * ny + utRb * nx;
        if (velR) {
            double inv = 1.0 / HfR;
            bR[1] += uRb * inv;
            bR[2] += vRb * inv;
            HfRb -= (uRb * uR + vRb * vR) * inv;
        }
    }
    double uLb = unLb * nx - utLb * ny, vLb = unLb * ny + utLb * nx;
    if (velL) {
        double inv = 1.0 / HfL;
        bL[1] += uLb * inv;
        bL[2] += vLb * inv;
        HfLb -= (uLb * uL + vLb * vL) * inv;
    }
    bL[0] += HfLb;
    bR[0] += HfRb;
}

// One thread per face (the face list: the lower-numbered cell owns an interior
// face, the cell a boundary face): R-bar of both cells -> Phi-bar, P-bar ->
// face-state adjoints.  FVb[(v*3+f)*nc + K] and zfb[f*nc + K] are the (cell,
// face) slots; each is written exactly once per residual.
__global__ void adj_flux_vjp_kernel(AdjMesh m, const double *FV, const double *Rb, double *FVb, double *zfb)
{
    const int nc = m.nc;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m.nfaces; q += gridDim.x * blockDim.x) {
        {
            const int K = m.faces[q] >> 2, f = m.faces[q] & 3;
            int j = m.nbr[f * nc + K];
            bool wall = j < 0;
            int fj = wall ? 0 : (m.nbrl[f * nc + K] & 3);
            if (!rb_nonzero(Rb, nc, K) && (wall || !rb_nonzero(Rb, nc, j))) {
                for (int v = 0; v < 3; v++) FVb[(v * 3 + f) * (size_t)nc + K] = 0.0;
                zfb[f * (size_t)nc + K] = 0.0;
                if (!wall) {
                    for (int v = 0; v < 3; v++) FVb[(v * 3 + fj) * (size_t)nc + j] = 0.0;
                    zfb[fj * (size_t)nc + j] = 0.0;
                }
                continue;
            }
            double nx = G(m, GEO_NX + f, K), ny = G(m, GEO_NY + f, K), l = G(m, GEO_LEN + f, K);
            double aL = G(m, GEO_AREA, K);
            double cLf = -l / aL;
            double Pb[3], PLb, PRb = 0.0;
            double RLH = Rb[K], RLU = Rb[nc + K], RLV = Rb[2 * (size_t)nc + K];
            Pb[0] = cLf * RLH;
            Pb[1] = cLf * RLU;
            Pb[2] = cLf * RLV;
            PLb = cLf * (RLU * nx + RLV * ny);
            double HfR = 0.0, HufR = 0.0, HvfR = 0.0, zR = 0.0;
            if (!wall) {
                double cRf = l / G(m, GEO_AREA, j);
                double RRH = Rb[j], RRU = Rb[nc + j], RRV = Rb[2 * (size_t)nc + j];
                Pb[0] += cRf * RRH;
                Pb[1] += cRf * RRU;
                Pb[2] += cRf * RRV;
                PRb = cRf * (RRU * nx + RRV * ny);
                HfR = FV[(0 * 3 + fj) * (size_t)nc + j];
                HufR = FV[(1 * 3 + fj) * (size_t)nc + j];
                HvfR = FV[(2 * 3 + fj) * (size_t)nc + j];
                zR = bed_under(m, j, fj);
            }
            double bL[4], bR[4];
            flux_vjp(m, FV[(0 * 3 + f) * (size_t)nc + K], FV[(1 * 3 + f) * (size_t)nc + K],
                     FV[(2 * 3 + f) * (size_t)nc + K], bed_under(m, K, f), HfR, HufR, HvfR, zR, nx, ny, wall, Pb, PLb,
                     PRb, bL, bR, 0.0, wall ? -j : 0);
            for (int v = 0; v < 3; v++) FVb[(v * 3 + f) * (size_t)nc + K] = bL[v];
            zfb[f * (size_t)nc + K] = bL[3];
            if (!wall) {
                for (int v = 0; v < 3; v++) FVb[(v * 3 + fj) * (size_t)nc + j] = bR[v];
                zfb[fj * (size_t)nc + j] = bR[3];
            }
        }
    }
}

// Per cell: reverse of the reconstruction.  own[7][nc] = (H, Hu, Hv, z_K)-bar of
// the cell itself, then the adjoints of its three face beds; send[(f*4+k)*nc + K]
// = the (H, Hu, Hv, z)-bar that cell K passes to its face-f neighbour.  The
// flux slots' bed adjoint (zfb) belongs to the bed under the face value: the
// face bed where the cell reconstructed, its cell bed otherwise.  A cell that
// reconstructed also carries the centred source g sum_f l_f z_f (eta_K - z_f/2)
// n_f of its momentum residual R = -(1/|K|)(... + source): with
// q_f = -(g/|K|) l_f (n_f . (R-bar_Hu, R-bar_Hv)), eta-bar_K += sum_f q_f z_f and
// z_f-bar += q_f (eta_K - z_f).
__global__ void adj_recon_vjp_kernel(AdjMesh m, const double *w, const double *Rb, const double *FVb,
                                     const double *zfb, double *own, double *send)
{
    const int nc = m.nc;
    for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < nc; K += gridDim.x * blockDim.x) {
        double fb[3][3];   // [v][f]
        bool any = m.rec[K] && (!is_zero(Rb[nc + K]) || !is_zero(Rb[2 * (size_t)nc + K]));
        for (int v = 0; v < 3; v++)
            for (int f = 0; f < 3; f++) {
                fb[v][f] = FVb[(v * 3 + f) * (size_t)nc + K];
                any = any || !is_zero(fb[v][f]);
            }
        double zsl[3];
        for (int f = 0; f < 3; f++) zsl[f] = zfb[f * (size_t)nc + K];
        if (!any) {                      // nothing flows back through the reconstruction
            own[K] = 0.0;
            own[nc + K] = 0.0;
            own[2 * (size_t)nc + K] = 0.0;
            const bool rk = m.rec[K];
            own[3 * (size_t)nc + K] = rk ? 0.0 : (zsl[0] + zsl[1]) + zsl[2];
            for (int f = 0; f < 3; f++) own[(4 + f) * (size_t)nc + K] = rk ? zsl[f] : 0.0;
            for (int q = 0; q < 12; q++) send[q * (size_t)nc + K] = 0.0;
            continue;
        }
        ReconFwd R;
        double Hf[3], Huf[3], Hvf[3];
        recon_forward(m, w, K, R, Hf, Huf, Hvf);
        double Hb = 0.0, Hub = 0.0, Hvb = 0.0, zb = 0.0, zfbK[3] = {0.0, 0.0, 0.0};
        double qnb[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};   // [f][v]
        if (!R.recon) {
            zb = (zsl[0] + zsl[1]) + zsl[2];
            for (int f = 0; f < 3; f++) { Hb += fb[0][f]; Hub += fb[1][f]; Hvb += fb[2][f]; }
        } else {
            double qKb[3] = {0, 0, 0};
            for (int f = 0; f < 3; f++) zfbK[f] = zsl[f] - fb[0][f];      // H_f = eta_f - z_f
            {
                // the centred source
                const double c = -m.g / G(m, GEO_AREA, K);
                const double rbu = Rb[nc + K], rbv = Rb[2 * (size_t)nc + K];
                const double eK = w[K] + m.z[K];
                double eb = 0.0;
                for (int f = 0; f < 3; f++) {
                    const double zff = m.zf[f * nc + K];
                    const double q = c * (G(m, GEO_LEN + f, K) * (G(m, GEO_NX + f, K) * rbu + G(m, GEO_NY + f, K) * rbv));
                    eb += q * zff;
                    zfbK[f] += q * (eK - zff);
                }
                Hb += eb;
                zb += eb;
            }
            for (int v = 0; v < 3; v++) {
                double ab = 0.0, Db[3];
                for (int f = 0; f < 3; f++) {
                    qKb[v] += fb[v][f];
                    ab += fb[v][f] * R.D[v][f];
                    Db[f] = fb[v][f] * R.alpha[v];
                }
                const int fa = R.fa[v];
                if (fa >= 0) {
                    // (faces picked by compare and select, not by index: indexed
                    // arrays would live in local memory)
                    const double D = fa == 0 ? R.D[v][0] : fa == 1 ? R.D[v][1] : R.D[v][2];
                    double iD = 1.0 / D;
                    double rb = ab * iD;
#pragma unroll
                    for (int f = 0; f < 3; f++)
                        if (f == fa) Db[f] -= rb * R.r[v] * iD;
                    int idx = is_pos(D) ? R.imax[v] : R.imin[v];
                    if (idx < 0) qKb[v] += rb;
#pragma unroll
                    for (int f = 0; f < 3; f++)
                        if (f == idx) qnb[f][v] += rb;
                    qKb[v] -= rb;
                }
                double gxb = 0.0, gyb = 0.0;
                for (int f = 0; f < 3; f++) {
                    gxb += Db[f] * G(m, GEO_FX + f, K);
                    gyb += Db[f] * G(m, GEO_FY + f, K);
                }
                for (int f = 0; f < 3; f++) {
                    double db = gxb * G(m, GEO_WX + f, K) + gyb * G(m, GEO_WY + f, K);
                    qnb[f][v] += db;
                    qKb[v] -= db;
                }
            }
            for (int f = 0; f < 3; f++) {
                if (!R.wall[f]) continue;
                if (R.open[f]) {                 // ghost = the cell's own values
                    qKb[0] += qnb[f][0];
                    Hub += qnb[f][1];
                    Hvb += qnb[f][2];
                    qnb[f][0] = qnb[f][1] = qnb[f][2] = 0.0;
                    continue;
                }
                double nx = G(m, GEO_NX + f, K), ny = G(m, GEO_NY + f, K);
                qKb[0] += qnb[f][0];
                double mnb = -2.0 * nx * qnb[f][1] - 2.0 * ny * qnb[f][2];
                Hub += qnb[f][1] + mnb * nx;
                Hvb += qnb[f][2] + mnb * ny;
                qnb[f][0] = qnb[f][1] = qnb[f][2] = 0.0;
            }
            Hb += qKb[0];
            zb += qKb[0];
            Hub += qKb[1];
            Hvb += qKb[2];
        }
        own[K] = Hb;
        own[nc + K] = Hub;
        own[2 * (size_t)nc + K] = Hvb;
        own[3 * (size_t)nc + K] = zb;
        for (int f = 0; f < 3; f++) own[(4 + f) * (size_t)nc + K] = zfbK[f];
        for (int f = 0; f < 3; f++) {
            send[(f * 4 + 0) * (size_t)nc + K] = qnb[f][0];     // eta-bar -> H-bar and z-bar
            send[(f * 4 + 1) * (size_t)nc + K] = qnb[f][1];
            send[(f * 4 + 2) * (size_t)nc + K] = qnb[f][2];
            send[(f * 4 + 3) * (size_t)nc + K] = qnb[f][0];
        }
    }
}

// wb[3][nc] += own + sum over faces of what the face neighbour sent; zb[nc] (cell
// beds) likewise; zb rows 1..3 (face beds) += the cell's own face-bed adjoints.
__global__ void adj_gather_kernel(AdjMesh m, const double *own, const double *send, double *wb, double *zb)
{
    const int nc = m.nc;
    for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < nc; K += gridDim.x * blockDim.x) {
        double a[4] = {own[K], own[nc + K], own[2 * (size_t)nc + K], own[3 * (size_t)nc + K]};
        for (int f = 0; f < 3; f++) {
            int j = m.nbr[f * nc + K];
            if (j < 0) continue;
            int fj = m.nbrl[f * nc + K] & 3;
            for (int k = 0; k < 4; k++) a[k] += send[(fj * 4 + k) * (size_t)nc + j];
        }
        wb[K] += a[0];
        wb[nc + K] += a[1];
        wb[2 * (size_t)nc + K] += a[2];
        zb[K] += a[3];
        for (int f = 0; f < 3; f++) zb[(1 + f) * (size_t)nc + K] += own[(4 + f) * (size_t)nc + K];
    }
}

// Dry fix after a stage (forward: H < 0 empties the cell; H <= H_threshold zeroes
// the momentum): its adjoint masks the incoming adjoint.
__device__ __forceinline__ void dry_fix_mask(double Hpre, double hthr, double &Hb, double &Hub, double &Hvb)
{
    if (is_neg(Hpre)) { Hb = 0.0; Hub = 0.0; Hvb = 0.0; }
    else if (!gt_nn(Hpre, hthr)) { Hub = 0.0; Hvb = 0.0; }
}

// w1 = fix(w + dt R0), keeping the pre-fix depth for the mask.
__global__ void adj_stage1_kernel(int nc, double dt, double hthr, const double *w, const double *R0, double *w1,
                                  double *H1pre)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += gridDim.x * blockDim.x) {
        double H = w[k] + dt * R0[k];
        double Hu = w[nc + k] + dt * R0[nc + k];
        double Hv = w[2 * (size_t)nc + k] + dt * R0[2 * (size_t)nc + k];
        H1pre[k] = H;
        if (is_neg(H)) { H = 0.0; Hu = 0.0; Hv = 0.0; }
        else if (!gt_nn(H, hthr)) { Hu = 0.0; Hv = 0.0; }
        w1[k] = H;
        w1[nc + k] = Hu;
        w1[2 * (size_t)nc + k] = Hv;
    }
}

// Reverse of stage 2: w^{n+1} = fix(w/2 + (w1 + dt R1)/2), with the dry-fix
// branch recorded by the forward stage-2 kernel (0 none, 1 momentum cut, 2
// emptied).  From wb (adjoint of w^{n+1}): wb_n = wb_1 = 1/2 wbpre, Rb = dt/2 wbpre.
__global__ void adj_stage2_rev_kernel(int nc, double dt, const uint8_t *mask2, const double *wb, double *wbn,
                                      double *wb1, double *Rb)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += gridDim.x * blockDim.x) {
        uint8_t br = mask2[k];
        double b[3] = {wb[k], wb[nc + k], wb[2 * (size_t)nc + k]};
        if (br == 2) { b[0] = 0.0; b[1] = 0.0; b[2] = 0.0; }
        else if (br == 1) { b[1] = 0.0; b[2] = 0.0; }
        for (int c = 0; c < 3; c++) {
            wbn[c * (size_t)nc + k] = 0.5 * b[c];
            wb1[c * (size_t)nc + k] = 0.5 * b[c];
            Rb[c * (size_t)nc + k] = 0.5 * dt * b[c];
        }
    }
}

// Reverse of stage 1: w1 = fix(w + dt R0).  wbn += wb1pre, Rb = dt wb1pre.
__global__ void adj_stage1_rev_kernel(int nc, double dt, double hthr, const double *H1pre, const double *wb1,
                                      double *wbn, double *Rb)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += gridDim.x * blockDim.x) {
        double b0 = wb1[k], b1 = wb1[nc + k], b2 = wb1[2 * (size_t)nc + k];
        dry_fix_mask(H1pre[k], hthr, b0, b1, b2);
        double b[3] = {b0, b1, b2};
        for (int c = 0; c < 3; c++) {
            wbn[c * (size_t)nc + k] += b[c];
            Rb[c * (size_t)nc + k] = dt * b[c];
        }
    }
}

// Gauge functional J = sum weights * (H + z) at the gauge cells: its adjoint.
__global__ void adj_gauge_kernel(int n_gauges, const int32_t *cells, const double *weights, int nc, double *wb,
                                 double *zb)
{
    // serial over gauges: two gauges may share a cell
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int g = 0; g < n_gauges; g++) {
            int c = cells[g];
            wb[c] += weights[g];
            zb[c] += weights[g];
        }
    (void)nc;
}

// ---------------------------------------------------------------------------
// Adjoint through the CFL time step (Sec. 2.3 rule, vg_adj_forward with dt = 0):
// dt = cfl |K*| / (3 l_f* a_f*) for the cell K* of smallest bound and its face
// f* of largest l_f a_f, so dt-bar reaches the state only through the wave
// speed of that one face: a-bar = -dt-bar dt / a.  dt-bar itself is
// sum (w1-bar . R0) + sum (w-bar^{n+1}_pre . R1 / 2), the two stages' use of dt.
// ---------------------------------------------------------------------------

// Forward wave speed of one face, the forward kernels' arithmetic.
__device__ double face_speed(const AdjMesh &m, double HfL, double HufL, double HvfL, double zL, double HfR,
                             double HufR, double HvfR, double zR, double nx, double ny, bool wall, int bnd)
{
    const double g = m.g, hthr = m.hthr;
    double uL = 0.0, vL = 0.0;
    if (gt_nn(HfL, hthr)) { uL = HufL / HfL; vL = HvfL / HfL; }
    double unL = uL * nx + vL * ny;
    double HsL, HsR, unR;
    if (wall && bnd == 3) {
        HsL = max0((HfL + zL) - zL);
        const double cL = sqrt(g * HsL), c0 = sqrt(g * max0(0.0 - zL));
        const double Rp = unL + 2.0 * cL, Rm = 0.0 - 2.0 * c0;
        unR = 0.5 * (Rp + Rm);
        const double cg = max0(0.25 * (Rp - Rm));
        HsR = cg * cg / g;
    } else if (wall) {
        HsL = max0((HfL + zL) - zL);
        HsR = HsL;
        unR = bnd == 2 ? unL : -unL;
    } else {
        double uR = 0.0, vR = 0.0;
        if (gt_nn(HfR, hthr)) { uR = HufR / HfR; vR = HvfR / HfR; }
        unR = uR * nx + vR * ny;
        double zs = smax(zL, zR);
        HsL = max0((HfL + zL) - zs);
        HsR = max0((HfR + zR) - zs);
    }
    if (is_zero(HsL) && is_zero(HsR)) return 0.0;
    double cL = sqrt(g * HsL), cR = sqrt(g * HsR), sL, sR;
    if (is_zero(HsL)) {
        sL = unR - 2.0 * cR;
        sR = unR + cR;
    } else if (is_zero(HsR)) {
        sL = unL - cL;
        sR = unL + 2.0 * cL;
    } else {
        double us = 0.5 * (unL + unR) + (cL - cR);
        double cs = 0.5 * (cL + cR) - 0.25 * (unR - unL);
        sL = smin(unL - cL, us - cs);
        sR = smax(us + cs, unR + cR);
    }
    return smax(fabs(sL), fabs(sR));
}

// The face states of face f of cell K (and its neighbour across it) from FV.
struct FaceIn {
    double HfL, HufL, HvfL, zL, HfR, HufR, HvfR, zR, nx, ny, l;
    int j, fj;
    bool wall;
    int bnd;                 // boundary kind: 1 wall, 2 open, 3 absorbing (0: interior)
};
__device__ FaceIn face_in(const AdjMesh &m, const double *FV, int K, int f)
{
    const int nc = m.nc;
    FaceIn r;
    r.j = m.nbr[f * nc + K];
    r.wall = r.j < 0;
    r.bnd = r.wall ? -r.j : 0;
    r.fj = r.wall ? 0 : (m.nbrl[f * nc + K] & 3);
    r.HfL = FV[(0 * 3 + f) * (size_t)nc + K];
    r.HufL = FV[(1 * 3 + f) * (size_t)nc + K];
    r.HvfL = FV[(2 * 3 + f) * (size_t)nc + K];
    r.zL = bed_under(m, K, f);
    r.HfR = r.HufR = r.HvfR = r.zR = 0.0;
    if (!r.wall) {
        r.HfR = FV[(0 * 3 + r.fj) * (size_t)nc + r.j];
        r.HufR = FV[(1 * 3 + r.fj) * (size_t)nc + r.j];
        r.HvfR = FV[(2 * 3 + r.fj) * (size_t)nc + r.j];
        r.zR = bed_under(m, r.j, r.fj);
    }
    r.nx = G(m, GEO_NX + f, K);
    r.ny = G(m, GEO_NY + f, K);
    r.l = G(m, GEO_LEN + f, K);
    return r;
}

// max_f l_f a_f of cell K (forward order, a tie keeping the earlier face) and its face.
__device__ double cell_speed(const AdjMesh &m, const double *FV, int K, int &fmax_out)
{
    double am = 0.0;
    fmax_out = -1;
    for (int f = 0; f < 3; f++) {
        FaceIn q = face_in(m, FV, K, f);
        double la = q.l * face_speed(m, q.HfL, q.HufL, q.HvfL, q.zL, q.HfR, q.HufR, q.HvfR, q.zR, q.nx, q.ny, q.wall,
                                     q.bnd);
        if (gt_nn(la, am)) { am = la; fmax_out = f; }
    }
    return am;
}

__device__ __forceinline__ bool cfl_less(double b1, int o1, double b2, int o2)
{
    return b1 < b2 || (b1 == b2 && o1 < o2);
}

// Per CTA: the cell of smallest bound |K| / (3 max_f l_f a_f) (ties: lowest
// original id) -> part_b, part_o, part_k [gridDim].
__global__ void adj_cfl_part_kernel(AdjMesh m, const double *FV, const int32_t *orig, double *part_b, int *part_o,
                                    int *part_k)
{
    __shared__ double sb[256];
    __shared__ int so[256], sk[256];
    const int nc = m.nc, tid = threadIdx.x;
    double bb = INFINITY;
    int bo = 0x7fffffff, bk = -1;
    for (int K = blockIdx.x * blockDim.x + tid; K < nc; K += gridDim.x * blockDim.x) {
        int f;
        double am = cell_speed(m, FV, K, f);
        if (!is_pos(am)) continue;
        double b = G(m, GEO_AREA, K) / (3.0 * am);
        if (cfl_less(b, orig[K], bb, bo)) { bb = b; bo = orig[K]; bk = K; }
    }
    sb[tid] = bb; so[tid] = bo; sk[tid] = bk;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s && cfl_less(sb[tid + s], so[tid + s], sb[tid], so[tid])) {
            sb[tid] = sb[tid + s]; so[tid] = so[tid + s]; sk[tid] = sk[tid + s];
        }
        __syncthreads();
    }
    if (tid == 0) { part_b[blockIdx.x] = sb[0]; part_o[blockIdx.x] = so[0]; part_k[blockIdx.x] = sk[0]; }
}

// dt-bar's face: one thread reduces the parts, finds the face f* of the chosen
// cell and adds the wave-speed adjoint's contribution to both sides' face slots.
__global__ void adj_cfl_face_kernel(AdjMesh m, const double *FV, int nparts, const double *part_b,
                                    const int *part_o, const int *part_k, const double *dtbar, double cfl,
                                    double dt_max, double *FVb, double *zfb)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double bb = INFINITY;
    int bo = 0x7fffffff, K = -1;
    for (int q = 0; q < nparts; q++)
        if (part_k[q] >= 0 && cfl_less(part_b[q], part_o[q], bb, bo)) { bb = part_b[q]; bo = part_o[q]; K = part_k[q]; }
    if (K < 0) return;                                   // nothing moves: dt = dt_max or 0
    const double dtc = cfl * bb;
    if (dt_max > 0.0 && dt_max < dtc) return;            // clamped by dt_max: no dependence
    int f;
    cell_speed(m, FV, K, f);
    const FaceIn q = face_in(m, FV, K, f);
    const double a = face_speed(m, q.HfL, q.HufL, q.HvfL, q.zL, q.HfR, q.HufR, q.HvfR, q.zR, q.nx, q.ny, q.wall,
                                q.bnd);
    const double ab = -(*dtbar) * dtc / a;
    const double P0[3] = {0.0, 0.0, 0.0};
    double bL[4], bR[4];
    flux_vjp(m, q.HfL, q.HufL, q.HvfL, q.zL, q.HfR, q.HufR, q.HvfR, q.zR, q.nx, q.ny, q.wall, P0, 0.0, 0.0, bL, bR, ab,
             q.bnd);
    const int nc = m.nc;
    for (int v = 0; v < 3; v++) FVb[(v * 3 + f) * (size_t)nc + K] += bL[v];
    zfb[f * (size_t)nc + K] += bL[3];
    if (!q.wall) {
        for (int v = 0; v < 3; v++) FVb[(v * 3 + q.fj) * (size_t)nc + q.j] += bR[v];
        zfb[q.fj * (size_t)nc + q.j] += bR[3];
    }
}

// Deterministic dot product: per-CTA partial sums, then one thread adds them in
// order, times scale, into *acc (reset: replaces it).
__global__ void adj_dot_part_kernel(int64_t n, const double *a, const double *b, double *part)
{
    __shared__ double sh[256];
    const int tid = threadIdx.x;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + tid; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += a[i] * b[i];
    sh[tid] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (tid < k) sh[tid] += sh[tid + k];
        __syncthreads();
    }
    if (tid == 0) part[blockIdx.x] = sh[0];
}

__global__ void adj_dot_final_kernel(int nparts, const double *part, double scale, double *acc, int reset)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int q = 0; q < nparts; q++) s += part[q];
    *acc = reset ? s * scale : *acc + s * scale;
}

// ---------------------------------------------------------------------------
// Moving bed: the beds of step n are z_K(t_n) = -(1/3) sum_{v in K} d_v(t_n) and
// z_f(t_n) = -(1/2) sum_{v on f} d_v(t_n), d_v(t) = depth0_v - uplift_v R((t -
// onset_v) / rise).  With zs the adjoints of that step's beds (its residuals
// and gauge record; row 0 cell beds, rows 1..3 face beds), per vertex
// s_v = sum over the cells K around v of zs_K / 3 + (zs of K's two faces at v) / 2,
// in a fixed order, and
//   uplift-bar_v += s_v R,   onset-bar_v += -s_v uplift_v R',
//   t-bar_n = sum_v s_v uplift_v R'      (R' = dR/dt = 1 / rise inside the ramp),
// the last summed per CTA into part (adaptive steps carry it to every earlier dt).
// ---------------------------------------------------------------------------
__global__ void adj_bed_vertex_kernel(int nv, int ncs, const int32_t *vptr, const int32_t *vcell, const double *zs,
                                      const double *uplift, const double *onset, double rise, double t, double *gU,
                                      double *gOn, double *part)
{
    __shared__ double sh[256];
    const int tid = threadIdx.x;
    double tb = 0.0;
    for (int v = blockIdx.x * blockDim.x + tid; v < nv; v += gridDim.x * blockDim.x) {
        double sv = 0.0;
        for (int k = vptr[v]; k < vptr[v + 1]; k++) {
            const int K = vcell[k] >> 2, j = vcell[k] & 3;
            // faces j (vertices j, j+1) and j+2 (vertices j+2, j) of K touch vertex j
            sv += zs[K] / 3.0 + (zs[(size_t)(1 + j) * ncs + K] + zs[(size_t)(1 + (j + 2) % 3) * ncs + K]) / 2.0;
        }
        double R, Rp = 0.0;
        if (rise > 0.0) {
            const double x = __dsub_rn(t, onset[v]) / rise;
            R = fmin(1.0, fmax(0.0, x));
            if (x > 0.0 && x < 1.0) Rp = 1.0 / rise;
        } else {
            R = t >= onset[v] ? 1.0 : 0.0;
        }
        gU[v] += sv * R;
        const double q = sv * uplift[v] * Rp;
        gOn[v] -= q;
        tb += q;
    }
    sh[tid] = tb;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (tid < k) sh[tid] += sh[tid + k];
        __syncthreads();
    }
    if (tid == 0) part[blockIdx.x] = sh[0];
}

__global__ void adj_axpy_kernel(int64_t n, const double *x, double *y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

__global__ void adj_scalar_add_kernel(double *y, const double *x)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *y += *x;
}

int grid_of(int n) { return (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096; }
// The two heavy reverse kernels run 128-thread CTAs: at 110 / 146 registers a
// thread that fits 4 / 3 CTAs per SM (16 / 12 warps) where 256-thread CTAs fit
// 2 / 1.
constexpr int kVjpThreads = 128;
int grid_vjp(int n) { return (n + kVjpThreads - 1) / kVjpThreads < 8192 ? (n + kVjpThreads - 1) / kVjpThreads : 8192; }

AdjMesh adj_mesh(const DevPtrs &d, const StepParams &p)
{
    AdjMesh m;
    m.nc = (int)d.nc;
    m.order = p.order;
    m.geo = static_cast<const double *>(d.geo);
    m.z = static_cast<const double *>(d.z);
    m.zf = static_cast<const double *>(d.zf);
    m.rec = nullptr;
    m.nbr = d.nbr;
    m.nbrl = d.nbrl;
    m.faces = d.adj_faces;
    m.nfaces = (int)d.n_adj_faces;
    m.g = p.g;
    m.half_g = 0.5 * p.g;
    m.hthr = p.hthr;
    return m;
}

}  // namespace

// Adds the VJP of the residual at w: (wb, zb) += (dR/dw, dR/dz)^T Rb, zb [4][nc]
// = (cell beds, face beds of faces 0..2).  rec: the stage's reconstruction flags.
// Scratch: FV, FVb [9][nc], zfb [3][nc], own [7][nc], send [12][nc].
int adjoint_residual_vjp(const DevPtrs &d, const StepParams &p, const double *w, const uint8_t *rec, const double *Rb,
                         double *wb, double *zb, double *FV, bool fv_given, double *FVb, double *zfb, double *own,
                         double *send, void *stream, const AdjCfl *cfl)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    AdjMesh m = adj_mesh(d, p);
    m.rec = rec;
    if (!rec) return (int)cudaErrorInvalidValue;
    int grid = grid_of(m.nc);
    if (!fv_given) adj_face_values_kernel<<<grid, 256, 0, s>>>(m, w, Rb, FV);
    if (!m.faces) return (int)cudaErrorInvalidValue;     // the face list is built by vg_adj_backward
    adj_flux_vjp_kernel<<<grid_vjp(m.nfaces), kVjpThreads, 0, s>>>(m, FV, Rb, FVb, zfb);
    if (cfl) {
        adj_cfl_part_kernel<<<kAdjCflParts, 256, 0, s>>>(m, FV, cfl->orig, cfl->part_b, cfl->part_o, cfl->part_k);
        adj_cfl_face_kernel<<<1, 32, 0, s>>>(m, FV, kAdjCflParts, cfl->part_b, cfl->part_o, cfl->part_k, cfl->dtbar,
                                             cfl->cfl, cfl->dt_max, FVb, zfb);
    }
    adj_recon_vjp_kernel<<<grid_vjp(m.nc), kVjpThreads, 0, s>>>(m, w, Rb, FVb, zfb, own, send);
    adj_gather_kernel<<<grid, 256, 0, s>>>(m, own, send, wb, zb);
    return (int)cudaGetLastError();
}

int adjoint_stage1(int nc, double dt, double hthr, const double *w, const double *R0, double *w1, double *H1pre,
                   void *stream)
{
    adj_stage1_kernel<<<grid_of(nc), 256, 0, static_cast<cudaStream_t>(stream)>>>(nc, dt, hthr, w, R0, w1, H1pre);
    return (int)cudaGetLastError();
}

int adjoint_stage2_rev(int nc, double dt, const uint8_t *mask2, const double *wb, double *wbn, double *wb1,
                       double *Rb, void *stream)
{
    adj_stage2_rev_kernel<<<grid_of(nc), 256, 0, static_cast<cudaStream_t>(stream)>>>(nc, dt, mask2, wb, wbn, wb1,
                                                                                       Rb);
    return (int)cudaGetLastError();
}

int adjoint_stage1_rev(int nc, double dt, double hthr, const double *H1pre, const double *wb1, double *wbn,
                       double *Rb, void *stream)
{
    adj_stage1_rev_kernel<<<grid_of(nc), 256, 0, static_cast<cudaStream_t>(stream)>>>(nc, dt, hthr, H1pre, wb1, wbn,
                                                                                       Rb);
    return (int)cudaGetLastError();
}

int adjoint_dot(int64_t n, const double *a, const double *b, double scale, double *acc, bool reset, double *part,
                void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    adj_dot_part_kernel<<<kAdjCflParts, 256, 0, s>>>(n, a, b, part);
    adj_dot_final_kernel<<<1, 32, 0, s>>>(kAdjCflParts, part, scale, acc, reset ? 1 : 0);
    return (int)cudaGetLastError();
}

int adjoint_bed_flush(int nc, int nv, const int32_t *vptr, const int32_t *vcell, double *zs, const double *uplift,
                      const double *onset, double rise, double t, double *gU, double *gOn, double *zb_total,
                      double *tsum, double *part, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    adj_bed_vertex_kernel<<<kAdjCflParts, 256, 0, s>>>(nv, nc, vptr, vcell, zs, uplift, onset, rise, t, gU, gOn, part);
    adj_dot_final_kernel<<<1, 32, 0, s>>>(kAdjCflParts, part, 1.0, tsum, 0);
    adj_axpy_kernel<<<grid_of(4 * nc), 256, 0, s>>>(4 * (int64_t)nc, zs, zb_total);
    return (int)cudaGetLastError();
}

int adjoint_scalar_add(double *y, const double *x, void *stream)
{
    adj_scalar_add_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(y, x);
    return (int)cudaGetLastError();
}

int adjoint_gauge(int n_gauges, const int32_t *cells, const double *weights, int nc, double *wb, double *zb,
                  void *stream)
{
    adj_gauge_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(n_gauges, cells, weights, nc, wb, zb);
    return (int)cudaGetLastError();
}

}  // namespace vg
