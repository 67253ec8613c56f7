/*
 * volna_oracle.c -- plain, slow FP64 CPU oracle of one explicit time step of the
 * cell-centred finite-volume scheme for the 2D nonlinear shallow water equations
 * of Giles et al., "Performance analysis of Volna-OP2" (Sec. 2).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load or call this file.  It shares no code, header,
 * table or helper with the CUDA library and never calls it.
 *
 * Build with -O2 -ffp-contract=off: no multiply-add contraction, so every
 * expression rounds exactly as written.  Loops over cells and edges may run
 * under OpenMP; each thread writes only its own cells, so results do not depend
 * on the thread count.
 *
 * The method, step by step (each function cites what it follows):
 *   geometry            cell area, centroid, outward unit normals, face midpoints
 *   bed                 z_K = -(mean of the three vertex depths), and the bed at
 *                       each face midpoint z_f = -(mean of its two vertex depths):
 *                       the piecewise linear bed of the vertex depths    (Sec. 2.1)
 *   reconstruction      least-squares gradient + Barth-Jespersen limiter,
 *                       skipped in the wet/dry zone; face depths stand on the
 *                       face beds                                        (Sec. 2.4, Eq. recon)
 *   interface           hydrostatic reconstruction of the two face depths (reading of
 *                       the wet/dry treatment named in Sec. 2.1), with the
 *                       centred bed-slope source of its second-order form
 *   numerical flux      HLL with the wave speeds of Sec. 2.2, dry-bed speeds
 *   wall                ghost state with mirrored normal velocity        (Sec. 2.5)
 *   open boundary       transmissive ghost (the cell's own state); reading, see
 *                       vo_set_open
 *   residual            edge fluxes gathered per cell in a fixed local order (Sec. 2.2)
 *   time step           CFL condition (reading of Sec. 2.3), SSP-RK(2,2) (Sec. 2.3)
 *   moving bed          time-dependent bathymetry h(x, y, t) of Sec. 2.1, read as a
 *                       kinematic rupture applied after each step        (vo_bed_at)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define VO_OK 0
#define VO_EINVAL (-1)
#define VO_ENOMEM (-2)

/* Scalar type of everything that depends on the water state or the bed.  It is
   double here; the oracle's discrete adjoint compiles this same file with a
   taping scalar type (oracle/volna_oracle_ad.cpp).  vo_val() is the value. */
#ifndef VO_REAL_DEFINED
typedef double vo_real;
#define vo_val(x) (x)
#endif

typedef struct vo_params {
    double g;            /* gravity, m s^-2 (the paper does not state it: 9.81) */
    double cfl;          /* Courant number of the time-step rule            */
    double h_threshold;  /* dry threshold H_threshold (Sec. 2.4)             */
    double dt_fixed;     /* > 0: use this time step instead of the CFL rule   */
    double dt_max;       /* > 0: upper clamp on the time step                 */
    double t_end;        /* > 0: the last step ends exactly at t_end          */
    int32_t order;       /* 1: first order (no reconstruction); 2: MUSCL      */
    int32_t limiter;     /* 1: Barth-Jespersen (Sec. 2.4); 0: none (alpha = 1),
                            only for the convergence pins of the reconstruction */
} vo_params;

typedef struct vo_mesh {
    int64_t nv, nc;
    int64_t n_flipped;   /* clockwise input triangles that were reoriented */
    int32_t *vtx;        /* [nc][3] vertex ids in local order              */
    int32_t *nbr;        /* [nc][3] neighbour across face f, -1 wall, -2 open, -3 absorbing */
    int32_t *nbr_face;   /* [nc][3] the same face seen from the neighbour   */
    vo_real *z;                                 /* [nc] bed                 */
    vo_real *zf;                                /* [nc][3] bed at the face midpoints */
    double *area, *cx, *cy;                     /* [nc]                     */
    double *nx, *ny, *len, *fx, *fy;            /* [nc][3] per face         */
    double *dx, *dy, *wx, *wy;                  /* [nc][3] LSQ stencil      */
    /* work arrays of the residual */
    vo_real *Hf, *Huf, *Hvf;                    /* [nc][3] face values      */
    vo_real *zfe;                               /* [nc][3] bed under each face value */
    int32_t *rec;                               /* [nc] 1 where the cell reconstructed */
    vo_real *slot;                              /* [nc][3][6] edge results  */
    vo_real *R0, *R1, *W1, *amax;               /* [3][nc], [3][nc], [3][nc], [nc] */
} vo_mesh;

void vo_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int vo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void vo_default_params(vo_params *p)
{
    p->g = 9.81;
    p->cfl = 0.9;
    p->h_threshold = 1e-5;
    p->dt_fixed = 0.0;
    p->dt_max = 0.0;
    p->t_end = 0.0;
    p->order = 2;
    p->limiter = 1;
}

void vo_mesh_free(vo_mesh *m)
{
    if (!m) return;
    free(m->vtx); free(m->nbr); free(m->nbr_face);
    free(m->z); free(m->zf); free(m->zfe); free(m->rec); free(m->area); free(m->cx); free(m->cy);
    free(m->nx); free(m->ny); free(m->len); free(m->fx); free(m->fy);
    free(m->dx); free(m->dy); free(m->wx); free(m->wy);
    free(m->Hf); free(m->Huf); free(m->Hvf); free(m->slot);
    free(m->R0); free(m->R1); free(m->W1); free(m->amax);
    free(m);
}

/*
 * Build the mesh: orientation, local face order, face adjacency and geometry.
 *
 * Local order: each triangle is made counter-clockwise (a clockwise input is
 * reoriented and counted), then rotated so that its first vertex has the
 * smallest input vertex id.  Face f joins local vertices f and f+1 (mod 3).
 * This fixes every summation order independently of how cells are numbered.
 *
 * Returns VO_EINVAL for an out-of-range or repeated vertex id, a zero-area
 * triangle, or an edge shared by more than two triangles (or twice in the same
 * direction).
 */
int vo_mesh_build(int64_t nv, const double *xy, int64_t nc, const int32_t *tri,
                  const vo_real *depth_v, vo_mesh **out)
{
    *out = NULL;
    if (nv < 3 || nc < 1 || !xy || !tri || !depth_v) return VO_EINVAL;
    vo_mesh *m = (vo_mesh *)calloc(1, sizeof(vo_mesh));
    if (!m) return VO_ENOMEM;
    m->nv = nv;
    m->nc = nc;
    size_t n3 = (size_t)nc * 3;
#define VO_ALLOC(p, n, T) do { (p) = (T *)malloc(sizeof(T) * (size_t)(n)); if (!(p)) { vo_mesh_free(m); return VO_ENOMEM; } } while (0)
#define VO_ALLOC_R(p, n, T) VO_ALLOC(p, n, T)
    VO_ALLOC(m->vtx, n3, int32_t);
    VO_ALLOC(m->nbr, n3, int32_t);
    VO_ALLOC(m->nbr_face, n3, int32_t);
    VO_ALLOC_R(m->z, nc, vo_real);
    VO_ALLOC_R(m->zf, n3, vo_real);
    VO_ALLOC_R(m->zfe, n3, vo_real);
    VO_ALLOC(m->rec, nc, int32_t);
    VO_ALLOC(m->area, nc, double);
    VO_ALLOC(m->cx, nc, double);
    VO_ALLOC(m->cy, nc, double);
    VO_ALLOC(m->nx, n3, double);
    VO_ALLOC(m->ny, n3, double);
    VO_ALLOC(m->len, n3, double);
    VO_ALLOC(m->fx, n3, double);
    VO_ALLOC(m->fy, n3, double);
    VO_ALLOC(m->dx, n3, double);
    VO_ALLOC(m->dy, n3, double);
    VO_ALLOC(m->wx, n3, double);
    VO_ALLOC(m->wy, n3, double);
    VO_ALLOC_R(m->Hf, n3, vo_real);
    VO_ALLOC_R(m->Huf, n3, vo_real);
    VO_ALLOC_R(m->Hvf, n3, vo_real);
    VO_ALLOC_R(m->slot, n3 * 6, vo_real);
    VO_ALLOC_R(m->R0, n3, vo_real);
    VO_ALLOC_R(m->R1, n3, vo_real);
    VO_ALLOC_R(m->W1, n3, vo_real);
    VO_ALLOC_R(m->amax, nc, vo_real);

    /* orientation and local order */
    for (int64_t c = 0; c < nc; c++) {
        int32_t a = tri[3 * c], b = tri[3 * c + 1], d = tri[3 * c + 2];
        if (a < 0 || b < 0 || d < 0 || a >= nv || b >= nv || d >= nv || a == b || b == d || a == d) {
            vo_mesh_free(m);
            return VO_EINVAL;
        }
        double s = (xy[2 * b] - xy[2 * a]) * (xy[2 * d + 1] - xy[2 * a + 1])
                 - (xy[2 * b + 1] - xy[2 * a + 1]) * (xy[2 * d] - xy[2 * a]);
        if (s == 0.0) { vo_mesh_free(m); return VO_EINVAL; }
        int32_t v[3] = {a, b, d};
        if (s < 0.0) { v[1] = d; v[2] = b; m->n_flipped++; }
        int k0 = 0;
        if (v[1] < v[k0]) k0 = 1;
        if (v[2] < v[k0]) k0 = 2;
        for (int k = 0; k < 3; k++) m->vtx[3 * c + k] = v[(k0 + k) % 3];
    }

    /* face adjacency through the cells around each vertex */
    int64_t *start = (int64_t *)calloc((size_t)nv + 1, sizeof(int64_t));
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * n3);
    if (!start || !list) { free(start); free(list); vo_mesh_free(m); return VO_ENOMEM; }
    for (size_t i = 0; i < n3; i++) start[m->vtx[i] + 1]++;
    for (int64_t v = 0; v < nv; v++) start[v + 1] += start[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    if (!fill) { free(start); free(list); vo_mesh_free(m); return VO_ENOMEM; }
    memcpy(fill, start, sizeof(int64_t) * (size_t)nv);
    for (int64_t c = 0; c < nc; c++)
        for (int k = 0; k < 3; k++) list[fill[m->vtx[3 * c + k]]++] = (int32_t)c;
    free(fill);
    int bad = 0;
    for (int64_t c = 0; c < nc && !bad; c++) {
        for (int f = 0; f < 3; f++) {
            int32_t p = m->vtx[3 * c + f], q = m->vtx[3 * c + (f + 1) % 3];
            int found = 0;
            m->nbr[3 * c + f] = -1;
            m->nbr_face[3 * c + f] = -1;
            for (int64_t i = start[p]; i < start[p + 1]; i++) {
                int32_t d = list[i];
                if (d == c) continue;
                for (int g = 0; g < 3; g++) {
                    int32_t a = m->vtx[3 * (int64_t)d + g], b = m->vtx[3 * (int64_t)d + (g + 1) % 3];
                    if (a == q && b == p) {          /* the same edge, opposite direction */
                        found++;
                        m->nbr[3 * c + f] = d;
                        m->nbr_face[3 * c + f] = g;
                    } else if (a == p && b == q) {   /* same direction: not a manifold */
                        bad = 1;
                    }
                }
            }
            if (found > 1) bad = 1;
        }
    }
    free(start);
    free(list);
    if (bad) { vo_mesh_free(m); return VO_EINVAL; }

    /* per-cell geometry and bed */
    for (int64_t c = 0; c < nc; c++) {
        const int32_t *v = m->vtx + 3 * c;
        double ax = xy[2 * v[0]], ay = xy[2 * v[0] + 1];
        double bx = xy[2 * v[1]], by = xy[2 * v[1] + 1];
        double qx = xy[2 * v[2]], qy = xy[2 * v[2] + 1];
        m->area[c] = 0.5 * ((bx - ax) * (qy - ay) - (by - ay) * (qx - ax));
        if (!(m->area[c] > 0.0)) { vo_mesh_free(m); return VO_EINVAL; }
        m->cx[c] = ((ax + bx) + qx) / 3.0;
        m->cy[c] = ((ay + by) + qy) / 3.0;
        m->z[c] = -((depth_v[v[0]] + depth_v[v[1]]) + depth_v[v[2]]) / 3.0;
        for (int f = 0; f < 3; f++) {
            int32_t p = v[f], q = v[(f + 1) % 3];
            double ex = xy[2 * q] - xy[2 * p];
            double ey = xy[2 * q + 1] - xy[2 * p + 1];
            double l = sqrt(ex * ex + ey * ey);
            m->len[3 * c + f] = l;
            m->zf[3 * c + f] = -(depth_v[p] + depth_v[q]) / 2.0;
            m->nx[3 * c + f] = ey / l;        /* outward: right of p -> q for a CCW cell */
            m->ny[3 * c + f] = -ex / l;
            m->fx[3 * c + f] = 0.5 * (xy[2 * p] + xy[2 * q]) - m->cx[c];
            m->fy[3 * c + f] = 0.5 * (xy[2 * p + 1] + xy[2 * q + 1]) - m->cy[c];
        }
    }
    /* least-squares stencil: neighbour centroids, or the centroid mirrored across a wall */
    for (int64_t c = 0; c < nc; c++) {
        double Mxx = 0.0, Mxy = 0.0, Myy = 0.0;
        for (int f = 0; f < 3; f++) {
            int64_t i = 3 * c + f;
            int32_t j = m->nbr[i];
            if (j >= 0) {
                m->dx[i] = m->cx[j] - m->cx[c];
                m->dy[i] = m->cy[j] - m->cy[c];
            } else {
                double dn = m->fx[i] * m->nx[i] + m->fy[i] * m->ny[i];
                m->dx[i] = 2.0 * dn * m->nx[i];
                m->dy[i] = 2.0 * dn * m->ny[i];
            }
            Mxx = Mxx + m->dx[i] * m->dx[i];
            Mxy = Mxy + m->dx[i] * m->dy[i];
            Myy = Myy + m->dy[i] * m->dy[i];
        }
        double det = Mxx * Myy - Mxy * Mxy;
        for (int f = 0; f < 3; f++) {
            int64_t i = 3 * c + f;
            m->wx[i] = (Myy * m->dx[i] - Mxy * m->dy[i]) / det;
            m->wy[i] = (Mxx * m->dy[i] - Mxy * m->dx[i]) / det;
        }
    }
    *out = m;
    return VO_OK;
}

/* --------------------------------------------------------------------------
 * Numerical flux (Sec. 2.2)
 * -------------------------------------------------------------------------- */

/*
 * HLL flux in the face's normal frame.  Each side is (H, u_n, u_t): depth,
 * velocity along the unit normal from L to R, and along t = (-n_y, n_x).
 * Conserved variables in this frame are w = (H, H u_n, H u_t) and the physical
 * flux is F(w) = (H u_n, H u_n^2 + g H^2 / 2, H u_n u_t).
 *
 * Wave speeds follow Sec. 2.2 (after Zhou 2002):
 *   s_L = min(u_nL - c_L, u*_n - c*),  s_R = max(u*_n + c*, u_nR + c_R),
 *   u*_n = (u_nL + u_nR)/2 + c_L - c_R,  c* = (c_L + c_R)/2 - (u_nR - u_nL)/4,
 *   c = sqrt(g H).
 * When one side is dry the textbook dry-bed speeds apply (reading of the
 * shoreline Riemann problem named in Sec. 2.1): L dry: s_L = u_nR - 2 c_R,
 * s_R = u_nR + c_R; R dry: s_L = u_nL - c_L, s_R = u_nL + 2 c_L.  Both dry:
 * zero flux.  F = F_L if s_L >= 0, F* if s_L < 0 <= s_R, F_R if s_R < 0, with
 *   F* = (s_R F_L - s_L F_R + s_L s_R (w_R - w_L)) / (s_R - s_L).
 * *amax receives max(|s_L|, |s_R|).
 */
/* The two HLL wave speeds (s_L, s_R) of the normal-frame states; see below. */
void vo_hll_speeds(double g, vo_real HL, vo_real unL, vo_real HR, vo_real unR, vo_real s[2])
{
    vo_real cL = sqrt(g * HL);
    vo_real cR = sqrt(g * HR);
    if (HL == 0.0) {
        s[0] = unR - 2.0 * cR;
        s[1] = unR + cR;
    } else if (HR == 0.0) {
        s[0] = unL - cL;
        s[1] = unL + 2.0 * cL;
    } else {
        vo_real us = 0.5 * (unL + unR) + (cL - cR);
        vo_real cs = 0.5 * (cL + cR) - 0.25 * (unR - unL);
        s[0] = fmin(unL - cL, us - cs);
        s[1] = fmax(us + cs, unR + cR);
    }
}

void vo_hll_normal(double g, vo_real HL, vo_real unL, vo_real utL,
                   vo_real HR, vo_real unR, vo_real utR, vo_real F[3], vo_real *amax)
{
    if (HL == 0.0 && HR == 0.0) {
        F[0] = 0.0; F[1] = 0.0; F[2] = 0.0;
        *amax = 0.0;
        return;
    }
    vo_real s[2];
    vo_hll_speeds(g, HL, unL, HR, unR, s);
    vo_real sL = s[0], sR = s[1];
    vo_real qL = HL * unL, qR = HR * unR;
    vo_real FL[3] = {qL, qL * unL + 0.5 * g * HL * HL, qL * utL};
    vo_real FR[3] = {qR, qR * unR + 0.5 * g * HR * HR, qR * utR};
    vo_real wL[3] = {HL, qL, HL * utL};
    vo_real wR[3] = {HR, qR, HR * utR};
    if (sL >= 0.0) {
        for (int k = 0; k < 3; k++) F[k] = FL[k];
    } else if (sR >= 0.0) {
        vo_real den = sR - sL;
        for (int k = 0; k < 3; k++)
            F[k] = ((sR * FL[k] - sL * FR[k]) + (sL * sR) * (wR[k] - wL[k])) / den;
    } else {
        for (int k = 0; k < 3; k++) F[k] = FR[k];
    }
    *amax = fmax(fabs(sL), fabs(sR));
}

/*
 * Flux through one face, seen from the left cell (outward unit normal n).
 * Inputs are the two reconstructed face states (depth H_f, momenta) and the bed
 * each of them stands on (the face bed z_f for a cell that reconstructed, its
 * cell bed otherwise).  Interface depths follow the hydrostatic reconstruction:
 *   z* = max(z_L, z_R),  H*_s = max(0, H_{s,f} + z_s - z*);
 * the face velocity is m_f / H_f where H_f > H_threshold, else 0, and the HLL
 * states carry H* times that velocity.  A wall face (wall != 0) uses the ghost
 * state of Sec. 2.5: same depth and bed, normal velocity reversed, tangential
 * velocity kept.  An open face (wall == 2) uses the transmissive ghost of
 * vo_set_open: the left face state itself, velocity unchanged.  An absorbing
 * face (wall == 3) uses the characteristic ghost of vo_set_boundary: the
 * outgoing Riemann invariant u_n + 2c of the face state and the incoming
 * u_n - 2c of the sea at rest beyond the boundary (eta = 0 over the face's bed,
 * c_0 = sqrt(g max(0, -z_L))) give u_n,g = (R+ + R-)/2 and c_g = max(0, (R+ - R-)/4),
 * depth c_g^2 / g on the same bed, tangential velocity kept.  Outputs: Phi
 * (mass, x- and y-momentum flux along n), the two pressure corrections
 * P_s = g (H_{s,f}^2 - H*_s^2) / 2 and the wave speed.
 */
void vo_face_flux(double g, double hthr,
                  vo_real HfL, vo_real HufL, vo_real HvfL, vo_real zL,
                  vo_real HfR, vo_real HufR, vo_real HvfR, vo_real zR,
                  double nx, double ny, int wall,
                  vo_real Phi[3], vo_real *PL, vo_real *PR, vo_real *amax)
{
    vo_real uL = 0.0, vL = 0.0;
    if (HfL > hthr) { uL = HufL / HfL; vL = HvfL / HfL; }
    vo_real unL = uL * nx + vL * ny;
    vo_real utL = -uL * ny + vL * nx;
    vo_real HsL, HsR, unR, utR;
    if (wall == 3) {
        HsL = fmax(0.0, (HfL + zL) - zL);
        vo_real cL = sqrt(g * HsL), c0 = sqrt(g * fmax(0.0, 0.0 - zL));
        vo_real Rp = unL + 2.0 * cL, Rm = 0.0 - 2.0 * c0;
        unR = 0.5 * (Rp + Rm);
        vo_real cg = fmax(0.0, 0.25 * (Rp - Rm));
        HsR = cg * cg / g;
        utR = utL;
        HfR = HsR;
    } else if (wall) {
        HsL = fmax(0.0, (HfL + zL) - zL);
        HsR = HsL;
        unR = wall == 2 ? unL : -unL;
        utR = utL;
        HfR = HfL;
    } else {
        vo_real uR = 0.0, vR = 0.0;
        if (HfR > hthr) { uR = HufR / HfR; vR = HvfR / HfR; }
        unR = uR * nx + vR * ny;
        utR = -uR * ny + vR * nx;
        vo_real zs = fmax(zL, zR);
        HsL = fmax(0.0, (HfL + zL) - zs);
        HsR = fmax(0.0, (HfR + zR) - zs);
    }
    vo_real F[3];
    vo_hll_normal(g, HsL, unL, utL, HsR, unR, utR, F, amax);
    Phi[0] = F[0];
    Phi[1] = F[1] * nx - F[2] * ny;
    Phi[2] = F[1] * ny + F[2] * nx;
    *PL = 0.5 * g * (HfL * HfL - HsL * HsL);
    *PR = 0.5 * g * (HfR * HfR - HsR * HsR);
}

/* --------------------------------------------------------------------------
 * Reconstruction (Sec. 2.4)
 * -------------------------------------------------------------------------- */

/*
 * Face values of cell K.  The reconstructed variables are eta = H + z, Hu, Hv.
 * Each face neighbour contributes its cell value; a wall contributes the ghost
 * of Sec. 2.5 (same eta, momentum mirrored: m - 2 (m.n) n), an open or an
 * absorbing face the cell's own values (zero gradient across it).
 *
 * The cell reconstructs (Eq. recon: w(x_f) = w_K + alpha_K grad(w)_K . (x_f - x_K))
 * only when it and every face neighbour are wetter than H_threshold and every
 * reconstructed face depth H_f = eta_f - z_f stays above H_threshold, z_f being
 * the bed at the face midpoint (the face value stands on the linear bed, as
 * the reconstructed free surface does on the face); otherwise its face values
 * are its cell values, standing on the cell bed z_K (the threshold rule of
 * Sec. 2.4).  zfe[f] receives the bed under face value f; returns 1 if the
 * cell reconstructed.
 *   gradient: least squares over the three stencil offsets d_f,
 *             grad q = sum_f w_f (q_f - q_K) with w_f = M^-1 d_f, M = sum d d^T;
 *   limiter:  Barth-Jespersen per variable, alpha = min over faces of
 *             min(1, (q_max - q_K)/D_f) if D_f > 0, min(1, (q_min - q_K)/D_f) if
 *             D_f < 0, 1 if D_f = 0, with D_f = grad q . (x_f - x_K) and q_max,
 *             q_min over the cell and its stencil values (alpha = 1 when the
 *             limiter is switched off for a pin).
 */
int vo_reconstruct_cell(const vo_mesh *m, const vo_params *p, const vo_real *H,
                        const vo_real *Hu, const vo_real *Hv, int64_t K,
                        vo_real Hf[3], vo_real Huf[3], vo_real Hvf[3], vo_real zfe[3])
{
    double hthr = p->h_threshold;
    vo_real zK = m->z[K];
    vo_real qK[3] = {H[K] + zK, Hu[K], Hv[K]};
    vo_real qn[3][3];
    int recon = (p->order == 2) && (H[K] > hthr);
    for (int f = 0; f < 3; f++) {
        int64_t i = 3 * K + f;
        int32_t j = m->nbr[i];
        if (j >= 0) {
            qn[f][0] = H[j] + m->z[j];
            qn[f][1] = Hu[j];
            qn[f][2] = Hv[j];
            if (!(H[j] > hthr)) recon = 0;
        } else if (j == -2 || j == -3) {
            qn[f][0] = qK[0];
            qn[f][1] = qK[1];
            qn[f][2] = qK[2];
        } else {
            vo_real mn = Hu[K] * m->nx[i] + Hv[K] * m->ny[i];
            qn[f][0] = qK[0];
            qn[f][1] = Hu[K] - 2.0 * mn * m->nx[i];
            qn[f][2] = Hv[K] - 2.0 * mn * m->ny[i];
        }
    }
    if (recon) {
        vo_real face[3][3];
        for (int v = 0; v < 3; v++) {
            const double *wx = m->wx + 3 * K, *wy = m->wy + 3 * K;
            vo_real gx = (wx[0] * (qn[0][v] - qK[v]) + wx[1] * (qn[1][v] - qK[v])) + wx[2] * (qn[2][v] - qK[v]);
            vo_real gy = (wy[0] * (qn[0][v] - qK[v]) + wy[1] * (qn[1][v] - qK[v])) + wy[2] * (qn[2][v] - qK[v]);
            vo_real qmax = qK[v], qmin = qK[v];
            for (int f = 0; f < 3; f++) {
                qmax = fmax(qmax, qn[f][v]);
                qmin = fmin(qmin, qn[f][v]);
            }
            vo_real alpha = 1.0;
            for (int f = 0; f < 3 && p->limiter; f++) {
                vo_real D = gx * m->fx[3 * K + f] + gy * m->fy[3 * K + f];
                vo_real phi = 1.0;
                if (D > 0.0) phi = fmin(1.0, (qmax - qK[v]) / D);
                else if (D < 0.0) phi = fmin(1.0, (qmin - qK[v]) / D);
                alpha = fmin(alpha, phi);
            }
            for (int f = 0; f < 3; f++) {
                vo_real D = gx * m->fx[3 * K + f] + gy * m->fy[3 * K + f];
                face[f][v] = qK[v] + alpha * D;
            }
        }
        for (int f = 0; f < 3; f++) {
            Hf[f] = face[f][0] - m->zf[3 * K + f];
            if (!(Hf[f] > hthr)) recon = 0;
        }
        if (recon) {
            for (int f = 0; f < 3; f++) {
                Huf[f] = face[f][1];
                Hvf[f] = face[f][2];
                zfe[f] = m->zf[3 * K + f];
            }
            return 1;
        }
    }
    for (int f = 0; f < 3; f++) {
        Hf[f] = H[K];
        Huf[f] = Hu[K];
        Hvf[f] = Hv[K];
        zfe[f] = zK;
    }
    return 0;
}

/* --------------------------------------------------------------------------
 * Residual L(w) (Sec. 2.2) and time step (Sec. 2.3)
 * -------------------------------------------------------------------------- */

/* A face is computed once, by the cell that owns it: the lower-numbered of the
   two cells, or the only cell at a wall. */
static int owns(const vo_mesh *m, int64_t K, int f)
{
    int32_t j = m->nbr[3 * K + f];
    return j < 0 || K < j;
}

/*
 * R = L(w): for every cell K,
 *   R_K = -(1/|K|) { sum_f l_f [ Phi_f + (0, P_{K,f} n_f) ] + (0, S_K) },
 * summed over the local faces f = 0, 1, 2 in that order, with Phi_f the flux out
 * of K (the owner's edge flux, negated for the other cell), P_{K,f} the
 * pressure correction on K's side, and, for a cell that reconstructed, the
 * centred bed-slope source of the second-order hydrostatic reconstruction
 * (Audusse et al. 2004, written over the faces of a triangle)
 *   S_K = g sum_f l_f z_f (eta_K - z_f / 2) n_f,   eta_K = H_K + z_K,
 * the integral over K of g (eta_K - z) grad z for the linear bed, in the form
 * that cancels the faces' hydrostatic pressures g (eta - z_f)^2 / 2 exactly
 * when eta is constant (lake at rest).  A cell that did not reconstruct stands
 * on its flat cell bed and has no such term.  amax[K] = max_f l_f a_f (NULL:
 * skipped).
 */
void vo_residual(vo_mesh *m, const vo_params *p, const vo_real *H, const vo_real *Hu,
                 const vo_real *Hv, vo_real *RH, vo_real *RHu, vo_real *RHv, vo_real *amax)
{
    int64_t nc = m->nc;
    double g = p->g, hthr = p->h_threshold;
#pragma omp parallel for schedule(static)
    for (int64_t K = 0; K < nc; K++)
        m->rec[K] = vo_reconstruct_cell(m, p, H, Hu, Hv, K, m->Hf + 3 * K, m->Huf + 3 * K, m->Hvf + 3 * K,
                                        m->zfe + 3 * K);

#pragma omp parallel for schedule(static)
    for (int64_t K = 0; K < nc; K++) {
        for (int f = 0; f < 3; f++) {
            if (!owns(m, K, f)) continue;
            int64_t i = 3 * K + f;
            int32_t j = m->nbr[i];
            vo_real *s = m->slot + 6 * i;
            if (j >= 0) {
                int64_t k = 3 * (int64_t)j + m->nbr_face[i];
                vo_face_flux(g, hthr, m->Hf[i], m->Huf[i], m->Hvf[i], m->zfe[i],
                             m->Hf[k], m->Huf[k], m->Hvf[k], m->zfe[k],
                             m->nx[i], m->ny[i], 0, s, s + 3, s + 4, s + 5);
            } else {
                vo_face_flux(g, hthr, m->Hf[i], m->Huf[i], m->Hvf[i], m->zfe[i],
                             0.0, 0.0, 0.0, 0.0, m->nx[i], m->ny[i], j == -2 ? 2 : j == -3 ? 3 : 1, s, s + 3, s + 4, s + 5);
            }
        }
    }

#pragma omp parallel for schedule(static)
    for (int64_t K = 0; K < nc; K++) {
        vo_real aH = 0.0, aHu = 0.0, aHv = 0.0, am = 0.0;
        for (int f = 0; f < 3; f++) {
            int64_t i = 3 * K + f;
            vo_real P0, P1, P2, P, a;
            if (owns(m, K, f)) {
                const vo_real *s = m->slot + 6 * i;
                P0 = s[0]; P1 = s[1]; P2 = s[2]; P = s[3]; a = s[5];
            } else {
                const vo_real *s = m->slot + 6 * (3 * (int64_t)m->nbr[i] + m->nbr_face[i]);
                P0 = -s[0]; P1 = -s[1]; P2 = -s[2]; P = s[4]; a = s[5];
            }
            double l = m->len[i];
            aH = aH + l * P0;
            aHu = aHu + l * (P1 + P * m->nx[i]);
            aHv = aHv + l * (P2 + P * m->ny[i]);
            am = fmax(am, l * a);
        }
        if (m->rec[K]) {
            vo_real eK = H[K] + m->z[K];
            for (int f = 0; f < 3; f++) {
                int64_t i = 3 * K + f;
                vo_real s = g * (m->len[i] * (m->zf[i] * (eK - 0.5 * m->zf[i])));
                aHu = aHu + s * m->nx[i];
                aHv = aHv + s * m->ny[i];
            }
        }
        RH[K] = -aH / m->area[K];
        RHu[K] = -aHu / m->area[K];
        RHv[K] = -aHv / m->area[K];
        if (amax) amax[K] = am;
    }
}

/*
 * Time step of the stage-1 state (reading of the CFL condition of Sec. 2.3):
 *   dt = CFL * min_K |K| / (3 max_f l_f a_f)
 * over cells with a nonzero wave speed, then clamped to dt_max (if > 0) and to
 * the time left before t_end (if > 0).  dt_fixed > 0 replaces the CFL rule.
 * With no moving wave anywhere the step is dt_max (0 when unset).
 */
vo_real vo_time_step(const vo_mesh *m, const vo_params *p, const vo_real *amax, double t)
{
    vo_real dt;
    if (p->dt_fixed > 0.0) {
        dt = p->dt_fixed;
    } else {
        /* the minimum runs over the cells in order, a tie keeping the earlier cell */
        vo_real mn = INFINITY;
        int any = 0;
        for (int64_t K = 0; K < m->nc; K++)
            if (vo_val(amax[K]) > 0.0) {
                mn = fmin(mn, m->area[K] / (3.0 * amax[K]));
                any = 1;
            }
        if (any) dt = p->cfl * mn;
        else dt = p->dt_max > 0.0 ? p->dt_max : 0.0;
    }
    if (p->dt_max > 0.0) dt = fmin(dt, (vo_real)p->dt_max);
    if (p->t_end > 0.0 && t + vo_val(dt) > p->t_end) dt = p->t_end - t;
    if (vo_val(dt) < 0.0) dt = 0.0;
    return dt;
}

/* After each stage: a negative depth is counted and the cell emptied; at or
   below H_threshold the momentum is zeroed. */
static int64_t dry_fix(int64_t nc, double hthr, vo_real *H, vo_real *Hu, vo_real *Hv)
{
    int64_t neg = 0;
#pragma omp parallel for schedule(static) reduction(+ : neg)
    for (int64_t K = 0; K < nc; K++) {
        if (H[K] < 0.0) {
            neg++;
            H[K] = 0.0; Hu[K] = 0.0; Hv[K] = 0.0;
        } else if (H[K] <= hthr) {
            Hu[K] = 0.0; Hv[K] = 0.0;
        }
    }
    return neg;
}

/*
 * One SSP-RK(2,2) step (Sec. 2.3), in place on (H, Hu, Hv):
 *   w1 = w + dt L(w);  w <- 1/2 w + 1/2 (w1 + dt L(w1)),
 * the same dt in both stages, each stage followed by the dry fix.  t is the
 * time at the start; returns dt (the state-dependent scalar); *neg_count is
 * added to.
 */
vo_real vo_step_dt(vo_mesh *m, const vo_params *p, vo_real *H, vo_real *Hu, vo_real *Hv, double t,
                   int64_t *neg_count)
{
    int64_t nc = m->nc;
    vo_real *R0 = m->R0, *R1 = m->R1, *W1 = m->W1;
    vo_real *H1 = W1, *Hu1 = W1 + nc, *Hv1 = W1 + 2 * nc;
    vo_residual(m, p, H, Hu, Hv, R0, R0 + nc, R0 + 2 * nc, m->amax);
    vo_real dt = vo_time_step(m, p, m->amax, t);
#pragma omp parallel for schedule(static)
    for (int64_t K = 0; K < nc; K++) {
        H1[K] = H[K] + dt * R0[K];
        Hu1[K] = Hu[K] + dt * R0[nc + K];
        Hv1[K] = Hv[K] + dt * R0[2 * nc + K];
    }
    int64_t neg = dry_fix(nc, p->h_threshold, H1, Hu1, Hv1);
    vo_residual(m, p, H1, Hu1, Hv1, R1, R1 + nc, R1 + 2 * nc, NULL);
#pragma omp parallel for schedule(static)
    for (int64_t K = 0; K < nc; K++) {
        H[K] = 0.5 * H[K] + 0.5 * (H1[K] + dt * R1[K]);
        Hu[K] = 0.5 * Hu[K] + 0.5 * (Hu1[K] + dt * R1[nc + K]);
        Hv[K] = 0.5 * Hv[K] + 0.5 * (Hv1[K] + dt * R1[2 * nc + K]);
    }
    neg += dry_fix(nc, p->h_threshold, H, Hu, Hv);
    if (neg_count) *neg_count += neg;
    return dt;
}

/* vo_step_dt with the time advanced in place: *t += dt, *dt_out = dt. */
void vo_step(vo_mesh *m, const vo_params *p, vo_real *H, vo_real *Hu, vo_real *Hv,
             double *t, double *dt_out, int64_t *neg_count)
{
    vo_real dt = vo_step_dt(m, p, H, Hu, Hv, *t, neg_count);
    *t += vo_val(dt);
    if (dt_out) *dt_out = vo_val(dt);
}

/* n steps; dts (may be NULL) receives each step's dt.  Gauges (may be NULL):
   eta at the n_gauges cells gauge_cells[] after every step into
   gauge_eta[step][g].  Returns the number of steps taken. */
int64_t vo_run(vo_mesh *m, const vo_params *p, vo_real *H, vo_real *Hu, vo_real *Hv,
               double *t, int64_t n_steps, double *dts, int64_t *neg_count,
               int32_t n_gauges, const int32_t *gauge_cells, vo_real *gauge_eta)
{
    for (int64_t s = 0; s < n_steps; s++) {
        double dt;
        vo_step(m, p, H, Hu, Hv, t, &dt, neg_count);
        if (dts) dts[s] = dt;
        for (int32_t g = 0; g < n_gauges && gauge_eta; g++) {
            int32_t c = gauge_cells[g];
            gauge_eta[s * (int64_t)n_gauges + g] = H[c] + m->z[c];
        }
    }
    return n_steps;
}

/*
 * Moving bed.  Sec. 2.1 writes the depth as time dependent, h(x, y, t), with
 * H = h + eta conserved by the mass equation.  Reading (the paper gives no
 * source model): a kinematic rupture in which vertex v rises by uplift_v,
 * linearly over `rise` seconds from its onset time,
 *     depth_v(t) = depth0_v - uplift_v R((t - onset_v) / rise),
 *     R(s) = min(1, max(0, s))           (rise = 0: R = 1 once t >= onset_v),
 * and the cell bed is z_K(t) = -(mean of its vertices' depths), the face bed
 * z_f(t) = -(mean of its two vertices' depths), as at set-up.
 * The bed moves between steps: after the step that ends at t^{n+1} the beds
 * are set to z(t^{n+1}) with H unchanged, so the free surface eta = H + z
 * follows the bed and no mass is created.
 */
static vo_real ramp(vo_real t, vo_real onset, double rise)
{
    if (rise > 0.0) return fmin((vo_real)1.0, fmax((vo_real)0.0, (t - onset) / rise));
    return vo_val(t) >= vo_val(onset) ? 1.0 : 0.0;
}

/* The source arrays and the time have the state-dependent scalar type, so
   that the taped build differentiates the run with respect to them (with
   adaptive steps the time itself depends on the state). */
void vo_bed_at(vo_mesh *m, const vo_real *depth0, const vo_real *uplift, const vo_real *onset, double rise,
               vo_real t)
{
#pragma omp parallel for schedule(static)
    for (int64_t K = 0; K < m->nc; K++) {
        vo_real d[3];
        for (int k = 0; k < 3; k++) {
            int32_t v = m->vtx[3 * K + k];
            d[k] = depth0[v] - uplift[v] * ramp(t, onset[v], rise);
        }
        m->z[K] = -((d[0] + d[1]) + d[2]) / 3.0;
        for (int f = 0; f < 3; f++) m->zf[3 * K + f] = -(d[f] + d[(f + 1) % 3]) / 2.0;
    }
}

/* vo_run with a moving bed: the beds are first set to z(t) at the start time,
   then after every step to z at the step's end time (before the gauges). */
int64_t vo_run_bed(vo_mesh *m, const vo_params *p, vo_real *H, vo_real *Hu, vo_real *Hv,
                   double *t, int64_t n_steps, double *dts, int64_t *neg_count,
                   int32_t n_gauges, const int32_t *gauge_cells, vo_real *gauge_eta,
                   const vo_real *depth0, const vo_real *uplift, const vo_real *onset, double rise)
{
    vo_bed_at(m, depth0, uplift, onset, rise, *t);
    for (int64_t s = 0; s < n_steps; s++) {
        double dt;
        vo_step(m, p, H, Hu, Hv, t, &dt, neg_count);
        vo_bed_at(m, depth0, uplift, onset, rise, *t);
        if (dts) dts[s] = dt;
        for (int32_t g = 0; g < n_gauges && gauge_eta; g++) {
            int32_t c = gauge_cells[g];
            gauge_eta[s * (int64_t)n_gauges + g] = H[c] + m->z[c];
        }
    }
    return n_steps;
}

/*
 * Open (transmissive) boundary.  The paper's code has walls (Sec. 2.5) and defers
 * other boundary conditions to Dutykh et al. 2011.  Reading: a boundary face
 * marked open takes as ghost the cell's own state, unchanged (zero-gradient
 * extrapolation): the reconstruction sees no difference across it, and the
 * face flux is the HLL flux between the face state and itself, i.e. the
 * physical flux of the face state, so waves leave with little reflection.
 * The ghost's position in the least-squares stencil stays the mirrored one.
 * Marks the n boundary edges edges[k] = (a, b) (vertex ids, either order) open
 * and every other boundary face a wall.  VO_EINVAL if an edge is not a
 * boundary face of the mesh (nothing is changed then).
 */
int vo_set_boundary(vo_mesh *m, int64_t n, const int32_t *edges, const int32_t *kinds);

int vo_set_open(vo_mesh *m, int64_t n, const int32_t *edges)
{
    return vo_set_boundary(m, n, edges, NULL);
}

/*
 * Boundary kinds per edge: kinds[k] = 1 wall, 2 open (vo_set_open), 3 absorbing
 * (kinds NULL: all open); every other boundary face a wall.  Absorbing reading:
 * the paper defers such conditions to Dutykh et al. 2011; here the
 * characteristic condition of a sea at rest (eta = 0) beyond the boundary, the
 * ghost of vo_face_flux (wall == 3), with the open face's zero-gradient ghost
 * in the reconstruction.  VO_EINVAL for an edge that is not a boundary face or
 * an unknown kind (nothing is changed then).
 */
int vo_set_boundary(vo_mesh *m, int64_t n, const int32_t *edges, const int32_t *kinds)
{
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1) * 2);
    if (!mark) return VO_ENOMEM;
    for (int64_t k = 0; k < n; k++) {
        int32_t a = edges[2 * k], b = edges[2 * k + 1];
        int64_t found = -1;
        for (int64_t i = 0; i < 3 * m->nc && found < 0; i++) {
            if (m->nbr[i] >= 0) continue;
            int64_t K = i / 3;
            int f = (int)(i % 3);
            int32_t p = m->vtx[3 * K + f], q = m->vtx[3 * K + (f + 1) % 3];
            if ((p == a && q == b) || (p == b && q == a)) found = i;
        }
        if (found < 0) { free(mark); return VO_EINVAL; }
        mark[k] = (int32_t)found;
    }
    for (int64_t k = 0; k < n; k++)
        if (kinds && (kinds[k] < 1 || kinds[k] > 3)) { free(mark); return VO_EINVAL; }
    for (int64_t i = 0; i < 3 * m->nc; i++)
        if (m->nbr[i] < 0) m->nbr[i] = -1;
    for (int64_t k = 0; k < n; k++) m->nbr[mark[k]] = kinds ? -kinds[k] : -2;
    free(mark);
    return VO_OK;
}

/* The cell containing each point (boundary included; among several, the lowest
   cell id).  -1 when no cell contains it. */
void vo_locate(const vo_mesh *m, const double *xy, int32_t n, const double *pts, int32_t *cells)
{
    for (int32_t k = 0; k < n; k++) {
        double px = pts[2 * k], py = pts[2 * k + 1];
        cells[k] = -1;
        for (int64_t c = 0; c < m->nc; c++) {
            int inside = 1;
            for (int f = 0; f < 3 && inside; f++) {
                int32_t a = m->vtx[3 * c + f], b = m->vtx[3 * c + (f + 1) % 3];
                double o = (xy[2 * b] - xy[2 * a]) * (py - xy[2 * a + 1])
                         - (xy[2 * b + 1] - xy[2 * a + 1]) * (px - xy[2 * a]);
                if (o < 0.0) inside = 0;
            }
            if (inside) { cells[k] = (int32_t)c; break; }
        }
    }
}

/* Accessors: copy a per-cell or per-face array out (what: see the switch). */
int vo_mesh_get(const vo_mesh *m, int what, void *out)
{
    size_t n1 = (size_t)m->nc, n3 = 3 * (size_t)m->nc;
    switch (what) {
    case 0: memcpy(out, m->vtx, n3 * sizeof(int32_t)); return 0;
    case 1: memcpy(out, m->nbr, n3 * sizeof(int32_t)); return 0;
    case 2: memcpy(out, m->nbr_face, n3 * sizeof(int32_t)); return 0;
    case 3: memcpy(out, m->z, n1 * sizeof(double)); return 0;
    case 4: memcpy(out, m->area, n1 * sizeof(double)); return 0;
    case 5: memcpy(out, m->cx, n1 * sizeof(double)); return 0;
    case 6: memcpy(out, m->cy, n1 * sizeof(double)); return 0;
    case 7: memcpy(out, m->nx, n3 * sizeof(double)); return 0;
    case 8: memcpy(out, m->ny, n3 * sizeof(double)); return 0;
    case 9: memcpy(out, m->len, n3 * sizeof(double)); return 0;
    case 10: memcpy(out, m->fx, n3 * sizeof(double)); return 0;
    case 11: memcpy(out, m->fy, n3 * sizeof(double)); return 0;
    case 12: memcpy(out, m->wx, n3 * sizeof(double)); return 0;
    case 13: memcpy(out, m->wy, n3 * sizeof(double)); return 0;
    case 14: memcpy(out, m->dx, n3 * sizeof(double)); return 0;
    case 15: memcpy(out, m->dy, n3 * sizeof(double)); return 0;
    case 16: memcpy(out, m->zf, n3 * sizeof(double)); return 0;
    default: return VO_EINVAL;
    }
}

int64_t vo_mesh_n_flipped(const vo_mesh *m) { return m->n_flipped; }
int64_t vo_mesh_nc(const vo_mesh *m) { return m->nc; }
