// The oracle's discrete adjoint.  TEST INFRASTRUCTURE.
//
// volna_oracle.c is compiled a second time here with its scalar type vo_real
// set to the taping type of ad_tape.hpp: the forward run is the oracle's own
// arithmetic, and one reverse sweep of the tape gives the exact derivative of
// that program (branches frozen where the run took them) -- an adjoint written
// by no one, against which the hand-written GPU adjoint is compared.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ad_tape.hpp"

#define VO_REAL_DEFINED
typedef adouble vo_real;
#define vo_val(x) ((x).v)

namespace vo_ad_impl {
#include "volna_oracle.c"
}

using vo_ad_impl::vo_mesh;
using vo_ad_impl::vo_params;

// Boundary edges and their kinds (vo_set_boundary: 1 wall, 2 open, 3
// absorbing) applied to every mesh the entry points below build; empty: all
// boundary faces are walls.
static std::vector<int32_t> g_bnd_edges, g_bnd_kinds;

static int apply_boundary(vo_mesh *m)
{
    if (g_bnd_kinds.empty()) return 0;
    return vo_ad_impl::vo_set_boundary(m, (int64_t)g_bnd_kinds.size(), g_bnd_edges.data(), g_bnd_kinds.data());
}

extern "C" {

/* The boundary edges [n][2] (vertex ids) and kinds [n] (NULL: all open) of the
 * following calls; n = 0: walls. */
int vo_ad_set_boundary(int64_t n, const int32_t *edges, const int32_t *kinds)
{
    if (n < 0) n = 0;
    g_bnd_edges.assign(edges, edges + 2 * n);
    g_bnd_kinds.assign((size_t)n, 2);
    if (kinds) g_bnd_kinds.assign(kinds, kinds + n);
    return 0;
}

/* The open boundary edges [n][2] (vertex ids) of the following calls; n = 0: walls. */
int vo_ad_set_open(int64_t n, const int32_t *edges)
{
    return vo_ad_set_boundary(n, edges, nullptr);
}

/*
 * Linear gauge functional and its gradient through n_steps SSP-RK(2,2) steps
 * with the fixed time step dt, or (dt <= 0) the CFL time step of each step
 * (Sec. 2.3 rule with the given cfl), differentiated through the minimum:
 *   J = sum_{n = 0..n_steps} sum_g weights[n][g] * eta_g(t_n),
 * eta_g = H + z of gauge cell g (after step n; n = 0 is the initial state).
 * Inputs: the mesh (as vo_mesh_build), per-vertex depth, the initial state,
 * g / H_threshold / order / cfl.  Outputs: eta_out[n_steps + 1][G] and
 * dts_out[n_steps] (may be NULL), *J, and dJ/dH0, dJ/dHu0, dJ/dHv0 [nc] and
 * dJ/ddepth_v [nv].
 * Returns 0, or a negative code for a rejected mesh.
 */
int vo_ad_gauge_gradient(int64_t nv, const double *xy, int64_t nc, const int32_t *tri, const double *depth_v,
                         const double *H0, const double *Hu0, const double *Hv0, double g, double hthr, int order,
                         double cfl, double dt, int64_t n_steps, int32_t n_gauges, const int32_t *gauge_cells,
                         const double *weights, double *eta_out, double *dts_out, double *J_out, double *gH0,
                         double *gHu0, double *gHv0, double *gdepth)
{
    VoTape &tape = vo_tape();
    tape.clear();
    std::vector<adouble> depth(nv), H(nc), Hu(nc), Hv(nc);
    for (int64_t v = 0; v < nv; v++) depth[v] = adouble::variable(depth_v[v]);
    for (int64_t k = 0; k < nc; k++) H[k] = adouble::variable(H0[k]);
    for (int64_t k = 0; k < nc; k++) Hu[k] = adouble::variable(Hu0[k]);
    for (int64_t k = 0; k < nc; k++) Hv[k] = adouble::variable(Hv0[k]);
    vo_mesh *m = nullptr;
    int rc = vo_ad_impl::vo_mesh_build(nv, xy, nc, tri, depth.data(), &m);
    if (rc) return rc;
    if ((rc = apply_boundary(m))) { vo_ad_impl::vo_mesh_free(m); return rc; }
    vo_params p;
    vo_ad_impl::vo_default_params(&p);
    p.g = g;
    p.h_threshold = hthr;
    p.order = order;
    p.cfl = cfl;
    p.dt_fixed = dt > 0.0 ? dt : 0.0;
    adouble J = 0.0;
    double t = 0.0;
    int64_t neg = 0;
    for (int64_t n = 0; n <= n_steps; n++) {
        if (n > 0) {
            double dtn = 0.0;
            vo_ad_impl::vo_step(m, &p, H.data(), Hu.data(), Hv.data(), &t, &dtn, &neg);
            if (dts_out) dts_out[n - 1] = dtn;
        }
        for (int32_t k = 0; k < n_gauges; k++) {
            int32_t c = gauge_cells[k];
            adouble eta = H[c] + m->z[c];
            if (eta_out) eta_out[n * n_gauges + k] = eta.v;
            J = J + weights[n * n_gauges + k] * eta;
        }
    }
    *J_out = J.v;
    std::vector<double> adj(tape.size(), 0.0);
    if (J.i >= 0) adj[J.i] = 1.0;
    tape.reverse(adj);
    // variables were pushed first, in the order depth, H, Hu, Hv
    for (int64_t v = 0; v < nv; v++) gdepth[v] = adj[v];
    for (int64_t k = 0; k < nc; k++) gH0[k] = adj[nv + k];
    for (int64_t k = 0; k < nc; k++) gHu0[k] = adj[nv + nc + k];
    for (int64_t k = 0; k < nc; k++) gHv0[k] = adj[nv + 2 * nc + k];
    vo_ad_impl::vo_mesh_free(m);
    tape.clear();
    tape.a0.shrink_to_fit(); tape.a1.shrink_to_fit(); tape.d0.shrink_to_fit(); tape.d1.shrink_to_fit();
    return 0;
}

/*
 * The same functional with a moving bed (vo_bed_at: depth_v(t) = depth_v -
 * uplift_v R((t - onset_v) / rise), applied at the start and after every step)
 * and its gradient, adding dJ/duplift_v and dJ/donset_v [nv] to the outputs of
 * vo_ad_gauge_gradient.
 */
int vo_ad_gauge_gradient_bed(int64_t nv, const double *xy, int64_t nc, const int32_t *tri, const double *depth_v,
                             const double *H0, const double *Hu0, const double *Hv0, double g, double hthr,
                             int order, double cfl, double dt, int64_t n_steps, int32_t n_gauges,
                             const int32_t *gauge_cells, const double *weights, const double *uplift_v,
                             const double *onset_v, double rise, double *eta_out, double *dts_out, double *J_out,
                             double *gH0, double *gHu0, double *gHv0, double *gdepth, double *guplift,
                             double *gonset)
{
    VoTape &tape = vo_tape();
    tape.clear();
    std::vector<adouble> depth(nv), H(nc), Hu(nc), Hv(nc), up(nv), on(nv);
    for (int64_t v = 0; v < nv; v++) depth[v] = adouble::variable(depth_v[v]);
    for (int64_t k = 0; k < nc; k++) H[k] = adouble::variable(H0[k]);
    for (int64_t k = 0; k < nc; k++) Hu[k] = adouble::variable(Hu0[k]);
    for (int64_t k = 0; k < nc; k++) Hv[k] = adouble::variable(Hv0[k]);
    for (int64_t v = 0; v < nv; v++) up[v] = adouble::variable(uplift_v[v]);
    for (int64_t v = 0; v < nv; v++) on[v] = adouble::variable(onset_v[v]);
    vo_mesh *m = nullptr;
    int rc = vo_ad_impl::vo_mesh_build(nv, xy, nc, tri, depth.data(), &m);
    if (rc) return rc;
    if ((rc = apply_boundary(m))) { vo_ad_impl::vo_mesh_free(m); return rc; }
    vo_params p;
    vo_ad_impl::vo_default_params(&p);
    p.g = g;
    p.h_threshold = hthr;
    p.order = order;
    p.cfl = cfl;
    p.dt_fixed = dt > 0.0 ? dt : 0.0;
    adouble J = 0.0;
    adouble t = 0.0;       // with adaptive steps the time, and so the bed, depend on the state
    int64_t neg = 0;
    vo_ad_impl::vo_bed_at(m, depth.data(), up.data(), on.data(), rise, t);
    for (int64_t n = 0; n <= n_steps; n++) {
        if (n > 0) {
            adouble dtn = vo_ad_impl::vo_step_dt(m, &p, H.data(), Hu.data(), Hv.data(), t.v, &neg);
            t = t + dtn;
            vo_ad_impl::vo_bed_at(m, depth.data(), up.data(), on.data(), rise, t);
            if (dts_out) dts_out[n - 1] = dtn.v;
        }
        for (int32_t k = 0; k < n_gauges; k++) {
            int32_t c = gauge_cells[k];
            adouble eta = H[c] + m->z[c];
            if (eta_out) eta_out[n * n_gauges + k] = eta.v;
            J = J + weights[n * n_gauges + k] * eta;
        }
    }
    *J_out = J.v;
    std::vector<double> adj(tape.size(), 0.0);
    if (J.i >= 0) adj[J.i] = 1.0;
    tape.reverse(adj);
    for (int64_t v = 0; v < nv; v++) gdepth[v] = adj[v];
    for (int64_t k = 0; k < nc; k++) gH0[k] = adj[nv + k];
    for (int64_t k = 0; k < nc; k++) gHu0[k] = adj[nv + nc + k];
    for (int64_t k = 0; k < nc; k++) gHv0[k] = adj[nv + 2 * nc + k];
    for (int64_t v = 0; v < nv; v++) guplift[v] = adj[nv + 3 * nc + v];
    for (int64_t v = 0; v < nv; v++) gonset[v] = adj[2 * nv + 3 * nc + v];
    vo_ad_impl::vo_mesh_free(m);
    tape.clear();
    tape.a0.shrink_to_fit(); tape.a1.shrink_to_fit(); tape.d0.shrink_to_fit(); tape.d1.shrink_to_fit();
    return 0;
}

}  // extern "C"
