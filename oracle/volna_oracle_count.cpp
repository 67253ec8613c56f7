// The oracle compiled with the operation-counting scalar of op_count.hpp.
// TEST INFRASTRUCTURE: counts the floating-point operations of one SSP-RK(2,2)
// step (Sec. 2.3) of the oracle's own arithmetic on a given state.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "op_count.hpp"

#define VO_REAL_DEFINED
typedef cdouble vo_real;
#define vo_val(x) ((x).v)

namespace vo_count_impl {
#include "volna_oracle.c"
}

extern "C" {

/*
 * One adaptive step (CFL rule of Sec. 2.3) from (H0, Hu0, Hv0) on the mesh
 * (as vo_mesh_build); counts[6] receives the additions, subtractions,
 * multiplications, divisions, square roots and min/max/abs operations on
 * state-dependent values, *dt_out the step.  Returns 0 or a negative code.
 */
int vo_count_step(int64_t nv, const double *xy, int64_t nc, const int32_t *tri, const double *depth_v,
                  const double *H0, const double *Hu0, const double *Hv0, double g, double hthr, double cfl,
                  int64_t counts[6], double *dt_out)
{
    vo_count_impl::vo_mesh *m = nullptr;
    cdouble *depth = (cdouble *)malloc(sizeof(cdouble) * nv);
    cdouble *w = (cdouble *)malloc(sizeof(cdouble) * 3 * nc);
    if (!depth || !w) { free(depth); free(w); return -2; }
    for (int64_t v = 0; v < nv; v++) depth[v] = cdouble(depth_v[v]);
    int rc = vo_count_impl::vo_mesh_build(nv, xy, nc, tri, depth, &m);
    if (rc) { free(depth); free(w); return rc; }
    for (int64_t k = 0; k < nc; k++) {
        w[k] = cdouble(H0[k]);
        w[nc + k] = cdouble(Hu0[k]);
        w[2 * nc + k] = cdouble(Hv0[k]);
    }
    vo_count_impl::vo_params p;
    vo_count_impl::vo_default_params(&p);
    p.g = g;
    p.h_threshold = hthr;
    p.cfl = cfl;
    vo_counts() = VoOpCounts();
    double t = 0.0, dt = 0.0;
    int64_t neg = 0;
    vo_count_impl::vo_step(m, &p, w, w + nc, w + 2 * nc, &t, &dt, &neg);
    const VoOpCounts &c = vo_counts();
    counts[0] = c.add; counts[1] = c.sub; counts[2] = c.mul;
    counts[3] = c.div; counts[4] = c.sqrt; counts[5] = c.minmax;
    if (dt_out) *dt_out = dt;
    vo_count_impl::vo_mesh_free(m);
    free(depth);
    free(w);
    return 0;
}

}  // extern "C"
