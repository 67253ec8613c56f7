// Small kernels around the step: the per-step epilogue (time, gauges, reset of
// the CFL minimum), state import/export with the cell permutation, and the
// diagnostics reduction.
#include "step_kernels.cuh"

namespace vg {

namespace {

template <typename real>
__device__ __forceinline__ unsigned long long inf_bits();
template <> __device__ __forceinline__ unsigned long long inf_bits<float>() { return (unsigned long long)__float_as_uint(CUDART_INF_F); }
template <> __device__ __forceinline__ unsigned long long inf_bits<double>() { return (unsigned long long)__double_as_longlong(CUDART_INF); }

// Epilogue of one step: t += dt (Sec. 2.3), gauge record (Sec. 3 virtual gauges:
// eta = H + z of each gauge cell), reset of the CFL minimum for the next step.
template <typename real>
__global__ void post_step_kernel(DevPtrs d, StepParams p, const real *w)
{
    __shared__ long long rec;
    DevScalars *sc = d.sc;
    if (threadIdx.x == 0) {
        double dt = step_dt<real>(sc, p.cfl, p.dt_fixed, p.dt_max, p.t_end);
        sc->dt = dt;
        rec = -1;
        if (!isfinite(dt)) sc->flags |= FLAG_NONFINITE_DT;
        if (dt > 0.0) {
            sc->t = sc->t + dt;
            sc->steps += 1;
            if (d.n_gauges > 0 && sc->steps % p.gauge_every == 0) {
                if (sc->n_rec < d.ring_cap) {
                    rec = sc->n_rec;
                    sc->n_rec = rec + 1;
                    d.ring_t[rec] = sc->t;
                } else {
                    sc->flags |= FLAG_RING_FULL;
                }
            }
        }
        sc->dtmin_bits = inf_bits<real>();
    }
    __syncthreads();
    if (rec >= 0) {
        const real *z = static_cast<const real *>(d.z);
        for (int g = threadIdx.x; g < d.n_gauges; g += blockDim.x) {
            int32_t c = d.gauge_cells[g];
            d.ring_eta[rec * d.n_gauges + g] = EtaForm<real>::value ? (double)w[c] : (double)(w[c] + z[c]);
        }
    }
}

template <typename real>
__global__ void record_gauges_kernel(DevPtrs d, const real *w)
{
    DevScalars *sc = d.sc;
    long long rec = sc->n_rec;
    if (rec >= d.ring_cap) {
        if (threadIdx.x == 0) sc->flags |= FLAG_RING_FULL;
        return;
    }
    const real *z = static_cast<const real *>(d.z);
    for (int g = threadIdx.x; g < d.n_gauges; g += blockDim.x) {
        int32_t c = d.gauge_cells[g];
        d.ring_eta[rec * d.n_gauges + g] = EtaForm<real>::value ? (double)w[c] : (double)(w[c] + z[c]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        d.ring_t[rec] = sc->t;
        sc->n_rec = rec + 1;
    }
}

// Moving bed (time-dependent depth of Sec. 2.1, read as a kinematic rupture):
// depth_v(t) = depth0_v - uplift_v R((t - onset_v) / rise), R(s) = min(1, max(0, s))
// (rise = 0: a step at onset), cell bed z_K = -(mean of its vertices' depths) and face
// beds z_f = -(mean of the face's two vertex depths),
// applied with H unchanged.  The products and sums are rounded one by one
// (__dmul_rn / __dadd_rn are never contracted), as written.
__device__ __forceinline__ double bed_ramp(double t, double onset, double rise)
{
    if (rise > 0.0) return fmin(1.0, fmax(0.0, __dsub_rn(t, onset) / rise));
    return t >= onset ? 1.0 : 0.0;
}

template <typename real>
__global__ void bed_update_kernel(DevPtrs d, StepParams p, real *w, int at_step_end, double t_set)
{
    const double t = at_step_end ? d.sc->t + step_dt<real>(d.sc, p.cfl, p.dt_fixed, p.dt_max, p.t_end) : t_set;
    real *z = static_cast<real *>(const_cast<void *>(d.z));
    void *zf = const_cast<void *>(d.zf);
    double *z64 = const_cast<double *>(d.z64);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < d.nc; k += (int64_t)gridDim.x * blockDim.x) {
        double dv[3];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const int32_t v = d.bed_vtx[j * d.nc + k];
            dv[j] = __dsub_rn(d.bed_depth0[v], __dmul_rn(d.bed_uplift[v], bed_ramp(t, d.bed_onset[v], d.bed_rise)));
        }
        const double zn = -(__dadd_rn(__dadd_rn(dv[0], dv[1]), dv[2]) / 3.0);
        // face beds: -(mean of the face's two vertex depths); FP32 keeps z_f - z_K
        // of faces 0 and 1
        double zfn[3];
#pragma unroll
        for (int f = 0; f < 3; f++) zfn[f] = -(__dadd_rn(dv[f], dv[(f + 1) % 3]) / 2.0);
        if (EtaForm<real>::value)
            reinterpret_cast<float2 *>(zf)[k] = make_float2((float)(zfn[0] - zn), (float)(zfn[1] - zn));
        else
            for (int f = 0; f < 3; f++) reinterpret_cast<double *>(zf)[f * d.nc + k] = zfn[f];
        if (EtaForm<real>::value) {
            // eta form: keep H = eta - z; a dry cell (eta == z) stays exactly dry
            const real zo = z[k], zr = (real)zn;
            if (w && zr != zo) {
                const real e = w[k];
                w[k] = e - zo <= real(0) ? zr : (e - zo) + zr;
            }
            z[k] = zr;
            z64[k] = zn;
        } else {
            z[k] = (real)zn;
        }
    }
}

// State in (original order, H) -> internal order, stored form (H, or eta = H + z
// formed with the FP64 bed before rounding to FP32, so still water at a common
// level gets exactly the same eta everywhere).
template <typename real, typename src_t>
__global__ void import_state_kernel(int64_t nc, const int32_t *old_of_new, const src_t *H,
                                    const src_t *Hu, const src_t *Hv, const double *z, real *w, DevScalars *sc)
{
    bool bad = false;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nc; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = old_of_new[k];
        src_t h = H[o], hu = Hu[o], hv = Hv[o];
        if (!(h >= src_t(0)) || !isfinite(h) || !isfinite(hu) || !isfinite(hv)) bad = true;
        w[k] = EtaForm<real>::value ? (real)((double)h + (double)z[k]) : (real)h;
        w[nc + k] = (real)hu;
        w[2 * nc + k] = (real)hv;
    }
    if (bad) atomicOr(&sc->flags, FLAG_BAD_INPUT);
}

// Internal order, stored form -> original order, H.  In the eta form a cell is
// dry when eta <= z in the kernels' own (rounded) bed, and then H is exactly 0.
template <typename real, typename dst_t>
__global__ void export_state_kernel(int64_t nc, const int32_t *old_of_new, const real *w, const real *zr,
                                    const double *z, dst_t *H, dst_t *Hu, dst_t *Hv)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nc; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = old_of_new[k];
        double h = (double)w[k];
        if (EtaForm<real>::value) h = (w[k] - zr[k] <= real(0)) ? 0.0 : fmax(0.0, h - z[k]);
        H[o] = (dst_t)h;
        Hu[o] = (dst_t)w[nc + k];
        Hv[o] = (dst_t)w[2 * nc + k];
    }
}

// The same two conversions with one thread per V consecutive ORIGINAL cells o
// (k = new_of_old[o]): the host-order arrays are read or written contiguously,
// 16 bytes per thread and array (V = 4 floats or 2 doubles), so they can be
// pinned host memory that the kernel reads or writes in place over the CPU-GPU
// link (the internal-order side is scattered in HBM instead).  vec = false (a
// host array not 16-byte aligned) takes every cell one at a time.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

template <typename real, typename src_t>
__device__ __forceinline__ void import_one(int64_t nc, int64_t k, src_t h, src_t hu, src_t hv, double zk,
                                           real *w, bool &bad)
{
    if (!(h >= src_t(0)) || !isfinite(h) || !isfinite(hu) || !isfinite(hv)) bad = true;
    w[k] = EtaForm<real>::value ? (real)((double)h + zk) : (real)h;
    w[nc + k] = (real)hu;
    w[2 * nc + k] = (real)hv;
}

// zo: the FP64 bed in the original order (contiguous reads), or null (z[k]).
template <typename real, typename src_t>
__global__ void import_state_orig_kernel(int64_t nc, const int32_t *new_of_old, const src_t *H, const src_t *Hu,
                                         const src_t *Hv, const double *z, const double *zo, real *w,
                                         DevScalars *sc, bool vec)
{
    constexpr int V = 16 / sizeof(src_t);
    using vt = typename Vec16<src_t>::type;
    bool bad = false;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t ng = vec ? nc / V : 0;
    for (int64_t gi = tid; gi < ng; gi += stride) {
        const vt h = reinterpret_cast<const vt *>(H)[gi], hu = reinterpret_cast<const vt *>(Hu)[gi],
                 hv = reinterpret_cast<const vt *>(Hv)[gi];
        const src_t *ph = reinterpret_cast<const src_t *>(&h), *phu = reinterpret_cast<const src_t *>(&hu),
                    *phv = reinterpret_cast<const src_t *>(&hv);
#pragma unroll
        for (int j = 0; j < V; j++) {
            const int64_t o = gi * V + j, k = new_of_old[o];
            import_one<real, src_t>(nc, k, ph[j], phu[j], phv[j],
                                    EtaForm<real>::value ? (zo ? zo[o] : z[k]) : 0.0, w, bad);
        }
    }
    for (int64_t o = ng * V + tid; o < nc; o += stride) {
        const int64_t k = new_of_old[o];
        import_one<real, src_t>(nc, k, H[o], Hu[o], Hv[o], EtaForm<real>::value ? (zo ? zo[o] : z[k]) : 0.0, w,
                                bad);
    }
    if (bad) atomicOr(&sc->flags, FLAG_BAD_INPUT);
}

// H of internal cell k in the destination type (the eta form is dry at eta <= z
// in the kernels' own rounded bed, and then H is exactly 0).
template <typename real, typename dst_t>
__device__ __forceinline__ void export_one(int64_t nc, int64_t k, const real *w, real zrk, double zk, dst_t &h,
                                           dst_t &hu, dst_t &hv)
{
    double x = (double)w[k];
    if (EtaForm<real>::value) x = (w[k] - zrk <= real(0)) ? 0.0 : fmax(0.0, x - zk);
    h = (dst_t)x;
    hu = (dst_t)w[nc + k];
    hv = (dst_t)w[2 * nc + k];
}

// zro / zo: the kernels' bed and the FP64 bed in the original order, or null.
template <typename real, typename dst_t>
__global__ void export_state_orig_kernel(int64_t nc, const int32_t *new_of_old, const real *w, const real *zr,
                                         const double *z, const real *zro, const double *zo, dst_t *H, dst_t *Hu,
                                         dst_t *Hv, bool vec)
{
    constexpr int V = 16 / sizeof(dst_t);
    using vt = typename Vec16<dst_t>::type;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t ng = vec ? nc / V : 0;
    for (int64_t gi = tid; gi < ng; gi += stride) {
        vt h, hu, hv;
        dst_t *ph = reinterpret_cast<dst_t *>(&h), *phu = reinterpret_cast<dst_t *>(&hu),
              *phv = reinterpret_cast<dst_t *>(&hv);
#pragma unroll
        for (int j = 0; j < V; j++) {
            const int64_t o = gi * V + j, k = new_of_old[o];
            real zrk = real(0);
            double zk = 0.0;
            if (EtaForm<real>::value) { zrk = zro ? zro[o] : zr[k]; zk = zo ? zo[o] : z[k]; }
            export_one<real, dst_t>(nc, k, w, zrk, zk, ph[j], phu[j], phv[j]);
        }
        reinterpret_cast<vt *>(H)[gi] = h;
        reinterpret_cast<vt *>(Hu)[gi] = hu;
        reinterpret_cast<vt *>(Hv)[gi] = hv;
    }
    for (int64_t o = ng * V + tid; o < nc; o += stride) {
        const int64_t k = new_of_old[o];
        real zrk = real(0);
        double zk = 0.0;
        if (EtaForm<real>::value) { zrk = zro ? zro[o] : zr[k]; zk = zo ? zo[o] : z[k]; }
        export_one<real, dst_t>(nc, k, w, zrk, zk, H[o], Hu[o], Hv[o]);
    }
}

constexpr int DIAG_BLOCKS = 1024;

// Fixed grid, fixed reduction tree: the sums do not depend on timing.
template <typename real>
__global__ void diag_partial_kernel(int64_t nc, const real *w, const double *z, const real *geo, double hthr,
                                    double *part)
{
    __shared__ double s_mass[256], s_min[256], s_dry[256];
    double mass = 0.0, mn = CUDART_INF, dry = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nc; k += (int64_t)gridDim.x * blockDim.x) {
        double h = (double)w[k];
        if (EtaForm<real>::value) h = h - z[k];
        double area = EtaForm<real>::value ? (double)geo[(size_t)k * G32 + G32_AREA] : (double)geo[GEO_AREA * nc + k];
        mass += area * h;
        mn = fmin(mn, h);
        dry += h <= hthr ? 1.0 : 0.0;
    }
    s_mass[threadIdx.x] = mass; s_min[threadIdx.x] = mn; s_dry[threadIdx.x] = dry;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_mass[threadIdx.x] += s_mass[threadIdx.x + o];
            s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
            s_dry[threadIdx.x] += s_dry[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = s_mass[0];
        part[3 * blockIdx.x + 1] = s_min[0];
        part[3 * blockIdx.x + 2] = s_dry[0];
    }
}

__global__ void diag_final_kernel(const double *part, int n, double *out)
{
    if (threadIdx.x == 0) {
        double mass = 0.0, mn = CUDART_INF, dry = 0.0;
        for (int i = 0; i < n; i++) {
            mass += part[3 * i];
            mn = fmin(mn, part[3 * i + 1]);
            dry += part[3 * i + 2];
        }
        out[0] = mass; out[1] = mn; out[2] = dry;
    }
}

int grid_for(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 4096); }

}  // namespace

int launch_post_step(const DevPtrs &d, const StepParams &p, const void *w, int precision, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 64) post_step_kernel<double><<<1, 128, 0, s>>>(d, p, static_cast<const double *>(w));
    else post_step_kernel<float><<<1, 128, 0, s>>>(d, p, static_cast<const float *>(w));
    return (int)cudaGetLastError();
}

int launch_bed_update(const DevPtrs &d, const StepParams &p, void *w, int precision, bool at_step_end,
                      double t_set, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = grid_for(d.nc);
    if (precision == 64)
        bed_update_kernel<double><<<blocks, 256, 0, s>>>(d, p, static_cast<double *>(w), at_step_end, t_set);
    else
        bed_update_kernel<float><<<blocks, 256, 0, s>>>(d, p, static_cast<float *>(w), at_step_end, t_set);
    return (int)cudaGetLastError();
}

int util_preload()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, (const void *)post_step_kernel<double>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void *)post_step_kernel<float>);
    return (int)e;
}

int launch_record_gauges(const DevPtrs &d, const void *w, int precision, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 64) record_gauges_kernel<double><<<1, 128, 0, s>>>(d, static_cast<const double *>(w));
    else record_gauges_kernel<float><<<1, 128, 0, s>>>(d, static_cast<const float *>(w));
    return (int)cudaGetLastError();
}

int launch_import_state(const DevPtrs &d, const int32_t *old_of_new, const void *H, const void *Hu,
                        const void *Hv, int src_is_double, void *w, int precision, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int grid = grid_for(d.nc);
    if (precision == 64) {
        const double *z = d.z64;
        if (src_is_double)
            import_state_kernel<double, double><<<grid, 256, 0, s>>>(d.nc, old_of_new, (const double *)H, (const double *)Hu, (const double *)Hv, z, (double *)w, d.sc);
        else
            import_state_kernel<double, float><<<grid, 256, 0, s>>>(d.nc, old_of_new, (const float *)H, (const float *)Hu, (const float *)Hv, z, (double *)w, d.sc);
    } else {
        const double *z = d.z64;
        if (src_is_double)
            import_state_kernel<float, double><<<grid, 256, 0, s>>>(d.nc, old_of_new, (const double *)H, (const double *)Hu, (const double *)Hv, z, (float *)w, d.sc);
        else
            import_state_kernel<float, float><<<grid, 256, 0, s>>>(d.nc, old_of_new, (const float *)H, (const float *)Hu, (const float *)Hv, z, (float *)w, d.sc);
    }
    return (int)cudaGetLastError();
}

static bool aligned16(const void *a, const void *b, const void *c)
{
    return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(c)) & 15) == 0;
}

int launch_import_state_orig(const DevPtrs &d, const int32_t *new_of_old, const void *H, const void *Hu,
                             const void *Hv, int src_is_double, void *w, int precision, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = grid_for(d.nc);
    const double *z = d.z64, *zo = d.z64_orig;
    const bool vec = aligned16(H, Hu, Hv);
    if (precision == 64) {
        if (src_is_double)
            import_state_orig_kernel<double, double><<<grid, 256, 0, s>>>(d.nc, new_of_old, (const double *)H, (const double *)Hu, (const double *)Hv, z, zo, (double *)w, d.sc, vec);
        else
            import_state_orig_kernel<double, float><<<grid, 256, 0, s>>>(d.nc, new_of_old, (const float *)H, (const float *)Hu, (const float *)Hv, z, zo, (double *)w, d.sc, vec);
    } else {
        if (src_is_double)
            import_state_orig_kernel<float, double><<<grid, 256, 0, s>>>(d.nc, new_of_old, (const double *)H, (const double *)Hu, (const double *)Hv, z, zo, (float *)w, d.sc, vec);
        else
            import_state_orig_kernel<float, float><<<grid, 256, 0, s>>>(d.nc, new_of_old, (const float *)H, (const float *)Hu, (const float *)Hv, z, zo, (float *)w, d.sc, vec);
    }
    return (int)cudaGetLastError();
}

int launch_export_state_orig(const DevPtrs &d, const int32_t *new_of_old, const void *w, int precision, void *H,
                             void *Hu, void *Hv, int dst_is_double, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = grid_for(d.nc);
    const bool vec = aligned16(H, Hu, Hv);
    const double *zo = d.z64_orig;
    if (precision == 64) {
        if (dst_is_double)
            export_state_orig_kernel<double, double><<<grid, 256, 0, s>>>(d.nc, new_of_old, (const double *)w, (const double *)d.z, d.z64, nullptr, zo, (double *)H, (double *)Hu, (double *)Hv, vec);
        else
            export_state_orig_kernel<double, float><<<grid, 256, 0, s>>>(d.nc, new_of_old, (const double *)w, (const double *)d.z, d.z64, nullptr, zo, (float *)H, (float *)Hu, (float *)Hv, vec);
    } else {
        const float *zro = static_cast<const float *>(d.z_orig);
        if (dst_is_double)
            export_state_orig_kernel<float, double><<<grid, 256, 0, s>>>(d.nc, new_of_old, (const float *)w, (const float *)d.z, d.z64, zro, zo, (double *)H, (double *)Hu, (double *)Hv, vec);
        else
            export_state_orig_kernel<float, float><<<grid, 256, 0, s>>>(d.nc, new_of_old, (const float *)w, (const float *)d.z, d.z64, zro, zo, (float *)H, (float *)Hu, (float *)Hv, vec);
    }
    return (int)cudaGetLastError();
}

int launch_export_state(const DevPtrs &d, const int32_t *old_of_new, const void *w, int precision,
                        void *H, void *Hu, void *Hv, int dst_is_double, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int grid = grid_for(d.nc);
    if (precision == 64) {
        const double *z = d.z64;
        if (dst_is_double)
            export_state_kernel<double, double><<<grid, 256, 0, s>>>(d.nc, old_of_new, (const double *)w, (const double *)d.z, z, (double *)H, (double *)Hu, (double *)Hv);
        else
            export_state_kernel<double, float><<<grid, 256, 0, s>>>(d.nc, old_of_new, (const double *)w, (const double *)d.z, z, (float *)H, (float *)Hu, (float *)Hv);
    } else {
        const double *z = d.z64;
        if (dst_is_double)
            export_state_kernel<float, double><<<grid, 256, 0, s>>>(d.nc, old_of_new, (const float *)w, (const float *)d.z, z, (double *)H, (double *)Hu, (double *)Hv);
        else
            export_state_kernel<float, float><<<grid, 256, 0, s>>>(d.nc, old_of_new, (const float *)w, (const float *)d.z, z, (float *)H, (float *)Hu, (float *)Hv);
    }
    return (int)cudaGetLastError();
}

int launch_diagnostics(const DevPtrs &d, const void *w, int precision, double hthr, double *part,
                       double *out, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 64)
        diag_partial_kernel<double><<<DIAG_BLOCKS, 256, 0, s>>>(d.nc, (const double *)w, d.z64, (const double *)d.geo, hthr, part);
    else
        diag_partial_kernel<float><<<DIAG_BLOCKS, 256, 0, s>>>(d.nc, (const float *)w, d.z64, (const float *)d.geo, hthr, part);
    diag_final_kernel<<<1, 32, 0, s>>>(part, DIAG_BLOCKS, out);
    return (int)cudaGetLastError();
}

}  // namespace vg
