// C ABI of the volna_gb library (declared in include/volna_gb.h): contexts,
// device memory, state transfer with the cell permutation, gauges, and the
// step loop (two persistent stage kernels and an epilogue per step, replayed
// from a CUDA graph two steps at a time).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/volna_gb.h"
#include "vg_internal.h"

using namespace vg;

namespace {

constexpr int kRingCap = 2048;       // gauge records held on the device between drains
constexpr int kDiagBlocks = 1024;
constexpr int kKernels = 7;
const char *kKernelNames[kKernels] = {"stage1", "stage2", "post_step", "bed_update",
                                      "rk_update1", "residual_w1", "rk_update2"};

}  // namespace

struct vg_ctx {
    int precision = 64;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    vg_params prm{};
    bool has_mesh = false, has_state = false;
    HostMesh hm;

    // device memory
    void *geo = nullptr, *z = nullptr, *w[2] = {nullptr, nullptr}, *R0 = nullptr;
    void *zf = nullptr;               // face beds (layout: DevPtrs::zf)
    void *rk_w1 = nullptr, *rk_R1 = nullptr;   // [3][nc] each: w1 and R(w1) of the unfused RK stages
    double *z64 = nullptr;
    float *z_orig = nullptr;          // FP32: the bed in the original cell order (state import/export)
    double *z64_orig = nullptr;
    bool zorig_ok = false;            // the two copies match z (false once a moving bed was set)
    int32_t *nbr = nullptr, *halo_ptr = nullptr, *halo_n1 = nullptr, *halo_ids = nullptr, *old_of_new = nullptr;
    int32_t *new_of_old = nullptr, *fq_ptr = nullptr, *adj_faces = nullptr;
    int64_t n_adj_faces = 0;          // built by the first adjoint sweep of a mesh
    uint16_t *nbrl = nullptr, *ring1_nbr = nullptr, *fq = nullptr;
    DevScalars *sc = nullptr;
    int32_t *gauge_cells = nullptr;
    double *ring_t = nullptr, *ring_eta = nullptr;
    double *diag_part = nullptr, *diag_out = nullptr;
    void *staging = nullptr;          // [3][nc] doubles for host transfers
    int64_t dev_bytes = 0;
    int cur = 0;

    int32_t n_gauges = 0;
    std::vector<int32_t> gauge_orig;
    std::vector<double> rec_t, rec_eta;

    // vertex depths of the static bed (mesh upload / vg_set_depth) and the
    // moving bed (vg_set_bed_motion): device copies while it is on
    std::vector<double> depth_v;
    bool bed_on = false;
    int64_t n_open = 0;                 // open or absorbing boundary faces (vg_set_boundary)
    int32_t *bed_vtx = nullptr;
    double *bed_depth0 = nullptr, *bed_uplift = nullptr, *bed_onset = nullptr;
    double bed_rise = 0.0;

    LaunchCfg cfg1{}, cfg2{};
    cudaGraphExec_t graph2 = nullptr;
    bool graph_dirty = true;
    int64_t launches = 0;

    // discrete adjoint: checkpoints of the last vg_adj_forward run
    std::vector<void *> ckpt;
    int64_t adj_n = 0, adj_every = 0;
    double adj_dt = 0.0;                // > 0 fixed step; 0: the CFL steps below
    double adj_cfl = 0.0, adj_dt_max = 0.0;
    std::vector<double> adj_dts;        // each step's dt (the CFL steps of the forward run)
    double adj_t0 = 0.0;                // time of the forward run's first state
    bool adj_bed = false;               // the forward run had a moving bed
    std::vector<double> adj_gU, adj_gOn;   // its uplift / onset gradients (last backward pass)
    int32_t adj_slots = 0;              // > 0: binomial checkpointing with this many state slots
    bool profile = false;
    double prof_ms[kKernels] = {0, 0, 0, 0};
    int64_t prof_n[kKernels] = {0, 0, 0, 0};
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kernel;
    size_t ev_used = 0;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) { if (cudaGetDevice(&prev) != cudaSuccess) prev = -1; cudaSetDevice(dev); }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

int fail(vg_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(vg_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, VG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define VG_CUDA(ctx, call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

int dmalloc(vg_ctx *c, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, VG_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    c->dev_bytes += (int64_t)bytes;
    return VG_OK;
}

template <typename T>
void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void free_adjoint(vg_ctx *c)
{
    for (void *p : c->ckpt) cudaFree(p);
    c->ckpt.clear();
    c->adj_n = 0;
}

void free_mesh(vg_ctx *c)
{
    free_adjoint(c);
    if (c->graph2) { cudaGraphExecDestroy(c->graph2); c->graph2 = nullptr; }
    if (c->z64 == c->z) c->z64 = nullptr;
    dfree(c->geo); dfree(c->z); dfree(c->zf); dfree(c->z64); dfree(c->w[0]); dfree(c->w[1]); dfree(c->R0);
    dfree(c->rk_w1); dfree(c->rk_R1);
    dfree(c->z_orig); dfree(c->z64_orig); c->zorig_ok = false;
    dfree(c->nbr); dfree(c->halo_ptr); dfree(c->halo_n1); dfree(c->halo_ids); dfree(c->ring1_nbr);
    dfree(c->old_of_new); dfree(c->new_of_old); dfree(c->nbrl); dfree(c->fq_ptr); dfree(c->fq);
    dfree(c->adj_faces); c->n_adj_faces = 0;
    dfree(c->gauge_cells); dfree(c->ring_t); dfree(c->ring_eta); dfree(c->staging);
    dfree(c->bed_vtx); dfree(c->bed_depth0); dfree(c->bed_uplift); dfree(c->bed_onset);
    c->bed_on = false;
    c->n_open = 0;
    c->depth_v.clear();
    c->dev_bytes = 0;
    c->has_mesh = c->has_state = false;
    c->n_gauges = 0;
    c->gauge_orig.clear();
    c->rec_t.clear();
    c->rec_eta.clear();
    c->graph_dirty = true;
}

size_t real_size(const vg_ctx *c) { return c->precision == 64 ? 8 : 4; }

DevPtrs dev_ptrs(const vg_ctx *c)
{
    DevPtrs d{};
    d.nc = c->hm.nc;
    d.block = c->hm.block;
    {
        // default: one thread per block cell.  (FP64 with two threads per cell, one
        // CTA of 512 threads per SM, was 5-8 % slower than two CTAs of 256 that
        // take turns at the barriers.)
        const int t = c->prm.block_threads;
        d.threads = (t >= c->hm.block && t <= 2 * c->hm.block && t <= 512) ? t : c->hm.block;
    }
    d.fp64_fast = c->precision == 64 && !c->prm.fp64_literal;
    d.nblocks = c->hm.nblocks;
    d.max_halo = c->hm.max_halo;
    d.max_ring1 = c->hm.max_ring1;
    d.n_gauges = c->n_gauges;
    d.ring_cap = kRingCap;
    d.geo = c->geo;
    d.z = c->z;
    d.zf = c->zf;
    d.z64 = c->z64;
    const bool zo = c->zorig_ok && !c->bed_on;
    d.z_orig = zo ? c->z_orig : nullptr;
    d.z64_orig = zo ? c->z64_orig : nullptr;
    d.bed_vtx = c->bed_vtx;
    d.bed_depth0 = c->bed_depth0;
    d.bed_uplift = c->bed_uplift;
    d.bed_onset = c->bed_onset;
    d.bed_rise = c->bed_rise;
    d.nbr = c->nbr;
    d.nbrl = c->nbrl;
    d.halo_ptr = c->halo_ptr;
    d.halo_n1 = c->halo_n1;
    d.halo_ids = c->halo_ids;
    d.ring1_nbr = c->ring1_nbr;
    d.fq_ptr = c->fq_ptr;
    d.fq = c->fq;
    d.adj_faces = c->adj_faces;
    d.n_adj_faces = c->n_adj_faces;
    d.R0 = c->R0;
    d.sc = c->sc;
    d.gauge_cells = c->gauge_cells;
    d.ring_t = c->ring_t;
    d.ring_eta = c->ring_eta;
    return d;
}

StepParams step_params(const vg_ctx *c)
{
    StepParams p{};
    p.g = c->prm.g;
    p.cfl = c->prm.cfl;
    p.hthr = c->prm.h_threshold;
    p.dt_fixed = c->prm.dt_fixed;
    p.dt_max = c->prm.dt_max;
    p.t_end = c->prm.t_end;
    p.order = c->prm.order;
    p.gauge_every = c->prm.gauge_every;
    p.fp64_fast = c->precision == 64 && !c->prm.fp64_literal;
    return p;
}

// Converts host doubles to the context precision into `dst` (device), via staging.
int upload_real(vg_ctx *c, void *dst, const double *src, size_t n)
{
    if (c->precision == 64) {
        VG_CUDA(c, cudaMemcpy(dst, src, n * 8, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> tmp(n);
        for (size_t i = 0; i < n; i++) tmp[i] = (float)src[i];
        VG_CUDA(c, cudaMemcpy(dst, tmp.data(), n * 4, cudaMemcpyHostToDevice));
    }
    return VG_OK;
}

// FP32: the bed (as the kernels round it, and in FP64) in the original cell
// order, so that the state import / export kernels, one thread per original
// cell, read it contiguously instead of at scattered internal positions.
int upload_bed_orig(vg_ctx *c)
{
    c->zorig_ok = false;
    if (c->precision == 64) return VG_OK;
    const HostMesh &m = c->hm;
    int rc;
    if (!c->z_orig && (rc = dmalloc(c, (void **)&c->z_orig, 4 * m.nc))) return rc;
    if (!c->z64_orig && (rc = dmalloc(c, (void **)&c->z64_orig, 8 * m.nc))) return rc;
    std::vector<double> zo(m.nc);
    std::vector<float> zf(m.nc);
    for (int64_t o = 0; o < m.nc; o++) {
        zo[o] = m.z[m.new_of_old[o]];
        zf[o] = (float)zo[o];             // the rounding of upload_real
    }
    VG_CUDA(c, cudaMemcpy(c->z64_orig, zo.data(), 8 * m.nc, cudaMemcpyHostToDevice));
    VG_CUDA(c, cudaMemcpy(c->z_orig, zf.data(), 4 * m.nc, cudaMemcpyHostToDevice));
    c->zorig_ok = true;
    return VG_OK;
}

// Face beds of the host mesh in the device layout: FP64 [3][nc] as they are;
// FP32 [nc][2] the differences z_f - z_K of faces 0 and 1, formed in FP64.
int upload_face_beds(vg_ctx *c)
{
    const HostMesh &m = c->hm;
    const int64_t n = m.nc;
    int rc;
    if (!c->zf && (rc = dmalloc(c, &c->zf, c->precision == 64 ? 8 * 3 * n : 8 * n))) return rc;
    if (c->precision == 64) {
        VG_CUDA(c, cudaMemcpy(c->zf, m.zf.data(), 8 * 3 * n, cudaMemcpyHostToDevice));
    } else {
        std::vector<float> d(2 * (size_t)n);
        for (int64_t k = 0; k < n; k++)
            for (int f = 0; f < 2; f++) d[2 * k + f] = (float)(m.zf[f * (size_t)n + k] - m.z[k]);
        VG_CUDA(c, cudaMemcpy(c->zf, d.data(), 4 * d.size(), cudaMemcpyHostToDevice));
    }
    return VG_OK;
}

// Block partition arrays (re-uploaded when block_cells changes).
int upload_partition(vg_ctx *c)
{
    const HostMesh &m = c->hm;
    dfree(c->halo_ptr); dfree(c->halo_n1); dfree(c->halo_ids); dfree(c->ring1_nbr); dfree(c->nbrl);
    dfree(c->fq_ptr); dfree(c->fq);
    int rc;
    size_t nh = std::max<size_t>(1, m.halo_ids.size());
    if ((rc = dmalloc(c, (void **)&c->fq_ptr, 4 * (m.nblocks + 1)))) return rc;
    if ((rc = dmalloc(c, (void **)&c->fq, 2 * m.fq.size()))) return rc;
    VG_CUDA(c, cudaMemcpy(c->fq_ptr, m.fq_ptr.data(), 4 * (m.nblocks + 1), cudaMemcpyHostToDevice));
    VG_CUDA(c, cudaMemcpy(c->fq, m.fq.data(), 2 * m.fq.size(), cudaMemcpyHostToDevice));
    if ((rc = dmalloc(c, (void **)&c->nbrl, 2 * 3 * m.nc))) return rc;
    if ((rc = dmalloc(c, (void **)&c->halo_ptr, 4 * (m.nblocks + 1)))) return rc;
    if ((rc = dmalloc(c, (void **)&c->halo_n1, 4 * m.nblocks))) return rc;
    if ((rc = dmalloc(c, (void **)&c->halo_ids, 4 * nh))) return rc;
    if ((rc = dmalloc(c, (void **)&c->ring1_nbr, 2 * 3 * nh))) return rc;
    VG_CUDA(c, cudaMemcpy(c->nbrl, m.nbrl.data(), 2 * 3 * m.nc, cudaMemcpyHostToDevice));
    VG_CUDA(c, cudaMemcpy(c->halo_ptr, m.halo_ptr.data(), 4 * (m.nblocks + 1), cudaMemcpyHostToDevice));
    VG_CUDA(c, cudaMemcpy(c->halo_n1, m.halo_n1.data(), 4 * m.nblocks, cudaMemcpyHostToDevice));
    if (!m.halo_ids.empty()) {
        VG_CUDA(c, cudaMemcpy(c->halo_ids, m.halo_ids.data(), 4 * m.halo_ids.size(), cudaMemcpyHostToDevice));
        VG_CUDA(c, cudaMemcpy(c->ring1_nbr, m.ring1_nbr.data(), 2 * m.ring1_nbr.size(), cudaMemcpyHostToDevice));
    }
    return VG_OK;
}

int upload_mesh_arrays(vg_ctx *c)
{
    const HostMesh &m = c->hm;
    size_t rs = real_size(c);
    int rc;
    if ((rc = dmalloc(c, &c->geo, c->precision == 64 ? 8 * GEO_ROWS * m.nc : 4 * 16 * m.nc))) return rc;
    if ((rc = dmalloc(c, &c->z, rs * m.nc))) return rc;
    if ((rc = dmalloc(c, &c->w[0], rs * 3 * m.nc))) return rc;
    if ((rc = dmalloc(c, &c->w[1], rs * 3 * m.nc))) return rc;
    if ((rc = dmalloc(c, &c->R0, rs * 3 * m.nc))) return rc;
    if ((rc = dmalloc(c, (void **)&c->nbr, 4 * 3 * m.nc))) return rc;
    if ((rc = dmalloc(c, (void **)&c->old_of_new, 4 * m.nc))) return rc;
    if ((rc = dmalloc(c, (void **)&c->new_of_old, 4 * m.nc))) return rc;
    if ((rc = dmalloc(c, (void **)&c->ring_t, 8 * kRingCap))) return rc;
    if (c->precision == 64) {
        if ((rc = upload_real(c, c->geo, m.geo.data(), m.geo.size()))) return rc;
    } else {
        // FP32 record per cell (16 floats): rows 0 and 1 of M_fj = w_j . (x_f - x_K)
        // formed in FP64, the area, face lengths and normals:
        //   M00 M01 M02 M10 | M11 M12 area l0 | nx0 ny0 nx1 ny1 | nx2 ny2 l1 l2
        const int64_t n = m.nc;
        std::vector<float> r(16 * (size_t)n, 0.0f);
        for (int64_t k = 0; k < n; k++) {
            auto G = [&](int row) { return m.geo[(size_t)row * n + k]; };
            float *o = &r[16 * (size_t)k];
            for (int f = 0; f < 2; f++)
                for (int j = 0; j < 3; j++)
                    o[3 * f + j] = (float)(G(GEO_WX + j) * G(GEO_FX + f) + G(GEO_WY + j) * G(GEO_FY + f));
            o[6] = (float)G(GEO_AREA);
            for (int f = 0; f < 3; f++) {
                o[8 + 2 * f] = (float)G(GEO_NX + f);
                o[9 + 2 * f] = (float)G(GEO_NY + f);
                o[f == 0 ? 7 : 13 + f] = (float)G(GEO_LEN + f);
            }
        }
        VG_CUDA(c, cudaMemcpy(c->geo, r.data(), 4 * r.size(), cudaMemcpyHostToDevice));
    }
    if ((rc = upload_real(c, c->z, m.z.data(), m.z.size()))) return rc;
    if ((rc = upload_face_beds(c))) return rc;
    if (c->precision == 64) {
        c->z64 = static_cast<double *>(c->z);
    } else {
        if ((rc = dmalloc(c, (void **)&c->z64, 8 * m.nc))) return rc;
        VG_CUDA(c, cudaMemcpy(c->z64, m.z.data(), 8 * m.nc, cudaMemcpyHostToDevice));
    }
    if ((rc = upload_bed_orig(c))) return rc;
    VG_CUDA(c, cudaMemcpy(c->nbr, m.nbr.data(), 4 * 3 * m.nc, cudaMemcpyHostToDevice));
    VG_CUDA(c, cudaMemcpy(c->old_of_new, m.old_of_new.data(), 4 * m.nc, cudaMemcpyHostToDevice));
    VG_CUDA(c, cudaMemcpy(c->new_of_old, m.new_of_old.data(), 4 * m.nc, cudaMemcpyHostToDevice));
    return upload_partition(c);
}

size_t stage_smem(const vg_ctx *c, int block, int max_halo, int max_ring1)
{
    return c->precision == 64 ? stage_smem_f64(block, max_halo, max_ring1)
                              : stage_smem_f32(block, max_halo, max_ring1);
}

// Halve the block size until the stage kernels' shared memory (block + two-ring
// halo) fits the device; scattered meshes without renumbering have halos of
// about nine times the block.
int fit_blocks(vg_ctx *c)
{
    int limit = 0;
    VG_CUDA(c, cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    while (stage_smem(c, c->hm.block, c->hm.max_halo, c->hm.max_ring1) > (size_t)limit) {
        if (c->hm.block <= 32)
            return fail(c, VG_EINVAL, "mesh blocks need more shared memory than the device has; renumber the mesh");
        int rc = partition_blocks(c->hm, c->hm.block / 2, c->err);
        if (rc) return rc;
    }
    return VG_OK;
}

int configure_launch(vg_ctx *c)
{
    DevPtrs d = dev_ptrs(c);
    int e = c->precision == 64 ? stage_config_f64(d, 1, c->cfg1) : stage_config_f32(d, 1, c->cfg1);
    if (e) return cuda_fail(c, (cudaError_t)e, "stage 1 launch configuration");
    e = c->precision == 64 ? stage_config_f64(d, 2, c->cfg2) : stage_config_f32(d, 2, c->cfg2);
    if (e) return cuda_fail(c, (cudaError_t)e, "stage 2 launch configuration");
    return VG_OK;
}

void reset_scalars_host(vg_ctx *c, DevScalars &s, double t)
{
    std::memset(&s, 0, sizeof(s));
    s.t = t;
    if (c->precision == 64) {
        double inf = INFINITY;
        std::memcpy(&s.dtmin_bits, &inf, 8);
    } else {
        float inf = INFINITY;
        uint32_t b;
        std::memcpy(&b, &inf, 4);
        s.dtmin_bits = b;
    }
}

int ev_begin(vg_ctx *c, int kernel)
{
    if (!c->profile) return VG_OK;
    if (c->ev_used + 2 > c->ev.size()) {
        for (int k = 0; k < 64; k++) {
            cudaEvent_t e;
            VG_CUDA(c, cudaEventCreate(&e));
            c->ev.push_back(e);
        }
        c->ev_kernel.resize(c->ev.size() / 2 + 1);
    }
    c->ev_kernel[c->ev_used / 2] = kernel;
    VG_CUDA(c, cudaEventRecord(c->ev[c->ev_used], c->stream));
    return VG_OK;
}

int ev_end(vg_ctx *c)
{
    if (!c->profile) return VG_OK;
    VG_CUDA(c, cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
    c->ev_used += 2;
    return VG_OK;
}

int ev_collect(vg_ctx *c)
{
    if (!c->profile) return VG_OK;
    for (size_t i = 0; i < c->ev_used; i += 2) {
        float ms = 0;
        VG_CUDA(c, cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
        int k = c->ev_kernel[i / 2];
        c->prof_ms[k] += ms;
        c->prof_n[k] += 1;
    }
    c->ev_used = 0;
    return VG_OK;
}

// Kernels one step launches.
int step_kernels(const vg_ctx *c) { return (c->bed_on ? 4 : 3) + (c->prm.rk_unfused ? 2 : 0); }

// Queue one step reading w[src] and writing w[1 - src].
int enqueue_step(vg_ctx *c, int src)
{
    DevPtrs d = dev_ptrs(c);
    StepParams p = step_params(c);
    void *s = (void *)c->stream;
    const void *win = c->w[src];
    void *wout = c->w[1 - src];
    int e, rc;
    if ((rc = ev_begin(c, 0))) return rc;
    e = c->precision == 64 ? launch_stage1_f64(d, p, win, c->cfg1, s) : launch_stage1_f32(d, p, win, c->cfg1, s);
    if (e) return cuda_fail(c, (cudaError_t)e, "stage 1 launch");
    if ((rc = ev_end(c))) return rc;
    if (c->prm.rk_unfused) {
        // the stage updates as kernels of their own (w1 and R(w1) through memory)
        for (int part = 0; part < 3; part++) {
            if ((rc = ev_begin(c, 4 + part))) return rc;
            e = c->precision == 64 ? launch_rk_unfused_f64(d, p, part, win, wout, c->rk_w1, c->rk_R1, c->cfg1, s)
                                   : launch_rk_unfused_f32(d, p, part, win, wout, c->rk_w1, c->rk_R1, c->cfg1, s);
            if (e) return cuda_fail(c, (cudaError_t)e, "unfused RK stage launch");
            if ((rc = ev_end(c))) return rc;
        }
    } else {
        if ((rc = ev_begin(c, 1))) return rc;
        e = c->precision == 64 ? launch_stage2_f64(d, p, win, wout, c->cfg2, s)
                               : launch_stage2_f32(d, p, win, wout, c->cfg2, s);
        if (e) return cuda_fail(c, (cudaError_t)e, "stage 2 launch");
        if ((rc = ev_end(c))) return rc;
    }
    if (c->bed_on) {
        // the bed of the step's end time, with H kept, before the gauges record
        if ((rc = ev_begin(c, 3))) return rc;
        e = launch_bed_update(d, p, wout, c->precision, true, 0.0, s);
        if (e) return cuda_fail(c, (cudaError_t)e, "bed update launch");
        if ((rc = ev_end(c))) return rc;
    }
    if ((rc = ev_begin(c, 2))) return rc;
    e = launch_post_step(d, p, wout, c->precision, s);
    if (e) return cuda_fail(c, (cudaError_t)e, "post-step launch");
    if ((rc = ev_end(c))) return rc;
    return VG_OK;
}

int build_graph(vg_ctx *c)
{
    if (c->graph2) { cudaGraphExecDestroy(c->graph2); c->graph2 = nullptr; }
    bool prof = c->profile;
    c->profile = false;
    cudaGraph_t g = nullptr;
    VG_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(c, 0);
    if (!rc) rc = enqueue_step(c, 1);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->profile = prof;
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph2, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    c->graph_dirty = false;
    return VG_OK;
}

int read_scalars(vg_ctx *c, DevScalars &s)
{
    VG_CUDA(c, cudaMemcpyAsync(&s, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(c, cudaStreamSynchronize(c->stream));
    return VG_OK;
}

// Move the device gauge records to the host and empty the device ring.
int drain_gauges(vg_ctx *c, DevScalars &s)
{
    if (c->n_gauges > 0 && s.n_rec > 0) {
        size_t n = (size_t)s.n_rec, G = (size_t)c->n_gauges;
        size_t t0 = c->rec_t.size();
        c->rec_t.resize(t0 + n);
        c->rec_eta.resize((t0 + n) * G);
        VG_CUDA(c, cudaMemcpyAsync(c->rec_t.data() + t0, c->ring_t, n * 8, cudaMemcpyDeviceToHost, c->stream));
        VG_CUDA(c, cudaMemcpyAsync(c->rec_eta.data() + t0 * G, c->ring_eta, n * G * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    static const long long zero = 0;
    VG_CUDA(c, cudaMemcpyAsync(&c->sc->n_rec, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream));
    VG_CUDA(c, cudaStreamSynchronize(c->stream));
    s.n_rec = 0;
    return VG_OK;
}

int check_flags(vg_ctx *c, const DevScalars &s, int64_t neg_before)
{
    if (s.flags & FLAG_NONFINITE_STATE) return fail(c, VG_ENONFINITE, "a non-finite value appeared in the state");
    if (s.flags & FLAG_NONFINITE_DT) return fail(c, VG_ENONFINITE, "the time step is not finite");
    if (s.flags & FLAG_RING_FULL) return fail(c, VG_ESTATE, "gauge ring overflow");
    if (c->prm.strict_positivity && s.neg_count > neg_before)
        return fail(c, VG_ENEGDEPTH, "a stage produced a negative depth (" + std::to_string(s.neg_count - neg_before) + " cells)");
    return VG_OK;
}

int validate_params(const vg_params *p, std::string &why)
{
    if (!(p->g > 0) || !std::isfinite(p->g)) { why = "g must be > 0"; return VG_EINVAL; }
    if (!(p->cfl > 0) || !std::isfinite(p->cfl)) { why = "cfl must be > 0"; return VG_EINVAL; }
    if (!(p->h_threshold >= 0) || !std::isfinite(p->h_threshold)) { why = "h_threshold must be >= 0"; return VG_EINVAL; }
    if (!(p->dt_fixed >= 0) || !(p->dt_max >= 0) || !(p->t_end >= 0)) { why = "dt_fixed, dt_max, t_end must be >= 0"; return VG_EINVAL; }
    if (p->order != 1 && p->order != 2) { why = "order must be 1 or 2"; return VG_EINVAL; }
    if (p->gauge_every < 1) { why = "gauge_every must be >= 1"; return VG_EINVAL; }
    if (p->block_cells != 0 && (p->block_cells < 32 || p->block_cells > 512 || p->block_cells % 32)) {
        why = "block_cells must be 0 or a multiple of 32 in [32, 512]";
        return VG_EINVAL;
    }
    int bc = p->block_cells ? p->block_cells : 256;
    if (p->block_threads != 0 && (p->block_threads % 32 || p->block_threads < bc || p->block_threads > 2 * bc ||
                                  p->block_threads > 512)) {
        why = "block_threads must be 0 or a multiple of 32 from block_cells to min(2 block_cells, 512)";
        return VG_EINVAL;
    }
    if (p->fp64_literal != 0 && p->fp64_literal != 1) { why = "fp64_literal must be 0 or 1"; return VG_EINVAL; }
    if (p->rk_unfused != 0 && p->rk_unfused != 1) { why = "rk_unfused must be 0 or 1"; return VG_EINVAL; }
    return VG_OK;
}

// The unfused RK stages' w1 and R(w1), allocated once a context with a mesh asks
// for them (never during a step, which a CUDA graph may be capturing).
int ensure_rk_buffers(vg_ctx *c)
{
    if (!c->has_mesh || !c->prm.rk_unfused) return VG_OK;
    const size_t bytes = 3 * (size_t)c->hm.nc * real_size(c);
    int rc;
    if (!c->rk_w1 && (rc = dmalloc(c, &c->rk_w1, bytes))) return rc;
    if (!c->rk_R1 && (rc = dmalloc(c, &c->rk_R1, bytes))) return rc;
    return VG_OK;
}

int record_now(vg_ctx *c)
{
    if (c->n_gauges <= 0 || !c->has_state) return VG_OK;
    int e = launch_record_gauges(dev_ptrs(c), c->w[c->cur], c->precision, (void *)c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e, "gauge record launch");
    c->launches++;
    return VG_OK;
}

}  // namespace

namespace vg {

// Accessors used by the batched ensemble (batch.cpp).
DevPtrs ctx_dev_ptrs(vg_ctx *c) { return dev_ptrs(c); }
StepParams ctx_step_params(vg_ctx *c) { return step_params(c); }
const HostMesh &ctx_host_mesh(vg_ctx *c) { return c->hm; }
const int32_t *ctx_old_of_new(vg_ctx *c) { return c->old_of_new; }
int ctx_staging(vg_ctx *c, double **staging)
{
    if (!c->staging) {
        int rc = dmalloc(c, &c->staging, 8 * 3 * c->hm.nc);
        if (rc) return rc;
    }
    *staging = static_cast<double *>(c->staging);
    return VG_OK;
}

}  // namespace vg

extern "C" {

int vg_version(void) { return 10000; }

const char *vg_strerror(int code)
{
    switch (code) {
    case VG_OK: return "ok";
    case VG_EINVAL: return "invalid argument";
    case VG_ENOMEM: return "out of memory";
    case VG_ECUDA: return "CUDA error";
    case VG_ENONFINITE: return "non-finite state or time step";
    case VG_ENEGDEPTH: return "negative depth";
    case VG_ETIMEOUT: return "device wait timed out";
    case VG_ESTATE: return "call out of order";
    default: return "unknown status";
    }
}

int vg_default_params(vg_params *p)
{
    if (!p) return VG_EINVAL;
    p->g = 9.81;
    p->cfl = 0.9;
    p->h_threshold = 1e-5;
    p->dt_fixed = 0.0;
    p->dt_max = 0.0;
    p->t_end = 0.0;
    p->order = 2;
    p->gauge_every = 1;
    p->strict_positivity = 0;
    p->block_cells = 0;
    p->block_threads = 0;
    p->fp64_literal = 1;
    p->rk_unfused = 0;
    return VG_OK;
}

int vg_create(vg_ctx **out, int precision, int device, void *cuda_stream)
{
    if (!out) return VG_EINVAL;
    *out = nullptr;
    if (precision != 32 && precision != 64) return VG_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return VG_ECUDA;
    }
    vg_ctx *c = new (std::nothrow) vg_ctx();
    if (!c) return VG_ENOMEM;
    c->precision = precision;
    c->device = device;
    vg_default_params(&c->prm);
    DeviceGuard guard(device);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return VG_ECUDA; }
        c->own_stream = true;
    }
    if (cudaMalloc((void **)&c->sc, sizeof(DevScalars)) != cudaSuccess ||
        cudaMalloc((void **)&c->diag_part, 8 * 3 * kDiagBlocks) != cudaSuccess ||
        cudaMalloc((void **)&c->diag_out, 8 * 4) != cudaSuccess) {
        vg_destroy(c);
        return VG_ENOMEM;
    }
    DevScalars s;
    reset_scalars_host(c, s, 0.0);
    if (cudaMemcpy(c->sc, &s, sizeof(s), cudaMemcpyHostToDevice) != cudaSuccess) { vg_destroy(c); return VG_ECUDA; }
    *out = c;
    return VG_OK;
}

void vg_destroy(vg_ctx *c)
{
    if (!c) return;
    DeviceGuard guard(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_mesh(c);
    dfree(c->sc);
    dfree(c->diag_part);
    dfree(c->diag_out);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *vg_last_error(vg_ctx *c) { return c ? c->err.c_str() : "NULL context"; }

int vg_mesh_upload(vg_ctx *c, int64_t nv, const double *xy, int64_t nc, const int32_t *tri,
                   const double *depth_v, int renumber)
{
    if (!c) return VG_EINVAL;
    DeviceGuard guard(c->device);
    cudaStreamSynchronize(c->stream);
    free_mesh(c);
    int block = c->prm.block_cells ? c->prm.block_cells : 256;
    int rc = prepare_mesh(nv, xy, nc, tri, depth_v, renumber, block, c->hm, c->err);
    if (rc) return rc;
    if ((rc = fit_blocks(c))) return rc;
    if ((rc = upload_mesh_arrays(c))) { free_mesh(c); return rc; }
    if ((rc = configure_launch(c))) { free_mesh(c); return rc; }
    {
        // the no-allocation step's scratch and kernels are resolved here, so that
        // vg_step_noalloc itself loads and allocates nothing
        int e = noalloc_prepare(c->device);
        if (!e) e = util_preload();
        if (e) { free_mesh(c); return cuda_fail(c, (cudaError_t)e, "no-allocation step set-up"); }
    }
    c->depth_v.assign(depth_v, depth_v + nv);
    c->has_mesh = true;
    c->has_state = false;
    c->cur = 0;
    int rc_rk = ensure_rk_buffers(c);
    if (rc_rk) { free_mesh(c); return rc_rk; }
    return VG_OK;
}

int vg_get_permutation(vg_ctx *c, int32_t *new_of_old)
{
    if (!c || !new_of_old) return VG_EINVAL;
    if (!c->has_mesh) return fail(c, VG_ESTATE, "no mesh");
    std::memcpy(new_of_old, c->hm.new_of_old.data(), 4 * c->hm.nc);
    return VG_OK;
}

int vg_get_flipped(vg_ctx *c, int64_t *n)
{
    if (!c || !n) return VG_EINVAL;
    if (!c->has_mesh) return fail(c, VG_ESTATE, "no mesh");
    *n = c->hm.n_flipped;
    return VG_OK;
}

int vg_set_params(vg_ctx *c, const vg_params *p)
{
    if (!c || !p) return VG_EINVAL;
    std::string why;
    if (validate_params(p, why)) return fail(c, VG_EINVAL, why);
    DeviceGuard guard(c->device);
    int old_block = c->prm.block_cells ? c->prm.block_cells : 256;
    int new_block = p->block_cells ? p->block_cells : 256;
    bool threads_changed = p->block_threads != c->prm.block_threads || p->fp64_literal != c->prm.fp64_literal;
    c->prm = *p;
    c->graph_dirty = true;
    if (c->has_mesh && threads_changed && new_block == old_block) {
        cudaStreamSynchronize(c->stream);
        int rc = configure_launch(c);
        if (rc) return rc;
    }
    if (c->has_mesh && new_block != old_block) {
        cudaStreamSynchronize(c->stream);
        int rc = partition_blocks(c->hm, new_block, c->err);
        if (rc) return rc;
        if ((rc = fit_blocks(c))) return rc;
        if ((rc = upload_partition(c))) return rc;
        if ((rc = configure_launch(c))) return rc;
    }
    return ensure_rk_buffers(c);
}

int vg_get_params(vg_ctx *c, vg_params *p)
{
    if (!c || !p) return VG_EINVAL;
    *p = c->prm;
    return VG_OK;
}

// The device address of a host buffer the kernels may read or write in place
// (pinned, mapped host memory), or NULL (pageable memory: copy through staging).
static const void *mapped_view(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Stores a state given in the original cell order.  host_order: one thread per
// original cell, so the source may be pinned host memory read in place over the
// CPU-GPU link; otherwise one thread per internal cell gathers from device arrays.
static int set_state_impl(vg_ctx *c, const void *H, const void *Hu, const void *Hv, bool src_double, bool host_order,
                          double t)
{
    DevScalars s;
    reset_scalars_host(c, s, t);
    VG_CUDA(c, cudaMemcpyAsync(c->sc, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream));
    c->cur = 0;
    if (c->bed_on) {
        // the moving bed at the state's time, before the state is stored over it
        int e = launch_bed_update(dev_ptrs(c), step_params(c), nullptr, c->precision, false, t, (void *)c->stream);
        if (e) return cuda_fail(c, (cudaError_t)e, "bed update launch");
        c->launches++;
    }
    int e = host_order ? launch_import_state_orig(dev_ptrs(c), c->new_of_old, H, Hu, Hv, src_double, c->w[0],
                                                  c->precision, (void *)c->stream)
                       : launch_import_state(dev_ptrs(c), c->old_of_new, H, Hu, Hv, src_double, c->w[0], c->precision,
                                             (void *)c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e, "state import launch");
    c->launches++;
    DevScalars r;
    int rc = read_scalars(c, r);
    if (rc) return rc;
    if (r.flags & FLAG_BAD_INPUT) {
        c->has_state = false;
        return fail(c, VG_EINVAL, "state has a negative or non-finite depth, or non-finite momentum");
    }
    c->has_state = true;
    c->rec_t.clear();
    c->rec_eta.clear();
    if ((rc = record_now(c))) return rc;
    return VG_OK;
}

// Host arrays of FP64 (dbl) or FP32 values.  Pinned buffers are read in place by
// the import kernel (contiguous over the link, scattered stores in HBM; a DMA to
// a staging buffer followed by a gather per internal cell measured slower for
// FP32 at 40M cells in random order: scattered 4-byte reads miss L2, while the
// scattered stores merge there); pageable ones go through a device staging copy.
static int set_state_host(vg_ctx *c, const void *H, const void *Hu, const void *Hv, bool dbl, double t)
{
    if (!c || !H || !Hu || !Hv) return VG_EINVAL;
    if (!c->has_mesh) return fail(c, VG_ESTATE, "no mesh");
    if (!std::isfinite(t)) return fail(c, VG_EINVAL, "t must be finite");
    DeviceGuard guard(c->device);
    const int64_t nc = c->hm.nc;
    const size_t bytes = (dbl ? 8 : 4) * (size_t)nc;
    int rc;
    const void *mH = mapped_view(H), *mHu = mapped_view(Hu), *mHv = mapped_view(Hv);
    if (mH && mHu && mHv) return set_state_impl(c, mH, mHu, mHv, dbl, true, t);
    if (!c->staging && (rc = dmalloc(c, &c->staging, 8 * 3 * nc))) return rc;
    char *st = static_cast<char *>(c->staging);
    VG_CUDA(c, cudaMemcpyAsync(st, H, bytes, cudaMemcpyHostToDevice, c->stream));
    VG_CUDA(c, cudaMemcpyAsync(st + bytes, Hu, bytes, cudaMemcpyHostToDevice, c->stream));
    VG_CUDA(c, cudaMemcpyAsync(st + 2 * bytes, Hv, bytes, cudaMemcpyHostToDevice, c->stream));
    return set_state_impl(c, st, st + bytes, st + 2 * bytes, dbl, false, t);
}

int vg_set_state(vg_ctx *c, const double *H, const double *Hu, const double *Hv, double t)
{
    return set_state_host(c, H, Hu, Hv, true, t);
}

int vg_set_state_f32(vg_ctx *c, const float *H, const float *Hu, const float *Hv, double t)
{
    return set_state_host(c, H, Hu, Hv, false, t);
}

int vg_set_state_dev(vg_ctx *c, const void *H, const void *Hu, const void *Hv, double t)
{
    if (!c || !H || !Hu || !Hv) return VG_EINVAL;
    if (!c->has_mesh) return fail(c, VG_ESTATE, "no mesh");
    if (!std::isfinite(t)) return fail(c, VG_EINVAL, "t must be finite");
    DeviceGuard guard(c->device);
    return set_state_impl(c, H, Hu, Hv, c->precision == 64, false, t);
}

// Host arrays of FP64 (dbl) or FP32 values.  Pinned buffers are written in place
// by the export kernel; pageable ones go through a device staging copy.
static int get_state_host(vg_ctx *c, void *H, void *Hu, void *Hv, bool dbl, double *t)
{
    if (!c || !H || !Hu || !Hv) return VG_EINVAL;
    if (!c->has_state) return fail(c, VG_ESTATE, "no state");
    DeviceGuard guard(c->device);
    const int64_t nc = c->hm.nc;
    const size_t bytes = (dbl ? 8 : 4) * (size_t)nc;
    int rc;
    void *mH = const_cast<void *>(mapped_view(H)), *mHu = const_cast<void *>(mapped_view(Hu));
    void *mHv = const_cast<void *>(mapped_view(Hv));
    if (mH && mHu && mHv) {
        int e = launch_export_state_orig(dev_ptrs(c), c->new_of_old, c->w[c->cur], c->precision, mH, mHu, mHv, dbl,
                                         (void *)c->stream);
        if (e) return cuda_fail(c, (cudaError_t)e, "state export launch");
        c->launches++;
        DevScalars s;
        if ((rc = read_scalars(c, s))) return rc;     // synchronises the stream
        if (t) *t = s.t;
        return VG_OK;
    }
    if (!c->staging && (rc = dmalloc(c, &c->staging, 8 * 3 * nc))) return rc;
    char *st = static_cast<char *>(c->staging);
    int e = launch_export_state(dev_ptrs(c), c->old_of_new, c->w[c->cur], c->precision, st, st + bytes,
                                st + 2 * bytes, dbl, (void *)c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e, "state export launch");
    c->launches++;
    VG_CUDA(c, cudaMemcpyAsync(H, st, bytes, cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(c, cudaMemcpyAsync(Hu, st + bytes, bytes, cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(c, cudaMemcpyAsync(Hv, st + 2 * bytes, bytes, cudaMemcpyDeviceToHost, c->stream));
    DevScalars s;
    if ((rc = read_scalars(c, s))) return rc;
    if (t) *t = s.t;
    return VG_OK;
}

int vg_get_state(vg_ctx *c, double *H, double *Hu, double *Hv, double *t)
{
    return get_state_host(c, H, Hu, Hv, true, t);
}

int vg_get_state_f32(vg_ctx *c, float *H, float *Hu, float *Hv, double *t)
{
    return get_state_host(c, H, Hu, Hv, false, t);
}

int vg_get_state_dev(vg_ctx *c, void *H, void *Hu, void *Hv)
{
    if (!c || !H || !Hu || !Hv) return VG_EINVAL;
    if (!c->has_state) return fail(c, VG_ESTATE, "no state");
    DeviceGuard guard(c->device);
    int e = launch_export_state(dev_ptrs(c), c->old_of_new, c->w[c->cur], c->precision, H, Hu, Hv,
                                c->precision == 64, (void *)c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e, "state export launch");
    c->launches++;
    VG_CUDA(c, cudaStreamSynchronize(c->stream));
    return VG_OK;
}

int vg_set_gauges(vg_ctx *c, int32_t n, const double *xy)
{
    if (!c || n < 0 || (n > 0 && !xy)) return VG_EINVAL;
    if (!c->has_mesh) return fail(c, VG_ESTATE, "no mesh");
    DeviceGuard guard(c->device);
    std::vector<int32_t> cells(n);
    locate_points(c->hm, n, xy, cells.data());
    for (int32_t k = 0; k < n; k++)
        if (cells[k] < 0) return fail(c, VG_EINVAL, "gauge " + std::to_string(k) + " lies outside the mesh");
    cudaStreamSynchronize(c->stream);
    dfree(c->gauge_cells);
    dfree(c->ring_eta);
    c->n_gauges = 0;
    c->gauge_orig = cells;
    c->rec_t.clear();
    c->rec_eta.clear();
    c->graph_dirty = true;
    if (n == 0) return VG_OK;
    std::vector<int32_t> internal(n);
    for (int32_t k = 0; k < n; k++) internal[k] = c->hm.new_of_old[cells[k]];
    int rc;
    if ((rc = dmalloc(c, (void **)&c->gauge_cells, 4 * n))) return rc;
    if ((rc = dmalloc(c, (void **)&c->ring_eta, 8 * (size_t)n * kRingCap))) return rc;
    VG_CUDA(c, cudaMemcpy(c->gauge_cells, internal.data(), 4 * n, cudaMemcpyHostToDevice));
    c->n_gauges = n;
    static const long long zero = 0;
    VG_CUDA(c, cudaMemcpyAsync(&c->sc->n_rec, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream));
    return record_now(c);
}

int vg_get_gauge_cells(vg_ctx *c, int32_t *cells)
{
    if (!c || (!cells && !c->gauge_orig.empty())) return VG_EINVAL;
    std::copy(c->gauge_orig.begin(), c->gauge_orig.end(), cells);
    return VG_OK;
}

int vg_step(vg_ctx *c, int64_t n_steps)
{
    if (!c || n_steps < 0) return VG_EINVAL;
    if (!c->has_mesh || !c->has_state) return fail(c, VG_ESTATE, "mesh and state must be set before stepping");
    DeviceGuard guard(c->device);
    DevScalars s;
    int rc = read_scalars(c, s);
    if (rc) return rc;
    if ((rc = drain_gauges(c, s))) return rc;
    int64_t neg_before = s.neg_count;
    int64_t chunk_max = c->n_gauges > 0 ? (int64_t)(kRingCap - 1) * c->prm.gauge_every : n_steps;
    if (chunk_max < 1) chunk_max = 1;
    while (n_steps > 0) {
        int64_t chunk = std::min(n_steps, chunk_max);
        n_steps -= chunk;
        int64_t left = chunk;
        if (c->profile) {
            while (left > 0) {
                if ((rc = enqueue_step(c, c->cur))) return rc;
                c->cur = 1 - c->cur;
                c->launches += step_kernels(c);
                left--;
            }
        } else {
            if (c->graph_dirty && (rc = build_graph(c))) return rc;
            if (c->cur == 1 && left > 0) {
                if ((rc = enqueue_step(c, 1))) return rc;
                c->cur = 0;
                c->launches += step_kernels(c);
                left--;
            }
            while (left >= 2) {
                VG_CUDA(c, cudaGraphLaunch(c->graph2, c->stream));
                c->launches += 2 * step_kernels(c);
                left -= 2;
            }
            if (left == 1) {
                if ((rc = enqueue_step(c, 0))) return rc;
                c->cur = 1;
                c->launches += step_kernels(c);
            }
        }
        if ((rc = read_scalars(c, s))) return rc;
        if ((rc = ev_collect(c))) return rc;
        if ((rc = drain_gauges(c, s))) return rc;
        if ((rc = check_flags(c, s, neg_before))) return rc;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "vg_step");
    return VG_OK;
}

int vg_advance_to(vg_ctx *c, double t_target)
{
    if (!c || !std::isfinite(t_target)) return VG_EINVAL;
    if (!c->has_mesh || !c->has_state) return fail(c, VG_ESTATE, "mesh and state must be set before stepping");
    vg_params saved = c->prm;
    vg_params p = saved;
    if (!(p.t_end > 0) || p.t_end > t_target) p.t_end = t_target;
    c->prm = p;
    c->graph_dirty = true;
    int rc = VG_OK;
    for (int iter = 0; iter < 1000000; iter++) {
        DevScalars s;
        if ((rc = read_scalars(c, s))) break;
        if (s.t >= p.t_end) break;
        double t_before = s.t;
        if ((rc = vg_step(c, 64))) break;
        if ((rc = read_scalars(c, s))) break;
        if (s.t <= t_before) { rc = fail(c, VG_ESTATE, "time does not advance (zero time step)"); break; }
    }
    c->prm = saved;
    c->graph_dirty = true;
    return rc;
}

int vg_get_gauges(vg_ctx *c, double *t, double *eta, int64_t cap, int64_t *n_rec)
{
    if (!c || cap < 0) return VG_EINVAL;
    DeviceGuard guard(c->device);
    if (c->has_mesh) {
        DevScalars s;
        int rc = read_scalars(c, s);
        if (rc) return rc;
        if ((rc = drain_gauges(c, s))) return rc;
    }
    int64_t n = (int64_t)c->rec_t.size();
    if (n_rec) *n_rec = n;
    int64_t k = std::min(n, cap);
    if (t) std::memcpy(t, c->rec_t.data(), 8 * k);
    if (eta) std::memcpy(eta, c->rec_eta.data(), 8 * k * c->n_gauges);
    return VG_OK;
}

int vg_get_diagnostics(vg_ctx *c, vg_diag *d)
{
    if (!c || !d) return VG_EINVAL;
    std::memset(d, 0, sizeof(*d));
    d->launches = c->launches;
    d->n_records = (int64_t)c->rec_t.size();
    if (!c->has_mesh || !c->has_state) return VG_OK;
    DeviceGuard guard(c->device);
    int e = launch_diagnostics(dev_ptrs(c), c->w[c->cur], c->precision, c->prm.h_threshold, c->diag_part,
                               c->diag_out, (void *)c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e, "diagnostics launch");
    c->launches += 2;
    double out[3];
    VG_CUDA(c, cudaMemcpyAsync(out, c->diag_out, 8 * 3, cudaMemcpyDeviceToHost, c->stream));
    DevScalars s;
    int rc = read_scalars(c, s);
    if (rc) return rc;
    if ((rc = drain_gauges(c, s))) return rc;
    d->t = s.t;
    d->last_dt = s.dt;
    d->mass = out[0];
    d->min_H = out[1];
    d->dry_count = (int64_t)out[2];
    d->steps = s.steps;
    d->neg_count = s.neg_count;
    d->launches = c->launches;
    d->n_records = (int64_t)c->rec_t.size();
    return VG_OK;
}

int vg_profile(vg_ctx *c, int enable)
{
    if (!c) return VG_EINVAL;
    c->profile = enable != 0;
    for (int k = 0; k < kKernels; k++) { c->prof_ms[k] = 0; c->prof_n[k] = 0; }
    c->ev_used = 0;
    return VG_OK;
}

int vg_get_profile(vg_ctx *c, int32_t n, const char **names, int64_t *launches, double *ms, int32_t *n_out)
{
    if (!c || n < 0) return VG_EINVAL;
    for (int k = 0; k < kKernels && k < n; k++) {
        if (names) names[k] = kKernelNames[k];
        if (launches) launches[k] = c->prof_n[k];
        if (ms) ms[k] = c->prof_ms[k];
    }
    if (n_out) *n_out = kKernels;
    return VG_OK;
}

int vg_set_depth(vg_ctx *c, const double *depth_v)
{
    if (!c || !depth_v) return VG_EINVAL;
    if (!c->has_mesh) return fail(c, VG_ESTATE, "no mesh");
    if (c->bed_on)
        return fail(c, VG_ESTATE, "a moving bed is set; remove it (vg_set_bed_motion with uplift NULL) first");
    DeviceGuard guard(c->device);
    HostMesh &m = c->hm;
    for (int64_t v = 0; v < m.nv; v++)
        if (!std::isfinite(depth_v[v])) return fail(c, VG_EINVAL, "non-finite depth");
    std::string err;
    if (bed_arrays(m, depth_v, err)) return fail(c, VG_EINVAL, err);
    cudaStreamSynchronize(c->stream);
    int rc = upload_real(c, c->z, m.z.data(), m.z.size());
    if (rc) return rc;
    if ((rc = upload_face_beds(c))) return rc;
    if (c->precision != 64) VG_CUDA(c, cudaMemcpy(c->z64, m.z.data(), 8 * m.nc, cudaMemcpyHostToDevice));
    if ((rc = upload_bed_orig(c))) return rc;
    c->depth_v.assign(depth_v, depth_v + m.nv);
    c->graph_dirty = true;
    return VG_OK;
}

int vg_set_open_boundary(vg_ctx *c, int64_t n, const int32_t *edges)
{
    return vg_set_boundary(c, n, edges, nullptr);
}

int vg_set_boundary(vg_ctx *c, int64_t n, const int32_t *edges, const int32_t *kinds)
{
    if (!c || n < 0 || (n > 0 && !edges)) return VG_EINVAL;
    for (int64_t e = 0; kinds && e < n; e++)
        if (kinds[e] < VG_BOUNDARY_WALL || kinds[e] > VG_BOUNDARY_ABSORBING)
            return fail(c, VG_EINVAL, "boundary kind " + std::to_string(kinds[e]) + " of edge " + std::to_string(e));
    if (!c->has_mesh) return fail(c, VG_ESTATE, "no mesh");
    DeviceGuard guard(c->device);
    HostMesh &m = c->hm;
    const int64_t nc = m.nc;
    // boundary faces by their (sorted) original vertex pair
    std::unordered_map<uint64_t, int64_t> face_of;
    for (int64_t k = 0; k < nc; k++) {
        const int32_t *v = &m.vtx[3 * (size_t)m.old_of_new[k]];
        for (int f = 0; f < 3; f++) {
            if (m.nbr[f * nc + k] >= 0) continue;
            uint32_t a = (uint32_t)v[f], b = (uint32_t)v[(f + 1) % 3];
            if (a > b) std::swap(a, b);
            face_of[((uint64_t)a << 32) | b] = f * nc + k;
        }
    }
    std::vector<int64_t> open(n);
    for (int64_t e = 0; e < n; e++) {
        uint32_t a = (uint32_t)edges[2 * e], b = (uint32_t)edges[2 * e + 1];
        if (a > b) std::swap(a, b);
        auto it = face_of.find(((uint64_t)a << 32) | b);
        if (it == face_of.end())
            return fail(c, VG_EINVAL, "edge " + std::to_string(e) + " is not a boundary edge of the mesh");
        open[e] = it->second;
    }
    for (auto &kv : face_of) m.nbr[kv.second] = -1;
    int64_t n_open = 0;
    for (int64_t e = 0; e < n; e++) {
        const int kind = kinds ? kinds[e] : VG_BOUNDARY_OPEN;
        m.nbr[open[e]] = -kind;                     // -1 wall, -2 open, -3 absorbing
        n_open += kind != VG_BOUNDARY_WALL;
    }
    VG_CUDA(c, cudaStreamSynchronize(c->stream));
    int rc = partition_blocks(m, m.block, c->err);
    if (rc) return rc;
    if ((rc = upload_partition(c))) return rc;
    VG_CUDA(c, cudaMemcpy(c->nbr, m.nbr.data(), 4 * 3 * (size_t)nc, cudaMemcpyHostToDevice));
    c->n_open = n_open;
    c->graph_dirty = true;
    return VG_OK;
}

int vg_set_bed_motion(vg_ctx *c, const double *uplift_v, const double *onset_v, double rise)
{
    if (!c) return VG_EINVAL;
    if (!c->has_mesh) return fail(c, VG_ESTATE, "no mesh");
    if (uplift_v && (!onset_v || !(rise >= 0.0) || !std::isfinite(rise)))
        return fail(c, VG_EINVAL, "onset times and a finite rise time >= 0 are required");
    DeviceGuard guard(c->device);
    const HostMesh &m = c->hm;
    const int64_t nv = m.nv, nc = m.nc;
    if (uplift_v)
        for (int64_t v = 0; v < nv; v++)
            if (!std::isfinite(uplift_v[v]) || !std::isfinite(onset_v[v]))
                return fail(c, VG_EINVAL, "non-finite uplift or onset at vertex " + std::to_string(v));
    VG_CUDA(c, cudaStreamSynchronize(c->stream));
    DevScalars sc;
    int rc = read_scalars(c, sc);
    if (rc) return rc;
    if (!c->bed_vtx) {
        std::vector<int32_t> bv(3 * (size_t)nc);
        for (int64_t k = 0; k < nc; k++)
            for (int j = 0; j < 3; j++) bv[j * (size_t)nc + k] = m.vtx[3 * (size_t)m.old_of_new[k] + j];
        if ((rc = dmalloc(c, (void **)&c->bed_vtx, 4 * bv.size()))) return rc;
        if ((rc = dmalloc(c, (void **)&c->bed_depth0, 8 * nv))) return rc;
        if ((rc = dmalloc(c, (void **)&c->bed_uplift, 8 * nv))) return rc;
        if ((rc = dmalloc(c, (void **)&c->bed_onset, 8 * nv))) return rc;
        VG_CUDA(c, cudaMemcpy(c->bed_vtx, bv.data(), 4 * bv.size(), cudaMemcpyHostToDevice));
    }
    VG_CUDA(c, cudaMemcpy(c->bed_depth0, c->depth_v.data(), 8 * nv, cudaMemcpyHostToDevice));
    if (uplift_v) {
        VG_CUDA(c, cudaMemcpy(c->bed_uplift, uplift_v, 8 * nv, cudaMemcpyHostToDevice));
        VG_CUDA(c, cudaMemcpy(c->bed_onset, onset_v, 8 * nv, cudaMemcpyHostToDevice));
        c->bed_rise = rise;
    } else {
        // back to the static bed: zero uplift evaluated once, then the motion is off
        VG_CUDA(c, cudaMemset(c->bed_uplift, 0, 8 * nv));
        VG_CUDA(c, cudaMemset(c->bed_onset, 0, 8 * nv));
        c->bed_rise = 0.0;
    }
    // the bed at the current time, keeping the state's total depth
    int e = launch_bed_update(dev_ptrs(c), step_params(c), c->has_state ? c->w[c->cur] : nullptr, c->precision,
                              false, sc.t, (void *)c->stream);
    if (e) return cuda_fail(c, (cudaError_t)e, "bed update launch");
    c->launches++;
    VG_CUDA(c, cudaStreamSynchronize(c->stream));
    c->bed_on = uplift_v != nullptr;
    if (c->bed_on) c->zorig_ok = false;     // the bed will move: import / export read z itself
    if (!c->bed_on) {
        dfree(c->bed_vtx); dfree(c->bed_depth0); dfree(c->bed_uplift); dfree(c->bed_onset);
    }
    c->graph_dirty = true;
    return VG_OK;
}

int vg_adj_forward(vg_ctx *c, int64_t n_steps, double dt, int64_t checkpoint_every)
{
    if (!c || n_steps < 1 || !(dt >= 0) || !std::isfinite(dt) || checkpoint_every < 0) return VG_EINVAL;
    if (c->precision != 64) return fail(c, VG_EINVAL, "the adjoint runs in FP64 contexts");
    if (!c->has_mesh || !c->has_state) return fail(c, VG_ESTATE, "mesh and state must be set");
    if (c->n_gauges < 1) return fail(c, VG_ESTATE, "the adjoint differentiates gauge records: set gauges first");
    DeviceGuard guard(c->device);
    free_adjoint(c);
    // default segment length: the one that minimises device memory, C checkpoints'
    // worth of recordings (per cell: face values of both stages, the segment state,
    // R0, R1 with CFL steps, flag bits) plus n_steps / C checkpoints of 24 bytes
    // each; every segment is recomputed once whatever C is
    const double rec_bytes = 8.0 * (18 + 3 + 3 + (dt > 0.0 ? 0 : 3)) + 3.0 / 8.0, ckpt_bytes = 24.0;
    int64_t C = checkpoint_every ? checkpoint_every
                                 : std::max<int64_t>(1, std::llround(std::sqrt((double)n_steps * ckpt_bytes / rec_bytes)));
    int64_t nck = (n_steps + C - 1) / C;
    size_t bytes = 8 * 3 * (size_t)c->hm.nc;
    for (int64_t k = 0; k < nck; k++) {
        void *p = nullptr;
        int rc = dmalloc(c, &p, bytes);
        if (rc) { free_adjoint(c); return rc; }
        c->ckpt.push_back(p);
    }
    double *dts_dev = nullptr;
    if (dmalloc(c, (void **)&dts_dev, 8 * (size_t)n_steps)) { free_adjoint(c); return VG_ENOMEM; }
    vg_params saved = c->prm;
    const LaunchCfg saved_cfg1 = c->cfg1, saved_cfg2 = c->cfg2;
    c->prm.dt_fixed = dt;               // 0: the CFL rule of every step
    c->prm.t_end = 0.0;
    c->prm.gauge_every = 1;
    c->prm.fp64_literal = 1;            // the adjoint reverses the literal form
    c->prm.rk_unfused = 0;
    c->graph_dirty = true;
    {
        int rc0 = configure_launch(c);
        if (rc0) { c->prm = saved; c->cfg1 = saved_cfg1; c->cfg2 = saved_cfg2; free_adjoint(c); return rc0; }
    }
    // restart the gauge record at the current state
    DevScalars s;
    int rc = read_scalars(c, s);
    const double t0 = s.t;
    if (!rc) rc = drain_gauges(c, s);
    c->rec_t.clear();
    c->rec_eta.clear();
    if (!rc) rc = record_now(c);
    for (int64_t n = 0; n < n_steps && !rc; n++) {
        if (n % C == 0) {
            cudaError_t e = cudaMemcpyAsync(c->ckpt[n / C], c->w[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) { rc = cuda_fail(c, e, "checkpoint copy"); break; }
        }
        if ((rc = enqueue_step(c, c->cur))) break;
        {
            cudaError_t e = cudaMemcpyAsync(dts_dev + n, &c->sc->dt, 8, cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) { rc = cuda_fail(c, e, "time-step record"); break; }
        }
        c->cur = 1 - c->cur;
        c->launches += step_kernels(c);
        if ((n + 1) % 1024 == 0) {
            if ((rc = read_scalars(c, s))) break;
            if ((rc = drain_gauges(c, s))) break;
        }
    }
    if (!rc) rc = read_scalars(c, s);
    if (!rc) rc = drain_gauges(c, s);
    if (!rc) rc = check_flags(c, s, 0);
    c->adj_dts.assign(n_steps, dt);
    if (!rc) {
        cudaError_t e = cudaMemcpy(c->adj_dts.data(), dts_dev, 8 * (size_t)n_steps, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "time-step read-back");
    }
    dfree(dts_dev);
    c->prm = saved;
    c->cfg1 = saved_cfg1;
    c->cfg2 = saved_cfg2;
    c->graph_dirty = true;
    if (rc) { free_adjoint(c); return rc; }
    c->adj_n = n_steps;
    c->adj_every = C;
    c->adj_dt = dt;
    c->adj_cfl = saved.cfl;
    c->adj_dt_max = saved.dt_max;
    c->adj_t0 = t0;
    c->adj_bed = c->bed_on;
    c->adj_gU.clear();
    c->adj_gOn.clear();
    c->adj_slots = 0;
    return VG_OK;
}

int vg_adj_forward_binomial(vg_ctx *c, int64_t n_steps, double dt, int32_t slots)
{
    if (!c || n_steps < 1 || slots < 1 || slots > 4096) return VG_EINVAL;
    int rc = vg_adj_forward(c, n_steps, dt, n_steps);     // keeps the first state only
    if (rc) return rc;
    c->adj_slots = slots;
    return VG_OK;
}

int vg_adj_backward(vg_ctx *c, const double *dJ_deta, double *dJ_dH0, double *dJ_dHu0, double *dJ_dHv0,
                    double *dJ_dz, double *dJ_ddepth)
{
    if (!c || !dJ_deta) return VG_EINVAL;
    if (c->adj_n < 1) return fail(c, VG_ESTATE, "call vg_adj_forward first");
    if (c->adj_bed && !c->bed_on) return fail(c, VG_ESTATE, "the moving bed of the forward run was removed");
    DeviceGuard guard(c->device);
    if (!c->adj_faces) {
        // every face once, owned by its lower-numbered cell (a boundary face by its
        // cell), for the flux VJP's one thread per face
        const HostMesh &hm = c->hm;
        std::vector<int32_t> fl;
        fl.reserve(2 * (size_t)hm.nc + 16);
        for (int64_t k = 0; k < hm.nc; k++)
            for (int f = 0; f < 3; f++) {
                const int32_t j = hm.nbr[f * hm.nc + k];
                if (j < 0 || j > k) fl.push_back((int32_t)((k << 2) | f));
            }
        int32_t *dev = nullptr;
        int e = dmalloc(c, (void **)&dev, 4 * std::max<size_t>(fl.size(), 1));
        if (e) return e;
        cudaError_t ce = cudaMemcpy(dev, fl.data(), 4 * fl.size(), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            c->dev_bytes -= (int64_t)(4 * std::max<size_t>(fl.size(), 1));
            dfree(dev);
            return cuda_fail(c, ce, "face list upload");
        }
        c->adj_faces = dev;                   // kept only once complete
        c->n_adj_faces = (int64_t)fl.size();
    }
    const int64_t N = c->adj_n, C = c->adj_every;
    const int nc = (int)c->hm.nc, G = c->n_gauges;
    const size_t w3 = 3 * (size_t)nc;
    const bool binomial = c->adj_slots > 0;
    const int64_t RC = binomial ? 1 : C;    // steps whose recordings are held at once
    // scratch (freed at the end)
    std::vector<void *> bufs;
    auto alloc = [&](size_t n_doubles, double **p) {
        void *q = nullptr;
        int rc = dmalloc(c, &q, 8 * n_doubles);
        if (!rc) { bufs.push_back(q); *p = static_cast<double *>(q); }
        return rc;
    };
    // seg: the segment's states, R0seg: their stage-1 residuals, m2seg: stage-2
    // dry-fix branches (all recorded by one forward recompute of the segment)
    double *W, *wb, *wbn, *wb1, *zb, *Rb, *w1, *H1pre, *FVb, *zfb, *own, *send, *seg, *R0seg, *wlast, *m2raw;
    double *recraw;  // reconstruction flags of both stages of every recorded step [RC][2][nc] (bytes)
    double *FVseg;   // face values of both stages of every step of the segment [C][2][9][nc]
    const bool adaptive = !(c->adj_dt > 0.0);
    double *R1seg = nullptr, *cflscr = nullptr;   // adaptive steps: stage-2 residuals; dt-bar and reduction scratch
    int rc = 0;
    if ((rc = alloc((size_t)(N + 1) * G, &W)) || (rc = alloc(w3, &wb)) || (rc = alloc(w3, &wbn)) ||
        (rc = alloc(w3, &wb1)) || (rc = alloc(4 * (size_t)nc, &zb)) || (rc = alloc(w3, &Rb)) || (rc = alloc(w3, &wlast)) ||
        (rc = alloc(w3, &w1)) || (rc = alloc(nc, &H1pre)) || (rc = alloc(18 * (size_t)nc * RC, &FVseg)) ||
        (rc = alloc(9 * (size_t)nc, &FVb)) || (rc = alloc(3 * (size_t)nc, &zfb)) || (rc = alloc(7 * (size_t)nc, &own)) ||
        (rc = alloc(12 * (size_t)nc, &send)) ||
        (rc = alloc(w3 * (size_t)(binomial ? 2 + c->adj_slots : C), &seg)) ||
        (rc = alloc(w3 * (size_t)RC, &R0seg)) || (rc = alloc(((size_t)nc * RC + 7) / 8, &m2raw)) ||
        (rc = alloc((2 * (size_t)nc * RC + 7) / 8, &recraw)) ||
        (adaptive && ((rc = alloc(w3 * (size_t)RC, &R1seg)) || (rc = alloc(8 + 3 * (size_t)kAdjCflParts, &cflscr))))) {
        for (void *q : bufs) cudaFree(q);
        return rc;
    }
    // moving bed: each step's own bed adjoint, the uplift / onset gradients, the
    // adjoint of time, and the cells around each vertex (fixed order)
    const bool bed = c->adj_bed;
    const int nv = (int)c->hm.nv;
    if (bed && nc >= (1 << 29)) {
        for (void *q : bufs) cudaFree(q);
        return fail(c, VG_EINVAL, "moving-bed adjoint: at most 2^29 - 1 cells");
    }
    double *zstep = nullptr, *gU = nullptr, *gOn = nullptr, *bedscr = nullptr;
    int32_t *vptr = nullptr, *vcell = nullptr;
    std::vector<double> tn;
    if (bed) {
        if ((rc = alloc(4 * (size_t)nc, &zstep)) || (rc = alloc(nv, &gU)) || (rc = alloc(nv, &gOn)) ||
            (rc = alloc(8 + (size_t)kAdjCflParts, &bedscr))) {
            for (void *q : bufs) cudaFree(q);
            return rc;
        }
        std::vector<int32_t> hp(nv + 1, 0), hc(3 * (size_t)nc);
        for (int k = 0; k < nc; k++)
            for (int j = 0; j < 3; j++) hp[c->hm.vtx[3 * (size_t)c->hm.old_of_new[k] + j] + 1]++;
        for (int v = 0; v < nv; v++) hp[v + 1] += hp[v];
        std::vector<int32_t> fill(hp.begin(), hp.end() - 1);
        for (int k = 0; k < nc; k++)          // internal ids in increasing order per vertex, with the
            for (int j = 0; j < 3; j++)        // vertex's local index: (cell << 2) | j
                hc[fill[c->hm.vtx[3 * (size_t)c->hm.old_of_new[k] + j]]++] = (k << 2) | j;
        double *vp = nullptr, *vc = nullptr;
        if ((rc = alloc(((size_t)nv + 2) / 2, &vp)) || (rc = alloc((3 * (size_t)nc + 1) / 2, &vc))) {
            for (void *q : bufs) cudaFree(q);
            return rc;
        }
        vptr = reinterpret_cast<int32_t *>(vp);
        vcell = reinterpret_cast<int32_t *>(vc);
        VG_CUDA(c, cudaMemcpy(vptr, hp.data(), 4 * hp.size(), cudaMemcpyHostToDevice));
        VG_CUDA(c, cudaMemcpy(vcell, hc.data(), 4 * hc.size(), cudaMemcpyHostToDevice));
        VG_CUDA(c, cudaMemsetAsync(gU, 0, 8 * (size_t)nv, c->stream));
        VG_CUDA(c, cudaMemsetAsync(gOn, 0, 8 * (size_t)nv, c->stream));
        VG_CUDA(c, cudaMemsetAsync(bedscr, 0, 8, c->stream));
        tn.resize(N + 1);
        tn[0] = c->adj_t0;
        for (int64_t n = 0; n < N; n++) tn[n + 1] = tn[n] + c->adj_dts[n];   // as the forward's epilogue
    }
    double *tsum = bed ? bedscr : nullptr, *bedpart = bed ? bedscr + 8 : nullptr;
    double *zacc;                          // where the bed adjoint goes: per step (moving bed) or total
    AdjCfl cfl{};
    double *dtbar = nullptr, *dotpart = nullptr;
    if (adaptive) {
        dtbar = cflscr;
        dotpart = cflscr + 8;
        cfl.orig = c->old_of_new;
        cfl.dtbar = dtbar;
        cfl.cfl = c->adj_cfl;
        cfl.dt_max = c->adj_dt_max;
        cfl.part_b = cflscr + 8 + kAdjCflParts;
        cfl.part_o = reinterpret_cast<int *>(cfl.part_b + kAdjCflParts);
        cfl.part_k = cfl.part_o + kAdjCflParts;
    }
    uint8_t *m2seg = reinterpret_cast<uint8_t *>(m2raw);
    uint8_t *recseg = reinterpret_cast<uint8_t *>(recraw);
    DevScalars *asc = nullptr;
    if ((rc = dmalloc(c, (void **)&asc, sizeof(DevScalars)))) {
        for (void *q : bufs) cudaFree(q);
        return rc;
    }
    bufs.push_back(asc);
    DevScalars s0;
    reset_scalars_host(c, s0, 0.0);
    StepParams p = step_params(c);
    p.dt_fixed = c->adj_dt;
    p.t_end = 0.0;
    p.dt_max = 0.0;
    const double hthr = p.hthr;
    void *st = (void *)c->stream;
    DevPtrs d = dev_ptrs(c);
    d.sc = asc;
    d.n_gauges = 0;
    d.fp64_fast = 0;                       // the literal form, as the forward run
    p.fp64_fast = 0;
    LaunchCfg lc1{}, lc2{};
    {
        int e1 = stage_config_f64(d, 1, lc1);
        if (!e1) e1 = stage_config_f64(d, 2, lc2);
        if (e1) {
            for (void *q : bufs) cudaFree(q);
            return cuda_fail(c, (cudaError_t)e1, "adjoint launch configuration");
        }
    }
#define ADJ_CHECK(call) do { int e_ = (call); if (e_) { rc = cuda_fail(c, (cudaError_t)e_, #call); goto done; } } while (0)
    {
        VG_CUDA(c, cudaMemcpyAsync(asc, &s0, sizeof(s0), cudaMemcpyHostToDevice, c->stream));
        VG_CUDA(c, cudaMemcpyAsync(W, dJ_deta, 8 * (size_t)(N + 1) * G, cudaMemcpyHostToDevice, c->stream));
        VG_CUDA(c, cudaMemsetAsync(wb, 0, 8 * w3, c->stream));
        VG_CUDA(c, cudaMemsetAsync(zb, 0, 8 * 4 * (size_t)nc, c->stream));
        zacc = bed ? zstep : zb;
        if (bed) VG_CUDA(c, cudaMemsetAsync(zstep, 0, 8 * 4 * (size_t)nc, c->stream));
        ADJ_CHECK(adjoint_gauge(G, c->gauge_cells, W + (size_t)N * G, nc, wb, zacc, st));
        if (bed)
            ADJ_CHECK(adjoint_bed_flush(nc, nv, vptr, vcell, zstep, c->bed_uplift, c->bed_onset, c->bed_rise, tn[N],
                                        gU, gOn, zb, tsum, bedpart, st));
        // one forward step n from win to wout, recording into recording slot r what
        // its reversal needs (stage-1 residual, face values of both stages, the
        // stage-2 dry-fix branches, with CFL steps the stage-2 residual)
        auto record_step = [&](int64_t n, const double *win, double *wout, int64_t r) -> int {
            DevPtrs dd = d;
            dd.R0 = R0seg + (size_t)r * w3;
            dd.mask2 = m2seg + (size_t)r * nc;
            dd.fv_out = FVseg + (size_t)r * 18 * nc;
            dd.rec_out = recseg + (size_t)r * 2 * nc;
            StepParams pn = p;
            pn.dt_fixed = c->adj_dts[n];        // the step the forward run took
            int e;
            if (bed && (e = launch_bed_update(d, p, nullptr, 64, false, tn[n], st))) return e;   // bed of step n
            if ((e = launch_stage1_f64(dd, pn, win, lc1, st))) return e;
            dd.fv_out = FVseg + ((size_t)r * 18 + 9) * nc;
            dd.rec_out = recseg + ((size_t)r * 2 + 1) * nc;
            if (adaptive) dd.r1_out = R1seg + (size_t)r * w3;
            return launch_stage2_f64(dd, pn, win, wout, lc2, st);
        };
        // one forward step without recordings (binomial schedule)
        auto advance_step = [&](int64_t n, const double *win, double *wout) -> int {
            DevPtrs dd = d;
            dd.R0 = R0seg;
            StepParams pn = p;
            pn.dt_fixed = c->adj_dts[n];
            int e;
            if (bed && (e = launch_bed_update(d, p, nullptr, 64, false, tn[n], st))) return e;
            if ((e = launch_stage1_f64(dd, pn, win, lc1, st))) return e;
            return launch_stage2_f64(dd, pn, win, wout, lc2, st);
        };
        // the reversal of step n from its state w and its recordings in slot r:
        // wb (adjoint of w^{n+1}) -> wb (adjoint of w^n)
        auto reverse_step = [&](int64_t n, const double *w, int64_t r) -> int {
            const double dtn = c->adj_dts[n];
            const double *R0 = R0seg + (size_t)r * w3;
            int e;
            if (bed) {
                if ((e = launch_bed_update(d, p, nullptr, 64, false, tn[n], st))) return e;     // bed of step n
                if ((e = (int)cudaMemsetAsync(zstep, 0, 8 * 4 * (size_t)nc, c->stream))) return e;
            }
            if ((e = adjoint_stage1(nc, dtn, hthr, w, R0, w1, H1pre, st))) return e;
            if ((e = adjoint_stage2_rev(nc, dtn, m2seg + (size_t)r * nc, wb, wbn, wb1, Rb, st))) return e;
            // dt-bar, stage 2: sum w-bar_pre . R1 / 2 = sum Rb . R1 / dt
            if (adaptive && (e = adjoint_dot((int64_t)w3, Rb, R1seg + (size_t)r * w3, 1.0 / dtn, dtbar, true,
                                             dotpart, st)))
                return e;
            double *FV0 = FVseg + (size_t)r * 18 * nc, *FV1 = FV0 + 9 * (size_t)nc;
            const uint8_t *rec0 = recseg + (size_t)r * 2 * nc, *rec1 = rec0 + nc;
            if ((e = adjoint_residual_vjp(d, p, w1, rec1, Rb, wb1, zacc, FV1, true, FVb, zfb, own, send, st))) return e;
            if ((e = adjoint_stage1_rev(nc, dtn, hthr, H1pre, wb1, wbn, Rb, st))) return e;
            // dt-bar, stage 1: sum w1-bar_pre . R0 = sum Rb . R0 / dt
            if (adaptive && (e = adjoint_dot((int64_t)w3, Rb, R0, 1.0 / dtn, dtbar, false, dotpart, st))) return e;
            // a moving bed: every later bed depends on this dt through the time
            if (adaptive && bed && (e = adjoint_scalar_add(dtbar, tsum, st))) return e;
            if ((e = adjoint_residual_vjp(d, p, w, rec0, Rb, wbn, zacc, FV0, true, FVb, zfb, own, send, st,
                                          adaptive ? &cfl : nullptr)))
                return e;
            if ((e = adjoint_gauge(G, c->gauge_cells, W + (size_t)n * G, nc, wbn, zacc, st))) return e;
            if (bed && (e = adjoint_bed_flush(nc, nv, vptr, vcell, zstep, c->bed_uplift, c->bed_onset, c->bed_rise,
                                              tn[n], gU, gOn, zb, tsum, bedpart, st)))
                return e;
            std::swap(wb, wbn);
            c->launches += (adaptive ? 17 : 11) + (bed ? 6 : 0);
            return 0;
        };
        if (!binomial) {
            // sqrt(N) segments: recompute each segment once from its checkpoint,
            // recording every step, then reverse it
            int64_t nseg = (N + C - 1) / C;
            for (int64_t sg = nseg - 1; sg >= 0; sg--) {
                int64_t a = sg * C, b = std::min(a + C, N);
                VG_CUDA(c, cudaMemcpyAsync(seg, c->ckpt[sg], 8 * w3, cudaMemcpyDeviceToDevice, c->stream));
                for (int64_t n = a; n < b; n++) {
                    double *win = seg + (size_t)(n - a) * w3;
                    double *wout = n + 1 < b ? win + w3 : wlast;
                    ADJ_CHECK(record_step(n, win, wout, n - a));
                }
                for (int64_t n = b - 1; n >= a; n--) ADJ_CHECK(reverse_step(n, seg + (size_t)(n - a) * w3, n - a));
            }
        } else {
            // binomial checkpointing: reverse [l, r) from the state at l with
            // `nfree` free state slots, splitting where the fewest forward steps
            // are recomputed (Griewank's binomial schedule, by dynamic programming
            // for up to 2048 steps, by halving beyond)
            const int S = c->adj_slots;
            double *tmp[2] = {seg, seg + w3};
            std::vector<double *> pool;
            for (int k = 0; k < S; k++) pool.push_back(seg + (size_t)(2 + k) * w3);
            const int64_t TD = std::min<int64_t>(N, 2048);
            std::vector<int64_t> F((size_t)(TD + 1) * (S + 1), 0), M((size_t)(TD + 1) * (S + 1), 1);
            auto at = [&](int64_t t, int sl) -> size_t { return (size_t)t * (S + 1) + sl; };
            for (int64_t t = 2; t <= TD; t++) {
                F[at(t, 0)] = t * (t - 1) / 2;
                for (int sl = 1; sl <= S; sl++) {
                    int64_t best = INT64_MAX, bm = 1;
                    for (int64_t m = 1; m < t; m++) {
                        int64_t cost = m + F[at(t - m, sl - 1)] + F[at(m, sl)];
                        if (cost < best) { best = cost; bm = m; }
                    }
                    F[at(t, sl)] = best;
                    M[at(t, sl)] = bm;
                }
            }
            auto split = [&](int64_t t, int sl) -> int64_t { return t <= TD ? M[at(t, sl)] : t / 2; };
            int err = 0;
            std::function<int(int64_t, int64_t, const double *, int)> rev;
            rev = [&](int64_t l, int64_t r, const double *wl, int nfree) -> int {
                int e;
                if (r - l == 1 || nfree == 0) {
                    // no free slot: recompute from l for each step, last first
                    for (int64_t k = r - 1; k >= l; k--) {
                        const double *cur = wl;
                        for (int64_t j = l; j < k; j++) {
                            double *dst = tmp[(j - l) & 1];
                            if ((e = advance_step(j, cur, dst))) return e;
                            cur = dst;
                        }
                        if ((e = record_step(k, cur, wlast, 0))) return e;
                        if ((e = reverse_step(k, cur, 0))) return e;
                    }
                    return 0;
                }
                const int64_t m = l + split(r - l, nfree);
                double *slot = pool.back();
                pool.pop_back();
                const double *cur = wl;
                for (int64_t j = l; j < m; j++) {
                    double *dst = j + 1 == m ? slot : tmp[(j - l) & 1];
                    if ((e = advance_step(j, cur, dst))) return e;
                    cur = dst;
                }
                e = rev(m, r, slot, nfree - 1);
                pool.push_back(slot);
                if (e) return e;
                return rev(l, m, wl, nfree);
            };
            err = rev(0, N, static_cast<const double *>(c->ckpt[0]), S);
            ADJ_CHECK(err);
        }
        if (bed) {
            // the context keeps the bed of the run's last time; the gradients stay on the host
            ADJ_CHECK(launch_bed_update(d, p, nullptr, 64, false, tn[N], st));
            c->adj_gU.resize(nv);
            c->adj_gOn.resize(nv);
            VG_CUDA(c, cudaMemcpyAsync(c->adj_gU.data(), gU, 8 * (size_t)nv, cudaMemcpyDeviceToHost, c->stream));
            VG_CUDA(c, cudaMemcpyAsync(c->adj_gOn.data(), gOn, 8 * (size_t)nv, cudaMemcpyDeviceToHost, c->stream));
        }
        // internal -> original order on the host
        std::vector<double> h(7 * (size_t)nc);
        VG_CUDA(c, cudaMemcpyAsync(h.data(), wb, 8 * w3, cudaMemcpyDeviceToHost, c->stream));
        VG_CUDA(c, cudaMemcpyAsync(h.data() + w3, zb, 8 * 4 * (size_t)nc, cudaMemcpyDeviceToHost, c->stream));
        VG_CUDA(c, cudaStreamSynchronize(c->stream));
        const std::vector<int32_t> &oon = c->hm.old_of_new;
        std::vector<double> zo(nc), zfo(3 * (size_t)nc);
        for (int k = 0; k < nc; k++) {
            int o = oon[k];
            if (dJ_dH0) dJ_dH0[o] = h[k];
            if (dJ_dHu0) dJ_dHu0[o] = h[nc + k];
            if (dJ_dHv0) dJ_dHv0[o] = h[2 * (size_t)nc + k];
            zo[o] = h[w3 + k];
            for (int f = 0; f < 3; f++) zfo[3 * (size_t)o + f] = h[w3 + (size_t)(1 + f) * nc + k];
        }
        if (dJ_dz) std::copy(zo.begin(), zo.end(), dJ_dz);
        if (dJ_ddepth) {
            // z_K = -(1/3) sum of its vertex depths, z_f = -(1/2) the sum over the
            // face's two vertices (face f joins local vertices f and f + 1)
            std::fill(dJ_ddepth, dJ_ddepth + c->hm.nv, 0.0);
            for (int o = 0; o < nc; o++)
                for (int k = 0; k < 3; k++)
                    dJ_ddepth[c->hm.vtx[3 * (size_t)o + k]] -=
                        zo[o] / 3.0 + (zfo[3 * (size_t)o + k] + zfo[3 * (size_t)o + (k + 2) % 3]) / 2.0;
        }
    }
done:
#undef ADJ_CHECK
    cudaStreamSynchronize(c->stream);
    for (void *q : bufs) cudaFree(q);
    return rc;
}

int vg_adj_bed_gradient(vg_ctx *c, double *dJ_duplift, double *dJ_donset)
{
    if (!c) return VG_EINVAL;
    if (c->adj_gU.empty()) return fail(c, VG_ESTATE, "no vg_adj_backward of a run with a moving bed");
    if (dJ_duplift) std::copy(c->adj_gU.begin(), c->adj_gU.end(), dJ_duplift);
    if (dJ_donset) std::copy(c->adj_gOn.begin(), c->adj_gOn.end(), dJ_donset);
    return VG_OK;
}

int vg_device_bytes(vg_ctx *c, int64_t *bytes)
{
    if (!c || !bytes) return VG_EINVAL;
    *bytes = c->dev_bytes;
    return VG_OK;
}

// One step whose scratch is the library's fixed device array (noalloc.cu):
// the ordinary stage kernels run with R0 and the step scalars pointed there.
int vg_step_noalloc(vg_ctx *c, const void *w_in, void *w_out, double t, double *dt_out)
{
    if (!c) return VG_EINVAL;
    if (!w_in || !w_out || w_in == w_out) return fail(c, VG_EINVAL, "w_in and w_out must be distinct device arrays");
    if (!std::isfinite(t)) return fail(c, VG_EINVAL, "t must be finite");
    if (!c->has_mesh) return fail(c, VG_ESTATE, "no mesh");
    if (c->bed_on)
        return fail(c, VG_ESTATE, "a moving bed is set: vg_step_noalloc steps a static bed (remove the motion first)");
    if (c->hm.nc > VG_NOALLOC_MAX_CELLS)
        return fail(c, VG_EINVAL, "vg_step_noalloc handles at most " + std::to_string(VG_NOALLOC_MAX_CELLS) +
                                      " cells; this mesh has " + std::to_string(c->hm.nc));
    DeviceGuard guard(c->device);
    void *scratch = nullptr;
    size_t bytes = 0;
    int e = noalloc_scratch(c->device, &scratch, &bytes);
    if (e) return cuda_fail(c, (cudaError_t)e, "cudaGetSymbolAddress of the no-allocation scratch");
    DevScalars *sc = static_cast<DevScalars *>(scratch);
    DevPtrs d = dev_ptrs(c);
    d.sc = sc;
    d.R0 = static_cast<unsigned char *>(scratch) + 256;
    d.n_gauges = 0;
    d.gauge_cells = nullptr;
    d.ring_t = nullptr;
    d.ring_eta = nullptr;
    StepParams p = step_params(c);
    void *s = (void *)c->stream;
    if ((e = noalloc_launch_init(sc, t, c->precision, s))) return cuda_fail(c, (cudaError_t)e, "scratch init launch");
    e = c->precision == 64 ? launch_stage1_f64(d, p, w_in, c->cfg1, s) : launch_stage1_f32(d, p, w_in, c->cfg1, s);
    if (e) return cuda_fail(c, (cudaError_t)e, "stage 1 launch");
    e = c->precision == 64 ? launch_stage2_f64(d, p, w_in, w_out, c->cfg2, s)
                           : launch_stage2_f32(d, p, w_in, w_out, c->cfg2, s);
    if (e) return cuda_fail(c, (cudaError_t)e, "stage 2 launch");
    if ((e = launch_post_step(d, p, w_out, c->precision, s))) return cuda_fail(c, (cudaError_t)e, "post-step launch");
    c->launches += 4;
    DevScalars r;
    VG_CUDA(c, cudaMemcpyAsync(&r, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (dt_out) *dt_out = r.dt;
    if (r.flags & FLAG_NONFINITE_STATE) return fail(c, VG_ENONFINITE, "a non-finite value appeared in the state");
    if (r.flags & FLAG_NONFINITE_DT) return fail(c, VG_ENONFINITE, "the time step is not finite");
    if (c->prm.strict_positivity && r.neg_count > 0)
        return fail(c, VG_ENEGDEPTH, "a stage produced a negative depth (" + std::to_string(r.neg_count) + " cells)");
    return VG_OK;
}

}  // extern "C"
