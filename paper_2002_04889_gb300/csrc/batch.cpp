// Batched ensembles (C ABI vg_batch_*): many scenarios on several meshes of
// uneven size, advanced together.  Each mesh is an internal context (mesh
// preparation, renumbering, geometry, partition); the batch owns the state
// slices of all scenarios ([2][S][3][nc] per mesh), their residual scratch, one
// device scalar record per scenario (time, dt, CFL minimum) and a device table
// of the meshes.  One batched step is three launches -- stage 1 and stage 2 over
// every (mesh, block) work item for all scenarios, and a per-scenario epilogue
// -- and the step loop is replayed from a CUDA graph two steps at a time.  A
// mesh may carry gauges (the same points for all its scenarios); each scenario
// then records eta there into a circular device ring after each of its steps
// (a fourth launch per step), and the host drains the rings whenever it reads
// the scenario scalars, at least every kBatchRingCap - 1 records.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/volna_gb.h"
#include "vg_internal.h"

using namespace vg;

namespace {
constexpr int kBatchRingCap = 64;     // records per scenario between two drains
}

struct vg_batch {
    int precision = 32;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    vg_params prm{};
    struct Mesh {
        vg_ctx *ctx = nullptr;
        int n_scen = 0;
        int first_entry = 0;
        void *w[2] = {nullptr, nullptr};
        void *R0 = nullptr;
        int n_gauges = 0;
        int32_t *gauge_cells = nullptr;    // device [G] internal cell ids
        double *ring_t = nullptr;          // device [n_scen][kBatchRingCap]
        double *ring_eta = nullptr;        // device [n_scen][kBatchRingCap][G]
        std::vector<int32_t> gauge_orig;   // containing cells, original ids
        std::vector<int64_t> drained;      // per scenario: records already on the host
        std::vector<std::vector<double>> rec_t, rec_eta;   // per scenario
    };
    std::vector<Mesh> meshes;
    std::vector<char> has_state;           // per scenario
    DevScalars *sc_all = nullptr;          // [n_entries + 1]
    int n_entries = 0;
    void *table[2] = {nullptr, nullptr};   // device BatchMesh arrays for both step parities
    int n_items = 0;
    int grid = 0;
    int ctas_per_sm = 0;                   // autotuned limit of resident CTAs per SM (0: as many as fit)
    int fit_per_sm = 0;                    // CTAs per SM that fit the current block size
    size_t smem = 0;
    int cur = 0;
    bool dirty = true;
    cudaGraphExec_t graph2 = nullptr;
    int64_t launches = 0;
    bool gauges = false;                   // some mesh has gauges
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) { if (cudaGetDevice(&prev) != cudaSuccess) prev = -1; cudaSetDevice(dev); }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

int bfail(vg_batch *b, int code, const std::string &msg)
{
    if (b) b->err = msg;
    return code;
}

int bcuda(vg_batch *b, cudaError_t e, const char *what)
{
    return bfail(b, VG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define VB_CUDA(b, call)                                         \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call);       \
    } while (0)

size_t rsize(const vg_batch *b) { return b->precision == 64 ? 8 : 4; }

void scalars_init(const vg_batch *b, DevScalars &s, double t)
{
    std::memset(&s, 0, sizeof(s));
    s.t = t;
    if (b->precision == 64) {
        double inf = INFINITY;
        std::memcpy(&s.dtmin_bits, &inf, 8);
    } else {
        float inf = INFINITY;
        uint32_t u;
        std::memcpy(&u, &inf, 4);
        s.dtmin_bits = u;
    }
}

int entry_of(vg_batch *b, int32_t mesh, int32_t scen, int &e)
{
    if (mesh < 0 || mesh >= (int)b->meshes.size()) return bfail(b, VG_EINVAL, "no such mesh");
    if (scen < 0 || scen >= b->meshes[mesh].n_scen) return bfail(b, VG_EINVAL, "no such scenario");
    e = b->meshes[mesh].first_entry + scen;
    return VG_OK;
}

// Rebuild the device tables and the launch configuration after a change of
// meshes, parameters or block size.
int rebuild(vg_batch *b)
{
    if (b->graph2) { cudaGraphExecDestroy(b->graph2); b->graph2 = nullptr; }
    size_t eb = b->precision == 64 ? batch_mesh_bytes_f64() : batch_mesh_bytes_f32();
    size_t nm = b->meshes.size();
    std::vector<unsigned char> host(eb * nm);
    int block = 0, max_halo = 0, max_ring1 = 0;
    for (int parity = 0; parity < 2; parity++) {
        int item = 0;
        for (size_t m = 0; m < nm; m++) {
            vg_batch::Mesh &M = b->meshes[m];
            DevPtrs d = ctx_dev_ptrs(M.ctx);
            d.R0 = M.R0;
            d.sc = b->sc_all + M.first_entry;
            d.n_gauges = M.n_gauges;
            d.gauge_cells = M.gauge_cells;
            d.ring_t = M.ring_t;
            d.ring_eta = M.ring_eta;
            d.ring_cap = kBatchRingCap;
            StepParams p = ctx_step_params(M.ctx);
            p.gauge_every = 1;
            if (b->precision == 64)
                fill_batch_mesh_f64(host.data() + m * eb, d, p, M.w[parity], M.w[1 - parity], M.n_scen, item, M.first_entry);
            else
                fill_batch_mesh_f32(host.data() + m * eb, d, p, M.w[parity], M.w[1 - parity], M.n_scen, item, M.first_entry);
            item += d.nblocks;
            if (block && block != d.block) return bfail(b, VG_EINVAL, "meshes of a batch must share one block size");
            if (d.block > 256) return bfail(b, VG_EINVAL, "batched ensembles use blocks of at most 256 cells");
            block = d.block;
            max_halo = std::max(max_halo, (int)d.max_halo);
            max_ring1 = std::max(max_ring1, (int)d.max_ring1);
        }
        b->n_items = item;
        if (b->table[parity]) cudaFree(b->table[parity]);
        VB_CUDA(b, cudaMalloc(&b->table[parity], eb * nm));
        VB_CUDA(b, cudaMemcpy(b->table[parity], host.data(), eb * nm, cudaMemcpyHostToDevice));
    }
    int e = b->precision == 64 ? batch_config_f64(block, max_halo, max_ring1, b->grid, b->smem, !b->prm.fp64_literal)
                               : batch_config_f32(block, max_halo, max_ring1, b->grid, b->smem);
    if (e) return bcuda(b, (cudaError_t)e, "batched launch configuration");
    {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        b->fit_per_sm = sms > 0 ? b->grid / sms : 1;
        if (b->ctas_per_sm > 0 && b->ctas_per_sm < b->fit_per_sm) b->grid = sms * b->ctas_per_sm;
    }
    if (b->grid > b->n_items) b->grid = b->n_items;
    b->gauges = false;
    for (auto &M : b->meshes) b->gauges = b->gauges || M.n_gauges > 0;
    b->dirty = false;
    return VG_OK;
}

StepParams batch_params(const vg_batch *b)
{
    StepParams p{};
    p.g = b->prm.g;
    p.cfl = b->prm.cfl;
    p.hthr = b->prm.h_threshold;
    p.dt_fixed = b->prm.dt_fixed;
    p.dt_max = b->prm.dt_max;
    p.t_end = b->prm.t_end;
    p.order = b->prm.order;
    p.gauge_every = b->prm.gauge_every > 0 ? b->prm.gauge_every : 1;
    p.fp64_fast = b->precision == 64 && !b->prm.fp64_literal;
    return p;
}

int enqueue_batch_step(vg_batch *b, int parity)
{
    int block = ctx_dev_ptrs(b->meshes[0].ctx).block;
    StepParams p = batch_params(b);
    int e = b->precision == 64
                ? launch_batch_step_f64(b->table[parity], (int)b->meshes.size(), b->n_items, b->n_entries, b->sc_all,
                                        block, b->grid, b->smem, p, b->gauges, (void *)b->stream)
                : launch_batch_step_f32(b->table[parity], (int)b->meshes.size(), b->n_items, b->n_entries, b->sc_all,
                                        block, b->grid, b->smem, p, b->gauges, (void *)b->stream);
    if (e) return bcuda(b, (cudaError_t)e, "batched step launch");
    b->launches += b->gauges ? 4 : 3;
    return VG_OK;
}

int build_batch_graph(vg_batch *b)
{
    if (b->graph2) { cudaGraphExecDestroy(b->graph2); b->graph2 = nullptr; }
    cudaGraph_t g = nullptr;
    int64_t saved = b->launches;
    VB_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_batch_step(b, 0);
    if (!rc) rc = enqueue_batch_step(b, 1);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    b->launches = saved;
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph2, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
    return VG_OK;
}

int ready(vg_batch *b)
{
    if (b->meshes.empty()) return bfail(b, VG_ESTATE, "no mesh in the batch");
    for (int e = 0; e < b->n_entries; e++)
        if (!b->has_state[e]) return bfail(b, VG_ESTATE, "scenario " + std::to_string(e) + " has no state");
    if (b->dirty) {
        int rc = rebuild(b);
        if (rc) return rc;
    }
    if (!b->graph2) {
        int rc = build_batch_graph(b);
        if (rc) return rc;
    }
    return VG_OK;
}

// n steps on the device (graph pairs; a single plain step to fix the parity).
int run_steps(vg_batch *b, int64_t n)
{
    int rc;
    if (b->cur == 1 && n > 0) {
        if ((rc = enqueue_batch_step(b, 1))) return rc;
        b->cur = 0;
        n--;
    }
    while (n >= 2) {
        VB_CUDA(b, cudaGraphLaunch(b->graph2, b->stream));
        b->launches += b->gauges ? 8 : 6;
        n -= 2;
    }
    if (n == 1) {
        if ((rc = enqueue_batch_step(b, 0))) return rc;
        b->cur = 1;
    }
    return VG_OK;
}

int drain(vg_batch *b, const std::vector<DevScalars> &s);

// Read every scenario's scalars, then drain the gauge rings.
int read_all(vg_batch *b, std::vector<DevScalars> &s)
{
    s.resize(b->n_entries + 1);
    VB_CUDA(b, cudaMemcpyAsync(s.data(), b->sc_all, sizeof(DevScalars) * (b->n_entries + 1), cudaMemcpyDeviceToHost,
                               b->stream));
    VB_CUDA(b, cudaStreamSynchronize(b->stream));
    return drain(b, s);
}

// Copy the gauge records written since the last drain to the host (per mesh one
// copy of each ring, then the new records of every scenario in order).
int drain(vg_batch *b, const std::vector<DevScalars> &s)
{
    std::vector<double> rt, re;
    for (auto &M : b->meshes) {
        if (M.n_gauges == 0) continue;
        bool any = false;
        for (int k = 0; k < M.n_scen; k++) {
            int64_t n = s[M.first_entry + k].n_rec - M.drained[k];
            if (n > kBatchRingCap) return bfail(b, VG_ESTATE, "gauge ring overflow");
            any = any || n > 0;
        }
        if (!any) continue;
        const size_t G = (size_t)M.n_gauges, cap = kBatchRingCap;
        rt.resize((size_t)M.n_scen * cap);
        re.resize((size_t)M.n_scen * cap * G);
        VB_CUDA(b, cudaMemcpyAsync(rt.data(), M.ring_t, 8 * rt.size(), cudaMemcpyDeviceToHost, b->stream));
        VB_CUDA(b, cudaMemcpyAsync(re.data(), M.ring_eta, 8 * re.size(), cudaMemcpyDeviceToHost, b->stream));
        VB_CUDA(b, cudaStreamSynchronize(b->stream));
        for (int k = 0; k < M.n_scen; k++) {
            const int64_t n_rec = s[M.first_entry + k].n_rec;
            for (int64_t r = M.drained[k]; r < n_rec; r++) {
                const size_t slot = (size_t)k * cap + (size_t)(r % kBatchRingCap);
                M.rec_t[k].push_back(rt[slot]);
                M.rec_eta[k].insert(M.rec_eta[k].end(), re.begin() + slot * G, re.begin() + (slot + 1) * G);
            }
            M.drained[k] = n_rec;
        }
    }
    return VG_OK;
}

// Record the gauges of scenario k of mesh M from its current state (at set_state
// and set_gauges), as record index 0 of a cleared ring.
int record_now(vg_batch *b, vg_batch::Mesh &M, int k)
{
    if (M.n_gauges == 0) return VG_OK;
    const int e = M.first_entry + k;
    static const long long zero = 0;
    VB_CUDA(b, cudaMemcpyAsync(&b->sc_all[e].n_rec, &zero, sizeof(zero), cudaMemcpyHostToDevice, b->stream));
    M.drained[k] = 0;
    M.rec_t[k].clear();
    M.rec_eta[k].clear();
    if (!b->has_state[e]) return VG_OK;
    DevPtrs d = ctx_dev_ptrs(M.ctx);
    d.sc = b->sc_all + e;
    d.n_gauges = M.n_gauges;
    d.gauge_cells = M.gauge_cells;
    d.ring_cap = kBatchRingCap;
    d.ring_t = M.ring_t + (size_t)k * kBatchRingCap;
    d.ring_eta = M.ring_eta + (size_t)k * kBatchRingCap * M.n_gauges;
    const int64_t nc = ctx_host_mesh(M.ctx).nc;
    const void *w = static_cast<unsigned char *>(M.w[b->cur]) + rsize(b) * 3 * (size_t)nc * k;
    int err = launch_record_gauges(d, w, b->precision, (void *)b->stream);
    if (err) return bcuda(b, (cudaError_t)err, "gauge record launch");
    b->launches++;
    return VG_OK;
}

void free_gauges(vg_batch::Mesh &M)
{
    if (M.gauge_cells) cudaFree(M.gauge_cells);
    if (M.ring_t) cudaFree(M.ring_t);
    if (M.ring_eta) cudaFree(M.ring_eta);
    M.gauge_cells = nullptr;
    M.ring_t = M.ring_eta = nullptr;
    M.n_gauges = 0;
}

int check(vg_batch *b, const std::vector<DevScalars> &s)
{
    unsigned flags = s[b->n_entries].flags;
    if (flags & FLAG_NONFINITE_STATE) return bfail(b, VG_ENONFINITE, "a non-finite value appeared in a scenario");
    if (flags & FLAG_NONFINITE_DT) return bfail(b, VG_ENONFINITE, "a scenario's time step is not finite");
    if (b->prm.strict_positivity && s[b->n_entries].neg_count > 0)
        return bfail(b, VG_ENEGDEPTH, "a stage produced a negative depth");
    return VG_OK;
}

void free_batch(vg_batch *b)
{
    if (b->graph2) cudaGraphExecDestroy(b->graph2);
    for (auto &M : b->meshes) {
        if (M.w[0]) cudaFree(M.w[0]);
        if (M.w[1]) cudaFree(M.w[1]);
        if (M.R0) cudaFree(M.R0);
        free_gauges(M);
        vg_destroy(M.ctx);
    }
    b->meshes.clear();
    if (b->sc_all) cudaFree(b->sc_all);
    for (int k = 0; k < 2; k++)
        if (b->table[k]) cudaFree(b->table[k]);
}

}  // namespace

extern "C" {

int vg_batch_create(vg_batch **out, int precision, int device, void *cuda_stream)
{
    if (!out) return VG_EINVAL;
    *out = nullptr;
    if (precision != 32 && precision != 64) return VG_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return VG_ECUDA;
    }
    vg_batch *b = new (std::nothrow) vg_batch();
    if (!b) return VG_ENOMEM;
    b->precision = precision;
    b->device = device;
    vg_default_params(&b->prm);
    DeviceGuard guard(device);
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return VG_ECUDA; }
        b->own_stream = true;
    }
    if (cudaMalloc((void **)&b->sc_all, sizeof(DevScalars)) != cudaSuccess) { vg_batch_destroy(b); return VG_ENOMEM; }
    DevScalars s;
    scalars_init(b, s, 0.0);
    cudaMemcpy(b->sc_all, &s, sizeof(s), cudaMemcpyHostToDevice);
    *out = b;
    return VG_OK;
}

void vg_batch_destroy(vg_batch *b)
{
    if (!b) return;
    DeviceGuard guard(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_batch(b);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *vg_batch_last_error(vg_batch *b) { return b ? b->err.c_str() : "NULL batch"; }

int vg_batch_set_params(vg_batch *b, const vg_params *p)
{
    if (!b || !p) return VG_EINVAL;
    DeviceGuard guard(b->device);
    for (auto &M : b->meshes) {
        int rc = vg_set_params(M.ctx, p);
        if (rc) return bfail(b, rc, vg_last_error(M.ctx));
    }
    b->prm = *p;
    b->dirty = true;
    return VG_OK;
}

int vg_batch_add_mesh(vg_batch *b, int64_t nv, const double *xy, int64_t nc, const int32_t *tri,
                      const double *depth_v, int renumber, int32_t n_scenarios, int32_t *mesh_id)
{
    if (!b || n_scenarios < 1) return VG_EINVAL;
    if (b->n_entries + n_scenarios > 512) return bfail(b, VG_EINVAL, "a batch holds at most 512 scenarios");
    DeviceGuard guard(b->device);
    cudaStreamSynchronize(b->stream);
    vg_batch::Mesh M;
    int rc = vg_create(&M.ctx, b->precision, b->device, (void *)b->stream);
    if (rc) return bfail(b, rc, "internal context creation failed");
    if ((rc = vg_set_params(M.ctx, &b->prm)) || (rc = vg_mesh_upload(M.ctx, nv, xy, nc, tri, depth_v, renumber))) {
        std::string msg = vg_last_error(M.ctx);
        vg_destroy(M.ctx);
        return bfail(b, rc, msg);
    }
    size_t bytes = rsize(b) * 3 * (size_t)nc * n_scenarios;
    if (cudaMalloc(&M.w[0], bytes) != cudaSuccess || cudaMalloc(&M.w[1], bytes) != cudaSuccess ||
        cudaMalloc(&M.R0, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (M.w[0]) cudaFree(M.w[0]);
        if (M.w[1]) cudaFree(M.w[1]);
        vg_destroy(M.ctx);
        return bfail(b, VG_ENOMEM, "state allocation failed");
    }
    M.n_scen = n_scenarios;
    M.first_entry = b->n_entries;
    M.drained.assign(n_scenarios, 0);
    M.rec_t.assign(n_scenarios, {});
    M.rec_eta.assign(n_scenarios, {});
    // grow the scalar array: [n_entries] scenarios + one batch-wide record
    DevScalars *sc = nullptr;
    int n_new = b->n_entries + n_scenarios;
    VB_CUDA(b, cudaMalloc((void **)&sc, sizeof(DevScalars) * (n_new + 1)));
    std::vector<DevScalars> host(n_new + 1);
    if (b->n_entries) VB_CUDA(b, cudaMemcpy(host.data(), b->sc_all, sizeof(DevScalars) * b->n_entries, cudaMemcpyDeviceToHost));
    for (int e = b->n_entries; e <= n_new; e++) scalars_init(b, host[e], 0.0);
    VB_CUDA(b, cudaMemcpy(sc, host.data(), sizeof(DevScalars) * (n_new + 1), cudaMemcpyHostToDevice));
    cudaFree(b->sc_all);
    b->sc_all = sc;
    b->n_entries = n_new;
    b->has_state.resize(n_new, 0);
    b->meshes.push_back(M);
    if (b->cur == 1) {
        // keep every mesh's current state in the same buffer index
        for (size_t m = 0; m + 1 < b->meshes.size(); m++)
            VB_CUDA(b, cudaMemcpy(b->meshes[m].w[0], b->meshes[m].w[1],
                                  rsize(b) * 3 * ctx_host_mesh(b->meshes[m].ctx).nc * b->meshes[m].n_scen,
                                  cudaMemcpyDeviceToDevice));
        b->cur = 0;
    }
    b->dirty = true;
    if (mesh_id) *mesh_id = (int32_t)b->meshes.size() - 1;
    return VG_OK;
}

int vg_batch_set_state(vg_batch *b, int32_t mesh, int32_t scen, const double *H, const double *Hu,
                       const double *Hv, double t)
{
    if (!b || !H || !Hu || !Hv || !std::isfinite(t)) return VG_EINVAL;
    int e, rc;
    if ((rc = entry_of(b, mesh, scen, e))) return rc;
    DeviceGuard guard(b->device);
    vg_batch::Mesh &M = b->meshes[mesh];
    int64_t nc = ctx_host_mesh(M.ctx).nc;
    double *st = nullptr;
    if ((rc = ctx_staging(M.ctx, &st))) return bfail(b, rc, "staging allocation failed");
    VB_CUDA(b, cudaMemcpyAsync(st, H, 8 * nc, cudaMemcpyHostToDevice, b->stream));
    VB_CUDA(b, cudaMemcpyAsync(st + nc, Hu, 8 * nc, cudaMemcpyHostToDevice, b->stream));
    VB_CUDA(b, cudaMemcpyAsync(st + 2 * nc, Hv, 8 * nc, cudaMemcpyHostToDevice, b->stream));
    DevScalars s;
    scalars_init(b, s, t);
    VB_CUDA(b, cudaMemcpyAsync(b->sc_all + e, &s, sizeof(s), cudaMemcpyHostToDevice, b->stream));
    DevPtrs d = ctx_dev_ptrs(M.ctx);
    d.sc = b->sc_all + e;
    void *dst = static_cast<unsigned char *>(M.w[b->cur]) + rsize(b) * 3 * (size_t)nc * scen;
    int err = launch_import_state(d, ctx_old_of_new(M.ctx), st, st + nc, st + 2 * nc, 1, dst, b->precision,
                                  (void *)b->stream);
    if (err) return bcuda(b, (cudaError_t)err, "state import launch");
    b->launches++;
    DevScalars r;
    VB_CUDA(b, cudaMemcpyAsync(&r, b->sc_all + e, sizeof(r), cudaMemcpyDeviceToHost, b->stream));
    VB_CUDA(b, cudaStreamSynchronize(b->stream));
    if (r.flags & FLAG_BAD_INPUT) {
        b->has_state[e] = 0;
        return bfail(b, VG_EINVAL, "state has a negative or non-finite depth, or non-finite momentum");
    }
    b->has_state[e] = 1;
    return record_now(b, M, scen);
}

int vg_batch_get_state(vg_batch *b, int32_t mesh, int32_t scen, double *H, double *Hu, double *Hv, double *t,
                       int64_t *steps)
{
    if (!b || !H || !Hu || !Hv) return VG_EINVAL;
    int e, rc;
    if ((rc = entry_of(b, mesh, scen, e))) return rc;
    if (!b->has_state[e]) return bfail(b, VG_ESTATE, "scenario has no state");
    DeviceGuard guard(b->device);
    vg_batch::Mesh &M = b->meshes[mesh];
    int64_t nc = ctx_host_mesh(M.ctx).nc;
    double *st = nullptr;
    if ((rc = ctx_staging(M.ctx, &st))) return bfail(b, rc, "staging allocation failed");
    const void *src = static_cast<unsigned char *>(M.w[b->cur]) + rsize(b) * 3 * (size_t)nc * scen;
    int err = launch_export_state(ctx_dev_ptrs(M.ctx), ctx_old_of_new(M.ctx), src, b->precision, st, st + nc,
                                  st + 2 * nc, 1, (void *)b->stream);
    if (err) return bcuda(b, (cudaError_t)err, "state export launch");
    b->launches++;
    VB_CUDA(b, cudaMemcpyAsync(H, st, 8 * nc, cudaMemcpyDeviceToHost, b->stream));
    VB_CUDA(b, cudaMemcpyAsync(Hu, st + nc, 8 * nc, cudaMemcpyDeviceToHost, b->stream));
    VB_CUDA(b, cudaMemcpyAsync(Hv, st + 2 * nc, 8 * nc, cudaMemcpyDeviceToHost, b->stream));
    DevScalars s;
    VB_CUDA(b, cudaMemcpyAsync(&s, b->sc_all + e, sizeof(s), cudaMemcpyDeviceToHost, b->stream));
    VB_CUDA(b, cudaStreamSynchronize(b->stream));
    if (t) *t = s.t;
    if (steps) *steps = s.steps;
    return VG_OK;
}

int vg_batch_step(vg_batch *b, int64_t n_steps)
{
    if (!b || n_steps < 0) return VG_EINVAL;
    DeviceGuard guard(b->device);
    int rc = ready(b);
    if (rc) return rc;
    // with gauges, drain before a ring can fill (at most one record per step)
    const int64_t every = b->prm.gauge_every > 0 ? b->prm.gauge_every : 1;
    const int64_t chunk_max = b->gauges ? (int64_t)(kBatchRingCap - 1) * every : std::max<int64_t>(n_steps, 1);
    std::vector<DevScalars> s;
    do {
        const int64_t chunk = std::min(n_steps, chunk_max);
        if ((rc = run_steps(b, chunk))) return rc;
        n_steps -= chunk;
        if ((rc = read_all(b, s))) return rc;
        if ((rc = check(b, s))) return rc;
    } while (n_steps > 0);
    return VG_OK;
}

int vg_batch_run(vg_batch *b, double t_end, int64_t max_steps, int64_t *steps_taken)
{
    if (!b || !(t_end > 0) || max_steps < 0) return VG_EINVAL;
    DeviceGuard guard(b->device);
    vg_params saved = b->prm;
    if (b->prm.t_end != t_end) {
        vg_params p = b->prm;
        p.t_end = t_end;
        int rc = vg_batch_set_params(b, &p);
        if (rc) return rc;
    }
    int rc = ready(b);
    int64_t taken = 0;
    std::vector<DevScalars> s;
    while (!rc && taken < max_steps) {
        int64_t chunk = std::min<int64_t>(16, max_steps - taken);
        if ((rc = run_steps(b, chunk))) break;
        taken += chunk;
        if ((rc = read_all(b, s))) break;
        if ((rc = check(b, s))) break;
        bool done = true;
        for (int e = 0; e < b->n_entries && done; e++) done = s[e].t >= t_end;
        if (done) break;
    }
    if (steps_taken) *steps_taken = taken;
    if (saved.t_end != t_end) {
        int rc2 = vg_batch_set_params(b, &saved);
        if (!rc) rc = rc2;
    }
    return rc;
}

int vg_batch_autotune(vg_batch *b, int32_t n_steps, int32_t *best_block, int32_t *best_ctas, double *best_ms)
{
    if (!b || n_steps < 1) return VG_EINVAL;
    DeviceGuard guard(b->device);
    int rc = ready(b);
    if (rc) return rc;
    {
        std::vector<DevScalars> s;      // drain, so that the trial steps overwrite no unread record
        if ((rc = read_all(b, s))) return rc;
    }
    // Save every scenario's state and scalars; each candidate block size runs
    // n_steps timed steps from the same state, which is restored afterwards.
    std::vector<void *> saved(b->meshes.size(), nullptr);
    void *sc_saved = nullptr;
    for (size_t m = 0; m < b->meshes.size(); m++) {
        size_t bytes = rsize(b) * 3 * ctx_host_mesh(b->meshes[m].ctx).nc * b->meshes[m].n_scen;
        VB_CUDA(b, cudaMalloc(&saved[m], bytes));
        VB_CUDA(b, cudaMemcpyAsync(saved[m], b->meshes[m].w[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream));
    }
    size_t sc_bytes = sizeof(DevScalars) * (b->n_entries + 1);
    VB_CUDA(b, cudaMalloc(&sc_saved, sc_bytes));
    VB_CUDA(b, cudaMemcpyAsync(sc_saved, b->sc_all, sc_bytes, cudaMemcpyDeviceToDevice, b->stream));
    const int candidates[3] = {64, 128, 256};
    int best = 0, best_c = 0;
    double best_t = INFINITY;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int cur0 = b->cur;
    for (int k = 0; k < 3 && !rc; k++) {
        vg_params p = b->prm;
        p.block_cells = candidates[k];
        if ((rc = vg_batch_set_params(b, &p))) break;
        b->ctas_per_sm = 0;
        b->dirty = true;
        if ((rc = ready(b))) break;
        const int fit = b->fit_per_sm;
        // as many CTAs per SM as fit, then one and two fewer
        for (int drop = 0; drop < 3 && !rc; drop++) {
            const int c = fit - drop;
            if (c < 1) break;
            b->ctas_per_sm = drop == 0 ? 0 : c;
            b->dirty = true;
            if ((rc = ready(b))) break;
            if ((rc = run_steps(b, 2))) break;      // warm-up
            cudaEventRecord(e0, b->stream);
            if ((rc = run_steps(b, n_steps))) break;
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_t) { best_t = ms; best = candidates[k]; best_c = b->ctas_per_sm; }
            for (size_t m = 0; m < b->meshes.size(); m++) {
                size_t bytes = rsize(b) * 3 * ctx_host_mesh(b->meshes[m].ctx).nc * b->meshes[m].n_scen;
                cudaMemcpyAsync(b->meshes[m].w[cur0], saved[m], bytes, cudaMemcpyDeviceToDevice, b->stream);
            }
            cudaMemcpyAsync(b->sc_all, sc_saved, sc_bytes, cudaMemcpyDeviceToDevice, b->stream);
            b->cur = cur0;
        }
    }
    cudaStreamSynchronize(b->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (void *p : saved) cudaFree(p);
    cudaFree(sc_saved);
    if (rc) return rc;
    vg_params p = b->prm;
    p.block_cells = best;
    if ((rc = vg_batch_set_params(b, &p))) return rc;
    b->ctas_per_sm = best_c;
    b->dirty = true;
    if (best_block) *best_block = best;
    if (best_ctas) *best_ctas = best_c;
    if (best_ms) *best_ms = best_t / n_steps;
    return VG_OK;
}

int vg_batch_set_gauges(vg_batch *b, int32_t mesh_id, int32_t n, const double *xy)
{
    if (!b || n < 0 || (n > 0 && !xy)) return VG_EINVAL;
    if (mesh_id < 0 || mesh_id >= (int)b->meshes.size()) return bfail(b, VG_EINVAL, "no such mesh");
    DeviceGuard guard(b->device);
    vg_batch::Mesh &M = b->meshes[mesh_id];
    const HostMesh &hm = ctx_host_mesh(M.ctx);
    std::vector<int32_t> cells(n);
    locate_points(hm, n, xy, cells.data());
    for (int32_t k = 0; k < n; k++)
        if (cells[k] < 0) return bfail(b, VG_EINVAL, "gauge " + std::to_string(k) + " lies outside the mesh");
    VB_CUDA(b, cudaStreamSynchronize(b->stream));
    free_gauges(M);
    M.gauge_orig = cells;
    b->dirty = true;
    if (b->graph2) { cudaGraphExecDestroy(b->graph2); b->graph2 = nullptr; }
    for (int k = 0; k < M.n_scen; k++) {
        M.drained[k] = 0;
        M.rec_t[k].clear();
        M.rec_eta[k].clear();
    }
    if (n == 0) return VG_OK;
    std::vector<int32_t> internal(n);
    for (int32_t k = 0; k < n; k++) internal[k] = hm.new_of_old[cells[k]];
    const size_t cap = kBatchRingCap;
    if (cudaMalloc((void **)&M.gauge_cells, 4 * (size_t)n) != cudaSuccess ||
        cudaMalloc((void **)&M.ring_t, 8 * (size_t)M.n_scen * cap) != cudaSuccess ||
        cudaMalloc((void **)&M.ring_eta, 8 * (size_t)M.n_scen * cap * n) != cudaSuccess) {
        cudaGetLastError();
        free_gauges(M);
        return bfail(b, VG_ENOMEM, "gauge ring allocation failed");
    }
    M.n_gauges = n;
    VB_CUDA(b, cudaMemcpy(M.gauge_cells, internal.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
    for (int k = 0; k < M.n_scen; k++) {
        int rc = record_now(b, M, k);
        if (rc) return rc;
    }
    return VG_OK;
}

int vg_batch_set_open_boundary(vg_batch *b, int32_t mesh_id, int64_t n, const int32_t *edges)
{
    return vg_batch_set_boundary(b, mesh_id, n, edges, nullptr);
}

int vg_batch_set_boundary(vg_batch *b, int32_t mesh_id, int64_t n, const int32_t *edges, const int32_t *kinds)
{
    if (!b) return VG_EINVAL;
    if (mesh_id < 0 || mesh_id >= (int)b->meshes.size()) return bfail(b, VG_EINVAL, "no such mesh");
    DeviceGuard guard(b->device);
    vg_ctx *ctx = b->meshes[mesh_id].ctx;
    int rc = vg_set_boundary(ctx, n, edges, kinds);
    if (rc) return bfail(b, rc, vg_last_error(ctx));
    b->dirty = true;
    if (b->graph2) { cudaGraphExecDestroy(b->graph2); b->graph2 = nullptr; }
    return VG_OK;
}

int vg_batch_get_gauges(vg_batch *b, int32_t mesh_id, int32_t scenario, double *t, double *eta, int64_t cap,
                        int64_t *n_rec)
{
    if (!b || cap < 0) return VG_EINVAL;
    int e, rc;
    if ((rc = entry_of(b, mesh_id, scenario, e))) return rc;
    DeviceGuard guard(b->device);
    std::vector<DevScalars> s;
    if ((rc = read_all(b, s))) return rc;
    const vg_batch::Mesh &M = b->meshes[mesh_id];
    const int64_t n = (int64_t)M.rec_t[scenario].size();
    if (n_rec) *n_rec = n;
    const int64_t k = std::min(n, cap);
    if (t && k) std::memcpy(t, M.rec_t[scenario].data(), 8 * k);
    if (eta && k) std::memcpy(eta, M.rec_eta[scenario].data(), 8 * k * M.n_gauges);
    return VG_OK;
}

int vg_batch_info(vg_batch *b, int32_t *n_meshes, int32_t *n_scenarios, int64_t *cells, int64_t *launches)
{
    if (!b) return VG_EINVAL;
    int64_t c = 0;
    for (auto &M : b->meshes) c += ctx_host_mesh(M.ctx).nc * M.n_scen;
    if (n_meshes) *n_meshes = (int32_t)b->meshes.size();
    if (n_scenarios) *n_scenarios = b->n_entries;
    if (cells) *cells = c;
    if (launches) *launches = b->launches;
    return VG_OK;
}

}  // extern "C"
