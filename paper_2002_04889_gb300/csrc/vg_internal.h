// Internal declarations of the volna_gb library: host mesh preparation, the
// device data layout, and the launch wrappers of the step kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace vg {

// Per-cell geometry rows, [GEO_ROWS][nc], in the order below (host, and the
// FP64 device copy; the FP32 device copy is a 16-float record per cell, formed
// from these rows at upload, layout beside the stage kernels).  Face f of a cell joins its local vertices f and f+1; the local order
// is counter-clockwise from the vertex with the smallest input id.
enum GeoRow : int {
    GEO_NX = 0,    // 3 rows: outward unit normal x of faces 0..2
    GEO_NY = 3,    // 3 rows: outward unit normal y
    GEO_LEN = 6,   // 3 rows: face length
    GEO_FX = 9,    // 3 rows: face midpoint minus centroid, x
    GEO_FY = 12,   // 3 rows: face midpoint minus centroid, y
    GEO_WX = 15,   // 3 rows: least-squares weight, x
    GEO_WY = 18,   // 3 rows: least-squares weight, y
    GEO_AREA = 21, // 1 row: cell area
    GEO_ROWS = 22
};

constexpr uint16_t NBR_WALL = 0xFFFF;   // wall face (ghost of Sec. 2.5); nbr = -1
constexpr uint16_t NBR_OPEN = 0xFFFE;   // open (transmissive) face; nbr = -2
constexpr uint16_t NBR_ABSORB = 0xFFFD; // absorbing (characteristic) face; nbr = -3; every code
                                        // >= NBR_ABSORB is a boundary face

// Host-side prepared mesh, cells in the library's (renumbered) order.
struct HostMesh {
    int64_t nc = 0, nv = 0;
    int64_t n_flipped = 0;
    int32_t block = 256;                 // cells per block
    int32_t nblocks = 0;
    int32_t max_halo = 0;                // max ring-1 + ring-2 cells of a block
    int32_t max_ring1 = 0;               // max ring-1 cells of a block
    std::vector<int32_t> new_of_old, old_of_new;
    std::vector<int32_t> vtx;            // [nc][3] local-order vertices (original cell order)
    std::vector<double> geo;             // [GEO_ROWS][nc]  (internal order)
    std::vector<double> z;               // [nc]            (internal order)
    std::vector<double> zf;              // [3][nc] bed at the face midpoints (internal order):
                                         // -(mean of the face's two vertex depths)
    std::vector<int32_t> nbr;            // [3][nc] internal neighbour ids, -1 wall, -2 open, -3 absorbing
    std::vector<uint16_t> nbrl;          // [3][nc] (local << 2 | face), NBR_WALL or NBR_OPEN
    std::vector<int32_t> halo_ptr;       // [nblocks + 1] into halo_ids / ring1_nbr
    std::vector<int32_t> halo_n1;        // [nblocks] ring-1 cells of each block
    std::vector<int32_t> halo_ids;       // per block: ring-1 then ring-2 cells (internal ids)
    std::vector<uint16_t> ring1_nbr;     // [3 * halo_ids.size()] local neighbour index of
                                         // each ring-1 cell (NBR_WALL / NBR_OPEN)
    std::vector<int32_t> fq_ptr;         // [nblocks + 1] into fq
    std::vector<uint16_t> fq;            // per block: its owned faces, (local cell << 2) | face
    std::vector<double> xy;              // [nv][2] copy for point location
};

// Builds everything in HostMesh.  Returns 0 or a VG_E* code with a message.
int prepare_mesh(int64_t nv, const double *xy, int64_t nc, const int32_t *tri,
                 const double *depth_v, int renumber, int block, HostMesh &m, std::string &err);

// Cell beds z [nc] and face beds zf [3][nc] (internal order) of the per-vertex
// depths: z_K = -(mean of the three vertex depths), z_f = -(mean of the face's two
// vertex depths), the piecewise linear bed (Sec. 2.1).  Returns 0, or VG_EINVAL
// for a non-finite bed.
int bed_arrays(HostMesh &m, const double *depth_v, std::string &err);

// Re-partitions an already prepared mesh into blocks of `block` cells.
int partition_blocks(HostMesh &m, int block, std::string &err);

// Cells containing each point (original ids; ties to the lowest id), -1 if none.
void locate_points(const HostMesh &m, int32_t n, const double *pts, int32_t *cells);

// Device scalars shared by the step kernels of one context.
struct DevScalars {
    double t;             // simulated time
    double dt;            // time step of the current step
    unsigned long long dtmin_bits;  // running min of the stage-1 CFL bound (bits of a
                                    // non-negative real: integer order = value order)
    long long steps;      // steps with dt > 0
    long long n_rec;      // gauge records in the device ring
    long long neg_count;  // negative depths met
    unsigned int flags;   // FLAG_* bits
    int pad;
};

enum : unsigned int {
    FLAG_NONFINITE_STATE = 1u,
    FLAG_NONFINITE_DT = 2u,
    FLAG_RING_FULL = 4u,
    FLAG_BAD_INPUT = 8u,
};

struct StepParams {
    double g, cfl, hthr, dt_fixed, dt_max, t_end;
    int order, gauge_every;
    int fp64_fast;          // FP64: the contracted build of the stage kernels (step_f64_fast.cu)
};

// Device pointers of one context (element type = the context's real).
struct DevPtrs {
    int64_t nc;
    int32_t block, nblocks, max_halo, max_ring1, n_gauges, ring_cap;
    int32_t threads;        // threads per CTA of the stage kernels (>= block)
    int32_t fp64_fast;      // FP64: launch the contracted build (step_f64_fast.cu), not the literal one
    const void *geo;        // FP64: [GEO_ROWS][nc]; FP32: [nc][16] record
    const void *z;          // [nc]
    const void *zf;         // face beds: FP64 [3][nc]; FP32 [nc][2] = (z_f - z_K) of faces 0
                            // and 1 (face 2: minus their sum, the face midpoints average
                            // to the centroid)
    const double *z64;      // [nc] FP64 bed (state import/export and diagnostics)
    const void *z_orig;     // FP32: [nc] the kernels' bed in the original cell order, or null
    const double *z64_orig; // FP32: [nc] the FP64 bed in the original cell order, or null
                            // (both current only while no moving bed has been set)
    const int32_t *nbr;     // [3][nc]
    const uint16_t *nbrl;   // [3][nc]
    const int32_t *halo_ptr;
    const int32_t *halo_n1;
    const int32_t *halo_ids;
    const uint16_t *ring1_nbr;
    const int32_t *fq_ptr;  // [nblocks + 1]
    const uint16_t *fq;     // owned faces of each block
    const int32_t *adj_faces;   // adjoint: every face once, (cell << 2) | face (cell = lower id or the boundary cell)
    int64_t n_adj_faces;
    void *R0;               // [3][nc] stage-1 residual (scratch)
    uint8_t *mask2;         // optional [nc]: stage-2 dry-fix branch per cell (adjoint)
    void *fv_out;           // optional [9][nc]: face values written by the stage kernels (adjoint)
    void *r1_out;           // optional [3][nc]: stage-2 residual written by the stage-2 kernel (adjoint)
    uint8_t *rec_out;       // optional [nc]: 1 where a cell reconstructed (its face values stand on
                            // the face beds), written by the stage kernels (adjoint)
    DevScalars *sc;
    const int32_t *gauge_cells;   // internal ids
    double *ring_t;               // [ring_cap]
    double *ring_eta;             // [ring_cap][n_gauges]
    // moving bed (vg_set_bed_motion): local-order vertices [3][nc] of each cell
    // (internal order) and per-vertex initial depth, uplift and onset time
    const int32_t *bed_vtx;
    const double *bed_depth0, *bed_uplift, *bed_onset;
    double bed_rise;
};

// Launch wrappers (defined in step_f32.cu / step_f64.cu).  w_in, w_out are
// [3][nc] state buffers.  Return cudaError_t as int.
struct LaunchCfg {
    int grid;        // persistent CTAs
    size_t smem;     // dynamic shared memory per CTA
};
size_t stage_smem_f32(int block, int max_halo, int max_ring1);
size_t stage_smem_f64(int block, int max_halo, int max_ring1);
int stage_config_f32(const DevPtrs &d, int stage, LaunchCfg &cfg);
int stage_config_f64(const DevPtrs &d, int stage, LaunchCfg &cfg);
int launch_stage1_f32(const DevPtrs &d, const StepParams &p, const void *w_in, const LaunchCfg &c, void *stream);
int launch_stage2_f32(const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, const LaunchCfg &c, void *stream);
int launch_stage1_f64(const DevPtrs &d, const StepParams &p, const void *w_in, const LaunchCfg &c, void *stream);
int launch_stage2_f64(const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, const LaunchCfg &c, void *stream);
// Unfused RK stages (vg_params.rk_unfused), after stage 1: part 0 writes
// w1 = w^n + dt R0 (dry fix) to w1, part 1 runs the stage-1 kernel on w1 into R1
// without its CFL bound (c1: stage 1's launch configuration), part 2 writes
// w^{n+1} = w^n / 2 + (w1 + dt R1) / 2 (dry fix) to w_out.
int launch_rk_unfused_f32(const DevPtrs &d, const StepParams &p, int part, const void *w_in, void *w_out, void *w1,
                          void *R1, const LaunchCfg &c1, void *stream);
int launch_rk_unfused_f64(const DevPtrs &d, const StepParams &p, int part, const void *w_in, void *w_out, void *w1,
                          void *R1, const LaunchCfg &c1, void *stream);
int launch_rk_unfused_f64_fast(const DevPtrs &d, const StepParams &p, int part, const void *w_in, void *w_out,
                               void *w1, void *R1, const LaunchCfg &c1, void *stream);

// The contracted FP64 build (step_f64_fast.cu); the *_f64 entry points above
// dispatch to it when DevPtrs::fp64_fast / StepParams::fp64_fast is set.
int stage_config_f64_fast(const DevPtrs &d, int stage, LaunchCfg &cfg);
int launch_stage1_f64_fast(const DevPtrs &d, const StepParams &p, const void *w_in, const LaunchCfg &c, void *stream);
int launch_stage2_f64_fast(const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, const LaunchCfg &c,
                           void *stream);
int batch_config_f64_fast(int block, int max_halo, int max_ring1, int &grid, size_t &smem);
int launch_batch_step_f64_fast(const void *table, int n_mesh, int n_items, int n_entries, DevScalars *sc_all,
                               int block, int grid, size_t smem, const StepParams &p, bool gauges, void *stream);

// Batched ensembles (step_f32.cu / step_f64.cu): the device table entry of one
// mesh, the launch configuration, and one batched step (stage 1, stage 2,
// epilogue) over all scenarios.  sc_all has n_entries scenario scalars plus one
// batch-wide record (negative-depth count, flags).
size_t batch_mesh_bytes_f32();
size_t batch_mesh_bytes_f64();
void fill_batch_mesh_f32(void *dst, const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, int n_scen,
                         int first_item, int first_entry);
void fill_batch_mesh_f64(void *dst, const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, int n_scen,
                         int first_item, int first_entry);
int batch_config_f32(int block, int max_halo, int max_ring1, int &grid, size_t &smem);
int batch_config_f64(int block, int max_halo, int max_ring1, int &grid, size_t &smem, bool fast);
int launch_batch_step_f32(const void *table, int n_mesh, int n_items, int n_entries, DevScalars *sc_all, int block,
                          int grid, size_t smem, const StepParams &p, bool gauges, void *stream);
int launch_batch_step_f64(const void *table, int n_mesh, int n_items, int n_entries, DevScalars *sc_all, int block,
                          int grid, size_t smem, const StepParams &p, bool gauges, void *stream);

// Discrete adjoint (adjoint_f64.cu, FP64 contexts).
// The CFL time step's dependence on the state (adaptive steps): orig = original
// cell ids [nc] (argmin ties), *dtbar = the step's dt adjoint, cfl / dt_max as in
// the forward run, part_* scratch of kAdjCflParts entries.
constexpr int kAdjCflParts = 1024;
struct AdjCfl {
    const int32_t *orig;
    const double *dtbar;
    double cfl, dt_max;
    double *part_b;
    int *part_o, *part_k;
};
// FV: the face values at w, precomputed by the forward stage kernel (fv_out)
// or, if fv_given is false, computed here into FV.  cfl (may be NULL): also
// the adjoint of the stage-1 CFL time step through the wave speed of the face
// that set it.
// rec: the reconstruction flags [nc] of the stage (recorded by the forward kernel
// with rec_out).  zb [4][nc] receives the bed adjoints: row 0 the cell beds z_K,
// rows 1..3 the face beds z_f of faces 0..2.
int adjoint_residual_vjp(const DevPtrs &d, const StepParams &p, const double *w, const uint8_t *rec, const double *Rb,
                         double *wb, double *zb, double *FV, bool fv_given, double *FVb, double *zfb, double *own,
                         double *send, void *stream, const AdjCfl *cfl = nullptr);
// *acc (= or +=) scale * sum_i a[i] b[i], deterministic; part: kAdjCflParts doubles.
int adjoint_dot(int64_t n, const double *a, const double *b, double scale, double *acc, bool reset, double *part,
                void *stream);
// Moving bed: one step's bed adjoint zs [4][nc] (cell beds, then the face beds of
// faces 0..2) at time t -> uplift / onset gradients gU, gOn [nv] (+=), zb_total
// [4][nc] (+= zs), *tsum (+= the adjoint of t); vptr [nv+1], vcell: the cells
// around each vertex as (cell << 2) | the vertex's local index in it.
int adjoint_bed_flush(int nc, int nv, const int32_t *vptr, const int32_t *vcell, double *zs, const double *uplift,
                      const double *onset, double rise, double t, double *gU, double *gOn, double *zb_total,
                      double *tsum, double *part, void *stream);
// *y += *x on the device.
int adjoint_scalar_add(double *y, const double *x, void *stream);
int adjoint_stage1(int nc, double dt, double hthr, const double *w, const double *R0, double *w1, double *H1pre,
                   void *stream);
int adjoint_stage2_rev(int nc, double dt, const uint8_t *mask2, const double *wb, double *wbn, double *wb1,
                       double *Rb, void *stream);
int adjoint_stage1_rev(int nc, double dt, double hthr, const double *H1pre, const double *wb1, double *wbn,
                       double *Rb, void *stream);
int adjoint_gauge(int n_gauges, const int32_t *cells, const double *weights, int nc, double *wb, double *zb,
                  void *stream);

// Utility kernels (util_kernels.cu).
int launch_post_step(const DevPtrs &d, const StepParams &p, const void *w, int precision, void *stream);
int launch_record_gauges(const DevPtrs &d, const void *w, int precision, void *stream);
// Moving bed: sets z (and z64) to the bed at time t -- the end time of the step
// being taken (sc->t + its dt) when at_step_end, else t_set -- keeping the total
// depth H of the state w (NULL: no state to keep).
int launch_bed_update(const DevPtrs &d, const StepParams &p, void *w, int precision, bool at_step_end,
                      double t_set, void *stream);
int launch_import_state(const DevPtrs &d, const int32_t *old_of_new, const void *H, const void *Hu,
                        const void *Hv, int src_is_double, void *w, int precision, void *stream);
int launch_export_state(const DevPtrs &d, const int32_t *old_of_new, const void *w, int precision,
                        void *H, void *Hu, void *Hv, int dst_is_double, void *stream);
// The same from / to FP64 arrays in host order that the kernel may access in
// place (device memory or mapped pinned host memory), one thread per original
// cell: contiguous on the host-order side.
int launch_import_state_orig(const DevPtrs &d, const int32_t *new_of_old, const void *H, const void *Hu,
                             const void *Hv, int src_is_double, void *w, int precision, void *stream);
int launch_export_state_orig(const DevPtrs &d, const int32_t *new_of_old, const void *w, int precision, void *H,
                             void *Hu, void *Hv, int dst_is_double, void *stream);
// No-allocation step scratch (noalloc.cu): the device address and size of the
// file-scope scratch array on `device`, and the kernel that clears its scalars.
int noalloc_scratch(int device, void **addr, size_t *bytes);
int noalloc_launch_init(void *scalars, double t, int precision, void *stream);
// Set-up at mesh upload: resolves the scratch address on `device` and loads the
// no-allocation kernels (no launch), so that a later step loads nothing.
int noalloc_prepare(int device);
// Loads the epilogue kernels (util_kernels.cu) without launching them.
int util_preload();

int launch_diagnostics(const DevPtrs &d, const void *w, int precision, double hthr, double *part,
                       double *out, void *stream);

}  // namespace vg

struct vg_ctx;
namespace vg {
DevPtrs ctx_dev_ptrs(vg_ctx *c);
StepParams ctx_step_params(vg_ctx *c);
const HostMesh &ctx_host_mesh(vg_ctx *c);
const int32_t *ctx_old_of_new(vg_ctx *c);
int ctx_staging(vg_ctx *c, double **staging);
}  // namespace vg
