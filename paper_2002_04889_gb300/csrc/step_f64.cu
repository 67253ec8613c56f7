// FP64 instantiation of the step kernels, literal form.  Built with
// --fmad=false: no multiply-add contraction, every expression rounds as
// written.  Its entry points dispatch to the contracted build
// (step_f64_fast.cu) when the context asks for it.
#include "step_kernels.cuh"

namespace vg {
size_t stage_smem_f64(int block, int max_halo, int max_ring1) { return stage_smem_bytes<double>(block, max_halo, max_ring1); }
int stage_config_f64(const DevPtrs &d, int stage, LaunchCfg &cfg)
{
    if (d.fp64_fast) return stage_config_f64_fast(d, stage, cfg);
    return stage_config<double, false>(d, stage, cfg);
}
int launch_stage1_f64(const DevPtrs &d, const StepParams &p, const void *w_in, const LaunchCfg &c, void *stream)
{
    if (d.fp64_fast) return launch_stage1_f64_fast(d, p, w_in, c, stream);
    return launch_stage<double, false>(d, p, 1, w_in, nullptr, c, stream);
}
int launch_stage2_f64(const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, const LaunchCfg &c, void *stream)
{
    if (d.fp64_fast) return launch_stage2_f64_fast(d, p, w_in, w_out, c, stream);
    return launch_stage<double, false>(d, p, 2, w_in, w_out, c, stream);
}
int launch_rk_unfused_f64(const DevPtrs &d, const StepParams &p, int part, const void *w_in, void *w_out, void *w1,
                          void *R1, const LaunchCfg &c1, void *stream)
{
    if (d.fp64_fast) return launch_rk_unfused_f64_fast(d, p, part, w_in, w_out, w1, R1, c1, stream);
    return launch_rk_unfused<double, false>(d, p, part, w_in, w_out, w1, R1, c1, stream);
}
size_t batch_mesh_bytes_f64() { return sizeof(BatchMesh<double>); }
void fill_batch_mesh_f64(void *dst, const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, int n_scen,
                         int first_item, int first_entry)
{
    fill_batch_mesh<double>(dst, d, p, w_in, w_out, n_scen, first_item, first_entry);
}
int batch_config_f64(int block, int max_halo, int max_ring1, int &grid, size_t &smem, bool fast)
{
    if (fast) return batch_config_f64_fast(block, max_halo, max_ring1, grid, smem);
    return batch_config<double, false>(block, max_halo, max_ring1, grid, smem);
}
int launch_batch_step_f64(const void *table, int n_mesh, int n_items, int n_entries, DevScalars *sc_all, int block,
                          int grid, size_t smem, const StepParams &p, bool gauges, void *stream)
{
    if (p.fp64_fast)
        return launch_batch_step_f64_fast(table, n_mesh, n_items, n_entries, sc_all, block, grid, smem, p, gauges,
                                          stream);
    return launch_batch_step<double, false>(table, n_mesh, n_items, n_entries, sc_all, block, grid, smem, p, gauges,
                                            stream);
}
}  // namespace vg
