// FP64 instantiation of the step kernels.  Built with --fmad=false: no
// multiply-add contraction, every expression rounds as written.
#include "step_kernels.cuh"

namespace vg {
size_t stage_smem_f64(int block, int max_halo, int max_ring1) { return stage_smem_bytes<double>(block, max_halo, max_ring1); }
int stage_config_f64(const DevPtrs &d, int stage, LaunchCfg &cfg) { return stage_config<double>(d, stage, cfg); }
int launch_stage1_f64(const DevPtrs &d, const StepParams &p, const void *w_in, const LaunchCfg &c, void *stream)
{
    return launch_stage<double>(d, p, 1, w_in, nullptr, c, stream);
}
int launch_stage2_f64(const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, const LaunchCfg &c, void *stream)
{
    return launch_stage<double>(d, p, 2, w_in, w_out, c, stream);
}
size_t batch_mesh_bytes_f64() { return sizeof(BatchMesh<double>); }
void fill_batch_mesh_f64(void *dst, const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, int n_scen,
                         int first_item, int first_entry)
{
    fill_batch_mesh<double>(dst, d, p, w_in, w_out, n_scen, first_item, first_entry);
}
int batch_config_f64(int block, int max_halo, int max_ring1, int &grid, size_t &smem)
{
    return batch_config<double>(block, max_halo, max_ring1, grid, smem);
}
int launch_batch_step_f64(const void *table, int n_mesh, int n_items, int n_entries, DevScalars *sc_all, int block,
                          int grid, size_t smem, const StepParams &p, bool gauges, void *stream)
{
    return launch_batch_step<double>(table, n_mesh, n_items, n_entries, sc_all, block, grid, smem, p, gauges, stream);
}
}  // namespace vg
