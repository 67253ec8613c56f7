// FP32 instantiation of the step kernels (multiply-add contraction allowed).
#include "step_kernels.cuh"

namespace vg {
size_t stage_smem_f32(int block, int max_halo, int max_ring1) { return stage_smem_bytes<float>(block, max_halo, max_ring1); }
int stage_config_f32(const DevPtrs &d, int stage, LaunchCfg &cfg) { return stage_config<float>(d, stage, cfg); }
int launch_stage1_f32(const DevPtrs &d, const StepParams &p, const void *w_in, const LaunchCfg &c, void *stream)
{
    return launch_stage<float>(d, p, 1, w_in, nullptr, c, stream);
}
int launch_stage2_f32(const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, const LaunchCfg &c, void *stream)
{
    return launch_stage<float>(d, p, 2, w_in, w_out, c, stream);
}
int launch_rk_unfused_f32(const DevPtrs &d, const StepParams &p, int part, const void *w_in, void *w_out, void *w1,
                          void *R1, const LaunchCfg &c1, void *stream)
{
    return launch_rk_unfused<float>(d, p, part, w_in, w_out, w1, R1, c1, stream);
}
size_t batch_mesh_bytes_f32() { return sizeof(BatchMesh<float>); }
void fill_batch_mesh_f32(void *dst, const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, int n_scen,
                         int first_item, int first_entry)
{
    fill_batch_mesh<float>(dst, d, p, w_in, w_out, n_scen, first_item, first_entry);
}
int batch_config_f32(int block, int max_halo, int max_ring1, int &grid, size_t &smem)
{
    return batch_config<float>(block, max_halo, max_ring1, grid, smem);
}
int launch_batch_step_f32(const void *table, int n_mesh, int n_items, int n_entries, DevScalars *sc_all, int block,
                          int grid, size_t smem, const StepParams &p, bool gauges, void *stream)
{
    return launch_batch_step<float>(table, n_mesh, n_items, n_entries, sc_all, block, grid, smem, p, gauges, stream);
}
}  // namespace vg
