// FP64 instantiation of the step kernels, contracted form (FAST = true): built
// without --fmad=false, so the compiler may fuse multiplies and adds, and the
// kernels divide once where the literal form divides several times by the same
// value.  Reached through the *_f64 entry points of step_f64.cu.
#include "step_kernels.cuh"

namespace vg {
int stage_config_f64_fast(const DevPtrs &d, int stage, LaunchCfg &cfg) { return stage_config<double, true>(d, stage, cfg); }
int launch_stage1_f64_fast(const DevPtrs &d, const StepParams &p, const void *w_in, const LaunchCfg &c, void *stream)
{
    return launch_stage<double, true>(d, p, 1, w_in, nullptr, c, stream);
}
int launch_stage2_f64_fast(const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, const LaunchCfg &c,
                           void *stream)
{
    return launch_stage<double, true>(d, p, 2, w_in, w_out, c, stream);
}
int launch_rk_unfused_f64_fast(const DevPtrs &d, const StepParams &p, int part, const void *w_in, void *w_out,
                               void *w1, void *R1, const LaunchCfg &c1, void *stream)
{
    return launch_rk_unfused<double, true>(d, p, part, w_in, w_out, w1, R1, c1, stream);
}
int batch_config_f64_fast(int block, int max_halo, int max_ring1, int &grid, size_t &smem)
{
    return batch_config<double, true>(block, max_halo, max_ring1, grid, smem);
}
int launch_batch_step_f64_fast(const void *table, int n_mesh, int n_items, int n_entries, DevScalars *sc_all,
                               int block, int grid, size_t smem, const StepParams &p, bool gauges, void *stream)
{
    return launch_batch_step<double, true>(table, n_mesh, n_items, n_entries, sc_all, block, grid, smem, p, gauges,
                                           stream);
}
}  // namespace vg
