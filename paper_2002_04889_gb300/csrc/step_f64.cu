// FP64 instantiation of the step kernels.  Built with --fmad=false: no
// multiply-add contraction, every expression rounds as written.
#include "step_kernels.cuh"

namespace vg {
int stage_config_f64(const DevPtrs &d, int stage, LaunchCfg &cfg) { return stage_config<double>(d, stage, cfg); }
int launch_stage1_f64(const DevPtrs &d, const StepParams &p, const void *w_in, const LaunchCfg &c, void *stream)
{
    return launch_stage<double>(d, p, 1, w_in, nullptr, c, stream);
}
int launch_stage2_f64(const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, const LaunchCfg &c, void *stream)
{
    return launch_stage<double>(d, p, 2, w_in, w_out, c, stream);
}
}  // namespace vg
