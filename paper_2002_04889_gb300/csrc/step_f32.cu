// FP32 instantiation of the step kernels (multiply-add contraction allowed).
#include "step_kernels.cuh"

namespace vg {
int stage_config_f32(const DevPtrs &d, int stage, LaunchCfg &cfg) { return stage_config<float>(d, stage, cfg); }
int launch_stage1_f32(const DevPtrs &d, const StepParams &p, const void *w_in, const LaunchCfg &c, void *stream)
{
    return launch_stage<float>(d, p, 1, w_in, nullptr, c, stream);
}
int launch_stage2_f32(const DevPtrs &d, const StepParams &p, const void *w_in, void *w_out, const LaunchCfg &c, void *stream)
{
    return launch_stage<float>(d, p, 2, w_in, w_out, c, stream);
}
}  // namespace vg
