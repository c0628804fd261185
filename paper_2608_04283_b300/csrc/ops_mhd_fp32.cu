// Kernel launchers and dispatch table of MHD-GLM in FP32 (see vk_host.cuh;
// MHD-GLM's precisions compile as separate units, each is large).
#include "vk_host.cuh"

const Ops* vk_ops_mhd_fp32() { return ops_of<MHDGLM<float>, float, float, 2>(); }
