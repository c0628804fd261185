// Kernel launchers and dispatch table of MHD-GLM in BF16 storage (see vk_host.cuh;
// MHD-GLM's precisions compile as separate units, each is large).
#include "vk_host.cuh"

const Ops* vk_ops_mhd_bf16() { return ops_of<MHDGLM<float>, __nv_bfloat16, float, 2>(); }
