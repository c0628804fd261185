// Kernel launchers and dispatch table of MHD-GLM in FP64 (see vk_host.cuh;
// MHD-GLM's precisions compile as separate units, each is large).
#include "vk_host.cuh"

const Ops* vk_ops_mhd_fp64() { return ops_of<MHDGLM<double>, double, double, 2>(); }
