// MHD-GLM dispatch by precision (the three tables are in ops_mhd_*.cu).
#include "vk_host.cuh"

const Ops* vk_ops_mhd_fp64();
const Ops* vk_ops_mhd_fp32();
const Ops* vk_ops_mhd_bf16();

const Ops* vk_ops_mhd(int dim, int prec) {
  if (dim != 2) return nullptr;
  if (prec == VKLB_FP64) return vk_ops_mhd_fp64();
  if (prec == VKLB_FP32) return vk_ops_mhd_fp32();
  return vk_ops_mhd_bf16();
}
