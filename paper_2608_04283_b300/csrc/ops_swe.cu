// Kernel launchers and dispatch table of one system (see vk_host.cuh).
#include "vk_host.cuh"

const Ops* vk_ops_swe(int dim, int prec) {
  return dim == 1 ? pick_prec<SWE, 1>(prec) : pick_prec<SWE, 2>(prec);
}
