// Kernel launchers and dispatch table of one system (see vk_host.cuh).
#include "vk_host.cuh"

const Ops* vk_ops_advect(int dim, int prec) {
  return dim == 1 ? pick_prec<Advect, 1>(prec) : pick_prec<Advect, 2>(prec);
}
