// Kernel launchers and dispatch table of one system (see vk_host.cuh).
#include "vk_host.cuh"

const Ops* vk_ops_euler(int dim, int prec) {
  return dim == 1 ? pick_prec<Euler, 1>(prec) : pick_prec<Euler, 2>(prec);
}
