// Device-resident control words of one simulation and the per-step scalars
// (lattice speed xi, cleaning speed c_h, time t) derived from them.
#pragma once
#include "vk_math.cuh"

namespace vk {

// Three rotating slots: step n reads slot n % 3 (maxima over U^n, t^n), reduces
// the maxima over U^{n+1} into slot (n+1) % 3 and clears slot (n+2) % 3, whose
// last reader was step n-1 (already finished: kernel boundary).
struct Ctl {
  unsigned long long m1[3];  // max over cells and directions of max_j |lambda_j| (no cleaning waves), double bits
  unsigned long long m2[3];  // MHD-GLM: max over cells and directions of c_f, double bits
  double t[3];               // time at the start of the step that reads the slot
  double xi_used[3];         // xi of the step that read the slot (for host queries)
  long long nsteps;          // steps taken (launches that reached t_end do not count)
  int32_t err;               // bit 0: non-physical state; bit 1: CFL violated (fixed xi)
  int32_t pad;
};

enum : int { ERR_NONPHYS = 1, ERR_CFL = 2, ERR_TIMEOUT = 4 };

struct StepScalars {
  double xi;   // lattice speed of this step
  double xinv; // 1 / xi
  double ch;   // cleaning speed of this step (MHD-GLM)
  double lam;  // max over the grid of max_j |lambda_j(U^n)| (with +-c_h for MHD-GLM)
  bool done;   // t_end reached: nothing to do
};

// xi of Eq. (29) (or the fixed xi); c_h = ch_factor * max c_f over the grid,
// refreshed every step with xi (the paper fixes neither the factor's use nor the
// refresh); and the landing rule of vklb_step_to, which the paper does not
// state: every remaining step takes xi_eff = m dx / (t_end - t) with
// m = ceil((t_end - t) xi / dx), so the steps stay evenly spread and the last
// ends on t_end.  Every thread of every block evaluates it from the same words,
// so all agree.
VK_HD StepScalars step_scalars(const Ctl* ctl, int slot, bool mhd, double ch_factor, double inv_nu,
                               double fixed_xi, double t_end, double dx) {
  StepScalars s;
  double m1 = bits_to_double(ctl->m1[slot]);
  double m2 = bits_to_double(ctl->m2[slot]);
  s.ch = mhd ? ch_factor * m2 : 0.0;
  double lam = mhd ? fmax(m1, s.ch) : m1;
  s.lam = lam;
  s.xi = fixed_xi > 0.0 ? fixed_xi : lam * inv_nu;
  s.done = false;
  if (t_end > 0.0) {
    double rem = t_end - ctl->t[slot];
    if (rem <= 1e-14 * fmax(1.0, fabs(t_end))) {
      s.done = true;
    } else {
      double m = ceil(rem * s.xi / dx - 1e-9);
      if (m < 1.0) m = 1.0;
      s.xi = m * dx / rem;
    }
  }
  s.xinv = 1.0 / s.xi;
  return s;
}

// Nodes of the characteristic faces of a 2D grid (cbx: the two x faces, cby:
// the two y faces), numbered for one thread each: the x faces' columns first
// (2 ny nodes, corners included), then the y faces' rows without those corners.
VK_HD int char_face_nodes(int nx, int ny, int cbx, int cby) {
  return (cbx ? 2 * ny : 0) + (cby ? 2 * (nx - (cbx ? 2 : 0)) : 0);
}
VK_HD void char_face_node(int id, int nx, int ny, int cbx, int cby, int& x, int& y) {
  if (cbx) {
    if (id < 2 * ny) {
      x = id < ny ? 0 : nx - 1;
      y = id < ny ? id : id - ny;
      return;
    }
    id -= 2 * ny;
  }
  const int w = nx - (cbx ? 2 : 0), x0 = cbx ? 1 : 0;
  y = id < w ? 0 : ny - 1;
  x = x0 + (id < w ? id : id - w);
}

}  // namespace vk
