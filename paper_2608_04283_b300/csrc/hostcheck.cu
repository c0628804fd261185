// Host-side evaluation of the device split functions, for CPU tests only.
//
// Builds libvklb_hostcheck.so.  It runs the same __host__ __device__ closed
// forms that the step kernels use (vk_systems.cuh) on the CPU so that tests can
// compare them with the FP64 oracle without a GPU.  It is not part of the
// simulation path: libvklb.so never calls it.
#include "vk_ctl.cuh"
#include "vk_systems.cuh"

namespace {
template <class Sys, class R>
void run(const Sys& sys, int d, int set, double k, double ch, const double* U, int64_t n,
         double* Fp, double* F, double* m1, double* m2) {
  const int P = Sys::P;
  for (int64_t i = 0; i < n; ++i) {
    R u[9], fp[9], f[9];
    for (int c = 0; c < P; ++c) u[c] = (R)U[c * n + i];
    sys.split(u, d, set, (R)k, (R)ch, fp, f);
    R a, b;
    sys.speeds(u, d, a, b);
    for (int c = 0; c < P; ++c) {
      Fp[c * n + i] = (double)fp[c];
      F[c * n + i] = (double)f[c];
    }
    m1[i] = (double)a;
    m2[i] = (double)b;
  }
}

template <class R>
int dispatch(int kind, int dim, int d, int set, double k, double lg, double ch, double gamma, double g,
             double ax, double ay, const double* U, int64_t n, double* Fp, double* F, double* m1,
             double* m2) {
  if (kind == 0) {
    if (dim == 1) { vk::Advect<R, 1> s; s.lg = (R)lg; s.a[0] = (R)ax; s.a[1] = (R)ay; run<vk::Advect<R, 1>, R>(s, d, set, k, ch, U, n, Fp, F, m1, m2); }
    else { vk::Advect<R, 2> s; s.lg = (R)lg; s.a[0] = (R)ax; s.a[1] = (R)ay; run<vk::Advect<R, 2>, R>(s, d, set, k, ch, U, n, Fp, F, m1, m2); }
  } else if (kind == 1) {
    if (dim == 1) { vk::SWE<R, 1> s; s.lg = (R)lg; s.g = (R)g; run<vk::SWE<R, 1>, R>(s, d, set, k, ch, U, n, Fp, F, m1, m2); }
    else { vk::SWE<R, 2> s; s.lg = (R)lg; s.g = (R)g; run<vk::SWE<R, 2>, R>(s, d, set, k, ch, U, n, Fp, F, m1, m2); }
  } else if (kind == 2) {
    if (dim == 1) { vk::Euler<R, 1> s; s.lg = (R)lg; s.gamma = (R)gamma; run<vk::Euler<R, 1>, R>(s, d, set, k, ch, U, n, Fp, F, m1, m2); }
    else { vk::Euler<R, 2> s; s.lg = (R)lg; s.gamma = (R)gamma; run<vk::Euler<R, 2>, R>(s, d, set, k, ch, U, n, Fp, F, m1, m2); }
  } else if (kind == 3) {
    if (dim != 2) return -8;
    vk::MHDGLM<R> s; s.lg = (R)lg; s.gamma = (R)gamma; run<vk::MHDGLM<R>, R>(s, d, set, k, ch, U, n, Fp, F, m1, m2);
  } else {
    return -1;
  }
  return 0;
}
}  // namespace

// lg: alpha's normaliser, 0 for the cell's own max |lambda|, else this grid-wide value.
extern "C" int vklb_hc_split(int kind, int dim, int d, int precision, int set, double k, double lg, double ch,
                             double gamma, double g, double ax, double ay, const double* U,
                             int64_t n, double* Fp, double* F, double* m1, double* m2) {
  if (precision == 0) return dispatch<double>(kind, dim, d, set, k, lg, ch, gamma, g, ax, ay, U, n, Fp, F, m1, m2);
  return dispatch<float>(kind, dim, d, set, k, lg, ch, gamma, g, ax, ay, U, n, Fp, F, m1, m2);
}

// Characteristic-boundary right-hand side P diag(lambda_j outgoing) P^-1 dU of the
// 1D systems (Eqs. 33-35) at n states; U, dU, out: [p][n].
namespace {
template <class Sys, class R>
void run_bc(const Sys& sys, const double* U, const double* dU, int side, int64_t n, double* out) {
  const int P = Sys::P;
  for (int64_t i = 0; i < n; ++i) {
    R u[3], du[3], o[3];
    for (int c = 0; c < P; ++c) {
      u[c] = (R)U[c * n + i];
      du[c] = (R)dU[c * n + i];
    }
    sys.char_rhs(u, du, side, o);
    for (int c = 0; c < P; ++c) out[c * n + i] = (double)o[c];
  }
}
template <class R>
int bc_dispatch(int kind, int side, double gamma, double g, double ax, const double* U, const double* dU, int64_t n,
                double* out) {
  const double lg = 0.0;
  if (kind == 0) { vk::Advect<R, 1> s; s.lg = (R)lg; s.a[0] = (R)ax; s.a[1] = 0; run_bc<vk::Advect<R, 1>, R>(s, U, dU, side, n, out); }
  else if (kind == 1) { vk::SWE<R, 1> s; s.lg = (R)lg; s.g = (R)g; run_bc<vk::SWE<R, 1>, R>(s, U, dU, side, n, out); }
  else if (kind == 2) { vk::Euler<R, 1> s; s.lg = (R)lg; s.gamma = (R)gamma; run_bc<vk::Euler<R, 1>, R>(s, U, dU, side, n, out); }
  else return -8;
  return 0;
}
}  // namespace

extern "C" int vklb_hc_char_rhs(int kind, int precision, int side, double gamma, double g, double ax,
                                const double* U, const double* dU, int64_t n, double* out) {
  if (precision == 0) return bc_dispatch<double>(kind, side, gamma, g, ax, U, dU, n, out);
  return bc_dispatch<float>(kind, side, gamma, g, ax, U, dU, n, out);
}

// Both-direction split and the step epilogue of the 2D systems, as the step
// kernels call them: Fp1, F1, Fp2, F2 [p][n]; m1, m2 [n]; ok[n] = physical.
namespace {
template <class Sys, class R>
void run2(const Sys& sys, int set, double k, double ch, const double* U, int64_t n, double* Fp1, double* F1,
          double* Fp2, double* F2, double* m1, double* m2, int* ok) {
  const int P = Sys::P;
  for (int64_t i = 0; i < n; ++i) {
    R u[9], a[9], b[9], c[9], d[9];
    for (int q = 0; q < P; ++q) u[q] = (R)U[q * n + i];
    sys.split2(u, set, (R)k, (R)ch, a, b, c, d);
    R e1, e2;
    ok[i] = sys.epilogue(u, e1, e2) ? 1 : 0;
    for (int q = 0; q < P; ++q) {
      Fp1[q * n + i] = (double)a[q];
      F1[q * n + i] = (double)b[q];
      Fp2[q * n + i] = (double)c[q];
      F2[q * n + i] = (double)d[q];
    }
    m1[i] = (double)e1;
    m2[i] = (double)e2;
  }
}
template <class R>
int dispatch2(int kind, int set, double k, double lg, double ch, double gamma, double g, double ax, double ay,
              const double* U, int64_t n, double* Fp1, double* F1, double* Fp2, double* F2, double* m1, double* m2, int* ok) {
  if (kind == 0) { vk::Advect<R, 2> s; s.lg = (R)lg; s.a[0] = (R)ax; s.a[1] = (R)ay; run2<vk::Advect<R, 2>, R>(s, set, k, ch, U, n, Fp1, F1, Fp2, F2, m1, m2, ok); }
  else if (kind == 1) { vk::SWE<R, 2> s; s.lg = (R)lg; s.g = (R)g; run2<vk::SWE<R, 2>, R>(s, set, k, ch, U, n, Fp1, F1, Fp2, F2, m1, m2, ok); }
  else if (kind == 2) { vk::Euler<R, 2> s; s.lg = (R)lg; s.gamma = (R)gamma; run2<vk::Euler<R, 2>, R>(s, set, k, ch, U, n, Fp1, F1, Fp2, F2, m1, m2, ok); }
  else if (kind == 3) { vk::MHDGLM<R> s; s.lg = (R)lg; s.gamma = (R)gamma; run2<vk::MHDGLM<R>, R>(s, set, k, ch, U, n, Fp1, F1, Fp2, F2, m1, m2, ok); }
  else return -1;
  return 0;
}
}  // namespace

extern "C" int vklb_hc_split2(int kind, int precision, int set, double k, double lg, double ch, double gamma,
                              double g, double ax, double ay, const double* U, int64_t n, double* Fp1, double* F1,
                              double* Fp2, double* F2, double* m1, double* m2, int* ok) {
  if (precision == 0)
    return dispatch2<double>(kind, set, k, lg, ch, gamma, g, ax, ay, U, n, Fp1, F1, Fp2, F2, m1, m2, ok);
  return dispatch2<float>(kind, set, k, lg, ch, gamma, g, ax, ay, U, n, Fp1, F1, Fp2, F2, m1, m2, ok);
}

// Characteristic-boundary right-hand side along direction d of the 2D systems
// (the construction of Eqs. 33-35 applied per face), at n states; U, dU, out: [p][n].
namespace {
template <class Sys, class R>
void run_bc2(const Sys& sys, const double* U, const double* dU, int d, int side, double ch, int64_t n,
             double* out) {
  const int P = Sys::P;
  for (int64_t i = 0; i < n; ++i) {
    R u[9], du[9], o[9];
    for (int c = 0; c < P; ++c) {
      u[c] = (R)U[c * n + i];
      du[c] = (R)dU[c * n + i];
    }
    sys.char_rhs_d(u, du, d, side, (R)ch, o);
    for (int c = 0; c < P; ++c) out[c * n + i] = (double)o[c];
  }
}
template <class R>
int bc2_dispatch(int kind, int d, int side, double gamma, double g, double ax, double ay, double ch,
                 const double* U, const double* dU, int64_t n, double* out) {
  const double lg = 0.0;
  if (kind == 0) { vk::Advect<R, 2> s; s.lg = (R)lg; s.a[0] = (R)ax; s.a[1] = (R)ay; run_bc2<vk::Advect<R, 2>, R>(s, U, dU, d, side, ch, n, out); }
  else if (kind == 1) { vk::SWE<R, 2> s; s.lg = (R)lg; s.g = (R)g; run_bc2<vk::SWE<R, 2>, R>(s, U, dU, d, side, ch, n, out); }
  else if (kind == 2) { vk::Euler<R, 2> s; s.lg = (R)lg; s.gamma = (R)gamma; run_bc2<vk::Euler<R, 2>, R>(s, U, dU, d, side, ch, n, out); }
  else if (kind == 3) { vk::MHDGLM<R> s; s.lg = (R)lg; s.gamma = (R)gamma; run_bc2<vk::MHDGLM<R>, R>(s, U, dU, d, side, ch, n, out); }
  else return -8;
  return 0;
}
}  // namespace

// ch: the cleaning speed c_h (MHD-GLM only)
extern "C" int vklb_hc_char_rhs2d(int kind, int precision, int d, int side, double gamma, double g, double ax,
                                  double ay, double ch, const double* U, const double* dU, int64_t n, double* out) {
  if (precision == 0) return bc2_dispatch<double>(kind, d, side, gamma, g, ax, ay, ch, U, dU, n, out);
  return bc2_dispatch<float>(kind, d, side, gamma, g, ax, ay, ch, U, dU, n, out);
}

// The enumeration of the characteristic faces' nodes that the boundary passes
// use (one thread a node): xs, ys receive char_face_nodes() coordinates.
extern "C" int vklb_hc_char_faces(int nx, int ny, int cbx, int cby, int* xs, int* ys, int cap) {
  const int nb = vk::char_face_nodes(nx, ny, cbx, cby);
  if (nb > cap) return -1;
  for (int id = 0; id < nb; ++id) vk::char_face_node(id, nx, ny, cbx, cby, xs[id], ys[id]);
  return nb;
}
