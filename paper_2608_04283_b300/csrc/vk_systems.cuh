// Hyperbolic systems and their weighted upwind flux splitting, closed form.
//
// For each system, split(U, d) returns the physical flux F = F^(d)(U) and
//     F+ = sum_j alpha(lambda_j) phi_j r_j,   phi = P^-1 F          (Eqs. 16, 25, 26)
// with alpha of Eq. (27) normalised by max_j |lambda_j|; F- = F - F+ (Eq. 11).
// Over what that maximum runs the paper leaves open: each system carries `lg`,
// 0 for the cell's own maximum along the direction, or the grid-wide maximum of
// the step (the number Eq. 29 divides by nu) for every cell.  The
// eigen-structures are written in closed form:
//   * shallow water (Eq. 52): r = (1, u -+ c, v), phi_{1,3} = h (u -+ c/2) / 2, and
//     the shear wave carries no flux (phi_2 = 0);
//   * Euler (Eq. 54): homogeneous of degree one, so phi_j = lambda_j l_j.U and
//     F+ = rho/(2 gamma) [w1 (1, u-a, v, H-ua) + 2(gamma-1) w2 (1, u, v, q^2/2)
//                         + w3 (1, u+a, v, H+ua)],  w_j = alpha_j lambda_j;
//   * MHD-GLM (Eq. 58): the 9x9 Jacobian is block upper triangular in
//     (rho, m, E, B_t | B_n, psi).  The 7 MHD waves use primitive eigenvectors
//     with the Roe-Balsara normalisation (alpha_f, alpha_s, beta); the two
//     cleaning waves +-c_h have phi_+- = (psi +- c_h B_n)/2, and their coupling to
//     the MHD block enters through divided differences of alpha (see split_x).
// The y direction is the x direction applied to the state with x and y swapped.
#pragma once
#include "vk_math.cuh"

namespace vk {

// alpha's normaliser: the grid-wide lg when set, else the cell's own maximum
template <class R>
VK_HD R lam_norm(R lg, R local) {
  return lg > R(0) ? lg : local;
}

// ----------------------------------------------------------------- advection
template <class R, int DIM>
struct Advect {
  static constexpr int P = 1;
  static constexpr bool MHD = false;
  R a[2];
  R lg;   // alpha's normaliser: 0 = per cell and direction, else this grid-wide value
  VK_HD void split(const R* U, int d, int set, R k, R ch, R* Fp, R* F) const {
    R ad = a[d];
    F[0] = ad * U[0];
    R lm = lam_norm(lg, vabs(ad));
    R al = lm > R(0) ? alpha_w(ad, k / lm, set) : R(0.5);
    Fp[0] = al * F[0];
  }
  // m1: max |lambda| along d; m2: unused (fast speed of MHD)
  VK_HD void speeds(const R* U, int d, R& m1, R& m2) const { m1 = vabs(a[d]); m2 = R(0); }
  VK_HD bool physical(const R* U) const { return U[0] == U[0]; }
  VK_HD void split2(const R* U, int set, R k, R ch, R* Fp1, R* F1, R* Fp2, R* F2) const {
    split(U, 0, set, k, ch, Fp1, F1);
    split(U, 1, set, k, ch, Fp2, F2);
  }
  // CFL maxima over both directions and the physical-state test of U^{n+1}
  VK_HD bool epilogue(const R* U, R& m1, R& m2) const {
    m1 = vmax(vabs(a[0]), vabs(a[1]));
    m2 = R(0);
    return U[0] == U[0];
  }
  // Characteristic boundary (Eqs. 33-35): P diag(lambda_j, outgoing only) P^-1 dU.
  VK_HD void char_rhs(const R* U, const R* dU, int side, R* out) const {
    R l = a[0];
    bool out_going = side == 0 ? l < R(0) : l > R(0);
    out[0] = out_going ? l * dU[0] : R(0);
  }
  // The same along direction d of a 2D grid (a face normal to d).
  VK_HD void char_rhs_d(const R* U, const R* dU, int d, int side, R /*ch*/, R* out) const {
    R l = a[d];
    bool out_going = side == 0 ? l < R(0) : l > R(0);
    out[0] = out_going ? l * dU[0] : R(0);
  }
};

// ------------------------------------------------------------- shallow water
template <class R, int DIM>
struct SWE {
  static constexpr int P = DIM + 1;
  static constexpr bool MHD = false;
  R g;
  R lg;   // alpha's normaliser: 0 = per cell and direction, else this grid-wide value
  VK_HD void split(const R* U, int d, int set, R k, R ch, R* Fp, R* F) const {
    const int in = 1 + d;           // normal momentum
    const int it = 2 - d;           // tangential momentum (2D)
    R h = U[0];
    R ih = vrcp(h);
    R un = U[in] * ih;
    R c = vsqrt(g * h);
    F[0] = U[in];
    F[in] = U[in] * un + R(0.5) * g * h * h;
    R ut = R(0);
    if (DIM == 2) {
      ut = U[it] * ih;
      F[it] = U[in] * ut;
    }
    if (set == SET_CENTERED) {
      for (int i = 0; i < P; ++i) Fp[i] = R(0.5) * F[i];
      return;
    }
    R lmax = lam_norm(lg, vabs(un) + c);
    R kl = k * vrcp(lmax);
    R a1 = alpha_w(un - c, kl, set);
    R a3 = alpha_w(un + c, kl, set);
    R p1 = a1 * R(0.5) * h * (un - R(0.5) * c);   // alpha_1 phi_1
    R p3 = a3 * R(0.5) * h * (un + R(0.5) * c);   // alpha_3 phi_3
    Fp[0] = p1 + p3;
    Fp[in] = p1 * (un - c) + p3 * (un + c);
    if (DIM == 2) Fp[it] = (p1 + p3) * ut;
  }
  VK_HD void speeds(const R* U, int d, R& m1, R& m2) const {
    R h = U[0];
    m1 = vabs(U[1 + d] / h) + vsqrt(g * h);
    m2 = R(0);
  }
  VK_HD bool physical(const R* U) const { return U[0] > R(0); }
  // Both directions with shared primitives (2D).
  VK_HD void split2(const R* U, int set, R k, R ch, R* Fp1, R* F1, R* Fp2, R* F2) const {
    const R h = U[0], ih = vrcp(h);
    const R u = U[1] * ih, v = U[DIM == 2 ? 2 : 1] * ih;
    const R c = vsqrt(g * h);
    const R hh = R(0.5) * g * h * h;
    F1[0] = U[1];
    F1[1] = U[1] * u + hh;
    F2[0] = U[2];
    F2[2] = U[2] * v + hh;
    F1[2] = U[1] * v;
    F2[1] = U[2] * u;
    if (set == SET_CENTERED) {
      for (int i = 0; i < P; ++i) {
        Fp1[i] = R(0.5) * F1[i];
        Fp2[i] = R(0.5) * F2[i];
      }
      return;
    }
    const R hc = R(0.25) * h * c;   // h c / 4
    const R hu2 = R(0.5) * U[1], hv2 = R(0.5) * U[2];
    {
      const R kl = k * vrcp(lam_norm(lg, vabs(u) + c));
      const R p1 = alpha_w(u - c, kl, set) * (hu2 - hc);
      const R p3 = alpha_w(u + c, kl, set) * (hu2 + hc);
      const R ps = p1 + p3;
      Fp1[0] = ps;
      Fp1[1] = ps * u + (p3 - p1) * c;
      Fp1[2] = ps * v;
    }
    {
      const R kl = k * vrcp(lam_norm(lg, vabs(v) + c));
      const R p1 = alpha_w(v - c, kl, set) * (hv2 - hc);
      const R p3 = alpha_w(v + c, kl, set) * (hv2 + hc);
      const R ps = p1 + p3;
      Fp2[0] = ps;
      Fp2[2] = ps * v + (p3 - p1) * c;
      Fp2[1] = ps * u;
    }
  }
  VK_HD bool epilogue(const R* U, R& m1, R& m2) const {
    const R h = U[0], ih = vrcp(h);
    m1 = vmax(vabs(U[1] * ih), vabs(U[DIM == 2 ? 2 : 1] * ih)) + vsqrt(g * h);
    m2 = R(0);
    return h > R(0);
  }
  // Characteristic boundary (Eqs. 33-35), 1D: P diag(lambda_j, outgoing only) P^-1 dU
  // with r_{1,2} = (1, u -+ c), l_1 = (u + c, -1)/(2c), l_2 = (c - u, 1)/(2c).
  VK_HD void char_rhs(const R* U, const R* dU, int side, R* out) const {
    R h = U[0], u = U[1] / h, c = vsqrt(g * h);
    R i2c = R(0.5) / c;
    R w1 = ((u + c) * dU[0] - dU[1]) * i2c;
    R w2 = ((c - u) * dU[0] + dU[1]) * i2c;
    R l1 = u - c, l2 = u + c;
    R k1 = (side == 0 ? l1 < R(0) : l1 > R(0)) ? l1 * w1 : R(0);
    R k2 = (side == 0 ? l2 < R(0) : l2 > R(0)) ? l2 * w2 : R(0);
    out[0] = k1 + k2;
    out[1] = k1 * l1 + k2 * l2;
  }
  // 2D, along direction d (normal momentum n = 1 + d, tangential t = 2 - d):
  // r = (1, u_n - c, u_t), (0, 0, 1) (shear, lambda = u_n), (1, u_n + c, u_t);
  // dual rows ((u_n + c), -1, 0)/(2c), (-u_t, 0, 1), ((c - u_n), 1, 0)/(2c).
  VK_HD void char_rhs_d(const R* U, const R* dU, int d, int side, R /*ch*/, R* out) const {
    const int in = 1 + d, it = 2 - d;
    const R h = U[0], un = U[in] / h, ut = U[it] / h, c = vsqrt(g * h);
    const R i2c = R(0.5) / c;
    const R w1 = ((un + c) * dU[0] - dU[in]) * i2c;
    const R w2 = dU[it] - ut * dU[0];
    const R w3 = ((c - un) * dU[0] + dU[in]) * i2c;
    const R l1 = un - c, l2 = un, l3 = un + c;
    const R k1 = (side == 0 ? l1 < R(0) : l1 > R(0)) ? l1 * w1 : R(0);
    const R k2 = (side == 0 ? l2 < R(0) : l2 > R(0)) ? l2 * w2 : R(0);
    const R k3 = (side == 0 ? l3 < R(0) : l3 > R(0)) ? l3 * w3 : R(0);
    out[0] = k1 + k3;
    out[in] = k1 * l1 + k3 * l3;
    out[it] = (k1 + k3) * ut + k2;
  }
};

// ------------------------------------------------------------------- Euler
template <class R, int DIM>
struct Euler {
  static constexpr int P = DIM + 2;
  static constexpr bool MHD = false;
  R gamma;
  R lg;   // alpha's normaliser: 0 = per cell and direction, else this grid-wide value
  // Both directions with shared primitives (2D); w_j = alpha_j lambda_j as in split().
  VK_HD void split2(const R* U, int set, R k, R ch, R* Fp1, R* F1, R* Fp2, R* F2) const {
    const R rho = U[0], ir = vrcp(rho);
    const R u = U[1] * ir, v = U[2] * ir;
    const R q2 = u * u + v * v;
    const R E = U[3];
    const R gm1 = gamma - R(1);
    const R p = gm1 * (E - R(0.5) * rho * q2);
    const R Ep = E + p;
    F1[0] = U[1];
    F1[1] = U[1] * u + p;
    F1[2] = U[2] * u;
    F1[3] = u * Ep;
    F2[0] = U[2];
    F2[1] = U[1] * v;
    F2[2] = U[2] * v + p;
    F2[3] = v * Ep;
    if (set == SET_CENTERED) {
      for (int i = 0; i < 4; ++i) {
        Fp1[i] = R(0.5) * F1[i];
        Fp2[i] = R(0.5) * F2[i];
      }
      return;
    }
    const R a = vsqrt(gamma * p * ir);
    const R H = Ep * ir;
    const R s = R(0.5) * rho * vrcp(gamma);
    const R g2 = R(2) * gm1;
    const R hq = R(0.5) * q2;
    {
      const R kl = k * vrcp(lam_norm(lg, vabs(u) + a));
      const R l1 = u - a, l3 = u + a;
      const R w1 = alpha_w(l1, kl, set) * l1, w2 = alpha_w(u, kl, set) * u * g2, w3 = alpha_w(l3, kl, set) * l3;
      const R ws = s * (w1 + w2 + w3);
      Fp1[0] = ws;
      Fp1[1] = s * (w1 * l1 + w2 * u + w3 * l3);
      Fp1[2] = ws * v;
      Fp1[3] = s * ((w1 + w3) * H + (w3 - w1) * u * a + w2 * hq);
    }
    {
      const R kl = k * vrcp(lam_norm(lg, vabs(v) + a));
      const R l1 = v - a, l3 = v + a;
      const R w1 = alpha_w(l1, kl, set) * l1, w2 = alpha_w(v, kl, set) * v * g2, w3 = alpha_w(l3, kl, set) * l3;
      const R ws = s * (w1 + w2 + w3);
      Fp2[0] = ws;
      Fp2[2] = s * (w1 * l1 + w2 * v + w3 * l3);
      Fp2[1] = ws * u;
      Fp2[3] = s * ((w1 + w3) * H + (w3 - w1) * v * a + w2 * hq);
    }
  }
  VK_HD bool epilogue(const R* U, R& m1, R& m2) const {
    const R rho = U[0], ir = vrcp(rho);
    const R u = U[1] * ir, v = U[2] * ir;
    const R p = (gamma - R(1)) * (U[3] - R(0.5) * rho * (u * u + v * v));
    m1 = vmax(vabs(u), vabs(v)) + vsqrt(gamma * p * ir);
    m2 = R(0);
    return rho > R(0) && p > R(0);
  }
  VK_HD void split(const R* U, int d, int set, R k, R ch, R* Fp, R* F) const {
    const int in = 1 + d, it = 2 - d, ie = P - 1;
    R rho = U[0];
    R ir = vrcp(rho);
    R un = U[in] * ir;
    R ut = DIM == 2 ? U[it] * ir : R(0);
    R q2 = un * un + ut * ut;
    R E = U[ie];
    R p = (gamma - R(1)) * (E - R(0.5) * rho * q2);
    F[0] = U[in];
    F[in] = U[in] * un + p;
    if (DIM == 2) F[it] = U[it] * un;
    F[ie] = un * (E + p);
    if (set == SET_CENTERED) {
      for (int i = 0; i < P; ++i) Fp[i] = R(0.5) * F[i];
      return;
    }
    R a = vsqrt(gamma * p * ir);
    R H = (E + p) * ir;
    R lmax = lam_norm(lg, vabs(un) + a);
    R kl = k * vrcp(lmax);
    R l1 = un - a, l3 = un + a;
    R w1 = alpha_w(l1, kl, set) * l1;
    R w2 = alpha_w(un, kl, set) * un * R(2) * (gamma - R(1));
    R w3 = alpha_w(l3, kl, set) * l3;
    R s = R(0.5) * rho / gamma;
    R wsum = w1 + w2 + w3;
    Fp[0] = s * wsum;
    Fp[in] = s * (w1 * l1 + w2 * un + w3 * l3);
    if (DIM == 2) Fp[it] = s * wsum * ut;
    Fp[ie] = s * (w1 * (H - un * a) + w2 * R(0.5) * q2 + w3 * (H + un * a));
  }
  VK_HD void speeds(const R* U, int d, R& m1, R& m2) const {
    R rho = U[0];
    R un = U[1 + d] / rho;
    R ut = DIM == 2 ? U[2 - d] / rho : R(0);
    R p = (gamma - R(1)) * (U[P - 1] - R(0.5) * rho * (un * un + ut * ut));
    m1 = vabs(un) + vsqrt(gamma * p / rho);
    m2 = R(0);
  }
  VK_HD bool physical(const R* U) const {
    R rho = U[0];
    R ke = U[1] * U[1];
    if (DIM == 2) ke += U[2] * U[2];
    R p = (gamma - R(1)) * (U[P - 1] - R(0.5) * ke / rho);
    return rho > R(0) && p > R(0);
  }
  // Characteristic boundary (Eqs. 33-35), 1D Euler: r = (1, u-a, H-ua), (1, u, u^2/2),
  // (1, u+a, H+ua); with b1 = (gamma-1)/a^2, b2 = b1 u^2/2 the dual rows are
  // l1 = ((b2 + u/a), -(b1 u + 1/a), b1)/2, l2 = (1 - b2, b1 u, -b1),
  // l3 = ((b2 - u/a), -(b1 u - 1/a), b1)/2.
  VK_HD void char_rhs(const R* U, const R* dU, int side, R* out) const {
    R rho = U[0], u = U[1] / rho, E = U[2];
    R p = (gamma - R(1)) * (E - R(0.5) * rho * u * u);
    R a = vsqrt(gamma * p / rho), H = (E + p) / rho;
    R b1 = (gamma - R(1)) / (a * a), b2 = R(0.5) * u * u * b1, ia = R(1) / a;
    R w1 = R(0.5) * ((b2 + u * ia) * dU[0] - (b1 * u + ia) * dU[1] + b1 * dU[2]);
    R w2 = (R(1) - b2) * dU[0] + b1 * u * dU[1] - b1 * dU[2];
    R w3 = R(0.5) * ((b2 - u * ia) * dU[0] - (b1 * u - ia) * dU[1] + b1 * dU[2]);
    R lam[3] = {u - a, u, u + a};
    R k[3] = {w1, w2, w3};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      bool og = side == 0 ? lam[j] < R(0) : lam[j] > R(0);
      k[j] = og ? lam[j] * k[j] : R(0);
    }
    out[0] = k[0] + k[1] + k[2];
    out[1] = k[0] * (u - a) + k[1] * u + k[2] * (u + a);
    out[2] = k[0] * (H - u * a) + k[1] * R(0.5) * u * u + k[2] * (H + u * a);
  }
  // 2D, along direction d (normal n = 1 + d, tangential t = 2 - d), q^2 = u_n^2 + u_t^2:
  // r = (1, u_n - a, u_t, H - u_n a), (1, u_n, u_t, q^2/2) (entropy),
  // (0, 0, 1, u_t) (shear), (1, u_n + a, u_t, H + u_n a); with b1 = (gamma-1)/a^2,
  // b2 = b1 q^2/2 the dual rows are
  // ((b2 + u_n/a), -(b1 u_n + 1/a), -b1 u_t, b1)/2, (1 - b2, b1 u_n, b1 u_t, -b1),
  // (-u_t, 0, 1, 0), ((b2 - u_n/a), -(b1 u_n - 1/a), -b1 u_t, b1)/2.
  VK_HD void char_rhs_d(const R* U, const R* dU, int d, int side, R /*ch*/, R* out) const {
    const int in = 1 + d, it = 2 - d;
    const R rho = U[0], un = U[in] / rho, ut = U[it] / rho, E = U[3];
    const R q2 = un * un + ut * ut;
    const R p = (gamma - R(1)) * (E - R(0.5) * rho * q2);
    const R a = vsqrt(gamma * p / rho), H = (E + p) / rho;
    const R b1 = (gamma - R(1)) / (a * a), b2 = R(0.5) * q2 * b1, ia = R(1) / a;
    const R dr = dU[0], dn = dU[in], dt = dU[it], de = dU[3];
    R w[4];
    w[0] = R(0.5) * ((b2 + un * ia) * dr - (b1 * un + ia) * dn - b1 * ut * dt + b1 * de);
    w[1] = (R(1) - b2) * dr + b1 * un * dn + b1 * ut * dt - b1 * de;
    w[2] = dt - ut * dr;
    w[3] = R(0.5) * ((b2 - un * ia) * dr - (b1 * un - ia) * dn - b1 * ut * dt + b1 * de);
    const R lam[4] = {un - a, un, un, un + a};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool og = side == 0 ? lam[j] < R(0) : lam[j] > R(0);
      w[j] = og ? lam[j] * w[j] : R(0);
    }
    out[0] = w[0] + w[1] + w[3];
    out[in] = w[0] * (un - a) + w[1] * un + w[3] * (un + a);
    out[it] = (w[0] + w[1] + w[3]) * ut + w[2];
    out[3] = w[0] * (H - un * a) + w[1] * R(0.5) * q2 + w[2] * ut + w[3] * (H + un * a);
  }
};

// ----------------------------------------------------------------- MHD-GLM
// Fast-wave normalisation (alpha_f, alpha_s) of Roe & Balsara, computed from
//   d = c_f^2 - c_s^2 = sqrt((a^2 - bx^2)^2 + bt^2 (2 a^2 + 2 bx^2 + bt^2)),
// X = a^2 - c_s^2, Y = c_f^2 - a^2 with X Y = a^2 bt^2 (no cancellation):
//   alpha_f^2 = X / d, alpha_s^2 = Y / d.  At d = 0 (bt = 0, a = |bx|) all three
// speeds coincide and any basis of the eigenspace serves; alpha_f = alpha_s = 1/sqrt 2.
template <class T>
VK_HD void mhd_norm(T a2, T bx2, T bt2, T& af, T& as, T& d) {
  T dd = (a2 - bx2) * (a2 - bx2) + bt2 * (T(2) * a2 + T(2) * bx2 + bt2);
  d = vsqrt(dd);
  T b2 = bx2 + bt2;
  T X, Y;
  if (a2 >= b2) {
    X = T(0.5) * ((a2 - b2) + d);
    Y = X > T(0) ? a2 * bt2 * vrcp(X) : T(0);
  } else {
    Y = T(0.5) * ((b2 - a2) + d);
    X = Y > T(0) ? a2 * bt2 * vrcp(Y) : T(0);
  }
  if (d > T(0)) {
    const T id = vrcp(d);
    af = vsqrt(vmax(X * id, T(0)));
    as = vsqrt(vmax(Y * id, T(0)));
  } else {
    af = as = T(0.70710678118654752440);
  }
}

template <class R>
struct MHDGLM {
  static constexpr int P = 9;
  static constexpr bool MHD = true;
  R gamma;
  R lg;   // alpha's normaliser: 0 = per cell and direction, else this grid-wide value

  // Fast speed c_f along the normal whose field component is bn.
  VK_HD R fast(R rho, R p, R bn, R bb) const {
    R ir = R(1) / rho;
    R a2 = gamma * p * ir;
    R bx2 = bn * bn * ir;
    R bt2 = (bb - bn * bn) * ir;
    R dd = (a2 - bx2) * (a2 - bx2) + bt2 * (R(2) * a2 + R(2) * bx2 + bt2);
    return vsqrt(R(0.5) * (a2 + bx2 + bt2 + vsqrt(dd)));
  }

  VK_HD void speeds(const R* U, int d, R& m1, R& m2) const {
    R rho = U[0];
    R bb = U[5] * U[5] + U[6] * U[6] + U[7] * U[7];
    R ke = (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho;
    R p = (gamma - R(1)) * (U[4] - R(0.5) * ke - R(0.5) * bb);
    R cf = fast(rho, p, U[5 + d], bb);
    m1 = vabs(U[1 + d] / rho) + cf;
    m2 = cf;
  }

  VK_HD bool physical(const R* U) const {
    R rho = U[0];
    R bb = U[5] * U[5] + U[6] * U[6] + U[7] * U[7];
    R ke = (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho;
    R p = (gamma - R(1)) * (U[4] - R(0.5) * ke - R(0.5) * bb);
    return rho > R(0) && p > R(0);
  }

  // Both directions through one copy of split_x (a loop the compiler keeps):
  // the split is several kilobytes of code, and a second inlined copy costs
  // more in instruction-cache misses than the loop's register moves.  The
  // second pass keeps the first one's result and turns the state in place
  // (swapping (m_x, m_y) and (B_x, B_y)), so that no value is chosen by the
  // pass index at run time (a select per value and pass, measured 5 % of the
  // MHD-GLM step's instructions).
  VK_HD void split2(const R* U, int set, R k, R ch, R* Fp1, R* F1, R* Fp2, R* F2) const {
    R V[9], a[9], b[9], ax[9], bx[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) V[i] = U[i];
#pragma unroll 1
    for (int d = 0; d < 2; ++d) {
      if (d == 1) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          ax[i] = a[i];
          bx[i] = b[i];
        }
        R t = V[1];
        V[1] = V[2];
        V[2] = t;
        t = V[5];
        V[5] = V[6];
        V[6] = t;
      }
      split_x(V, set, k, ch, a, b);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      Fp1[i] = ax[i];
      F1[i] = bx[i];
    }
    Fp2[0] = a[0]; Fp2[1] = a[2]; Fp2[2] = a[1]; Fp2[3] = a[3]; Fp2[4] = a[4];
    Fp2[5] = a[6]; Fp2[6] = a[5]; Fp2[7] = a[7]; Fp2[8] = a[8];
    F2[0] = b[0]; F2[1] = b[2]; F2[2] = b[1]; F2[3] = b[3]; F2[4] = b[4];
    F2[5] = b[6]; F2[6] = b[5]; F2[7] = b[7]; F2[8] = b[8];
  }

  // m1 = max_d (|u_d| + c_f,d), m2 = max_d c_f,d, physical test of U^{n+1}
  VK_HD bool epilogue(const R* U, R& m1, R& m2) const {
    const R rho = U[0], ir = vrcp(rho);
    const R bx2 = U[5] * U[5], by2 = U[6] * U[6];
    const R bb = bx2 + by2 + U[7] * U[7];
    const R ke = (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) * ir;
    const R p = (gamma - R(1)) * (U[4] - R(0.5) * ke - R(0.5) * bb);
    const R a2 = gamma * p * ir, b2 = bb * ir, s = a2 + b2;
    const R cfx = vsqrt(R(0.5) * (s + vsqrt(vmax(s * s - R(4) * a2 * bx2 * ir, R(0)))));
    const R cfy = vsqrt(R(0.5) * (s + vsqrt(vmax(s * s - R(4) * a2 * by2 * ir, R(0)))));
    m1 = vmax(vabs(U[1] * ir) + cfx, vabs(U[2] * ir) + cfy);
    m2 = vmax(cfx, cfy);
    return rho > R(0) && p > R(0);
  }

  VK_HD void split(const R* Uin, int d, int set, R k, R ch, R* Fp, R* F) const {
    if (d == 0) {
      split_x(Uin, set, k, ch, Fp, F);
      return;
    }
    // y direction: swap (mx, my) and (Bx, By), split along x, swap back
    R U[9] = {Uin[0], Uin[2], Uin[1], Uin[3], Uin[4], Uin[6], Uin[5], Uin[7], Uin[8]};
    R a[9], b[9];
    split_x(U, set, k, ch, a, b);
    Fp[0] = a[0]; Fp[1] = a[2]; Fp[2] = a[1]; Fp[3] = a[3]; Fp[4] = a[4];
    Fp[5] = a[6]; Fp[6] = a[5]; Fp[7] = a[7]; Fp[8] = a[8];
    F[0] = b[0]; F[1] = b[2]; F[2] = b[1]; F[3] = b[3]; F[4] = b[4];
    F[5] = b[6]; F[6] = b[5]; F[7] = b[7]; F[8] = b[8];
  }

  // Characteristic boundary along direction d (Eqs. 33-35 on a face normal
  // to d): out = P Lambda^out P^-1 dU of the 9 x 9 Jacobian, the waves leaving
  // through a low face (side 0: lambda < 0) or a high face (side 1: lambda > 0).
  // The same eigen-structure as split_x with the weight alpha(lambda) replaced by
  // g(lambda) = lambda on outgoing waves, 0 on incoming ones, and the flux by
  // dU: for the block-triangular Jacobian g(A) dU = (sum_j c_j r_j,
  // sum_+- g(+-c_h) phi_+- (1, +-c_h)) with phi_+- = dB_n / 2 +- dpsi / (2 c_h)
  // and c_j = g_j l_j.dU_7 + l_j.ga sum_+- phi_+- (g_j - g_+-) / (lambda_j - lambda_+-).
  VK_HD void char_rhs_d(const R* Uin, const R* dUin, int d, int side, R ch, R* out) const {
    if (d == 0) {
      char_rhs_x(Uin, dUin, side, ch, out);
      return;
    }
    const R U[9] = {Uin[0], Uin[2], Uin[1], Uin[3], Uin[4], Uin[6], Uin[5], Uin[7], Uin[8]};
    const R dU[9] = {dUin[0], dUin[2], dUin[1], dUin[3], dUin[4], dUin[6], dUin[5], dUin[7], dUin[8]};
    R o[9];
    char_rhs_x(U, dU, side, ch, o);
    out[0] = o[0]; out[1] = o[2]; out[2] = o[1]; out[3] = o[3]; out[4] = o[4];
    out[5] = o[6]; out[6] = o[5]; out[7] = o[7]; out[8] = o[8];
  }

  VK_HD void char_rhs_x(const R* U, const R* dU, int side, R ch, R* out) const {
    const R rho = U[0];
    const R ir = R(1) / rho;
    const R u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
    const R bx = U[5], by = U[6], bz = U[7];
    const R bt2 = by * by + bz * bz;
    const R q2 = u * u + v * v + w * w;
    const R gm1 = gamma - R(1);
    const R p = gm1 * (U[4] - R(0.5) * rho * q2 - R(0.5) * (bx * bx + bt2));
    const R a2 = gamma * p * ir, bx2 = bx * bx * ir, btt = bt2 * ir;
    R af, as, dcs;
    mhd_norm<R>(a2, bx2, btt, af, as, dcs);
    if (sizeof(R) == 4 && !(dcs > R(1e-3) * (a2 + bx2 + btt))) {
      double af64, as64, d64;
      mhd_norm<double>((double)a2, (double)bx2, (double)btt, af64, as64, d64);
      af = (R)af64;
      as = (R)as64;
    }
    const R cf2 = R(0.5) * (a2 + bx2 + btt + dcs);
    const R cf = vsqrt(cf2);
    const R cs = cf2 > R(0) ? vsqrt(a2 * bx2 / cf2) : R(0);
    const R ca = vsqrt(bx2), a = vsqrt(a2), sr = vsqrt(rho);
    R bty, btz;
    const R bt = vsqrt(bt2);
    if (bt > R(1e-30) * (vabs(bx) + R(1e-30))) {
      bty = by / bt;
      btz = bz / bt;
    } else {
      bty = btz = R(0.70710678118654752440);
    }
    const R s = bx >= R(0) ? R(1) : R(-1);
    auto og = [&](R l) -> bool { return side == 0 ? l < R(0) : l > R(0); };
    auto g = [&](R l) -> R { return og(l) ? l : R(0); };
    // divided difference (g(l1) - g(l2)) / (l1 - l2): exactly 1 when both waves
    // leave, 0 when both enter (g is l or 0 there), else the plain quotient
    // (one of the two is 0 and the speeds lie on either side of 0)
    auto gdd = [&](R l1, R g1, R l2, R g2) -> R {
      if (og(l1) == og(l2)) return og(l1) ? R(1) : R(0);
      return (g1 - g2) / (l1 - l2);
    };
    const R lam[7] = {u - cf, u - ca, u - cs, u, u + cs, u + ca, u + cf};
    R gl[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) gl[j] = g(lam[j]);
    const R gp = g(ch), gm = g(-ch);
    const R php = R(0.5) * (dU[5] + dU[8] / ch), phm = R(0.5) * (dU[5] - dU[8] / ch);
    // primitive increments of the MHD block of dU (B_n held), and of d F7 / d B_n
    const R ia2 = R(1) / a2;
    const R Gr = dU[0];
    const R Gu = (dU[1] - u * dU[0]) * ir, Gv = (dU[2] - v * dU[0]) * ir, Gw = (dU[3] - w * dU[0]) * ir;
    const R Gp = gm1 * (dU[4] + R(0.5) * q2 * dU[0] - (u * dU[1] + v * dU[2] + w * dU[3]) - (by * dU[6] + bz * dU[7]));
    const R Gy = dU[6], Gz = dU[7];
    const R hu = -gamma * bx * ir, hv = -by * ir, hw = -bz * ir;
    const R hp = gm1 * (v * by + w * bz), hy = -v, hz = -w;
    const R isr_a = R(1) / (sr * a), isr = R(1) / sr;
    const R Tu = R(0.5) * Gu * ia2, Tt = R(0.5) * s * (bty * Gv + btz * Gw) * ia2;
    const R Tp = R(0.5) * Gp * ia2 * ir, TB = R(0.5) * (bty * Gy + btz * Gz) * isr_a;
    const R Tq = R(0.5) * (-btz * Gv + bty * Gw), TQ = R(0.5) * s * (btz * Gy - bty * Gz) * isr;
    const R Hu = R(0.5) * hu * ia2, Ht = R(0.5) * s * (bty * hv + btz * hw) * ia2;
    const R Hp = R(0.5) * hp * ia2 * ir, HB = R(0.5) * (bty * hy + btz * hz) * isr_a;
    const R Hq = R(0.5) * (-btz * hv + bty * hw), HQ = R(0.5) * s * (btz * hy - bty * hz) * isr;
    R lG[7], lH[7];
    lG[0] = -(af * cf * Tu - as * cs * Tt) + af * Tp + as * TB;
    lG[6] = +(af * cf * Tu - as * cs * Tt) + af * Tp + as * TB;
    lG[2] = -(as * cs * Tu + af * cf * Tt) + as * Tp - af * TB;
    lG[4] = +(as * cs * Tu + af * cf * Tt) + as * Tp - af * TB;
    lG[1] = Tq - TQ;
    lG[5] = Tq + TQ;
    lG[3] = Gr - Gp * ia2;
    lH[0] = -(af * cf * Hu - as * cs * Ht) + af * Hp + as * HB;
    lH[6] = +(af * cf * Hu - as * cs * Ht) + af * Hp + as * HB;
    lH[2] = -(as * cs * Hu + af * cf * Ht) + as * Hp - af * HB;
    lH[4] = +(as * cs * Hu + af * cf * Ht) + as * Hp - af * HB;
    lH[1] = Hq - HQ;
    lH[5] = Hq + HQ;
    lH[3] = -hp * ia2;
    R cc[7];
#pragma unroll
    for (int j = 0; j < 7; ++j)
      cc[j] = gl[j] * lG[j] + lH[j] * (php * gdd(lam[j], gl[j], ch, gp) + phm * gdd(lam[j], gl[j], -ch, gm));
    const R fs = cc[6] + cc[0], fd = cc[6] - cc[0];
    const R ss = cc[4] + cc[2], sd = cc[4] - cc[2];
    const R as_ = cc[5] + cc[1], ad = cc[5] - cc[1];
    const R Sr = rho * (af * fs + as * ss) + cc[3];
    const R Su = af * cf * fd + as * cs * sd;
    const R tr = s * (-as * cs * fd + af * cf * sd);
    const R Sv = bty * tr - btz * as_;
    const R Sw = btz * tr + bty * as_;
    const R Sp = rho * a2 * (af * fs + as * ss);
    const R tb = sr * a * (as * fs - af * ss);
    const R Sy = bty * tb + s * sr * btz * ad;
    const R Sz = btz * tb - s * sr * bty * ad;
    out[0] = Sr;
    out[1] = u * Sr + rho * Su;
    out[2] = v * Sr + rho * Sv;
    out[3] = w * Sr + rho * Sw;
    out[4] = Sp / gm1 + R(0.5) * q2 * Sr + rho * (u * Su + v * Sv + w * Sw) + by * Sy + bz * Sz;
    out[6] = Sy;
    out[7] = Sz;
    out[5] = gp * php + gm * phm;
    out[8] = ch * (gp * php - gm * phm);
  }

  VK_HD void split_x(const R* U, int set, R k, R ch, R* Fp, R* F) const {
    const R rho = U[0];
    const R ir = vrcp(rho);
    const R u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
    const R E = U[4], bx = U[5], by = U[6], bz = U[7], psi = U[8];
    const R bt2 = by * by + bz * bz;
    const R bb = bx * bx + bt2;
    const R q2 = u * u + v * v + w * w;
    const R gm1 = gamma - R(1);
    const R p = gm1 * (E - R(0.5) * rho * q2 - R(0.5) * bb);
    const R pt = p + R(0.5) * bb;
    const R bu = bx * u + by * v + bz * w;
    // physical flux, Eq. (58), x component
    F[0] = U[1];
    F[1] = U[1] * u + pt - bx * bx;
    F[2] = U[2] * u - bx * by;
    F[3] = U[3] * u - bx * bz;
    F[4] = (E + pt) * u - bu * bx;
    F[5] = psi;
    F[6] = u * by - bx * v;
    F[7] = u * bz - bx * w;
    F[8] = ch * ch * bx;
    if (set == SET_CENTERED) {
      for (int i = 0; i < 9; ++i) Fp[i] = R(0.5) * F[i];
      return;
    }
    // wave speeds
    const R a2 = gamma * p * ir;
    const R bx2 = bx * bx * ir;
    const R btt = bt2 * ir;
    R af, as, dcs;
    mhd_norm<R>(a2, bx2, btt, af, as, dcs);
    if (sizeof(R) == 4 && !(dcs > R(1e-3) * (a2 + bx2 + btt))) {
      // near-degenerate fast/slow/Alfven speeds: normalise in FP64
      double af64, as64, d64;
      mhd_norm<double>((double)a2, (double)bx2, (double)btt, af64, as64, d64);
      af = (R)af64;
      as = (R)as64;
    }
    const R cf2 = R(0.5) * (a2 + bx2 + btt + dcs);
    const R cf = vsqrt(cf2);
    const R cs = cf2 > R(0) ? vsqrt(a2 * bx2 * vrcp(cf2)) : R(0);
    const R ca = vsqrt(bx2);
    const R a = vsqrt(a2);
    const R sr = vsqrt(rho);
    R bty, btz;
    const R bt = vsqrt(bt2);
    if (bt > R(1e-30) * (vabs(bx) + R(1e-30))) {
      R ib = vrcp(bt);
      bty = by * ib;
      btz = bz * ib;
    } else {
      bty = btz = R(0.70710678118654752440);
    }
    const R s = bx >= R(0) ? R(1) : R(-1);

    // sigmoid weights, normalised by the largest |lambda| of the cell (with
    // the cleaning waves), or by the grid-wide lg
    const R lmax = lam_norm(lg, vmax(vabs(u) + cf, ch));
    const R kl = k * vrcp(lmax);
    const R lam[7] = {u - cf, u - ca, u - cs, u, u + cs, u + ca, u + cf};
    R al[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) al[j] = alpha_w(lam[j], kl, set);
    const R alp = alpha_w(ch, kl, set), alm = alpha_w(-ch, kl, set);
    const R php = R(0.5) * (psi + ch * bx), phm = R(0.5) * (psi - ch * bx);

    // G = M^-1 F7 (primitive increments of the flux), ga = M^-1 dF7/dBx
    const R ia2 = vrcp(a2);
    const R Gr = F[0];
    const R Gu = (F[1] - u * F[0]) * ir, Gv = (F[2] - v * F[0]) * ir, Gw = (F[3] - w * F[0]) * ir;
    const R Gp = gm1 * (F[4] + R(0.5) * q2 * F[0] - (u * F[1] + v * F[2] + w * F[3]) - (by * F[6] + bz * F[7]));
    const R Gy = F[6], Gz = F[7];
    const R hu = -gamma * bx * ir, hv = -by * ir, hw = -bz * ir;
    const R hp = gm1 * (v * by + w * bz), hy = -v, hz = -w;

    // shared projections
    const R isr_a = vrcp(sr * a);
    const R Tu = R(0.5) * Gu * ia2, Tt = R(0.5) * s * (bty * Gv + btz * Gw) * ia2;
    const R Tp = R(0.5) * Gp * ia2 * ir, TB = R(0.5) * (bty * Gy + btz * Gz) * isr_a;
    const R Tq = R(0.5) * (-btz * Gv + bty * Gw), TQ = R(0.5) * s * (btz * Gy - bty * Gz) * vrcp(sr);
    const R Hu = R(0.5) * hu * ia2, Ht = R(0.5) * s * (bty * hv + btz * hw) * ia2;
    const R Hp = R(0.5) * hp * ia2 * ir, HB = R(0.5) * (bty * hy + btz * hz) * isr_a;
    const R Hq = R(0.5) * (-btz * hv + bty * hw), HQ = R(0.5) * s * (btz * hy - bty * hz) * vrcp(sr);

    // l_j . G and l_j . ga in the order of lam[]
    R lG[7], lH[7];
    lG[0] = -(af * cf * Tu - as * cs * Tt) + af * Tp + as * TB;   // fast -
    lG[6] = +(af * cf * Tu - as * cs * Tt) + af * Tp + as * TB;   // fast +
    lG[2] = -(as * cs * Tu + af * cf * Tt) + as * Tp - af * TB;   // slow -
    lG[4] = +(as * cs * Tu + af * cf * Tt) + as * Tp - af * TB;   // slow +
    lG[1] = Tq - TQ;                                              // Alfven -
    lG[5] = Tq + TQ;                                              // Alfven +
    lG[3] = Gr - Gp * ia2;                                        // entropy
    lH[0] = -(af * cf * Hu - as * cs * Ht) + af * Hp + as * HB;
    lH[6] = +(af * cf * Hu - as * cs * Ht) + af * Hp + as * HB;
    lH[2] = -(as * cs * Hu + af * cf * Ht) + as * Hp - af * HB;
    lH[4] = +(as * cs * Hu + af * cf * Ht) + as * Hp - af * HB;
    lH[1] = Hq - HQ;
    lH[5] = Hq + HQ;
    lH[3] = -hp * ia2;

    // coefficients c_j = alpha_j l_j.G + l_j.ga sum_+- phi_+- (alpha_j - alpha_+-)/(lam_j - lam_+-)
    // The plain quotients first (alpha_dd's branch for well separated speeds,
    // which is every wave when c_h is several times the fast speed); the
    // stable forms only where a speed comes within 0.05 lmax of +-c_h, or for
    // the other weight sets, in a branch a warp rarely enters.
    R cc[7];
    bool near = set != SET_WEIGHTED;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const R dp = lam[j] - ch, dm = lam[j] + ch;
      near = near || !(vabs(dp) > R(0.05) * lmax) || !(vabs(dm) > R(0.05) * lmax);
      const R ddp = (al[j] - alp) * vrcp(dp), ddm = (al[j] - alm) * vrcp(dm);
      cc[j] = al[j] * lG[j] + lH[j] * (php * ddp + phm * ddm);
    }
    if (near) {
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        R ddp = alpha_dd(al[j], lam[j], alp, ch, kl, lmax, set);
        R ddm = alpha_dd(al[j], lam[j], alm, -ch, kl, lmax, set);
        cc[j] = al[j] * lG[j] + lH[j] * (php * ddp + phm * ddm);
      }
    }
    // S = sum_j c_j r_j (primitive), then F+_7 = M S
    const R fs = cc[6] + cc[0], fd = cc[6] - cc[0];
    const R ss = cc[4] + cc[2], sd = cc[4] - cc[2];
    const R as_ = cc[5] + cc[1], ad = cc[5] - cc[1];
    const R Sr = rho * (af * fs + as * ss) + cc[3];
    const R Su = af * cf * fd + as * cs * sd;
    const R tr = s * (-as * cs * fd + af * cf * sd);
    const R Sv = bty * tr - btz * as_;
    const R Sw = btz * tr + bty * as_;
    const R Sp = rho * a2 * (af * fs + as * ss);
    const R tb = sr * a * (as * fs - af * ss);
    const R Sy = bty * tb + s * sr * btz * ad;
    const R Sz = btz * tb - s * sr * bty * ad;
    Fp[0] = Sr;
    Fp[1] = u * Sr + rho * Su;
    Fp[2] = v * Sr + rho * Sv;
    Fp[3] = w * Sr + rho * Sw;
    Fp[4] = Sp / gm1 + R(0.5) * q2 * Sr + rho * (u * Su + v * Sv + w * Sw) + by * Sy + bz * Sz;
    Fp[6] = Sy;
    Fp[7] = Sz;
    // cleaning block: e_+- = (1, +-c_h)
    Fp[5] = alp * php + alm * phm;
    Fp[8] = ch * (alp * php - alm * phm);
  }
};

}  // namespace vk
