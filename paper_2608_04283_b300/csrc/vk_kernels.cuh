// CUDA kernels of the VKLB step (Sec. 3.5, Fig. 5) for sm_103a.
//
// Layout in HBM (two buffers ping-pong between steps): D2Q5 in 32-cell bricks,
// component q p + k of cell (x, y) at ((y nxb + x / 32) 5p + q p + k) 32 + x % 32
// (brick_base below); D1Q3 in component planes f[(q p + k) nx + x].  The moment
// form (omega = 1) stores the p fields of U in bricks of p components.
//
// step2d_kernel: one launch = one step on D2Q5, periodic (Eq. 37).  (Its
// variants: step2d_lb_kernel, the same body with a register bound; step2d_u_kernel,
// the moment form; step2d_tma_kernel, rows staged by bulk copies; the batched
// kernel over a work-list of tiles of many simulations.)  A block owns
// a tile of TX columns x TY rows; each thread owns one column and marches up the
// tile.  Per cell it loads the 5p values of f^n (coalesced across the warp),
// forms U = sum_q f_q (Eq. 3), splits F^(1), F^(2) (Eqs. 25-27), builds the
// equilibria (Eq. 41), collides (Eq. 42) and streams by pull (Eq. 43):
//     f^{n+1}_q(x) = f*_q(x - v_q).
// The x neighbours' f*_1, f*_2 go through shared memory (three row buffers, one
// mbarrier phase per row); f*_4 of the row below and f*_5 of the row above stay in
// registers.  The 1-cell ring around the tile is recomputed for just the one
// component that streams inward (x ring: f*_1 / f*_2 from the x split only;
// y ring: f*_4 / f*_5 from the y split only).  Knowing every f^{n+1} of its tile,
// the block then forms U^{n+1} and reduces max_j |lambda_j| (and the MHD fast
// speed) into the control words, so xi_{n+1} (Eq. 29) is ready for the next
// launch with no second pass over f.
//
// step1d_kernel: D1Q3, one block runs many steps (tiny 1D grids are latency
// bound), with the characteristic boundary (Eqs. 33-36) or periodic wrap.
#pragma once
#include "vk_ctl.cuh"
#include "vk_systems.cuh"

namespace vk {

struct SysParams {
  double gamma, g, ax, ay;
};

template <class Sys> VK_HD Sys make_sys(const SysParams& s);
template <> VK_HD Advect<float, 1> make_sys(const SysParams& s) { Advect<float, 1> r; r.a[0] = (float)s.ax; r.a[1] = (float)s.ay; r.lg = 0.0f; return r; }
template <> VK_HD Advect<double, 1> make_sys(const SysParams& s) { Advect<double, 1> r; r.a[0] = s.ax; r.a[1] = s.ay; r.lg = 0.0; return r; }
template <> VK_HD Advect<float, 2> make_sys(const SysParams& s) { Advect<float, 2> r; r.a[0] = (float)s.ax; r.a[1] = (float)s.ay; r.lg = 0.0f; return r; }
template <> VK_HD Advect<double, 2> make_sys(const SysParams& s) { Advect<double, 2> r; r.a[0] = s.ax; r.a[1] = s.ay; r.lg = 0.0; return r; }
template <> VK_HD SWE<float, 1> make_sys(const SysParams& s) { SWE<float, 1> r; r.g = (float)s.g; r.lg = 0.0f; return r; }
template <> VK_HD SWE<double, 1> make_sys(const SysParams& s) { SWE<double, 1> r; r.g = s.g; r.lg = 0.0; return r; }
template <> VK_HD SWE<float, 2> make_sys(const SysParams& s) { SWE<float, 2> r; r.g = (float)s.g; r.lg = 0.0f; return r; }
template <> VK_HD SWE<double, 2> make_sys(const SysParams& s) { SWE<double, 2> r; r.g = s.g; r.lg = 0.0; return r; }
template <> VK_HD Euler<float, 1> make_sys(const SysParams& s) { Euler<float, 1> r; r.gamma = (float)s.gamma; r.lg = 0.0f; return r; }
template <> VK_HD Euler<double, 1> make_sys(const SysParams& s) { Euler<double, 1> r; r.gamma = s.gamma; r.lg = 0.0; return r; }
template <> VK_HD Euler<float, 2> make_sys(const SysParams& s) { Euler<float, 2> r; r.gamma = (float)s.gamma; r.lg = 0.0f; return r; }
template <> VK_HD Euler<double, 2> make_sys(const SysParams& s) { Euler<double, 2> r; r.gamma = s.gamma; r.lg = 0.0; return r; }
template <> VK_HD MHDGLM<float> make_sys(const SysParams& s) { MHDGLM<float> r; r.gamma = (float)s.gamma; r.lg = 0.0f; return r; }
template <> VK_HD MHDGLM<double> make_sys(const SysParams& s) { MHDGLM<double> r; r.gamma = s.gamma; r.lg = 0.0; return r; }

// Everything one step of one simulation needs.  The buffer pair is selected
// with src() / dst(), not indexed by the parity: an indexed member array would
// keep a copy of the struct (the batched kernels make one) in local memory.
template <class T>
struct StepArgs {
  T* f[2];         // ping-pong distribution buffers
  int parity;      // f[parity] holds f^n
  int nx, ny;
  int pitch;       // cells per padded row (a multiple of 32 in 2D: pitch / 32 bricks per row)
  double dx, c, omega, k, inv_nu, fixed_xi, t_end, ch_factor;
  int set;
  int anorm;       // alpha's normaliser: 0 per cell and direction, 1 grid-wide max |lambda| of the step
  int bc_lo, bc_hi;  // 1D: 0 periodic, 1 characteristic, 2 transmissive
  int cbx, cby;      // 2D: non-periodic boundaries on the x (y) faces
  int btr;           // 2D: those faces are transmissive (else characteristic)
  Ctl* ctl;
  int slot;        // n % 3
  SysParams sp;
  // Edge columns of the tiles (long-split march only; see halo_index): hl[b]
  // holds those of f[b]; hl_ok says hl[parity] matches f^n for this tile width.
  T* hl[2];
  int hl_ok;
  VK_HD T* src() const { return parity ? f[1] : f[0]; }
  VK_HD T* dst() const { return parity ? f[0] : f[1]; }
  VK_HD const T* halo_in() const { return hl_ok ? (parity ? hl[1] : hl[0]) : nullptr; }
  VK_HD T* halo_out() const { return parity ? hl[0] : hl[1]; }
};

// 2D distribution layout: 32-cell bricks.  Component k = q p + i of cell (x, y)
// is f[((y nxb + x / 32) 5p + k) 32 + x % 32], nxb = pitch / 32: a warp's access
// to one component of 32 neighbouring cells is one contiguous 32-element run,
// the 5p components of a brick follow each other (component stride kBrick, a
// compile-time immediate offset), and a tile row of whole bricks is one
// contiguous range.  1D grids keep component planes f[k nx + x].
constexpr int kBrick = 32;
VK_HD size_t brick_base(int x, int y, int nxb, int npl) {
  return ((((size_t)y * nxb + (x >> 5)) * npl) << 5) + (x & 31);
}
// Offset of component 0 of cell (x, y) and the stride between components of a
// state with Q components a field: Q = 3 (D1Q3) planes of pitch x ny; Q = 5
// (D2Q5 distributions) and Q = 1 (D2Q5 moment form) 32-cell bricks of Q p.
VK_HD size_t cell_base(int Q, int P, int x, int y, int pitch) {
  return Q != 3 ? brick_base(x, y, pitch / kBrick, Q * P) : (size_t)y * pitch + x;
}
VK_HD size_t comp_stride(int Q, int pitch, int ny) { return Q != 3 ? (size_t)kBrick : (size_t)pitch * ny; }

// Halo of the long-split march: the first (side 0) and last (side 1) column of
// every tile TX wide, the npl stored components of a cell contiguous, rows in
// order.  The step that writes f^{n+1} writes them too, so the next step reads
// its x ring (the neighbouring tiles' edge columns) as whole contiguous runs
// instead of one 4-byte value from each of npl brick lines a cell.
VK_HD size_t halo_index(int tile, int side, int y, int ny, int npl) {
  return (((size_t)tile * 2 + side) * ny + y) * npl;
}

// Which post-collision components a cell must produce (C_QX: f*_1 and f*_2).
enum CollideMode { C_FULL = 0, C_Q1 = 1, C_Q2 = 2, C_Q4 = 3, C_Q5 = 4, C_QX = 5 };

// Weighted equilibria of Eq. (41) from U, the components MODE needs:
//   e1 = c U + F(1,+)/xi, e2 = c U - F(1,-)/xi, e4 = c U + F(2,+)/xi,
//   e5 = c U - F(2,-)/xi, e3 = U - (e1 + e2 + e4 + e5) (= Eq. 41's rest term).
template <class Sys, class R, int MODE>
__device__ __forceinline__ void equilibria_d2q5(const Sys& sys, const R (&U)[Sys::P], R xinv, R c, int set, R k,
                                                R ch, R (&e)[5][Sys::P]) {
  constexpr int P = Sys::P;
  if (MODE == C_FULL) {
    R Fp1[P], F1[P], Fp2[P], F2[P];
    sys.split2(U, set, k, ch, Fp1, F1, Fp2, F2);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const R cu = c * U[i];
      e[0][i] = vfma(Fp1[i], xinv, cu);
      e[1][i] = vfma(Fp1[i] - F1[i], xinv, cu);
      e[3][i] = vfma(Fp2[i], xinv, cu);
      e[4][i] = vfma(Fp2[i] - F2[i], xinv, cu);
      e[2][i] = U[i] - ((e[0][i] + e[1][i]) + e[3][i] + e[4][i]);
    }
    return;
  }
  R Fp[P], F[P];
  if (MODE == C_Q1 || MODE == C_Q2 || MODE == C_QX) {
    sys.split(U, 0, set, k, ch, Fp, F);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      e[0][i] = vfma(Fp[i], xinv, c * U[i]);
      e[1][i] = vfma(Fp[i] - F[i], xinv, c * U[i]);
    }
  } else {
    sys.split(U, 1, set, k, ch, Fp, F);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      e[3][i] = vfma(Fp[i], xinv, c * U[i]);
      e[4][i] = vfma(Fp[i] - F[i], xinv, c * U[i]);
    }
  }
}

// Collision (Eq. 42) of one D2Q5 cell: load f, U = sum_q f_q (Eq. 3), the
// equilibria, relax f* = f + omega (f^eq - f).  At omega = 1 the post-collision
// state is the equilibrium itself, taken exactly (as the moment form takes it).
// omega is the same for the whole launch, so the test is one uniform branch
// rather than a select per component.
template <class Sys, class T, class R, int MODE, bool KEEP = false>
__device__ __forceinline__ void collide_d2q5(const Sys& sys, const T* __restrict__ fin, size_t plane,
                                             size_t idx, R xinv, R c, R om, int set, R k, R ch,
                                             R (&out)[5][Sys::P]) {
  constexpr int P = Sys::P;
  R f[5][P];
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const T* ptr = fin + (size_t)(q * P + i) * plane + idx;
      f[q][i] = KEEP ? Store<T>::ld_keep(ptr) : Store<T>::ld(ptr);
    }
  R U[P];
#pragma unroll
  for (int i = 0; i < P; ++i) U[i] = f[0][i] + f[1][i] + f[2][i] + f[3][i] + f[4][i];
  R e[5][P];
  equilibria_d2q5<Sys, R, MODE>(sys, U, xinv, c, set, k, ch, e);
  if (om == R(1)) {
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int i = 0; i < P; ++i) out[q][i] = e[q][i];
  } else {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      constexpr bool qx = MODE == C_Q1 || MODE == C_Q2 || MODE == C_QX, qy = MODE == C_Q4 || MODE == C_Q5;
      const bool need = MODE == C_FULL || ((q == 0 || q == 1) && qx) || ((q == 3 || q == 4) && qy);
      if (!need) continue;
#pragma unroll
      for (int i = 0; i < P; ++i) {
        // A long split (MHD-GLM) does not hold f in registers across it: f is
        // read again here (an L1 hit).  The short ones keep it.
        const R fv = Sys::P > 4 ? Store<T>::ld_again(fin + (size_t)(q * P + i) * plane + idx) : f[q][i];
        out[q][i] = fv + om * (e[q][i] - fv);
      }
    }
  }
}

template <class R> __device__ __forceinline__ R round_store(R v, const float*) { return v; }
template <class R> __device__ __forceinline__ R round_store(R v, const double*) { return v; }
template <class R> __device__ __forceinline__ R round_store(R v, const __nv_bfloat16*) {
  return (R)__bfloat162float(__float2bfloat16_rn((float)v));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide max of (a, b) and OR of bad (in the compute type); thread 0
// commits them to slot s1 as doubles.
template <class R>
__device__ __forceinline__ void commit_max(R a, R b, bool bad, Ctl* ctl, int s1) {
  __shared__ R red[2][32];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  a = warp_max(a);
  b = warp_max(b);
  if (bad) sbad = 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    a = lane < nw ? red[0][lane] : R(0);
    b = lane < nw ? red[1][lane] : R(0);
    a = warp_max(a);
    b = warp_max(b);
    if (lane == 0) {
      atomicMax(&ctl->m1[s1], double_to_bits((double)a));
      atomicMax(&ctl->m2[s1], double_to_bits((double)b));
      if (sbad) atomicOr(&ctl->err, ERR_NONPHYS);
    }
  }
}

// Per-step bookkeeping done once per launch by block 0: t^{n+1}, clearing the
// slot of step n+2, the fixed-xi CFL check.
__device__ __forceinline__ void step_bookkeeping(Ctl* ctl, int slot, const StepScalars& sc, double dx,
                                                 double fixed_xi, bool mhd) {
  const int s1 = (slot + 1) % 3, s2 = (slot + 2) % 3;
  ctl->nsteps += 1;
  ctl->t[s1] = ctl->t[slot] + dx / sc.xi;
  ctl->xi_used[slot] = sc.xi;
  ctl->m1[s2] = 0ull;
  ctl->m2[s2] = 0ull;
  if (fixed_xi > 0.0) {
    double lam = bits_to_double(ctl->m1[slot]);
    if (mhd) lam = fmax(lam, sc.ch);
    if (lam > fixed_xi * (1.0 + 1e-12)) atomicOr(&ctl->err, ERR_CFL);
  }
}

// The step's constants in the compute type, converted once per block by one
// thread and shared: FP64 conversions issue at a small fraction of the FP32
// rate on this part, so per-thread conversions would cost more than the march.
template <class Sys, class R>
struct BlockConsts {
  Sys sys;
  R xinv, ch, c, om, k;
};
template <class Sys, class R, class T>
__device__ __forceinline__ BlockConsts<Sys, R> block_consts(const StepArgs<T>& a, const StepScalars& sc) {
  BlockConsts<Sys, R> b;
  b.sys = make_sys<Sys>(a.sp);
  if (a.anorm) b.sys.lg = (R)sc.lam;
  b.xinv = (R)sc.xinv;
  b.ch = (R)sc.ch;
  b.c = (R)a.c;
  b.om = (R)a.omega;
  b.k = (R)a.k;
  return b;
}

// State forms of a D2Q5 simulation.  FORM 0 keeps the distributions f (5p
// components a cell); FORM 1, for omega = 1 only, keeps the moments U (p a
// cell): at omega = 1 the post-collision state is f^eq(U) (Eq. 42), so f after
// streaming is a function of the neighbours' U and a step is the finite-volume
// update of Thm 4.3, U^{n+1}(x) = sum_q f^eq_q(U^n(x - v_q)) (Eqs. 41, 43).
// Both march the same way; only the load and the store differ.
template <class Sys, int FORM>
struct StateForm {
  static constexpr int NS = FORM == 0 ? 5 * Sys::P : Sys::P;   // stored components a cell
};

// Post-collision components that MODE needs of the cell whose stored
// component j sits at fin[b + j * plane].
template <class Sys, class T, class R, int MODE, int FORM, bool KEEP = false>
__device__ __forceinline__ void cell_post_at(const Sys& sys, const T* __restrict__ fin, size_t plane, size_t b,
                                             R xinv, R c, R om, int set, R k, R ch, R (&o)[5][Sys::P]) {
  constexpr int P = Sys::P;
  if constexpr (FORM == 0) {
    collide_d2q5<Sys, T, R, MODE, KEEP>(sys, fin, plane, b, xinv, c, om, set, k, ch, o);
  } else {
    R U[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const T* ptr = fin + b + (size_t)i * plane;
      U[i] = KEEP ? Store<T>::ld_keep(ptr) : Store<T>::ld(ptr);
    }
    equilibria_d2q5<Sys, R, MODE>(sys, U, xinv, c, set, k, ch, o);
  }
}

// Post-collision components of cell (x, y) that MODE needs.
template <class Sys, class T, class R, int MODE, int FORM, bool KEEP = false>
__device__ __forceinline__ void cell_post(const Sys& sys, const T* __restrict__ fin, int x, int y, int nxb, R xinv,
                                          R c, R om, int set, R k, R ch, R (&o)[5][Sys::P]) {
  cell_post_at<Sys, T, R, MODE, FORM, KEEP>(sys, fin, kBrick, brick_base(x, y, nxb, StateForm<Sys, FORM>::NS), xinv,
                                            c, om, set, k, ch, o);
}

// The stored values of the cell at b (FORM 0: its 5p distributions; FORM 1:
// U in v[0]), loaded ahead of the arithmetic that uses them.
template <class Sys, class T, class R, int FORM>
__device__ __forceinline__ void load_stored(const T* __restrict__ fin, size_t b, R (&v)[5][Sys::P]) {
  constexpr int P = Sys::P;
  if constexpr (FORM == 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int i = 0; i < P; ++i) v[q][i] = Store<T>::ld(fin + b + (size_t)(q * P + i) * kBrick);
  } else {
#pragma unroll
    for (int i = 0; i < P; ++i) v[0][i] = Store<T>::ld(fin + b + (size_t)i * kBrick);
  }
}

// Post-collision components MODE needs from loaded stored values, the same
// arithmetic as cell_post_at (short splits: f held in registers).
template <class Sys, class R, int MODE, int FORM>
__device__ __forceinline__ void post_loaded(const Sys& sys, const R (&f)[5][Sys::P], R xinv, R c, R om, int set, R k,
                                            R ch, R (&o)[5][Sys::P]) {
  constexpr int P = Sys::P;
  static_assert(P <= 4, "long splits reload f");
  if constexpr (FORM == 0) {
    R U[P];
#pragma unroll
    for (int i = 0; i < P; ++i) U[i] = f[0][i] + f[1][i] + f[2][i] + f[3][i] + f[4][i];
    R e[5][P];
    equilibria_d2q5<Sys, R, MODE>(sys, U, xinv, c, set, k, ch, e);
    if (om == R(1)) {
#pragma unroll
      for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int i = 0; i < P; ++i) o[q][i] = e[q][i];
    } else {
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        constexpr bool qx = MODE == C_Q1 || MODE == C_Q2 || MODE == C_QX, qy = MODE == C_Q4 || MODE == C_Q5;
        const bool need = MODE == C_FULL || ((q == 0 || q == 1) && qx) || ((q == 3 || q == 4) && qy);
        if (!need) continue;
#pragma unroll
        for (int i = 0; i < P; ++i) o[q][i] = f[q][i] + om * (e[q][i] - f[q][i]);
      }
    }
  } else {
    equilibria_d2q5<Sys, R, MODE>(sys, f[0], xinv, c, set, k, ch, o);
  }
}

// A node on a characteristic (non-periodic) face: the step writes it from the
// periodic pull, the boundary pass overwrites it, and the CFL maximum of the
// step leaves it to that pass.
template <class T>
__device__ __forceinline__ bool on_char_face(const StepArgs<T>& a, int x, int y) {
  return (a.cbx && (x == 0 || x == a.nx - 1)) || (a.cby && (y == 0 || y == a.ny - 1));
}

// Per-cell vectors of P values in shared memory, cell-major: cell j of a row
// buffer starts at j * PP.  Where P values fill whole 16-byte words (4 floats,
// 2 doubles; 3 floats padded to 4) a cell moves as 16-byte accesses, which a
// warp serves without bank conflicts; otherwise PP is odd (P, or P + 1), so a
// warp's scalar accesses to one component hit 32 different banks.  Either way
// a component's address is the cell's base plus a constant, with no per-value
// index arithmetic.
template <class R, int P>
struct CellVec {
  static constexpr int VW = 16 / (int)sizeof(R);
  static constexpr bool VEC = P % VW == 0 || (P == 3 && VW == 4);
  static constexpr int PP = VEC ? (P + VW - 1) / VW * VW : (P % 2 ? P : P + 1);
  static __device__ __forceinline__ void put(R* p, const R (&v)[P]) {
    if constexpr (VEC && VW == 4) {
#pragma unroll
      for (int k = 0; k < PP; k += 4)
        *reinterpret_cast<float4*>(p + k) =
            make_float4(v[k], k + 1 < P ? v[k + 1] : R(0), k + 2 < P ? v[k + 2] : R(0), k + 3 < P ? v[k + 3] : R(0));
    } else if constexpr (VEC) {
#pragma unroll
      for (int k = 0; k < PP; k += 2) *reinterpret_cast<double2*>(p + k) = make_double2(v[k], v[k + 1]);
    } else {
#pragma unroll
      for (int i = 0; i < P; ++i) p[i] = v[i];
    }
  }
  static __device__ __forceinline__ void get(const R* p, R (&v)[P]) {
    if constexpr (VEC && VW == 4) {
#pragma unroll
      for (int k = 0; k < PP; k += 4) {
        const float4 t = *reinterpret_cast<const float4*>(p + k);
        v[k] = t.x;
        if (k + 1 < P) v[k + 1] = t.y;
        if (k + 2 < P) v[k + 2] = t.z;
        if (k + 3 < P) v[k + 3] = t.w;
      }
    } else if constexpr (VEC) {
#pragma unroll
      for (int k = 0; k < PP; k += 2) {
        const double2 t = *reinterpret_cast<const double2*>(p + k);
        v[k] = t.x;
        v[k + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < P; ++i) v[i] = p[i];
    }
  }
};

// Row buffer index of the next row: (i + 1) mod 3 without a division.
__device__ __forceinline__ int next3(int i) { return i == 2 ? 0 : i + 1; }
// A row or column index one step outside [0, n) wrapped periodically (Eq. 37).
__device__ __forceinline__ int wrap1(int j, int n) { return j < 0 ? j + n : (j >= n ? j - n : j); }

// Row barrier of both marches as an mbarrier: every thread arrives once a row
// iteration is done (its f*_1 / f*_2 written, the rows it read finished) and
// waits only where it next reads the others' values, so a thread that is ahead
// keeps working instead of idling at a block barrier.  A thread waits between
// any two of its arrivals, so it is never two phases ahead and the parity of
// the phase it waits on is unambiguous.  The wait is bounded (%globaltimer):
// giving up latches ERR_TIMEOUT and the march goes on without further waits,
// so it cannot hang.
__device__ __forceinline__ void rowbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void rowbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"((uint32_t)__cvta_generic_to_shared(bar)) : "memory");
}
__device__ __forceinline__ bool rowbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool rowbar_wait(uint64_t* bar, uint32_t parity) {
  if (rowbar_test(bar, parity)) return true;
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t i = 1;; ++i) {
    if (rowbar_test(bar, parity)) return true;
    if ((i & 63u) == 0) {
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 2000000000ull) return false;
    }
  }
}

// ------------------------------------------------------------------ D2Q5 step
// March over the rows of one tile, up or down.  Tiles of
// even row index march up and odd ones down, so the two tiles that share a
// boundary read the boundary rows (their own and the ring) at the same time,
// the second read then hitting L2.  Going up, f^{n+1}_4(y) = f*_4(y - 1) comes
// from the previous row and f^{n+1}_5(y) = f*_5(y + 1) from the next one; going
// down the two roles swap.
// DIR = +1 / -1 fixes the direction at compile time (two bodies; the small
// systems, whose code fits the instruction cache either way).
template <class Sys, class T, class R, int DIR, int FORM>
__device__ __forceinline__ void step2d_tile_dir(const StepArgs<T>& a, const BlockConsts<Sys, R>& bc, int bx,
                                                int by, int TX, int TY, unsigned char* smem) {
  constexpr int P = Sys::P;
  const bool up = DIR > 0;
  const Sys sys = bc.sys;
  const int tx = threadIdx.x;
  const int x0 = bx * TX, y0 = by * TY;
  const int nx = a.nx, ny = a.ny;
  const int w = min(TX, nx - x0), h = min(TY, ny - y0);
  const int x = x0 + tx;
  const bool act = tx < w;
  constexpr int NS = StateForm<Sys, FORM>::NS;
  const int nxb = a.pitch / kBrick;
  const T* __restrict__ fin = a.src();
  T* __restrict__ fout = a.dst();
  const int s1 = (a.slot + 1) % 3;
  const R xinv = bc.xinv, ch = bc.ch, c = bc.c, om = bc.om, kk = bc.k;
  const int set = a.set;
  auto row_of = [&](int r) -> int { return up ? y0 + r : y0 + h - 1 - r; };
  typedef CellVec<R, P> CV;
  constexpr int PP = CV::PP;

  R* rb1 = reinterpret_cast<R*>(smem);   // [3][TX][PP]  f*_1 of the row
  R* rb2 = rb1 + 3 * PP * TX;            // [3][TX][PP]  f*_2 of the row
  R* ringL = rb2 + 3 * PP * TX;          // [TY][PP]     f*_1 at x0 - 1, by tile row
  R* ringR = ringL + PP * TY;            // [TY][PP]     f*_2 at x0 + w

  __shared__ __align__(8) uint64_t rowbar;
  if (tx == 0) {
    rowbar_init(&rowbar, blockDim.x);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // The prologue: the ring row behind and the first row of this thread's
  // column are loaded together and collided; then the x ring (only the
  // component that streams into the tile, from the x split), read for all rows
  // long before the neighbouring tile reaches the later rows: the step streams
  // more bytes than L2 holds, so these loads ask L2 to keep their lines (else
  // they are fetched from DRAM twice).
  R fbp[P], f3c[P], fbc[P];
#pragma unroll
  for (int i = 0; i < P; ++i) fbp[i] = f3c[i] = fbc[i] = R(0);
  if (act) {
    R fb0[5][P], fr0[5][P];
    load_stored<Sys, T, R, FORM>(fin, brick_base(x, up ? wrap1(y0 - 1, ny) : wrap1(y0 + h, ny), nxb, NS), fb0);
    load_stored<Sys, T, R, FORM>(fin, brick_base(x, row_of(0), nxb, NS), fr0);
    R o[5][P];
    if (up) {
      post_loaded<Sys, R, C_Q4, FORM>(sys, fb0, xinv, c, om, set, kk, ch, o);
#pragma unroll
      for (int i = 0; i < P; ++i) fbp[i] = o[3][i];
    } else {
      post_loaded<Sys, R, C_Q5, FORM>(sys, fb0, xinv, c, om, set, kk, ch, o);
#pragma unroll
      for (int i = 0; i < P; ++i) fbp[i] = o[4][i];
    }
    post_loaded<Sys, R, C_FULL, FORM>(sys, fr0, xinv, c, om, set, kk, ch, o);
    CV::put(rb1 + tx * PP, o[0]);
    CV::put(rb2 + tx * PP, o[1]);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      f3c[i] = o[2][i];
      fbc[i] = up ? o[3][i] : o[4][i];
    }
  }
  for (int t = tx; t < 2 * h; t += blockDim.x) {
    const int side = t >= h;
    const int r = side ? t - h : t;
    const int xr = side ? wrap1(x0 + w, nx) : wrap1(x0 - 1, nx);
    R o[5][P];
    if (!side) {
      cell_post<Sys, T, R, C_Q1, FORM, true>(sys, fin, xr, y0 + r, nxb, xinv, c, om, set, kk, ch, o);
      CV::put(ringL + r * PP, o[0]);
    } else {
      cell_post<Sys, T, R, C_Q2, FORM, true>(sys, fin, xr, y0 + r, nxb, xinv, c, om, set, kk, ch, o);
      CV::put(ringR + r * PP, o[1]);
    }
  }

  R m1 = R(0), m2 = R(0);
  bool bad = false;
  int nb = 1, cb = 0;   // row buffers of rows r + 1 and r: (r + 1) mod 3, r mod 3
  // Software-pipelined rows: iteration r loads the stored values of row r + 1
  // first, and while they arrive finishes row r - 1 (the component streaming
  // from row r, its sum and the CFL epilogue) and as much of row r as does not
  // need row r + 1 (stores and partial sums of the other four components);
  // then row r + 1's collision.  Row r's f*_1 / f*_2 were published by the
  // row barrier's arrivals ending iteration r - 1; a thread waits on them only
  // after the loads and row r - 1's finish, which touch no shared memory.  The
  // three row buffers make one phase of slack safe: a thread past the wait of
  // iteration r writes buffer (r + 1) mod 3, while the slowest is still in
  // iteration r, reading buffer r mod 3.
  __syncthreads();
  constexpr int QB = up ? 3 : 4;   // component streaming from the row behind
  constexpr int QA = up ? 4 : 3;   // component streaming from the row ahead
  const T* tp = nullptr;
  R acc[P], held[P], fan[P];       // row r - 1's partial sums and its missing component
  auto finish_late = [&](int jr) {
    const size_t base = brick_base(x, jr, nxb, NS);
    R U[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      if constexpr (FORM == 0) {
        Store<T>::st(fout + (size_t)(QA * P + i) * kBrick + base, fan[i]);
        U[i] = up ? acc[i] + round_store(fan[i], tp) : (acc[i] + round_store(fan[i], tp)) + held[i];
      } else {
        const R u = up ? acc[i] + fan[i] : (acc[i] + fan[i]) + held[i];
        Store<T>::st(fout + (size_t)i * kBrick + base, u);
        U[i] = round_store(u, tp);
      }
    }
    if (!(a.cbx | a.cby) || !on_char_face(a, x, jr)) {   // periodic grids skip the face test
      R e1, e2;
      bad |= !sys.epilogue(U, e1, e2);
      m1 = vmax(m1, e1);
      m2 = vmax(m2, e2);
    }
  };
  bool waiting = true;
  for (int r = 0; r < h; ++r) {
    const int j = row_of(r);
    const bool nxt = r + 1 < h;
    R f3n[P], fbn[P];
    R fl[5][P];
    if (act) {
      const int jn = nxt ? row_of(r + 1) : (up ? wrap1(y0 + h, ny) : wrap1(y0 - 1, ny));
      load_stored<Sys, T, R, FORM>(fin, brick_base(x, jn, nxb, NS), fl);
      if (r > 0) finish_late(row_of(r - 1));
    }
    // row r's f*_1 / f*_2, written in iteration r - 1; every thread waits
    // (including those without a column), so that none arrives twice in a phase
    if (r > 0 && waiting && !rowbar_wait(&rowbar, (uint32_t)((r - 1) & 1))) {
      atomicOr(&a.ctl->err, ERR_TIMEOUT);
      waiting = false;
    }
    if (act) {
      const size_t base = brick_base(x, j, nxb, NS);
      const int rt = j - y0;
      // the x neighbours' components, picked by offset from one shared base (a
      // select between two pointers would lose their state space)
      R* const sm = rb1;
      R g0[P], g1[P];
      CV::get(sm + (tx == 0 ? (int)(ringL - sm) + rt * PP : (cb * TX + tx - 1) * PP), g0);
      CV::get(sm + (tx == w - 1 ? (int)(ringR - sm) + rt * PP : (int)(rb2 - sm) + (cb * TX + tx + 1) * PP), g1);
#pragma unroll
      for (int i = 0; i < P; ++i) {
        if constexpr (FORM == 0) {
          Store<T>::st(fout + (size_t)(0 * P + i) * kBrick + base, g0[i]);
          Store<T>::st(fout + (size_t)(1 * P + i) * kBrick + base, g1[i]);
          Store<T>::st(fout + (size_t)(2 * P + i) * kBrick + base, f3c[i]);
          Store<T>::st(fout + (size_t)(QB * P + i) * kBrick + base, fbp[i]);
          R sum = ((R(0) + round_store(g0[i], tp)) + round_store(g1[i], tp)) + round_store(f3c[i], tp);
          if (up) sum += round_store(fbp[i], tp);
          acc[i] = sum;
          held[i] = round_store(fbp[i], tp);
        } else {
          R sum = (g0[i] + g1[i]) + f3c[i];
          if (up) sum = sum + fbp[i];
          acc[i] = sum;
          held[i] = fbp[i];
        }
      }
      R o[5][P];
      if (nxt) {
        post_loaded<Sys, R, C_FULL, FORM>(sys, fl, xinv, c, om, set, kk, ch, o);
        CV::put(rb1 + (nb * TX + tx) * PP, o[0]);
        CV::put(rb2 + (nb * TX + tx) * PP, o[1]);
#pragma unroll
        for (int i = 0; i < P; ++i) {
          f3n[i] = o[2][i];
          fbn[i] = up ? o[3][i] : o[4][i];
          fan[i] = up ? o[4][i] : o[3][i];
        }
      } else {
        if (up) {
          post_loaded<Sys, R, C_Q5, FORM>(sys, fl, xinv, c, om, set, kk, ch, o);
#pragma unroll
          for (int i = 0; i < P; ++i) fan[i] = o[4][i];
        } else {
          post_loaded<Sys, R, C_Q4, FORM>(sys, fl, xinv, c, om, set, kk, ch, o);
#pragma unroll
          for (int i = 0; i < P; ++i) fan[i] = o[3][i];
        }
#pragma unroll
        for (int i = 0; i < P; ++i) f3n[i] = fbn[i] = R(0);
      }
    }
    rowbar_arrive(&rowbar);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      fbp[i] = fbc[i];
      f3c[i] = f3n[i];
      fbc[i] = fbn[i];
    }
    nb = next3(nb);
    cb = next3(cb);
  }
  if (act && h > 0) finish_late(row_of(h - 1));
  commit_max<R>(m1, m2, bad, a.ctl, s1);
}

// The same march for a system whose split is long (MHD-GLM: two 9-wave
// eigen-decompositions a cell), written so that the split's code appears as few
// times as possible: the direction is picked at run time, the ring rows behind
// and ahead of the tile go through the same call as the tile's rows (computing
// an x split they do not need, 2 rows a tile), and the x ring's two sides share
// one call.  Each inlined copy of the split is several kilobytes of code; with
// one copy per call site the march above holds ten, which overflow the
// instruction cache (measured: 68 % hit rate, instruction fetch the largest
// stall).  The registers go to the split: the column's march state waits in
// shared memory, and f is not held across the split (collide_d2q5); with both,
// the FP32 step of a 2048^2 grid went from 0.68 to 0.48 ms.  Rows in march
// order: R_-1 (the ring row behind), R_0 .. R_{h-1}, R_h (the ring row ahead);
// row r is finished once R_{r+1} is collided.
template <class Sys, class T, class R, int FORM, int TXC>
__device__ __forceinline__ void step2d_tile_one(const StepArgs<T>& a, const BlockConsts<Sys, R>& bc, int bx,
                                                int by, int TX_, int TY, unsigned char* smem, int set) {
  const int TX = TXC > 0 ? TXC : TX_;   // tile width, a compile-time constant where TXC > 0
  constexpr int P = Sys::P;
  const bool up = (by & 1) == 0;
  const Sys sys = bc.sys;
  const int tx = threadIdx.x;
  const int x0 = bx * TX, y0 = by * TY;
  const int nx = a.nx, ny = a.ny;
  const int w = min(TX, nx - x0), h = min(TY, ny - y0);
  const int x = x0 + tx;
  const bool act = tx < w;
  constexpr int NS = StateForm<Sys, FORM>::NS;
  const int nxb = a.pitch / kBrick;
  const T* __restrict__ fin = a.src();
  T* __restrict__ fout = a.dst();
  const int s1 = (a.slot + 1) % 3;
  const R xinv = bc.xinv, ch = bc.ch, c = bc.c, om = bc.om, kk = bc.k;

  // Component-major row buffers: with the tile width known at compile time
  // (TXC, the host's instantiation for 128-wide tiles) every component of a
  // row sits at a constant offset from one base; measured 8 % fewer
  // instructions than the width at run time and 4 % fewer than a cell-major
  // layout (MHD-GLM, FP32).
  R* rb1 = reinterpret_cast<R*>(smem);   // [3][P][TX]  f*_1 of the row
  R* rb2 = rb1 + 3 * P * TX;             // [3][P][TX]  f*_2 of the row
  R* ringL = rb2 + 3 * P * TX;           // [TY][P]     f*_1 at x0 - 1, by tile row
  R* ringR = ringL + P * TY;             // [TY][P]     f*_2 at x0 + w

  __shared__ __align__(8) uint64_t rowbar;
  if (tx == 0) {
    rowbar_init(&rowbar, blockDim.x);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool waiting = true;
  // x ring, read up front with the L2 keep policy (as in the march above):
  // from the halo of the neighbouring tiles when the last step wrote it (the
  // left ring is the left neighbour's last column, the right ring the right
  // neighbour's first), else from the bricks.  The loops stay rolled so that
  // the split is not copied.
  const T* __restrict__ hin = a.halo_in();
  T* __restrict__ hout = a.halo_out();
  const int nbx = (nx + TX - 1) / TX;
#pragma unroll 1
  for (int t = tx; t < 2 * h; t += blockDim.x) {
    const int side = t >= h;
    const int r = side ? t - h : t;
    const T* src = fin;
    size_t plane = kBrick, b;
    if (hin) {
      src = hin;
      plane = 1;
      b = halo_index(side ? (bx + 1) % nbx : (bx - 1 + nbx) % nbx, side ? 0 : 1, y0 + r, ny, NS);
    } else {
      b = brick_base(side ? (x0 + w) % nx : (x0 - 1 + nx) % nx, y0 + r, nxb, NS);
    }
    R o[5][P];
    cell_post_at<Sys, T, R, C_QX, FORM, true>(sys, src, plane, b, xinv, c, om, set, kk, ch, o);
    R* dst = side ? ringR : ringL;
#pragma unroll
    for (int i = 0; i < P; ++i) dst[r * P + i] = side ? o[1][i] : o[0][i];
  }

  // The march state of this thread's column lives in shared memory, not in
  // registers across the split: the component streaming along the march of the
  // last two rows (beh, by row parity) and f*_3 of the last row (f3s).  Only
  // the thread itself touches its column, so no barrier guards them.
  R* beh = ringR + P * TY;                // [2][P][TX]
  R* f3s = beh + 2 * P * TX;              // [P][TX]
  R m1 = R(0), m2 = R(0);
  bool bad = false;
  int nbr = 2, cbr = 1;   // (r + 3) % 3 and (r + 2) % 3
#pragma unroll 1
  for (int r = -1; r <= h; ++r) {
    R an[P], bn[P], f3n[P];
    if (act) {
      int jr = up ? y0 + r : y0 + h - 1 - r;
      jr = jr < 0 ? jr + ny : (jr >= ny ? jr - ny : jr);
      R o[5][P];
      cell_post<Sys, T, R, C_FULL, FORM>(sys, fin, x, jr, nxb, xinv, c, om, set, kk, ch, o);
      const int nb = nbr;
#pragma unroll
      for (int i = 0; i < P; ++i) {
        if (r >= 0 && r < h) {
          rb1[(nb * P + i) * TX + tx] = o[0][i];
          rb2[(nb * P + i) * TX + tx] = o[1][i];
        }
        f3n[i] = o[2][i];
        bn[i] = up ? o[3][i] : o[4][i];
        an[i] = up ? o[4][i] : o[3][i];
      }
    }
    if (r >= 1) {
      // finish row r - 1 of the march, once every thread is done with iteration
      // r - 1 (phase r - 1: a thread arrives from iteration 0 on, and waits
      // between any two of its arrivals, so none runs two phases ahead).  Row
      // r - 1's f*_1 / f*_2 were written in that iteration; the buffer this
      // iteration wrote before the wait, (r mod 3), was last read in iteration
      // r - 2, which the wait of iteration r - 1 saw finished.  Unlike a
      // barrier after the split, a thread whose split ran long no longer holds
      // up the others' finish.
      if (waiting && !rowbar_wait(&rowbar, (uint32_t)((r - 1) & 1))) {
        atomicOr(&a.ctl->err, ERR_TIMEOUT);
        waiting = false;
      }
      if (act) {
        const int rr = r - 1;
        const int j = up ? y0 + rr : y0 + h - 1 - rr;
        const int cb = cbr;
        const size_t base = brick_base(x, j, nxb, NS);
        const int rt = j - y0;
        const R* bp = beh + (r & 1) * P * TX;          // behind component of R_{r-2}
        // the tile's edge columns also go to the halo of f^{n+1}
        T* const h0 = hout && tx == 0 ? hout + halo_index(bx, 0, j, ny, NS) : nullptr;
        T* const h1 = hout && tx == w - 1 ? hout + halo_index(bx, 1, j, ny, NS) : nullptr;
        R U[P];
#pragma unroll
        for (int i = 0; i < P; ++i) {
          R g[5];
          g[0] = tx == 0 ? ringL[rt * P + i] : rb1[(cb * P + i) * TX + tx - 1];
          g[1] = tx == w - 1 ? ringR[rt * P + i] : rb2[(cb * P + i) * TX + tx + 1];
          g[2] = f3s[i * TX + tx];
          const R bv = bp[i * TX + tx];
          g[3] = up ? bv : an[i];
          g[4] = up ? an[i] : bv;
          const T* tp = nullptr;
          if constexpr (FORM == 0) {
            R acc = R(0);
#pragma unroll
            for (int q = 0; q < 5; ++q) {
              Store<T>::st(fout + (size_t)(q * P + i) * kBrick + base, g[q]);
              if (h0) Store<T>::st(h0 + q * P + i, g[q]);
              if (h1) Store<T>::st(h1 + q * P + i, g[q]);
              acc += round_store(g[q], tp);
            }
            U[i] = acc;
          } else {
            const R u = (((g[0] + g[1]) + g[2]) + g[3]) + g[4];
            Store<T>::st(fout + (size_t)i * kBrick + base, u);
            if (h0) Store<T>::st(h0 + i, u);
            if (h1) Store<T>::st(h1 + i, u);
            U[i] = round_store(u, tp);
          }
        }
        if (!on_char_face(a, x, j)) {
          R e1, e2;
          bad |= !sys.epilogue(U, e1, e2);
          m1 = vmax(m1, e1);
          m2 = vmax(m2, e2);
        }
      }
    }
    if (act) {
      R* bw = beh + (r & 1) * P * TX;                  // R_r's slot (R_{r-2}'s, just read)
#pragma unroll
      for (int i = 0; i < P; ++i) {
        bw[i * TX + tx] = bn[i];
        f3s[i * TX + tx] = f3n[i];
      }
    }
    if (r >= 0) rowbar_arrive(&rowbar);
    nbr = nbr == 2 ? 0 : nbr + 1;
    cbr = cbr == 2 ? 0 : cbr + 1;
  }
  commit_max<R>(m1, m2, bad, a.ctl, s1);
}

template <class Sys, class T, class R, int FORM = 0, int TXC = 0>
__device__ __forceinline__ void step2d_tile(const StepArgs<T>& a, int bx, int by, int TX, int TY,
                                            unsigned char* smem) {
  constexpr int NS = StateForm<Sys, FORM>::NS;
  const int tx = threadIdx.x;
  const int x0 = bx * TX, y0 = by * TY;
  // the step's scalars in FP64 by one thread per block (FP64 is slow on this
  // part), shared with the others
  __shared__ StepScalars s_sc;
  __shared__ BlockConsts<Sys, R> s_bc;
  if (tx == 0) {
    s_sc = step_scalars(a.ctl, a.slot, Sys::MHD, a.ch_factor, a.inv_nu, a.fixed_xi, a.t_end, a.dx);
    s_bc = block_consts<Sys, R>(a, s_sc);
  }
  __syncthreads();
  if (s_sc.done) {
    // t_end already reached: this launch is a no-op that keeps the ping-pong
    // consistent (f^{n+1} = f^n, same control words).
    const int w = min(TX, a.nx - x0), h = min(TY, a.ny - y0);
    T* const hout = Sys::P > 4 ? a.halo_out() : nullptr;   // the long-split march's halo
    if (tx < w)
      for (int r = 0; r < h; ++r)
        for (int i = 0; i < NS; ++i) {
          const size_t o = brick_base(x0 + tx, y0 + r, a.pitch / kBrick, NS) + (size_t)i * kBrick;
          const T v = a.src()[o];
          a.dst()[o] = v;
          if (hout && tx == 0) hout[halo_index(bx, 0, y0 + r, a.ny, NS) + i] = v;
          if (hout && tx == w - 1) hout[halo_index(bx, 1, y0 + r, a.ny, NS) + i] = v;
        }
    if (bx == 0 && by == 0 && tx == 0) {
      const int s1 = (a.slot + 1) % 3, s2 = (a.slot + 2) % 3;
      a.ctl->t[s1] = a.ctl->t[a.slot];
      a.ctl->m1[s1] = a.ctl->m1[a.slot];
      a.ctl->m2[s1] = a.ctl->m2[a.slot];
      a.ctl->m1[s2] = 0ull;
      a.ctl->m2[s2] = 0ull;
    }
    return;
  }
  if (bx == 0 && by == 0 && tx == 0) step_bookkeeping(a.ctl, a.slot, s_sc, a.dx, a.fixed_xi, Sys::MHD);
  if constexpr (Sys::P <= 4) {
    if (by & 1)
      step2d_tile_dir<Sys, T, R, -1, FORM>(a, s_bc, bx, by, TX, TY, smem);
    else
      step2d_tile_dir<Sys, T, R, +1, FORM>(a, s_bc, bx, by, TX, TY, smem);
  } else {
    // The weighted set (Eq. 41) gets its own copy of the march, compiled under
    // the test that selects it.  Measured for MHD-GLM (FP32 2048^2, with a block
    // barrier per row at the time): 321 us with this form, 327 us passing the
    // set as a literal in that copy, 336 us with one copy; the short splits
    // gain nothing.
    if (a.set == SET_WEIGHTED)
      step2d_tile_one<Sys, T, R, FORM, TXC>(a, s_bc, bx, by, TX, TY, smem, a.set);
    else
      step2d_tile_one<Sys, T, R, FORM, TXC>(a, s_bc, bx, by, TX, TY, smem, a.set);
  }
}

// ------------------------------------------------- D2Q5 step, bulk-copy rows
// Same arithmetic as step2d_tile, but the rows of f^n reach the block through
// shared memory by 1D bulk asynchronous copies (cp.async.bulk, the TMA engine):
// in the brick layout a tile row is one contiguous range, so one copy per row,
// D rows ahead, each stage completing on its own mbarrier.  There is one block barrier per row, as
// in the plain march: before it, thread 0 waits for the next row's copies, so
// the barrier also publishes that row to the block; after it, the lanes of warp
// 0 refill the stage just consumed.  Every mbarrier wait is bounded; a wait that
// gives up sets ERR_TIMEOUT and the block leaves the tile after all threads
// agree, waiting (bounded) for its copies still in flight.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Gives up after limit_ns nanoseconds of polling (checked every 64 polls).
constexpr uint64_t kWaitNs = 2000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0 && global_ns() - t0 > limit_ns) return false;
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives at, gives up after limit_ns and latches ERR_TIMEOUT in the error word,
// as the bulk-copy step does when a copy never lands.  Bounded: it cannot hang.
static __global__ void wait_selftest_kernel(Ctl* ctl, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, limit_ns)) atomicOr(&ctl->err, ERR_TIMEOUT);
  __syncthreads();
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <class T>
struct TmaLayout {
  int TX, TY, D;
  size_t stage_elems;       // elements of one stage (TX / 32 bricks of 5p x 32)
  size_t off_stage, off_rb, off_ring, bytes;
  template <class R, int P>
  VK_HD static TmaLayout make(int TX, int TY, int D) {
    TmaLayout L;
    L.TX = TX;
    L.TY = TY;
    L.D = D;
    L.stage_elems = (size_t)5 * P * TX;
    L.off_stage = 128;
    L.off_rb = L.off_stage + (size_t)D * L.stage_elems * sizeof(T);
    L.off_rb = (L.off_rb + 15) & ~(size_t)15;
    L.off_ring = L.off_rb + (size_t)4 * P * TX * sizeof(R);
    L.bytes = L.off_ring + (size_t)2 * P * TY * sizeof(R) + 16;
    return L;
  }
};

// The march over stream rows 0 .. h+1 (ring row behind, the h tile rows in
// march order, ring row ahead).  Iteration j collides row j from its stage and
// then writes stream row j-1, whose f*_1 / f*_2 exchange buffer the previous
// barrier published; so two exchange buffers suffice.  The x-ring cells are
// collided up front from global memory.  Tiles march up or down by tile-row
// parity.
template <class Sys, class T, class R>
__device__ __forceinline__ void step2d_tile_tma(const StepArgs<T>& a, int bx, int by, int TX, int TY, int D,
                                                unsigned char* smem) {
  constexpr int P = Sys::P;
  constexpr int NPL = 5 * P;
  const TmaLayout<T> L = TmaLayout<T>::template make<R, P>(TX, TY, D);
  const int tid = threadIdx.x;
  const int x0 = bx * TX, y0 = by * TY;
  const int nx = a.nx, ny = a.ny;
  const int nxb = a.pitch / kBrick;
  const int w = min(TX, nx - x0), h = min(TY, ny - y0);
  const int x = x0 + tid;
  const bool act = tid < w;
  const bool up = (by & 1) == 0;
  constexpr size_t plane = kBrick;   // component stride in the brick layout
  const T* __restrict__ fin = a.src();
  T* __restrict__ fout = a.dst();
  __shared__ StepScalars s_sc;
  __shared__ BlockConsts<Sys, R> s_bc;
  if (tid == 0) {
    s_sc = step_scalars(a.ctl, a.slot, Sys::MHD, a.ch_factor, a.inv_nu, a.fixed_xi, a.t_end, a.dx);
    s_bc = block_consts<Sys, R>(a, s_sc);
  }
  __syncthreads();
  const int s1 = (a.slot + 1) % 3;
  if (s_sc.done) {
    if (act)
      for (int r = 0; r < h; ++r)
        for (int i = 0; i < NPL; ++i) {
          const size_t o = brick_base(x, y0 + r, nxb, NPL) + (size_t)i * kBrick;
          fout[o] = fin[o];
        }
    if (bx == 0 && by == 0 && tid == 0) {
      const int s2 = (a.slot + 2) % 3;
      a.ctl->t[s1] = a.ctl->t[a.slot];
      a.ctl->m1[s1] = a.ctl->m1[a.slot];
      a.ctl->m2[s1] = a.ctl->m2[a.slot];
      a.ctl->m1[s2] = 0ull;
      a.ctl->m2[s2] = 0ull;
    }
    return;
  }
  if (bx == 0 && by == 0 && tid == 0) step_bookkeeping(a.ctl, a.slot, s_sc, a.dx, a.fixed_xi, Sys::MHD);
  const Sys sys = s_bc.sys;
  const R xinv = s_bc.xinv, ch = s_bc.ch, c = s_bc.c, om = s_bc.om, kk = s_bc.k;
  const int set = a.set;

  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  T* stages = reinterpret_cast<T*>(smem + L.off_stage);
  R* rb1 = reinterpret_cast<R*>(smem + L.off_rb);   // [2][P][TX]  f*_1 of the row
  R* rb2 = rb1 + 2 * P * TX;                       // [2][P][TX]  f*_2 of the row
  R* ringL = reinterpret_cast<R*>(smem + L.off_ring);  // [TY][P]  f*_1 at x0 - 1
  R* ringR = ringL + P * TY;                           // [TY][P]  f*_2 at x0 + w
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.off_ring + 2 * P * TY * sizeof(R));

  const int nrows = h + 2;
  // whole bricks of the tile row: (w + 31) / 32 of 5p x 32 elements
  const uint32_t row_bytes = (uint32_t)((size_t)((w + kBrick - 1) / kBrick) * NPL * kBrick * sizeof(T));
  auto row_y = [&](int j) -> int {
    if (j == 0) return up ? wrap1(y0 - 1, ny) : wrap1(y0 + h, ny);
    if (j == nrows - 1) return up ? wrap1(y0 + h, ny) : wrap1(y0 - 1, ny);
    return up ? y0 + j - 1 : y0 + h - j;
  };
  // thread 0: stream row j into stage j % D, one copy
  auto issue = [&](int j) {
    const int s = j % D;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bars[s], row_bytes);
    bulk_g2s(stages + (size_t)s * L.stage_elems, fin + brick_base(x0, row_y(j), nxb, NPL), row_bytes, &bars[s]);
  };

  if (tid == 0) {
    for (int s = 0; s < D; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
    *abort_flag = 0;
  }
  __syncthreads();
  if (tid == 0)
    for (int j = 0; j < min(D, nrows); ++j) issue(j);
  int issued = min(D, nrows);

  // x ring: only the component that streams into the tile, from the x split
  for (int t = tid; t < 2 * h; t += TX) {
    const int side = t >= h;
    const int r = side ? t - h : t;
    const int xr = side ? wrap1(x0 + w, nx) : wrap1(x0 - 1, nx);
    const size_t idx = brick_base(xr, y0 + r, nxb, NPL);
    R o[5][P];
    collide_d2q5<Sys, T, R, C_Q1, true>(sys, fin, plane, idx, xinv, c, om, set, kk, ch, o);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      if (side)
        ringR[i * TY + r] = o[1][i];
      else
        ringL[i * TY + r] = o[0][i];
    }
  }
  if (tid == 0 && !mbar_wait_bounded(&bars[0], 0u)) *abort_flag = 1;
  __syncthreads();   // row 0 and the ring published
  bool aborted = *abort_flag != 0;
  int waiting = 0;   // first row whose copies may still be in flight

  R fbp[P], f3c[P], fbc[P];
#pragma unroll
  for (int i = 0; i < P; ++i) fbp[i] = f3c[i] = fbc[i] = R(0);
  R m1 = R(0), m2 = R(0);
  bool bad = false;
  const size_t sidx = (size_t)(tid >> 5) * NPL * kBrick + (tid & 31);   // this column in a stage
  for (int j = 0; j < nrows && !aborted; ++j) {
    const T* st = stages + (size_t)(j % D) * L.stage_elems;
    if (act) {
      R o[5][P];
      if (j == 0) {
        if (up)
          collide_d2q5<Sys, T, R, C_Q4>(sys, st, plane, sidx, xinv, c, om, set, kk, ch, o);
        else
          collide_d2q5<Sys, T, R, C_Q5>(sys, st, plane, sidx, xinv, c, om, set, kk, ch, o);
      } else if (j <= h) {
        collide_d2q5<Sys, T, R, C_FULL>(sys, st, plane, sidx, xinv, c, om, set, kk, ch, o);
        const int nb = (j - 1) & 1;
#pragma unroll
        for (int i = 0; i < P; ++i) {
          rb1[(nb * P + i) * TX + tid] = o[0][i];
          rb2[(nb * P + i) * TX + tid] = o[1][i];
        }
      } else if (up) {
        collide_d2q5<Sys, T, R, C_Q5>(sys, st, plane, sidx, xinv, c, om, set, kk, ch, o);
      } else {
        collide_d2q5<Sys, T, R, C_Q4>(sys, st, plane, sidx, xinv, c, om, set, kk, ch, o);
      }
      if (j >= 2) {   // stream row j - 1 (a tile row) is complete
        const int yo = row_y(j - 1);
        const int rt = yo - y0;
        const int cb = (j - 2) & 1;
        const size_t base = brick_base(x, yo, nxb, NPL);
        R U[P];
#pragma unroll
        for (int i = 0; i < P; ++i) {
          R g[5];
          g[0] = tid == 0 ? ringL[i * TY + rt] : rb1[(cb * P + i) * TX + tid - 1];
          g[1] = tid == w - 1 ? ringR[i * TY + rt] : rb2[(cb * P + i) * TX + tid + 1];
          g[2] = f3c[i];
          g[3] = up ? fbp[i] : o[3][i];
          g[4] = up ? o[4][i] : fbp[i];
          const T* tp = nullptr;
          R acc = R(0);
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            Store<T>::st(fout + (size_t)(q * P + i) * plane + base, g[q]);
            acc += round_store(g[q], tp);
          }
          U[i] = acc;
        }
        R e1, e2;
        bad |= !sys.epilogue(U, e1, e2);
        m1 = vmax(m1, e1);
        m2 = vmax(m2, e2);
      }
      if (j <= h) {
#pragma unroll
        for (int i = 0; i < P; ++i) {
          fbp[i] = fbc[i];
          fbc[i] = up ? o[3][i] : o[4][i];
          if (j > 0) f3c[i] = o[2][i];   // (row 0 is a ring row: its collision has no f*_3)
        }
      }
    }
    if (tid == 0 && j + 1 < nrows && !mbar_wait_bounded(&bars[(j + 1) % D], (uint32_t)(((j + 1) / D) & 1)))
      *abort_flag = 1;
    __syncthreads();   // row j consumed; row j + 1 and the exchange buffer of row j published
    aborted = *abort_flag != 0;
    waiting = j + 1;
    if (!aborted && j + D < nrows) {
      if (tid == 0) issue(j + D);
      issued = j + D + 1;
    }
  }
  if (aborted) {
    // a wait gave up: report it and let the copies still in flight land first
    if (tid == 0) {
      atomicOr(&a.ctl->err, ERR_TIMEOUT);
      for (int j = waiting; j < issued; ++j) mbar_wait_bounded(&bars[j % D], (uint32_t)((j / D) & 1));
    }
    __syncthreads();
    return;
  }
  commit_max<R>(m1, m2, bad, a.ctl, s1);
}

template <class Sys, class T, class R, int TXC = 0>
__global__ void step2d_kernel(StepArgs<T> a, int TX, int TY) {
  extern __shared__ __align__(128) unsigned char smem[];
  step2d_tile<Sys, T, R, 0, TXC>(a, blockIdx.x, blockIdx.y, TX, TY, smem);
}

// The moment form (omega = 1): U in, U out, p components a cell.
template <class Sys, class T, class R, int TXC = 0>
__global__ void step2d_u_kernel(StepArgs<T> a, int TX, int TY) {
  extern __shared__ __align__(128) unsigned char smem[];
  step2d_tile<Sys, T, R, 1, TXC>(a, blockIdx.x, blockIdx.y, TX, TY, smem);
}

// Register bound of the plain step: blocks of at most 128 threads with at least
// `min_blocks` of them resident per SM (0 = no bound).  FP32 MHD-GLM needs about
// 170 registers a thread unbounded (3 blocks of 4 warps per SM); capped at 128
// (4 blocks) it fits without spills and runs faster.
template <class Sys, class R>
struct StepBound {
  static constexpr int min_blocks = 0;
};
template <>
struct StepBound<MHDGLM<float>, float> {
  static constexpr int min_blocks = 4;
};
// FP32 Euler (also with BF16 storage): 72 registers keep 7 blocks of 128
// threads resident, the occupancy its 128 x 8 tiles need to fill a 1024^2 grid
// in one wave; unbounded it takes 76 (6 blocks).
template <>
struct StepBound<Euler<float, 2>, float> {
  static constexpr int min_blocks = 7;
};

template <class Sys, class T, class R, int MINB, int FORM = 0, int TXC = 0>
__global__ void __launch_bounds__(128, MINB) step2d_lb_kernel(StepArgs<T> a, int TX, int TY) {
  extern __shared__ __align__(128) unsigned char smem[];
  step2d_tile<Sys, T, R, FORM, TXC>(a, blockIdx.x, blockIdx.y, TX, TY, smem);
}

template <class Sys, class T, class R>
__global__ void step2d_tma_kernel(StepArgs<T> a, int TX, int TY, int D) {
  extern __shared__ __align__(128) unsigned char smem[];
  step2d_tile_tma<Sys, T, R>(a, blockIdx.x, blockIdx.y, TX, TY, D, smem);
}

// Batched form: one launch advances every simulation of the batch by one step.
// work[b] = (simulation, tile x, tile y) of block b; desc[s] describes
// simulation s with its parity / slot at the batch's step 0; step_off moves them.
struct BatchWork {
  int sim, bx, by;
};

template <class Sys, class T, class R, int VARIANT, int TXC = 0>
__device__ __forceinline__ void step2d_batch_body(const StepArgs<T>* __restrict__ desc,
                                                  const BatchWork* __restrict__ work, int step_off, int TX, int TY,
                                                  int D, unsigned char* smem) {
  const BatchWork wk = work[blockIdx.x];
  StepArgs<T> a = desc[wk.sim];
  a.parity = (a.parity + step_off) & 1;
  a.slot = (a.slot + step_off) % 3;
  if constexpr (VARIANT == 1)
    step2d_tile_tma<Sys, T, R>(a, wk.bx, wk.by, TX, TY, D, smem);
  else if constexpr (VARIANT == 2)
    step2d_tile<Sys, T, R, 1, TXC>(a, wk.bx, wk.by, TX, TY, smem);   // moment form
  else
    step2d_tile<Sys, T, R, 0, TXC>(a, wk.bx, wk.by, TX, TY, smem);
}

template <class Sys, class T, class R, int VARIANT, int TXC = 0>
__global__ void step2d_batch_kernel(const StepArgs<T>* __restrict__ desc, const BatchWork* __restrict__ work,
                                    int step_off, int TX, int TY, int D) {
  extern __shared__ __align__(128) unsigned char smem[];
  step2d_batch_body<Sys, T, R, VARIANT, TXC>(desc, work, step_off, TX, TY, D, smem);
}

// The batched step with the plain step's register bound (StepBound), for blocks
// of at most 128 threads (plain and moment-form bodies).
template <class Sys, class T, class R, int VARIANT, int MINB, int TXC = 0>
__global__ void __launch_bounds__(128, MINB)
    step2d_batch_lb_kernel(const StepArgs<T>* __restrict__ desc, const BatchWork* __restrict__ work, int step_off,
                           int TX, int TY, int D) {
  extern __shared__ __align__(128) unsigned char smem[];
  step2d_batch_body<Sys, T, R, VARIANT, TXC>(desc, work, step_off, TX, TY, D, smem);
}

// ------------------------------------------------ 2D characteristic faces
// The construction of Eqs. (33)-(36) applied along the normal of every
// characteristic face of a D2Q5 grid, after the step kernel: the boundary node
// takes U_b^{n+1} = U_b^n - (1/xi_n) P Lambda^out P^-1 D U^n with the one-sided
// difference D towards the interior (a corner sums its two faces), and
// f^{n+1} = f^eq(U_b^{n+1}) with xi_{n+1}.  Boundary nodes are numbered: the
// x faces' columns (2 ny nodes) first, then the y faces' rows without the
// corners already counted (char_face_nodes / char_face_node, vk_ctl.cuh).

template <class Sys, class T, class R>
__device__ __forceinline__ void load_U(const T* __restrict__ f, int x, int y, int nxb, R (&U)[Sys::P]) {
  constexpr int P = Sys::P;
  const size_t b = brick_base(x, y, nxb, 5 * P);
#pragma unroll
  for (int i = 0; i < P; ++i) {
    R acc = R(0);
#pragma unroll
    for (int q = 0; q < 5; ++q) acc += Store<T>::ld(f + b + (size_t)(q * P + i) * kBrick);
    U[i] = acc;
  }
}

// Pass 1: U_b^{n+1} of every boundary node from f^n into Ub ([p][nb]), and its
// wave-speed maximum into the control slot of step n+1 (after the step kernel
// has reduced the interior's).
template <class Sys, class T, class R>
__global__ void char2d_state_kernel(StepArgs<T> a, R* __restrict__ Ub, int nb) {
  constexpr int P = Sys::P;
  const StepScalars sc = step_scalars(a.ctl, a.slot, Sys::MHD, a.ch_factor, a.inv_nu, a.fixed_xi, a.t_end, a.dx);
  if (sc.done) return;   // the step was a no-op (t_end reached): nothing to replace
  const Sys sys = make_sys<Sys>(a.sp);
  const int nxb = a.pitch / kBrick, nx = a.nx, ny = a.ny;
  const T* __restrict__ fin = a.src();
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  R m1 = R(0), m2 = R(0);
  bool bad = false;
  if (id < nb && a.btr) {
    // transmissive faces: U_b^{n+1} = U^{n+1} of the node one cell inwards along
    // each face it lies on (a corner: the diagonal one), from f^{n+1}
    int x, y;
    char_face_node(id, nx, ny, a.cbx, a.cby, x, y);
    const int xi = a.cbx && x == 0 ? 1 : (a.cbx && x == nx - 1 ? nx - 2 : x);
    const int yi = a.cby && y == 0 ? 1 : (a.cby && y == ny - 1 ? ny - 2 : y);
    R U[P];
    load_U<Sys, T, R>(a.dst(), xi, yi, nxb, U);
#pragma unroll
    for (int i = 0; i < P; ++i) Ub[(size_t)i * nb + id] = U[i];
    bad = !sys.epilogue(U, m1, m2);
  } else if (id < nb) {
    int x, y;
    char_face_node(id, nx, ny, a.cbx, a.cby, x, y);
    R U[P], rhs[P];
    load_U<Sys, T, R>(fin, x, y, nxb, U);
#pragma unroll
    for (int i = 0; i < P; ++i) rhs[i] = R(0);
#pragma unroll 1
    for (int d = 0; d < 2; ++d) {
      const bool face = d == 0 ? (a.cbx && (x == 0 || x == nx - 1)) : (a.cby && (y == 0 || y == ny - 1));
      if (!face) continue;
      const int side = (d == 0 ? x : y) == 0 ? 0 : 1;
      const int xn = d == 0 ? (side == 0 ? 1 : nx - 2) : x;
      const int yn = d == 1 ? (side == 0 ? 1 : ny - 2) : y;
      R Un[P], dU[P], t[P];
      load_U<Sys, T, R>(fin, xn, yn, nxb, Un);
#pragma unroll
      for (int i = 0; i < P; ++i) dU[i] = side == 0 ? Un[i] - U[i] : U[i] - Un[i];
      sys.char_rhs_d(U, dU, d, side, (R)sc.ch, t);
#pragma unroll
      for (int i = 0; i < P; ++i) rhs[i] += t[i];
    }
    const R xinv = (R)sc.xinv;
#pragma unroll
    for (int i = 0; i < P; ++i) {
      U[i] = U[i] - rhs[i] * xinv;
      Ub[(size_t)i * nb + id] = U[i];
    }
    bad = !sys.epilogue(U, m1, m2);
  }
  commit_max<R>(m1, m2, bad, a.ctl, (a.slot + 1) % 3);
}

// Pass 2: f^{n+1} = f^eq(U_b^{n+1}) (Eq. 36) at the boundary nodes, with xi_{n+1}
// (and alpha's grid-wide normaliser) from the completed slot of step n+1.
template <class Sys, class T, class R>
__global__ void char2d_feq_kernel(StepArgs<T> a, const R* __restrict__ Ub, int nb) {
  constexpr int P = Sys::P;
  const StepScalars sc = step_scalars(a.ctl, a.slot, Sys::MHD, a.ch_factor, a.inv_nu, a.fixed_xi, a.t_end, a.dx);
  if (sc.done) return;
  const StepScalars sn = step_scalars(a.ctl, (a.slot + 1) % 3, Sys::MHD, a.ch_factor, a.inv_nu, a.fixed_xi,
                                      -1.0, a.dx);
  Sys sys = make_sys<Sys>(a.sp);
  if (a.anorm) sys.lg = (R)sn.lam;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nb) return;
  int x, y;
  char_face_node(id, a.nx, a.ny, a.cbx, a.cby, x, y);
  R U[P], e[5][P];
#pragma unroll
  for (int i = 0; i < P; ++i) U[i] = Ub[(size_t)i * nb + id];
  equilibria_d2q5<Sys, R, C_FULL>(sys, U, (R)sn.xinv, (R)a.c, a.set, (R)a.k, (R)sn.ch, e);
  T* __restrict__ fout = a.dst();
  const size_t b = brick_base(x, y, a.pitch / kBrick, 5 * P);
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int i = 0; i < P; ++i) Store<T>::st(fout + b + (size_t)(q * P + i) * kBrick, e[q][i]);
}

// ------------------------------------------------------------------ D1Q3 steps
// Weighted set in 1D, Eqs. (22)-(24): f1 = c U + F+/xi, f3 = c U - F-/xi,
// f2 = (1 - 2c) U - (F+ - F-)/xi = U - f1 - f3.
template <class Sys, class R>
__device__ __forceinline__ void feq_d1q3(const Sys& sys, const R* U, R xinv, R c, int set, R k,
                                         R (&e)[3][Sys::P]) {
  constexpr int P = Sys::P;
  R Fp[P], F[P];
  sys.split(U, 0, set, k, R(0), Fp, F);
#pragma unroll
  for (int i = 0; i < P; ++i) {
    e[0][i] = c * U[i] + Fp[i] * xinv;
    e[2][i] = c * U[i] - (F[i] - Fp[i]) * xinv;
    e[1][i] = U[i] - (e[0][i] + e[2][i]);
  }
}

template <class Sys, class T, class R>
__global__ void step1d_kernel(StepArgs<T> a, int nsteps) {
  constexpr int P = Sys::P;
  Sys sys = make_sys<Sys>(a.sp);
  const int nx = a.nx;
  const size_t plane = (size_t)nx;
  const bool cl = a.bc_lo != 0, chi = a.bc_hi != 0;        // non-periodic ends
  const bool ccl = a.bc_lo == 1, cchi = a.bc_hi == 1;      // characteristic ones
  const bool trans = (cl && !ccl) || (chi && !cchi);      // a transmissive end
  __shared__ R Ub[2][P];
  __shared__ double red[32];
  int par = a.parity, slot = a.slot;
  volatile Ctl* vc = a.ctl;
  for (int st = 0; st < nsteps; ++st) {
    StepScalars sc = step_scalars(a.ctl, slot, false, 0.0, a.inv_nu, a.fixed_xi, a.t_end, a.dx);
    if (sc.done) break;
    const T* fin = a.f[par];
    T* fout = a.f[par ^ 1];
    const R xinv = (R)(1.0 / sc.xi), c = (R)a.c, om = (R)a.omega, kk = (R)a.k;
    sys.lg = a.anorm ? (R)sc.lam : R(0);
    // collide (Eq. 42) and push-stream (Eq. 43)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      R f[3][P], U[P], e[3][P];
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int s = 0; s < P; ++s) f[q][s] = Store<T>::ld(fin + (size_t)(q * P + s) * plane + i);
#pragma unroll
      for (int s = 0; s < P; ++s) U[s] = f[0][s] + f[1][s] + f[2][s];
      feq_d1q3<Sys, R>(sys, U, xinv, c, a.set, kk, e);
      int ip = i + 1, im = i - 1;
      bool okp = true, okm = true;
      if (ip == nx) { if (chi) okp = false; else ip = 0; }
      if (im < 0) { if (cl) okm = false; else im = nx - 1; }
#pragma unroll
      for (int s = 0; s < P; ++s) {
        R g0 = f[0][s] + om * (e[0][s] - f[0][s]);
        R g1 = f[1][s] + om * (e[1][s] - f[1][s]);
        R g2 = f[2][s] + om * (e[2][s] - f[2][s]);
        if (okp) Store<T>::st(fout + (size_t)(0 * P + s) * plane + ip, g0);
        Store<T>::st(fout + (size_t)(1 * P + s) * plane + i, g1);
        if (okm) Store<T>::st(fout + (size_t)(2 * P + s) * plane + im, g2);
      }
    }
    // characteristic boundaries (Eqs. 33-35): U_b^{n+1} from U^n at x_b and its neighbour
    if (threadIdx.x < 2 && ((threadIdx.x == 0 && ccl) || (threadIdx.x == 1 && cchi))) {
      const int side = threadIdx.x;
      const int ib = side == 0 ? 0 : nx - 1, in = side == 0 ? 1 : nx - 2;
      R Ubv[P], Un[P], dU[P], rhs[P];
#pragma unroll
      for (int s = 0; s < P; ++s) {
        Ubv[s] = Un[s] = R(0);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          Ubv[s] += Store<T>::ld(fin + (size_t)(q * P + s) * plane + ib);
          Un[s] += Store<T>::ld(fin + (size_t)(q * P + s) * plane + in);
        }
        dU[s] = side == 0 ? Un[s] - Ubv[s] : Ubv[s] - Un[s];
      }
      sys.char_rhs(Ubv, dU, side, rhs);
#pragma unroll
      for (int s = 0; s < P; ++s) Ub[side][s] = Ubv[s] - rhs[s] * xinv;
    }
    __syncthreads();
    // transmissive ends: U_b^{n+1} = U^{n+1} of the neighbour, now streamed
    if (trans) {
      if (threadIdx.x < 2 && ((threadIdx.x == 0 && cl && !ccl) || (threadIdx.x == 1 && chi && !cchi))) {
        const int side = threadIdx.x;
        const int in = side == 0 ? 1 : nx - 2;
#pragma unroll
        for (int s = 0; s < P; ++s)
          Ub[side][s] = Store<T>::ld(fout + (size_t)(0 * P + s) * plane + in) +
                        Store<T>::ld(fout + (size_t)(1 * P + s) * plane + in) +
                        Store<T>::ld(fout + (size_t)(2 * P + s) * plane + in);
      }
      __syncthreads();
    }
    // moments of f^{n+1} (Eq. 3) and the CFL max (Eq. 29)
    double m1 = 0.0;
    bool bad = false;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      R U[P];
      if (i == 0 && cl) {
#pragma unroll
        for (int s = 0; s < P; ++s) U[s] = Ub[0][s];
      } else if (i == nx - 1 && chi) {
#pragma unroll
        for (int s = 0; s < P; ++s) U[s] = Ub[1][s];
      } else {
#pragma unroll
        for (int s = 0; s < P; ++s)
          U[s] = Store<T>::ld(fout + (size_t)(0 * P + s) * plane + i) + Store<T>::ld(fout + (size_t)(1 * P + s) * plane + i) +
                 Store<T>::ld(fout + (size_t)(2 * P + s) * plane + i);
      }
      R l1, l2;
      sys.speeds(U, 0, l1, l2);
      m1 = fmax(m1, (double)l1);
      bad |= !sys.physical(U);
    }
    m1 = warp_max(m1);
    const bool wbad = __any_sync(0xffffffffu, bad);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) red[wid] = wbad ? -1.0 : m1;
    __syncthreads();
    if (threadIdx.x == 0) {
      double mm = 0.0;
      bool bb = false;
      for (int wv = 0; wv < nw; ++wv) {
        if (red[wv] < 0.0) bb = true;
        else mm = fmax(mm, red[wv]);
      }
      const int s1 = (slot + 1) % 3, s2 = (slot + 2) % 3;
      vc->t[s1] = vc->t[slot] + a.dx / sc.xi;
      vc->xi_used[slot] = sc.xi;
      vc->nsteps = vc->nsteps + 1;
      vc->m1[s1] = double_to_bits(mm);
      vc->m2[s1] = 0ull;
      vc->m1[s2] = 0ull;
      vc->m2[s2] = 0ull;
      if (bb) vc->err |= ERR_NONPHYS;
      if (a.fixed_xi > 0.0 && bits_to_double(vc->m1[slot]) > a.fixed_xi * (1.0 + 1e-12)) vc->err |= ERR_CFL;
    }
    __syncthreads();
    // boundary distributions f_q(x_b) = f_q^eq(U_b^{n+1}) (Eq. 36), taken with
    // xi_{n+1}, the lattice speed of the step that streams them
    if (threadIdx.x < 2 && ((threadIdx.x == 0 && cl) || (threadIdx.x == 1 && chi))) {
      const int side = threadIdx.x;
      const int ib = side == 0 ? 0 : nx - 1;
      const double ln = bits_to_double(vc->m1[(slot + 1) % 3]);
      const double xn = a.fixed_xi > 0.0 ? a.fixed_xi : ln * a.inv_nu;
      Sys sb = sys;
      if (a.anorm) sb.lg = (R)ln;   // the grid-wide max |lambda| of U^{n+1}
      R e[3][P];
      feq_d1q3<Sys, R>(sb, Ub[side], (R)(1.0 / xn), c, a.set, kk, e);
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int s = 0; s < P; ++s) Store<T>::st(fout + (size_t)(q * P + s) * plane + ib, e[q][s]);
    }
    __syncthreads();
    par ^= 1;
    slot = (slot + 1) % 3;
  }
}

// ------------------------------------------------------------- init / moments
// Max of the wave speeds over U (double, [p][cells]) into slot 0.
template <class Sys, class R, int DIM>
__global__ void init_max_kernel(const double* __restrict__ U, size_t cells, SysParams sp, Ctl* ctl) {
  constexpr int P = Sys::P;
  const Sys sys = make_sys<Sys>(sp);
  double m1 = 0.0, m2 = 0.0;
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
    R u[P];
#pragma unroll
    for (int s = 0; s < P; ++s) u[s] = (R)U[s * cells + i];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      R a, b;
      sys.speeds(u, d, a, b);
      m1 = fmax(m1, (double)a);
      m2 = fmax(m2, (double)b);
    }
    bad |= !sys.physical(u);
  }
  commit_max<double>(m1, m2, bad, ctl, 0);
}

// f_q = f_q^eq(U) (Eq. 2b) with xi_0, c_h^0 from slot 0.  U is dense [p][ny][nx];
// f in the lattice's layout (cell_base / comp_stride).
template <class Sys, class T, class R, int DIM, int FORM = 0>
__global__ void init_feq_kernel(const double* __restrict__ U, size_t cells, StepArgs<T> a) {
  constexpr int P = Sys::P;
  const StepScalars sc = step_scalars(a.ctl, 0, Sys::MHD, a.ch_factor, a.inv_nu, a.fixed_xi, -1.0, a.dx);
  Sys sys = make_sys<Sys>(a.sp);
  if (a.anorm) sys.lg = (R)sc.lam;
  const R xinv = (R)(1.0 / sc.xi), ch = (R)sc.ch, c = (R)a.c, kk = (R)a.k;
  T* f = a.f[a.parity];
  constexpr int Q = DIM == 1 ? 3 : (FORM == 0 ? 5 : 1);
  const size_t plane = comp_stride(Q, a.pitch, a.ny);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
    const size_t y = i / a.nx, x = i - y * a.nx;
    const size_t o = cell_base(Q, P, (int)x, (int)y, a.pitch);
    R u[P];
#pragma unroll
    for (int s = 0; s < P; ++s) u[s] = (R)U[s * cells + i];
    if (DIM == 1) {
      R e[3][P];
      feq_d1q3<Sys, R>(sys, u, xinv, c, a.set, kk, e);
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int s = 0; s < P; ++s) Store<T>::st(f + (size_t)(q * P + s) * plane + o, e[q][s]);
    } else {
      R Fp[P], F[P], e[5][P];
      sys.split(u, 0, a.set, kk, ch, Fp, F);
#pragma unroll
      for (int s = 0; s < P; ++s) {
        e[0][s] = c * u[s] + Fp[s] * xinv;
        e[1][s] = c * u[s] - (F[s] - Fp[s]) * xinv;
      }
      sys.split(u, 1, a.set, kk, ch, Fp, F);
#pragma unroll
      for (int s = 0; s < P; ++s) {
        e[3][s] = c * u[s] + Fp[s] * xinv;
        e[4][s] = c * u[s] - (F[s] - Fp[s]) * xinv;
        e[2][s] = u[s] - (e[0][s] + e[1][s] + e[3][s] + e[4][s]);
      }
      if constexpr (FORM == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
          for (int s = 0; s < P; ++s) Store<T>::st(f + (size_t)(q * P + s) * plane + o, e[q][s]);
      } else {
        // the moments of those distributions, summed in the order of the
        // distribution form's first collision
        const T* tp = nullptr;
#pragma unroll
        for (int s = 0; s < P; ++s) {
          const R u = (((round_store(e[0][s], tp) + round_store(e[1][s], tp)) + round_store(e[2][s], tp)) +
                       round_store(e[3][s], tp)) +
                      round_store(e[4][s], tp);
          Store<T>::st(f + (size_t)s * plane + o, u);
        }
      }
    }
  }
}

// U_k = sum_q f_q,k (Eq. 3), as double, dense [p][ny][nx] from f in the lattice's layout.
template <class T, int P, int Q>
__global__ void moments_kernel(const T* __restrict__ f, int nx, int ny, int pitch, double* __restrict__ U) {
  const size_t cells = (size_t)nx * ny, plane = comp_stride(Q, pitch, ny);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cells; i += (size_t)gridDim.x * blockDim.x) {
    const size_t y = i / nx, x = i - y * nx;
    const size_t o = cell_base(Q, P, (int)x, (int)y, pitch);
#pragma unroll
    for (int s = 0; s < P; ++s) {
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < Q; ++q) acc += (double)Store<T>::ld(f + (size_t)(q * P + s) * plane + o);
      U[s * cells + i] = acc;
    }
  }
}

// Conservation totals, pass 1: block b sums the cells of its fixed chunk in
// FP64 (fixed thread order, shuffle tree), writing part[s][b].
template <class T, int P, int Q>
__global__ void totals_pass1(const T* __restrict__ f, int nx, int ny, int pitch, double* __restrict__ part) {
  __shared__ double red[32];
  const size_t cells = (size_t)nx * ny, plane = comp_stride(Q, pitch, ny);
  const size_t chunk = (cells + gridDim.x - 1) / gridDim.x;
  const size_t lo = blockIdx.x * chunk, hi = min(cells, lo + chunk);
  for (int s = 0; s < P; ++s) {
    double acc = 0.0;
    for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const size_t y = i / nx, x = i - y * nx;
      const size_t o = cell_base(Q, P, (int)x, (int)y, pitch);
#pragma unroll
      for (int q = 0; q < Q; ++q) acc += (double)Store<T>::ld(f + (size_t)(q * P + s) * plane + o);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      part[(size_t)s * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// Pass 2: one thread per field sums the partials in block order.
static __global__ void totals_pass2(const double* __restrict__ part, int nblocks, int P, double scale,
                             double* __restrict__ out) {
  const int s = threadIdx.x;
  if (s >= P) return;
  double t = 0.0;
  for (int b = 0; b < nblocks; ++b) t += part[(size_t)s * nblocks + b];
  out[s] = t * scale;
}

}  // namespace vk
