// Host-side machinery shared by the translation units of libvklb.so: the
// simulation and batch records, the per-(system, precision, lattice) kernel
// launchers (Impl, BatchImpl) and their dispatch tables (Ops).  Each system's
// tables are instantiated in a translation unit of its own (ops_*.cu) so that
// the library compiles in parallel; vklb.cu holds the C ABI.
#pragma once
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "vk_kernels.cuh"
#include "vklb.h"

using namespace vk;

// kernel launches enqueued through the library (vklb_launch_count)
extern std::atomic<long long> g_launches;

const int kRedBlocks = 296;  // conservation-total pass 1: 2 blocks per SM on 148 SMs

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? VKLB_OK : VKLB_ERR_CUDA; }

// True the first time it is called for the current device with this mask:
// function attributes (the dynamic shared-memory limit) are set per device.
inline bool first_on_device(std::atomic<unsigned long long>& mask) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return true;
  }
  const unsigned long long bit = 1ull << dev;
  return (mask.fetch_or(bit) & bit) == 0;
}

struct Ops;

struct vklb_sim {
  int kind, lattice, dim, P, Q, prec, store_bytes;
  int64_t nx, ny, cells, pitch;
  double dx, ch_factor;
  SysParams sp;
  int set;
  int anorm;               // alpha's normaliser: 0 per cell, 1 grid-wide (vklb_alpha_norm)
  double c, k, omega, cfl, fixed_xi;
  double inv_nu;   // xi = inv_nu max|lambda|: 1 / cfl, or sqrt(3/2) / eta
  int bc_lo, bc_hi;
  int cbx, cby;            // 2D: non-periodic faces normal to x / y
  int btr;                 // 2D: those faces are transmissive (else characteristic)
  int nb;                  // 2D: boundary nodes of those faces (0: fully periodic)
  void* ub;                // 2D: [p][nb] boundary states U_b^{n+1} between the two boundary passes
  cudaStream_t stream;
  void* f[2];
  bool f_borrowed;         // f[] belong to the caller (vklb_create_borrowed): never freed here
  int cur;                 // f[cur] holds the current state
  long long launched;      // step launches so far (slot = launched % 3)
  Ctl* ctl;
  double* part;            // [p][kRedBlocks] partial sums
  double* dvec;            // [p] device totals
  double* stage;           // [p][cells] double staging for set_state / moments
  int tile_x, tile_y;
  int variant, stages;     // step kernel: 0 plain, 1 bulk-copy row pipeline with `stages` rows in flight
  int form;                // 0 distributions f, 1 moments U (omega = 1, D2Q5)
  int QS;                  // stored components a field: Q (form 0) or 1 (form 1)
  // halo of the long-split march (2D, p > 4): hl[b] holds the edge columns of
  // the tiles of f[b] (halo_index), for tiles hl_tx wide; hl_ok: hl[cur] is
  // the one of f[cur], written by the last step
  void* hl[2];
  size_t hl_bytes;
  int hl_tx, hl_ok;
  bool ready;
  const Ops* ops;
};

struct Ops {
  int (*init)(vklb_sim*, const double*);
  int (*step)(vklb_sim*, int64_t, double);   // enqueue n step launches with t_end
  int (*moments)(vklb_sim*, double*);
  int (*totals)(vklb_sim*, double*);
  int (*batch)(vklb_batch*, int64_t, int);
  size_t (*smem)(int variant, int p, int tx, int ty, int stages);
  int (*occupancy)(int variant, int tx, int ty, int stages);
  int (*batch_occupancy)(int variant, int tx, int ty, int stages);
  size_t real_bytes;
  size_t args_bytes;
};

struct vklb_batch {
  std::vector<vklb_sim*> sims;
  int tile_x, tile_y;
  void* d_desc;
  BatchWork* d_work;
  int nwork;
  int variant, stages;
  std::vector<unsigned char> h_desc;
  std::vector<BatchWork> h_work;   // host copy of the work-list (source of its async upload)
  cudaStream_t stream;
  const Ops* ops;
  int64_t graph_n;
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  cudaStream_t own;        // private stream: graphs cannot be captured on the legacy stream
  cudaEvent_t ev_in, ev_out;
};


// The dispatch table of each system, one translation unit each.
const Ops* vk_ops_advect(int dim, int prec);
const Ops* vk_ops_swe(int dim, int prec);
const Ops* vk_ops_euler(int dim, int prec);
const Ops* vk_ops_mhd(int dim, int prec);

namespace {

// Kernel selector: 0 plain distribution step, 1 bulk-copy distribution step,
// 2 moment-form step.
int kernel_variant(const vklb_sim* s) { return s->form == 1 ? 2 : s->variant; }

template <class T>
StepArgs<T> make_args(const vklb_sim* s, double t_end) {
  StepArgs<T> a;
  a.f[0] = (T*)s->f[0];
  a.f[1] = (T*)s->f[1];
  a.parity = s->cur;
  a.nx = (int)s->nx;
  a.ny = (int)s->ny;
  a.pitch = (int)s->pitch;
  a.dx = s->dx;
  a.c = s->c;
  a.omega = s->omega;
  a.k = s->k;
  a.inv_nu = s->inv_nu;
  a.fixed_xi = s->fixed_xi;
  a.t_end = t_end;
  a.ch_factor = s->ch_factor;
  a.set = s->set;
  a.anorm = s->anorm;
  a.bc_lo = s->bc_lo;
  a.bc_hi = s->bc_hi;
  a.cbx = s->cbx;
  a.cby = s->cby;
  a.btr = s->btr;
  a.ctl = s->ctl;
  a.slot = (int)(s->launched % 3);
  a.sp = s->sp;
  const bool hl = s->hl[0] && s->hl_tx == s->tile_x;
  a.hl[0] = hl ? (T*)s->hl[0] : nullptr;
  a.hl[1] = hl ? (T*)s->hl[1] : nullptr;
  a.hl_ok = hl && s->hl_ok;
  return a;
}

int grid_for(size_t cells, int block) {
  size_t g = (cells + block - 1) / block;
  if (g > 148 * 16) g = 148 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

template <class Sys, class T, class R, int DIM>
struct Impl {
  static constexpr int P = Sys::P;
  static constexpr int Q = DIM == 1 ? 3 : 5;

  static int init(vklb_sim* s, const double* dU) {
    StepArgs<T> a = make_args<T>(s, -1.0);
    a.parity = s->cur;
    const int blk = 256;
    init_max_kernel<Sys, R, DIM><<<grid_for(s->cells, blk), blk, 0, s->stream>>>(dU, (size_t)s->cells, s->sp, s->ctl);
    if constexpr (DIM == 2) {
      if (s->form == 1)
        init_feq_kernel<Sys, T, R, DIM, 1><<<grid_for(s->cells, blk), blk, 0, s->stream>>>(dU, (size_t)s->cells, a);
      else
        init_feq_kernel<Sys, T, R, DIM><<<grid_for(s->cells, blk), blk, 0, s->stream>>>(dU, (size_t)s->cells, a);
    } else {
      init_feq_kernel<Sys, T, R, DIM><<<grid_for(s->cells, blk), blk, 0, s->stream>>>(dU, (size_t)s->cells, a);
    }
    g_launches += 2;
    return cuda_status(cudaGetLastError());
  }

  // rows f*_1 / f*_2 (3 each) and the x ring; the long-split march (P > 4)
  // also keeps its column state (3 rows of P) in shared memory
  // row buffers [3][tx] x 2, the x ring [ty] x 2, and for the long-split march
  // its column state [3][tx], each entry a cell of CellVec<R, P>::PP values
  static size_t smem_bytes(int tx, int ty) {
    constexpr int PP = CellVec<R, P>::PP;
    return (size_t)(((P > 4) ? 9 : 6) * PP * tx + 2 * PP * ty) * sizeof(R);
  }
  static size_t smem_bytes_v(int variant, int tx, int ty, int d) {
    if (variant == 1) return TmaLayout<T>::template make<R, P>(tx, ty, d).bytes;
    return smem_bytes(tx, ty);
  }

  static int step(vklb_sim* s, int64_t n, double t_end) {
    if constexpr (DIM == 1) {
      // one block; as many threads as the grid has cells, within what the
      // kernel's registers allow per block
      static int max_blk = 0;
      if (max_blk == 0) {
        cudaFuncAttributes fa;
        max_blk = cudaFuncGetAttributes(&fa, step1d_kernel<Sys, T, R>) == cudaSuccess ? fa.maxThreadsPerBlock : 256;
        max_blk = max_blk / 32 * 32;
        if (max_blk < 32) max_blk = 32;
        cudaGetLastError();
      }
      int blk = (int)(((s->nx + 31) / 32) * 32);
      if (blk > max_blk) blk = max_blk;
      if (blk < 64 && max_blk >= 64) blk = 64;
      StepArgs<T> a = make_args<T>(s, t_end);
      // n steps in one launch; with t_end the kernel may stop early, so the
      // caller re-reads the step counter (vklb_step_to).
      step1d_kernel<Sys, T, R><<<1, blk, 0, s->stream>>>(a, (int)n);
      g_launches += 1;
      int st = cuda_status(cudaGetLastError());
      if (st) return st;
      if (t_end <= 0.0) {
        s->cur ^= (int)(n & 1);
        s->launched += n;
      }
      return VKLB_OK;
    } else {
      const int TX = s->tile_x, TY = s->tile_y, D = s->stages;
      const int kv = kernel_variant(s);
      const size_t sm = smem_bytes_v(kv, TX, TY, D);
      set_attributes();
      dim3 grid((unsigned)((s->nx + TX - 1) / TX), (unsigned)((s->ny + TY - 1) / TY));
      // the long-split march keeps the halo of its tiles' edge columns (p > 4,
      // not the bulk-copy step); with non-periodic faces the boundary passes
      // rewrite face nodes after the halo was written, so the next step reads
      // its x ring from the bricks
      const bool halo = P > 4 && kv != 1 && s->hl[0] && s->hl_tx == TX && s->nb == 0;
      for (int64_t i = 0; i < n; ++i) {
        StepArgs<T> a = make_args<T>(s, t_end);
        if (kv == 1)
          step2d_tma_kernel<Sys, T, R><<<grid, TX, sm, s->stream>>>(a, TX, TY, D);

        else if (wide128(TX))
          launch_plain<128>(kv, grid, TX, sm, s->stream, a, TY);
        else
          launch_plain<0>(kv, grid, TX, sm, s->stream, a, TY);
        if (s->nb > 0) {
          // the non-periodic faces (same step arguments: parity and slot of step n)
          const int bb = 128, gb = (s->nb + bb - 1) / bb;
          char2d_state_kernel<Sys, T, R><<<gb, bb, 0, s->stream>>>(a, (R*)s->ub, s->nb);
          char2d_feq_kernel<Sys, T, R><<<gb, bb, 0, s->stream>>>(a, (const R*)s->ub, s->nb);
          g_launches += 2;
        }
        s->cur ^= 1;
        s->launched += 1;
        s->hl_ok = halo;
      }
      g_launches += n;
      return cuda_status(cudaGetLastError());
    }
  }

  // the plain step takes the register-bounded instantiation when it has one
  // and the block fits its 128-thread bound
  static constexpr bool kBounded = StepBound<Sys, R>::min_blocks > 0;
  // the bounded instantiations exist only where they are launched
  template <int FORM, int TXC>
  static void launch_lb(dim3 grid, int TX, size_t sm, cudaStream_t st, const StepArgs<T>& a, int TY) {
    if constexpr (kBounded) step2d_lb_kernel<Sys, T, R, kMinBlocks, FORM, TXC><<<grid, TX, sm, st>>>(a, TX, TY);
  }
  static constexpr int kMinBlocks = kBounded ? StepBound<Sys, R>::min_blocks : 1;
  static bool bounded(int tx) { return kBounded && tx <= 128; }
  // The long-split march (p > 4) has instantiations with the tile width 128
  // (the default launch shape's and the server's) known at compile time:
  // measured 9 % fewer instructions for MHD-GLM than with the width at run time.
  static constexpr bool kWide128 = P > 4;
  static bool wide128(int tx) { return kWide128 && tx == 128; }
  // plain (kv 0) or moment-form (kv 2) step kernel, TXC as above
  template <int TXC>
  static void launch_plain(int kv, dim3 grid, int TX, size_t sm, cudaStream_t st, const StepArgs<T>& a, int TY) {
    if constexpr (TXC == 0 || kWide128) {
      if (kv == 2 && bounded(TX))
        launch_lb<1, TXC>(grid, TX, sm, st, a, TY);
      else if (kv == 2)
        step2d_u_kernel<Sys, T, R, TXC><<<grid, TX, sm, st>>>(a, TX, TY);
      else if (bounded(TX))
        launch_lb<0, TXC>(grid, TX, sm, st, a, TY);
      else
        step2d_kernel<Sys, T, R, TXC><<<grid, TX, sm, st>>>(a, TX, TY);
    }
  }

  static void set_attributes() {
    if constexpr (DIM == 2) {
      static std::atomic<unsigned long long> done{0};
      if (!first_on_device(done)) return;
      cudaFuncSetAttribute(step2d_tma_kernel<Sys, T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      set_plain_attributes<0>();
      if constexpr (kWide128) set_plain_attributes<128>();
    }
  }
  template <int TXC>
  static void set_plain_attributes() {
    cudaFuncSetAttribute(step2d_kernel<Sys, T, R, TXC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(step2d_u_kernel<Sys, T, R, TXC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if constexpr (kBounded) {
      cudaFuncSetAttribute(step2d_lb_kernel<Sys, T, R, kMinBlocks, 0, TXC>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(step2d_lb_kernel<Sys, T, R, kMinBlocks, 1, TXC>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
  }

  template <int FORM, int TXC>
  static cudaError_t occupancy_lb(int* nb, int tx, size_t sm) {
    if constexpr (kBounded)
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, step2d_lb_kernel<Sys, T, R, kMinBlocks, FORM, TXC>, tx,
                                                           sm);
    else
      return cudaErrorInvalidValue;
  }
  template <int TXC>
  static cudaError_t occupancy_plain(int* nb, int variant, int tx, size_t sm) {
    if constexpr (TXC == 0 || kWide128) {
      if (variant == 2 && bounded(tx)) return occupancy_lb<1, TXC>(nb, tx, sm);
      if (variant == 2) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, step2d_u_kernel<Sys, T, R, TXC>, tx, sm);
      if (bounded(tx)) return occupancy_lb<0, TXC>(nb, tx, sm);
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, step2d_kernel<Sys, T, R, TXC>, tx, sm);
    }
    return cudaErrorInvalidValue;
  }

  // resident blocks per SM of the step kernel a sim with this launch shape runs
  static int occupancy(int variant, int tx, int ty, int d) {
    if constexpr (DIM != 2) {
      return 0;
    } else {
      set_attributes();
      const size_t sm = smem_bytes_v(variant, tx, ty, d);
      int nb = 0;
      cudaError_t e;
      if (variant == 1)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step2d_tma_kernel<Sys, T, R>, tx, sm);
      else if (wide128(tx))
        e = occupancy_plain<128>(&nb, variant, tx, sm);
      else
        e = occupancy_plain<0>(&nb, variant, tx, sm);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return nb;
    }
  }

  static int moments(vklb_sim* s, double* dU) {
    const int blk = 256;
    if (s->form == 1)
      moments_kernel<T, P, 1><<<grid_for(s->cells, blk), blk, 0, s->stream>>>((const T*)s->f[s->cur], (int)s->nx,
                                                                              (int)s->ny, (int)s->pitch, dU);
    else
      moments_kernel<T, P, Q><<<grid_for(s->cells, blk), blk, 0, s->stream>>>((const T*)s->f[s->cur], (int)s->nx,
                                                                              (int)s->ny, (int)s->pitch, dU);
    g_launches += 1;
    return cuda_status(cudaGetLastError());
  }

  static int totals(vklb_sim* s, double* host) {
    if (s->form == 1)
      totals_pass1<T, P, 1><<<kRedBlocks, 256, 0, s->stream>>>((const T*)s->f[s->cur], (int)s->nx, (int)s->ny,
                                                               (int)s->pitch, s->part);
    else
      totals_pass1<T, P, Q><<<kRedBlocks, 256, 0, s->stream>>>((const T*)s->f[s->cur], (int)s->nx, (int)s->ny,
                                                               (int)s->pitch, s->part);
    double scale = DIM == 1 ? s->dx : s->dx * s->dx;
    totals_pass2<<<1, 32, 0, s->stream>>>(s->part, kRedBlocks, P, scale, s->dvec);
    g_launches += 2;
    int st = cuda_status(cudaGetLastError());
    if (st) return st;
    return cuda_status(cudaMemcpyAsync(host, s->dvec, sizeof(double) * P, cudaMemcpyDeviceToHost, s->stream));
  }
};

template <class Sys, class T, class R, int DIM>
struct BatchImpl {
  // the plain and moment-form bodies take the register-bounded instantiation
  // where the single-simulation step does (blocks of at most 128 threads)
  static constexpr bool kBounded = Impl<Sys, T, R, DIM>::kBounded;
  static constexpr int kMinBlocks = Impl<Sys, T, R, DIM>::kMinBlocks;
  static bool bounded(int variant, int tx) { return variant != 1 && Impl<Sys, T, R, DIM>::bounded(tx); }
  // tile width 128 at compile time for the long-split march (as Impl)
  static constexpr bool kWide128 = Impl<Sys, T, R, DIM>::kWide128;
  static bool wide128(int variant, int tx) { return variant != 1 && Impl<Sys, T, R, DIM>::wide128(tx); }
  template <int V, int TXC>
  static void launch_lb(const vklb_batch* b, int i, int TX, int TY, int D, size_t sm) {
    if constexpr (kBounded)
      step2d_batch_lb_kernel<Sys, T, R, V, kMinBlocks, TXC><<<b->nwork, TX, sm, b->own>>>(
          (const StepArgs<T>*)b->d_desc, b->d_work, i, TX, TY, D);
  }
  template <int V, int TXC>
  static cudaError_t occupancy_lb(int* nb, int tx, size_t sm) {
    if constexpr (kBounded) {
      cudaFuncSetAttribute(step2d_batch_lb_kernel<Sys, T, R, V, kMinBlocks, TXC>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, step2d_batch_lb_kernel<Sys, T, R, V, kMinBlocks, TXC>,
                                                           tx, sm);
    }
    return cudaErrorInvalidValue;
  }
  // plain (variant 0) or moment-form (variant 2) batched step, TXC as in Impl
  template <int TXC>
  static void launch_plain(vklb_batch* b, int i, int TX, int TY, int D, size_t sm) {
    if constexpr (TXC == 0 || kWide128) {
      const bool lb = bounded(b->variant, TX);
      if (b->variant == 2 && lb)
        launch_lb<2, TXC>(b, i, TX, TY, D, sm);
      else if (b->variant == 2)
        step2d_batch_kernel<Sys, T, R, 2, TXC><<<b->nwork, TX, sm, b->own>>>(
            (const StepArgs<T>*)b->d_desc, b->d_work, i, TX, TY, D);
      else if (lb)
        launch_lb<0, TXC>(b, i, TX, TY, D, sm);
      else
        step2d_batch_kernel<Sys, T, R, 0, TXC><<<b->nwork, TX, sm, b->own>>>(
            (const StepArgs<T>*)b->d_desc, b->d_work, i, TX, TY, D);
    }
  }
  template <int TXC>
  static void set_plain_attributes() {
    cudaFuncSetAttribute(step2d_batch_kernel<Sys, T, R, 0, TXC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(step2d_batch_kernel<Sys, T, R, 2, TXC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    if constexpr (kBounded) {
      cudaFuncSetAttribute(step2d_batch_lb_kernel<Sys, T, R, 0, kMinBlocks, TXC>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(step2d_batch_lb_kernel<Sys, T, R, 2, kMinBlocks, TXC>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
  }
  static void set_attributes() {
    cudaFuncSetAttribute(step2d_batch_kernel<Sys, T, R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    set_plain_attributes<0>();
    if constexpr (kWide128) set_plain_attributes<128>();
  }
  template <int TXC>
  static cudaError_t occupancy_plain(int* nb, int variant, int tx, size_t sm) {
    if constexpr (TXC == 0 || kWide128) {
      const bool lb = bounded(variant, tx);
      if (variant == 2)
        return lb ? occupancy_lb<2, TXC>(nb, tx, sm)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, step2d_batch_kernel<Sys, T, R, 2, TXC>, tx, sm);
      return lb ? occupancy_lb<0, TXC>(nb, tx, sm)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, step2d_batch_kernel<Sys, T, R, 0, TXC>, tx, sm);
    }
    return cudaErrorInvalidValue;
  }
  static void launch(vklb_batch* b, int64_t n) {
    if constexpr (DIM == 2) {
    const int TX = b->tile_x, TY = b->tile_y, D = b->stages;
    const size_t sm = Impl<Sys, T, R, DIM>::smem_bytes_v(b->variant, TX, TY, D);
    for (int64_t i = 0; i < n; ++i) {
      if (b->variant == 1)
        step2d_batch_kernel<Sys, T, R, 1><<<b->nwork, TX, sm, b->own>>>(
            (const StepArgs<T>*)b->d_desc, b->d_work, (int)i, TX, TY, D);
      else if (wide128(b->variant, TX))
        launch_plain<128>(b, (int)i, TX, TY, D, sm);
      else
        launch_plain<0>(b, (int)i, TX, TY, D, sm);
    }
    }
  }
  // resident blocks per SM of the batched step kernel at this launch shape
  static int occupancy(int variant, int tx, int ty, int d) {
    if constexpr (DIM != 2) {
      return 0;
    } else {
      const size_t sm = Impl<Sys, T, R, DIM>::smem_bytes_v(variant, tx, ty, d);
      set_attributes();
      int nb = 0;
      cudaError_t e =
          variant == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step2d_batch_kernel<Sys, T, R, 1>, tx, sm)
          : wide128(variant, tx) ? occupancy_plain<128>(&nb, variant, tx, sm)
                                 : occupancy_plain<0>(&nb, variant, tx, sm);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return nb;
    }
  }
  static int step(vklb_batch* b, int64_t n, int use_graph) {
    if constexpr (DIM != 2) {
      return VKLB_ERR_UNSUPPORTED;
    } else {
    static std::atomic<unsigned long long> attr_set{0};
    if (first_on_device(attr_set)) set_attributes();
    StepArgs<T>* h = (StepArgs<T>*)b->h_desc.data();
    for (size_t i = 0; i < b->sims.size(); ++i) {
      h[i] = make_args<T>(b->sims[i], -1.0);
      h[i].hl[0] = h[i].hl[1] = nullptr;   // batches keep no halo: the batch's tiles are its own
      h[i].hl_ok = 0;
    }
    // order after the work already queued on the simulations' streams
    int st = VKLB_OK;
    for (size_t i = 0; i < b->sims.size(); ++i) {
      if (i > 0 && b->sims[i]->stream == b->sims[i - 1]->stream) continue;
      if ((st = cuda_status(cudaEventRecord(b->ev_in, b->sims[i]->stream)))) return st;
      if ((st = cuda_status(cudaStreamWaitEvent(b->own, b->ev_in, 0)))) return st;
    }
    // pageable source: the runtime stages it before returning, so h may be reused
    if ((st = cuda_status(cudaMemcpyAsync(b->d_desc, h, b->h_desc.size(), cudaMemcpyHostToDevice, b->own)))) return st;
    if (use_graph) {
      if (!b->gexec || b->graph_n != n) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->gexec = nullptr;
        b->graph = nullptr;
        if ((st = cuda_status(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal)))) return st;
        launch(b, n);
        if ((st = cuda_status(cudaStreamEndCapture(b->own, &b->graph)))) return st;
        if ((st = cuda_status(cudaGraphInstantiate(&b->gexec, b->graph, 0)))) return st;
        b->graph_n = n;
      }
      if ((st = cuda_status(cudaGraphLaunch(b->gexec, b->own)))) return st;
    } else {
      launch(b, n);
    }
    g_launches += n;
    if ((st = cuda_status(cudaGetLastError()))) return st;
    // later work on the simulations' streams waits for the batch
    if ((st = cuda_status(cudaEventRecord(b->ev_out, b->own)))) return st;
    for (size_t i = 0; i < b->sims.size(); ++i) {
      if (i > 0 && b->sims[i]->stream == b->sims[i - 1]->stream) continue;
      if ((st = cuda_status(cudaStreamWaitEvent(b->sims[i]->stream, b->ev_out, 0)))) return st;
    }
    for (vklb_sim* s : b->sims) {
      s->cur ^= (int)(n & 1);
      s->launched += n;
      s->hl_ok = 0;
    }
    return VKLB_OK;
    }
  }
};

template <class Sys, class T, class R, int DIM>
size_t smem_of(int variant, int p, int tx, int ty, int stages) {
  return Impl<Sys, T, R, DIM>::smem_bytes_v(variant, tx, ty, stages);
}

template <class Sys, class T, class R, int DIM>
const Ops* ops_of() {
  static const Ops o = {&Impl<Sys, T, R, DIM>::init,    &Impl<Sys, T, R, DIM>::step,
                        &Impl<Sys, T, R, DIM>::moments, &Impl<Sys, T, R, DIM>::totals,
                        &BatchImpl<Sys, T, R, DIM>::step, &smem_of<Sys, T, R, DIM>,
                        &Impl<Sys, T, R, DIM>::occupancy, &BatchImpl<Sys, T, R, DIM>::occupancy,
                        sizeof(R),                        sizeof(StepArgs<T>)};
  return &o;
}

template <template <class, int> class S, int DIM>
const Ops* pick_prec(int prec) {
  if (prec == VKLB_FP64) return ops_of<S<double, DIM>, double, double, DIM>();
  if (prec == VKLB_FP32) return ops_of<S<float, DIM>, float, float, DIM>();
  return ops_of<S<float, DIM>, __nv_bfloat16, float, DIM>();
}

}  // namespace
