// Host side of libvklb.so: the C ABI declared in include/vklb.h.
//
// A simulation owns two device buffers of q * p * cells distributions (store
// type of its precision), one Ctl block of control words and small scratch
// buffers for reductions.  Every kernel runs on the simulation's stream; no call
// synchronises except those documented as synchronising.
#include <nvtx3/nvToolsExt.h>

#include "vk_host.cuh"

namespace {
// An NVTX range over one call of the C ABI (named after the call), so that a
// timeline profiler shows the host calls beside the kernels they enqueue; free
// when no tool is attached.
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
};
}  // namespace

std::atomic<long long> g_launches{0};

namespace {

const Ops* pick_ops(int kind, int dim, int prec) {
  if (kind == VKLB_ADVECT) return vk_ops_advect(dim, prec);
  if (kind == VKLB_SWE) return vk_ops_swe(dim, prec);
  if (kind == VKLB_EULER) return vk_ops_euler(dim, prec);
  if (kind == VKLB_MHD_GLM) return vk_ops_mhd(dim, prec);
  return nullptr;
}

int fields_of(int kind, int dim) {
  switch (kind) {
    case VKLB_ADVECT: return 1;
    case VKLB_SWE: return dim + 1;
    case VKLB_EULER: return dim + 2;
    case VKLB_MHD_GLM: return 9;
  }
  return 0;
}

int read_ctl(vklb_sim* s, Ctl* h) {
  int st = cuda_status(cudaMemcpyAsync(h, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  if (st) return st;
  return cuda_status(cudaStreamSynchronize(s->stream));
}

int err_of(const Ctl& h) {
  // a violated CFL bound (fixed xi) is the cause of any non-physical state after it
  if (h.err & ERR_TIMEOUT) return VKLB_ERR_TIMEOUT;
  if (h.err & ERR_CFL) return VKLB_ERR_CFL;
  if (h.err & ERR_NONPHYS) return VKLB_ERR_NONPHYSICAL;
  return VKLB_OK;
}

// A simulation's device buffers are stream-ordered allocations on its stream
// (cudaMallocAsync / cudaFreeAsync): creating or destroying one while other
// simulations run on other streams does not wait for their work.
void free_on(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}
void free_sim(vklb_sim* s) {
  if (!s) return;
  if (!s->f_borrowed) {
    free_on(s->f[0], s->stream);
    free_on(s->f[1], s->stream);
  }
  free_on(s->ctl, s->stream);
  free_on(s->part, s->stream);
  free_on(s->dvec, s->stream);
  free_on(s->stage, s->stream);
  free_on(s->ub, s->stream);
  free_on(s->hl[0], s->stream);
  free_on(s->hl[1], s->stream);
  delete s;
}

// Halo of the long-split march (2D systems with p > 4): two buffers of the
// tiles' first and last columns, sized for the current tile width; any change
// of the tiling or the form invalidates it until the next step writes it.
int halo_fit(vklb_sim* s) {
  s->hl_ok = 0;
  if (s->dim != 2 || s->P <= 4) return VKLB_OK;
  const size_t nbx = (size_t)((s->nx + s->tile_x - 1) / s->tile_x);
  const size_t need = nbx * 2 * (size_t)s->ny * (size_t)s->QS * s->P * s->store_bytes;
  if (need > s->hl_bytes) {
    free_on(s->hl[0], s->stream);
    free_on(s->hl[1], s->stream);
    s->hl[0] = s->hl[1] = nullptr;
    s->hl_bytes = 0;
    cudaError_t e = cudaMallocAsync(&s->hl[0], need, s->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&s->hl[1], need, s->stream);
    if (e != cudaSuccess) {
      free_on(s->hl[0], s->stream);
      free_on(s->hl[1], s->stream);
      s->hl[0] = s->hl[1] = nullptr;
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? VKLB_ERR_NOMEM : VKLB_ERR_CUDA;
    }
    s->hl_bytes = need;
  }
  s->hl_tx = s->tile_x;
  return VKLB_OK;
}

const uint32_t kMagic = 0x564b4c42u;  // "VKLB"
struct BlobHeader {
  uint32_t magic, kind, P, Q, prec, slot;
  int64_t nx, ny, launched;
};

}  // namespace

extern "C" {

const char* vklb_strerror(int status) {
  switch (status) {
    case VKLB_OK: return "ok";
    case VKLB_ERR_ARG: return "invalid argument";
    case VKLB_ERR_NOMEM: return "out of memory";
    case VKLB_ERR_CUDA: return "CUDA runtime error";
    case VKLB_ERR_NONPHYSICAL: return "non-physical state (NaN or non-positive depth/density/pressure)";
    case VKLB_ERR_CFL: return "fixed lattice speed below the largest wave speed (CFL violated)";
    case VKLB_ERR_TIMEOUT: return "bounded device wait gave up";
    case VKLB_ERR_STATE: return "call out of order";
    case VKLB_ERR_UNSUPPORTED: return "unsupported combination";
    case VKLB_ERR_LIMIT: return "request exceeds the fixed limits of the allocation-free entry point";
  }
  return "unknown status";
}

int64_t vklb_launch_count(void) { return g_launches.load(); }

int vklb_selftest_wait_timeout(int64_t limit_ns, void* cuda_stream) {
  if (limit_ns < 1000 || limit_ns > 100000000) return VKLB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Ctl* ctl = nullptr;
  if (cudaMalloc((void**)&ctl, sizeof(Ctl)) != cudaSuccess) {
    cudaGetLastError();
    return VKLB_ERR_NOMEM;
  }
  int rc = cuda_status(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
  if (!rc) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(ctl, (uint64_t)limit_ns);
    g_launches += 1;
    rc = cuda_status(cudaGetLastError());
  }
  Ctl h;
  if (!rc) rc = cuda_status(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
  cudaFree(ctl);
  if (rc) return rc;
  return err_of(h);
}

// Tile height that makes the grid fill whole waves of resident blocks: with
// `slots` = SMs x resident blocks per SM and gx tiles across, the first k for
// which ceil(ny / (k * floor(slots / gx))) <= 256 rows.
static int wave_fit_rows(vklb_sim* s, int tx, int* ty_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return VKLB_ERR_CUDA;
  }
  const int64_t gx = (s->nx + tx - 1) / tx;
  int ty = 16;
  for (int pass = 0; pass < 2; ++pass) {   // occupancy depends on ty through the ring buffers
    const int nb = s->ops->occupancy(kernel_variant(s), tx, ty, s->stages);
    if (nb < 1) return VKLB_ERR_ARG;
    int64_t rows = (int64_t)nb * sms / gx;
    if (rows < 1) rows = 1;
    for (int64_t k = 1;; ++k) {
      const int64_t t = (s->ny + k * rows - 1) / (k * rows);
      if (t <= 256) {
        ty = (int)(t < 1 ? 1 : t);
        break;
      }
    }
  }
  *ty_out = ty;
  return VKLB_OK;
}

// Bytes of one distribution buffer (q p values a cell on the padded grid).
static int64_t buffer_bytes_of(int32_t kind, int32_t lattice, const vklb_grid* grid, int32_t precision) {
  const int dim = grid->dim;
  if (!((lattice == VKLB_D1Q3 && dim == 1) || (lattice == VKLB_D2Q5 && dim == 2))) return -1;
  if (kind < VKLB_ADVECT || kind > VKLB_MHD_GLM || precision < VKLB_FP64 || precision > VKLB_BF16_STORE) return -1;
  const int64_t nx = grid->n[0], ny = dim == 2 ? grid->n[1] : 1;
  if (nx < 1 || ny < 1 || nx > (1 << 30) || ny > (1 << 30)) return -1;
  const int64_t pitch = dim == 2 ? ((nx + 31) / 32) * 32 : nx;
  const int64_t sb = precision == VKLB_FP64 ? 8 : (precision == VKLB_FP32 ? 4 : 2);
  return (int64_t)(dim == 1 ? 3 : 5) * fields_of(kind, dim) * pitch * ny * sb;
}

int vklb_buffer_bytes(int32_t kind, int32_t lattice, const vklb_grid* grid, int32_t precision, size_t* bytes) {
  if (!grid || !bytes) return VKLB_ERR_ARG;
  const int64_t b = buffer_bytes_of(kind, lattice, grid, precision);
  if (b < 0) return VKLB_ERR_ARG;
  *bytes = (size_t)b;
  return VKLB_OK;
}

static int create_impl(const vklb_system* sys, int32_t lattice, const vklb_grid* grid, const vklb_bc* bc,
                       const vklb_weight* weight, double dt, int32_t precision, void* cuda_stream,
                       void* const* f_buf, size_t buf_bytes, vklb_sim** out);

int vklb_create(const vklb_system* sys, int32_t lattice, const vklb_grid* grid, const vklb_bc* bc,
                const vklb_weight* weight, double dt, int32_t precision, void* cuda_stream, vklb_sim** out) {
  return create_impl(sys, lattice, grid, bc, weight, dt, precision, cuda_stream, nullptr, 0, out);
}

int vklb_create_borrowed(const vklb_system* sys, int32_t lattice, const vklb_grid* grid, const vklb_bc* bc,
                         const vklb_weight* weight, double dt, int32_t precision, void* cuda_stream,
                         void* const f_buf[2], size_t buf_bytes, vklb_sim** out) {
  if (!f_buf || !f_buf[0] || !f_buf[1] || !grid || !sys || !out) return VKLB_ERR_ARG;
  const int64_t need = buffer_bytes_of(sys->kind, lattice, grid, precision);
  if (need < 0 || buf_bytes < (size_t)need) return VKLB_ERR_ARG;
  const uintptr_t a = (uintptr_t)f_buf[0], b = (uintptr_t)f_buf[1];
  if ((a % 256) != 0 || (b % 256) != 0) return VKLB_ERR_ARG;          // whole bricks on 256-byte lines
  if ((a < b ? b - a : a - b) < (uintptr_t)need) return VKLB_ERR_ARG;   // the two must not overlap
  return create_impl(sys, lattice, grid, bc, weight, dt, precision, cuda_stream, f_buf, buf_bytes, out);
}

static int create_impl(const vklb_system* sys, int32_t lattice, const vklb_grid* grid, const vklb_bc* bc,
                       const vklb_weight* weight, double dt, int32_t precision, void* cuda_stream,
                       void* const* f_buf, size_t buf_bytes, vklb_sim** out) {
  if (!sys || !grid || !bc || !weight || !out) return VKLB_ERR_ARG;
  *out = nullptr;
  const int dim = grid->dim;
  if (!((lattice == VKLB_D1Q3 && dim == 1) || (lattice == VKLB_D2Q5 && dim == 2))) return VKLB_ERR_ARG;
  if (precision < VKLB_FP64 || precision > VKLB_BF16_STORE) return VKLB_ERR_ARG;
  if (weight->set < 0 || weight->set > 2) return VKLB_ERR_ARG;
  if (!(weight->omega > 0.0 && weight->omega <= 2.0)) return VKLB_ERR_ARG;   // Sec. 2.3
  if (!(weight->cfl > 0.0 && weight->cfl <= 1.0)) return VKLB_ERR_ARG;       // Eq. (28)
  if (!(weight->eta == 0.0 || (weight->eta > 0.0 && weight->eta < 1.0))) return VKLB_ERR_ARG;   // Sec. 2.3
  if (!(weight->k >= 0.0)) return VKLB_ERR_ARG;
  if (weight->alpha_norm != VKLB_ALPHA_LOCAL && weight->alpha_norm != VKLB_ALPHA_GLOBAL) return VKLB_ERR_ARG;
  const int64_t nx = grid->n[0], ny = dim == 2 ? grid->n[1] : 1;
  if (nx < 1 || ny < 1 || nx > (1 << 30) || ny > (1 << 30)) return VKLB_ERR_ARG;
  if (nx < 3 && dim == 1) return VKLB_ERR_ARG;
  const double dx = (grid->hi[0] - grid->lo[0]) / (double)nx;
  if (!(dx > 0.0)) return VKLB_ERR_ARG;
  if (dim == 2) {
    const double dy = (grid->hi[1] - grid->lo[1]) / (double)ny;
    if (!(fabs(dx - dy) <= 1e-12 * dx)) return VKLB_ERR_ARG;                  // Sec. 3.4
  }
  // one kind per axis (both ends alike), each periodic, characteristic or
  // transmissive; the non-periodic axes of a 2D grid all of one kind
  for (int i = 0; i < dim; ++i) {
    if (bc->lo[i] != bc->hi[i]) return VKLB_ERR_ARG;
    if (bc->lo[i] < VKLB_BC_PERIODIC || bc->lo[i] > VKLB_BC_TRANSMISSIVE) return VKLB_ERR_ARG;
  }
  if (dim == 2 && bc->lo[0] != VKLB_BC_PERIODIC && bc->lo[1] != VKLB_BC_PERIODIC && bc->lo[0] != bc->lo[1])
    return VKLB_ERR_ARG;
  // non-periodic 2D faces: at least 3 cells across a non-periodic axis
  const bool open2d = dim == 2 && (bc->lo[0] != VKLB_BC_PERIODIC || bc->lo[1] != VKLB_BC_PERIODIC);
  const Ops* ops = pick_ops(sys->kind, dim, precision);
  if (!ops) return VKLB_ERR_UNSUPPORTED;
  if (open2d && ((bc->lo[0] != VKLB_BC_PERIODIC && grid->n[0] < 3) ||
                 (bc->lo[1] != VKLB_BC_PERIODIC && grid->n[1] < 3)))
    return VKLB_ERR_ARG;
  if ((sys->kind == VKLB_EULER || sys->kind == VKLB_MHD_GLM) && !(sys->gamma > 1.0)) return VKLB_ERR_ARG;
  if (sys->kind == VKLB_SWE && !(sys->g > 0.0)) return VKLB_ERR_ARG;
  if (sys->kind == VKLB_MHD_GLM && !(sys->ch_factor > 0.0)) return VKLB_ERR_ARG;

  vklb_sim* s = new (std::nothrow) vklb_sim();
  if (!s) return VKLB_ERR_NOMEM;
  s->kind = sys->kind;
  s->lattice = lattice;
  s->dim = dim;
  s->P = fields_of(sys->kind, dim);
  s->Q = dim == 1 ? 3 : 5;
  s->prec = precision;
  s->store_bytes = precision == VKLB_FP64 ? 8 : (precision == VKLB_FP32 ? 4 : 2);
  s->nx = nx;
  s->ny = ny;
  s->cells = nx * ny;
  // 2D rows are padded to whole 32-cell bricks (the D2Q5 layout, see
  // brick_base): every brick starts on a 64-byte (bf16) / 128-byte (fp32) /
  // 256-byte (fp64) boundary, as coalescing and the bulk copies need.
  s->pitch = dim == 2 ? ((nx + 31) / 32) * 32 : nx;
  s->dx = dx;
  s->ch_factor = sys->ch_factor;
  s->sp.gamma = sys->gamma;
  s->sp.g = sys->g;
  s->sp.ax = sys->adv_speed[0];
  s->sp.ay = sys->adv_speed[1];
  s->set = weight->set;
  // centered set: c = 1/Q (Eqs. 8-10, 39); discontinuous set: c = 0 (Eqs. 12-14)
  s->c = weight->set == VKLB_SET_CENTERED ? 1.0 / s->Q : (weight->set == VKLB_SET_DISCONTINUOUS ? 0.0 : weight->c);
  s->k = weight->k;
  s->anorm = weight->alpha_norm == VKLB_ALPHA_GLOBAL ? 1 : 0;
  s->omega = weight->omega;
  s->cfl = weight->cfl;
  // Eq. (29), or the centered set's subcharacteristic condition (Sec. 2.3)
  s->inv_nu = weight->eta > 0.0 ? sqrt(1.5) / weight->eta : 1.0 / weight->cfl;
  s->fixed_xi = dt > 0.0 ? dx / dt : 0.0;
  s->bc_lo = bc->lo[0];
  s->bc_hi = bc->hi[0];
  s->cbx = dim == 2 && bc->lo[0] != VKLB_BC_PERIODIC;
  s->cby = dim == 2 && bc->lo[1] != VKLB_BC_PERIODIC;
  s->btr = dim == 2 && (bc->lo[0] == VKLB_BC_TRANSMISSIVE || bc->lo[1] == VKLB_BC_TRANSMISSIVE);
  s->nb = dim == 2 ? char_face_nodes((int)nx, (int)ny, s->cbx, s->cby) : 0;
  s->ub = nullptr;
  s->hl[0] = s->hl[1] = nullptr;
  s->hl_bytes = 0;
  s->hl_tx = 0;
  s->hl_ok = 0;
  s->stream = (cudaStream_t)cuda_stream;
  s->tile_x = 64;
  s->tile_y = 16;
  s->variant = 0;   // plain loads measure faster than the bulk-copy pipeline on B300 so far
  s->stages = 4;
  s->form = 0;
  s->QS = s->Q;
  s->ops = ops;
  const size_t fbytes = (size_t)s->Q * s->P * (size_t)s->pitch * s->ny * s->store_bytes;
  cudaError_t e = cudaSuccess;
  cudaStream_t st = s->stream;
  s->f_borrowed = f_buf != nullptr;
  if (s->f_borrowed) {
    s->f[0] = f_buf[0];
    s->f[1] = f_buf[1];
  }
  (void)buf_bytes;
  if ((!s->f_borrowed && (e = cudaMallocAsync(&s->f[0], fbytes, st)) != cudaSuccess) ||
      (!s->f_borrowed && (e = cudaMallocAsync(&s->f[1], fbytes, st)) != cudaSuccess) ||
      (e = cudaMallocAsync((void**)&s->ctl, sizeof(Ctl), st)) != cudaSuccess ||
      (e = cudaMallocAsync((void**)&s->part, sizeof(double) * s->P * kRedBlocks, st)) != cudaSuccess ||
      (e = cudaMallocAsync((void**)&s->dvec, sizeof(double) * s->P, st)) != cudaSuccess ||
      (e = cudaMallocAsync((void**)&s->stage, sizeof(double) * s->P * (size_t)s->cells, st)) != cudaSuccess ||
      (s->nb > 0 && (e = cudaMallocAsync(&s->ub, sizeof(double) * s->P * (size_t)s->nb, st)) != cudaSuccess)) {
    free_sim(s);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? VKLB_ERR_NOMEM : VKLB_ERR_CUDA;
  }
  // zero both buffers once: the row padding (pitch > nx) is never written by
  // the kernels, and a checkpoint blob must not carry stale device memory
  if ((e = cudaMemsetAsync(s->f[0], 0, fbytes, s->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(s->f[1], 0, fbytes, s->stream)) != cudaSuccess) {
    free_sim(s);
    cudaGetLastError();
    return VKLB_ERR_CUDA;
  }
  if (dim == 2) {   // default launch shape: 128-cell rows, height fitted to whole waves
    int ty = 16;
    if (wave_fit_rows(s, 128, &ty) == VKLB_OK) {
      s->tile_x = 128;
      s->tile_y = ty;
    }
  }
  if (int hs = halo_fit(s)) {
    free_sim(s);
    return hs;
  }
  *out = s;
  return VKLB_OK;
}

int vklb_destroy(vklb_sim* s) {
  if (!s) return VKLB_ERR_ARG;
  cudaStreamSynchronize(s->stream);   // this simulation's stream only
  free_sim(s);
  return cuda_status(cudaGetLastError());
}

int vklb_set_state(vklb_sim* s, const double* U, int32_t on_device) {
  CallRange range("vklb_set_state");
  if (!s || !U) return VKLB_ERR_ARG;
  const size_t bytes = sizeof(double) * s->P * (size_t)s->cells;
  int st = cuda_status(cudaMemcpyAsync(s->stage, U, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                       s->stream));
  if (st) return st;
  if ((st = cuda_status(cudaMemsetAsync(s->ctl, 0, sizeof(Ctl), s->stream)))) return st;
  s->cur = 0;
  s->launched = 0;
  s->hl_ok = 0;
  if ((st = s->ops->init(s, s->stage))) return st;
  if (!on_device) {
    // the caller may reuse U as soon as we return
    if ((st = cuda_status(cudaStreamSynchronize(s->stream)))) return st;
  }
  s->ready = true;
  return VKLB_OK;
}

int vklb_set_tiling(vklb_sim* s, int32_t tx, int32_t ty) {
  if (!s) return VKLB_ERR_ARG;
  if (tx == 0) tx = 128;
  if (ty == 0) ty = -1;
  if (ty == -1 && s->dim == 2 && tx >= 32 && tx <= 256 && tx % 32 == 0) {
    int st = wave_fit_rows(s, tx, &ty);
    if (st) return st;
  }
  if (tx < 32 || tx > 256 || (tx % 32) != 0 || ty < 1 || ty > 256) return VKLB_ERR_ARG;
  if (s->ops->smem(kernel_variant(s), s->P, tx, ty, s->stages) > 200 * 1024) return VKLB_ERR_ARG;
  const int old_tx = s->tile_x;
  s->tile_x = tx;
  s->tile_y = ty;
  if (tx != old_tx) return halo_fit(s);
  return VKLB_OK;
}

int vklb_set_variant(vklb_sim* s, int32_t variant, int32_t stages) {
  if (!s || variant < 0 || variant > 1) return VKLB_ERR_ARG;
  if (stages == 0) stages = 4;
  if (stages < 2 || stages > 8) return VKLB_ERR_ARG;
  if (s->dim != 2 && variant != 0) return VKLB_ERR_UNSUPPORTED;
  if (s->nb > 0 && variant == 1) return VKLB_ERR_UNSUPPORTED;   // characteristic faces: not the bulk-copy step
  if (s->form == 1 && variant != 0) return VKLB_ERR_UNSUPPORTED;
  if (s->ops->smem(variant, s->P, s->tile_x, s->tile_y, stages) > 200 * 1024) return VKLB_ERR_ARG;
  s->variant = variant;
  s->stages = stages;
  s->hl_ok = 0;
  return VKLB_OK;
}

int vklb_set_form(vklb_sim* s, int32_t form) {
  if (!s || (form != 0 && form != 1)) return VKLB_ERR_ARG;
  if (form == s->form) return VKLB_OK;
  if (s->f_borrowed) return VKLB_ERR_UNSUPPORTED;   // the caller's buffers keep their size
  if (form == 1 && s->dim != 2) return VKLB_ERR_UNSUPPORTED;
  if (form == 1 && s->nb > 0) return VKLB_ERR_UNSUPPORTED;
  if (form == 1 && s->omega != 1.0) return VKLB_ERR_ARG;   // f* = f^eq(U) holds at omega = 1 only
  if (form == 1 && s->variant != 0) return VKLB_ERR_UNSUPPORTED;
  int st = cuda_status(cudaStreamSynchronize(s->stream));
  if (st) return st;
  const int qs = form == 1 ? 1 : s->Q;
  const size_t fbytes = (size_t)qs * s->P * (size_t)s->pitch * s->ny * s->store_bytes;
  void* nf[2] = {nullptr, nullptr};
  cudaError_t e = cudaMallocAsync(&nf[0], fbytes, s->stream);
  if (e == cudaSuccess) e = cudaMallocAsync(&nf[1], fbytes, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(nf[0], 0, fbytes, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(nf[1], 0, fbytes, s->stream);
  if (e != cudaSuccess) {
    free_on(nf[0], s->stream);
    free_on(nf[1], s->stream);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? VKLB_ERR_NOMEM : VKLB_ERR_CUDA;
  }
  free_on(s->f[0], s->stream);
  free_on(s->f[1], s->stream);
  s->f[0] = nf[0];
  s->f[1] = nf[1];
  s->form = form;
  s->QS = qs;
  s->cur = 0;
  s->launched = 0;
  s->ready = false;   // the state must be set again
  int ty = 16;        // the default launch shape, refitted for this form's kernel
  if (wave_fit_rows(s, 128, &ty) == VKLB_OK) {
    s->tile_x = 128;
    s->tile_y = ty;
  }
  return halo_fit(s);
}

int vklb_step(vklb_sim* s, int64_t n) {
  CallRange range("vklb_step");
  if (!s || n < 0) return VKLB_ERR_ARG;
  if (!s->ready) return VKLB_ERR_STATE;
  if (n == 0) return VKLB_OK;
  return s->ops->step(s, n, -1.0);
}

int vklb_step_to(vklb_sim* s, double t_end) {
  CallRange range("vklb_step_to");
  if (!s || !(t_end > 0.0)) return VKLB_ERR_ARG;
  if (!s->ready) return VKLB_ERR_STATE;
  for (int iter = 0; iter < 1000; ++iter) {
    Ctl h;
    int st = read_ctl(s, &h);
    if (st) return st;
    if ((st = err_of(h))) return st;
    const int slot = (int)(s->launched % 3);
    StepScalars sc = step_scalars(&h, slot, s->kind == VKLB_MHD_GLM, s->ch_factor, s->inv_nu, s->fixed_xi, t_end, s->dx);
    if (sc.done) return VKLB_OK;
    // steps left if xi stayed as it is now
    double m = ceil((t_end - h.t[slot]) * sc.xi / s->dx - 1e-9);
    if (!std::isfinite(m) || !(sc.xi > 0.0)) return VKLB_ERR_NONPHYSICAL;
    if (m > 1e8) return VKLB_ERR_ARG;  // more than 1e8 steps left: refuse rather than enqueue them
    if (m < 1) m = 1;
    if (s->dim == 1) {
      const long long before = h.nsteps;
      int64_t chunk = (int64_t)m + 16;
      if ((st = s->ops->step(s, chunk, t_end))) return st;
      if ((st = read_ctl(s, &h))) return st;
      const long long took = h.nsteps - before;
      s->cur ^= (int)(took & 1);
      s->launched += took;
    } else {
      if ((st = s->ops->step(s, (int64_t)m, t_end))) return st;
    }
  }
  return VKLB_ERR_STATE;
}

int vklb_sync(vklb_sim* s) {
  if (!s) return VKLB_ERR_ARG;
  Ctl h;
  int st = read_ctl(s, &h);
  if (st) return st;
  return err_of(h);
}

int vklb_moments(vklb_sim* s, double* U, int32_t on_device) {
  CallRange range("vklb_moments");
  if (!s || !U) return VKLB_ERR_ARG;
  if (!s->ready) return VKLB_ERR_STATE;
  int st = s->ops->moments(s, s->stage);
  if (st) return st;
  const size_t bytes = sizeof(double) * s->P * (size_t)s->cells;
  if ((st = cuda_status(cudaMemcpyAsync(U, s->stage, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                        s->stream))))
    return st;
  return vklb_sync(s);
}

int vklb_conservation_totals(vklb_sim* s, double* totals) {
  CallRange range("vklb_conservation_totals");
  if (!s || !totals) return VKLB_ERR_ARG;
  if (!s->ready) return VKLB_ERR_STATE;
  int st = s->ops->totals(s, totals);
  if (st) return st;
  return vklb_sync(s);
}

int vklb_time(vklb_sim* s, double* t, int64_t* steps, double* xi) {
  if (!s) return VKLB_ERR_ARG;
  if (!s->ready) return VKLB_ERR_STATE;
  Ctl h;
  int st = read_ctl(s, &h);
  if (st) return st;
  const int slot = (int)(s->launched % 3);
  StepScalars sc = step_scalars(&h, slot, s->kind == VKLB_MHD_GLM, s->ch_factor, s->inv_nu, s->fixed_xi, -1.0, s->dx);
  if (t) *t = h.t[slot];
  if (steps) *steps = h.nsteps;
  if (xi) *xi = sc.xi;
  return err_of(h);
}

int vklb_info(const vklb_sim* s, vklb_info_t* info) {
  if (!s || !info) return VKLB_ERR_ARG;
  info->p = s->P;
  info->q = s->Q;
  info->precision = s->prec;
  info->store_bytes = s->store_bytes;
  info->cells = s->cells;
  info->bytes_per_lup = 2LL * s->QS * s->P * s->store_bytes;
  info->state_bytes = (int64_t)s->QS * s->P * s->pitch * s->ny * s->store_bytes;
  info->pitch = s->pitch;
  info->dx = s->dx;
  info->tile_x = s->tile_x;
  info->tile_y = s->tile_y;
  info->kernels_per_step = s->nb > 0 ? 3 : 1;
  info->variant = s->variant;
  info->blocks_per_sm = s->dim == 2 ? s->ops->occupancy(kernel_variant(s), s->tile_x, s->tile_y, s->stages) : 0;
  info->form = s->form;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    cudaGetLastError();
  info->sms = sms;
  return VKLB_OK;
}

int vklb_device_state(const vklb_sim* s, void** f_dev) {
  if (!s || !f_dev) return VKLB_ERR_ARG;
  *f_dev = s->f[s->cur];
  return VKLB_OK;
}

int vklb_poison_next(vklb_sim* s) {
  if (!s) return VKLB_ERR_ARG;
  const size_t bytes = (size_t)s->QS * s->P * s->pitch * s->ny * s->store_bytes;
  int st = cuda_status(cudaMemsetAsync(s->f[s->cur ^ 1], 0xFF, bytes, s->stream));
  if (st == VKLB_OK && s->hl[s->cur ^ 1])   // and the halo the next step writes
    st = cuda_status(cudaMemsetAsync(s->hl[s->cur ^ 1], 0xFF, s->hl_bytes, s->stream));
  return st;
}

int vklb_state_bytes(const vklb_sim* s, size_t* bytes) {
  if (!s || !bytes) return VKLB_ERR_ARG;
  *bytes = sizeof(BlobHeader) + sizeof(Ctl) + (size_t)s->QS * s->P * s->pitch * s->ny * s->store_bytes;
  return VKLB_OK;
}

int vklb_get_state(vklb_sim* s, void* blob, size_t bytes) {
  size_t need = 0;
  if (!s || !blob || vklb_state_bytes(s, &need) || bytes < need) return VKLB_ERR_ARG;
  if (!s->ready) return VKLB_ERR_STATE;
  BlobHeader hdr = {kMagic, (uint32_t)s->kind, (uint32_t)s->P, (uint32_t)s->QS, (uint32_t)s->prec,
                    (uint32_t)(s->launched % 3), s->nx, s->ny, s->launched};
  memcpy(blob, &hdr, sizeof(hdr));
  char* p = (char*)blob + sizeof(hdr);
  int st = cuda_status(cudaMemcpyAsync(p, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  if (st) return st;
  const size_t fb = (size_t)s->QS * s->P * s->pitch * s->ny * s->store_bytes;
  if ((st = cuda_status(cudaMemcpyAsync(p + sizeof(Ctl), s->f[s->cur], fb, cudaMemcpyDeviceToHost, s->stream)))) return st;
  if ((st = cuda_status(cudaStreamSynchronize(s->stream)))) return st;
  Ctl h;
  memcpy(&h, p, sizeof(h));
  return err_of(h);
}

int vklb_put_state(vklb_sim* s, const void* blob, size_t bytes) {
  size_t need = 0;
  if (!s || !blob || vklb_state_bytes(s, &need) || bytes < need) return VKLB_ERR_ARG;
  BlobHeader hdr;
  memcpy(&hdr, blob, sizeof(hdr));
  if (hdr.magic != kMagic || (int)hdr.kind != s->kind || (int)hdr.P != s->P || (int)hdr.Q != s->QS ||
      (int)hdr.prec != s->prec || hdr.nx != s->nx || hdr.ny != s->ny)
    return VKLB_ERR_ARG;
  const char* p = (const char*)blob + sizeof(hdr);
  int st = cuda_status(cudaMemcpyAsync(s->ctl, p, sizeof(Ctl), cudaMemcpyHostToDevice, s->stream));
  if (st) return st;
  s->cur = 0;
  s->launched = hdr.launched;
  s->hl_ok = 0;
  const size_t fb = (size_t)s->QS * s->P * s->pitch * s->ny * s->store_bytes;
  if ((st = cuda_status(cudaMemcpyAsync(s->f[0], p + sizeof(Ctl), fb, cudaMemcpyHostToDevice, s->stream)))) return st;
  if ((st = cuda_status(cudaStreamSynchronize(s->stream)))) return st;
  s->ready = true;
  return VKLB_OK;
}

// ------------------------------------------------------------------- batches
// The batch's device buffers are stream-ordered allocations on its own stream
// (cudaMallocAsync / cudaFreeAsync): creating and destroying a batch then never
// synchronises the device, so a server that rebuilds batches as its membership
// changes does not stall the other families' work.
static int batch_build_work(vklb_batch* b) {
  std::vector<BatchWork>& w = b->h_work;
  cudaStreamSynchronize(b->own);   // the previous list's upload has finished reading h_work
  w.clear();
  for (size_t i = 0; i < b->sims.size(); ++i) {
    const vklb_sim* s = b->sims[i];
    const int gx = (int)((s->nx + b->tile_x - 1) / b->tile_x), gy = (int)((s->ny + b->tile_y - 1) / b->tile_y);
    for (int by = 0; by < gy; ++by)
      for (int bx = 0; bx < gx; ++bx) w.push_back(BatchWork{(int)i, bx, by});
  }
  if (b->d_work) cudaFreeAsync(b->d_work, b->own);
  b->d_work = nullptr;
  if (cudaMallocAsync((void**)&b->d_work, sizeof(BatchWork) * w.size(), b->own) != cudaSuccess) {
    cudaGetLastError();
    return VKLB_ERR_NOMEM;
  }
  b->nwork = (int)w.size();
  int st = cuda_status(
      cudaMemcpyAsync(b->d_work, w.data(), sizeof(BatchWork) * w.size(), cudaMemcpyHostToDevice, b->own));
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->graph_n = 0;
  return st;
}

int vklb_batch_create(int32_t n, vklb_sim* const* sims, vklb_batch** out) {
  if (n < 1 || !sims || !out) return VKLB_ERR_ARG;
  *out = nullptr;
  const vklb_sim* s0 = sims[0];
  if (!s0 || s0->dim != 2) return VKLB_ERR_UNSUPPORTED;
  for (int i = 0; i < n; ++i) {
    const vklb_sim* s = sims[i];
    if (!s || !s->ready) return VKLB_ERR_STATE;
    if (s->nb > 0) return VKLB_ERR_UNSUPPORTED;   // characteristic faces: single-simulation steps only
    if (s->ops != s0->ops || s->set != s0->set || s->variant != s0->variant || s->stages != s0->stages ||
        s->form != s0->form)
      return VKLB_ERR_ARG;
  }
  vklb_batch* b = new (std::nothrow) vklb_batch();
  if (!b) return VKLB_ERR_NOMEM;
  b->sims.assign(sims, sims + n);
  b->tile_x = s0->tile_x;
  b->tile_y = s0->tile_y;
  b->variant = kernel_variant(s0);   // 2: the moment form
  b->stages = s0->stages;
  b->stream = s0->stream;
  b->ops = s0->ops;
  b->h_desc.resize(s0->ops->args_bytes * n);
  if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    vklb_batch_destroy(b);
    return VKLB_ERR_CUDA;
  }
  if (cudaMallocAsync(&b->d_desc, b->h_desc.size(), b->own) != cudaSuccess) {
    cudaGetLastError();
    vklb_batch_destroy(b);
    return VKLB_ERR_NOMEM;
  }
  int st = batch_build_work(b);
  if (st) {
    vklb_batch_destroy(b);
    return st;
  }
  *out = b;
  return VKLB_OK;
}

// Batch tile height for tile_y = -1: the members' grids differ, so no height
// makes the work-list a whole number of waves in general.  Over ty = 1..64 take
// the best (fill of the last wave) x (tile rows / (tile rows + the 2 ring rows
// each tile recomputes)), the larger ty on ties.
static int batch_fit_rows(vklb_batch* b, int tx, int* ty_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return VKLB_ERR_CUDA;
  }
  double best = -1.0;
  int best_ty = 8;
  for (int ty = 1; ty <= 64; ++ty) {
    const int nb = b->ops->batch_occupancy(b->variant, tx, ty, b->stages);
    if (nb < 1) continue;
    const double slots = (double)nb * sms;
    double blocks = 0.0;
    for (const vklb_sim* s : b->sims) blocks += (double)((s->nx + tx - 1) / tx) * (double)((s->ny + ty - 1) / ty);
    const double waves = std::ceil(blocks / slots);
    const double score = blocks / (waves * slots) * ((double)ty / (ty + 2));
    if (score >= best) {
      best = score;
      best_ty = ty;
    }
  }
  if (best < 0.0) return VKLB_ERR_ARG;
  *ty_out = best_ty;
  return VKLB_OK;
}

int vklb_batch_set_tiling(vklb_batch* b, int32_t tx, int32_t ty) {
  if (!b) return VKLB_ERR_ARG;
  if (tx == 0) tx = 64;
  if (ty == 0) ty = 16;
  if (ty == -1 && tx >= 32 && tx <= 256 && tx % 32 == 0) {
    int st = batch_fit_rows(b, tx, &ty);
    if (st) return st;
  }
  if (tx < 32 || tx > 256 || (tx % 32) != 0 || ty < 1 || ty > 256) return VKLB_ERR_ARG;
  if (b->ops->smem(b->variant, b->sims[0]->P, tx, ty, b->stages) > 200 * 1024) return VKLB_ERR_ARG;
  b->tile_x = tx;
  b->tile_y = ty;
  return batch_build_work(b);
}

int vklb_batch_step(vklb_batch* b, int64_t n, int32_t use_graph) {
  CallRange range("vklb_batch_step");
  if (!b || n < 0) return VKLB_ERR_ARG;
  if (n == 0) return VKLB_OK;
  // a member whose form, kernel variant or state changed since the batch was
  // made would be stepped with the wrong kernel over a differently sized buffer
  for (const vklb_sim* s : b->sims)
    if (!s->ready || kernel_variant(s) != b->variant || s->stages != b->stages) return VKLB_ERR_STATE;
  return b->ops->batch(b, n, use_graph);
}

int vklb_batch_destroy(vklb_batch* b) {
  if (!b) return VKLB_ERR_ARG;
  if (b->own) cudaStreamSynchronize(b->own);   // this batch's own work only
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->own) {
    if (b->d_desc) cudaFreeAsync(b->d_desc, b->own);
    if (b->d_work) cudaFreeAsync(b->d_work, b->own);
  }
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
  return VKLB_OK;
}

// ------------------------------------------------- allocation-free totals
// For callers that cannot allocate device memory themselves (for example a host
// process that only receives device pointers from another runtime, or code
// running where cudaMalloc is not permitted), conservation totals of a
// distribution buffer they own, with the partial sums kept in this file-scope
// device array instead of a cudaMalloc'd buffer.  Every GPU that loads the
// library holds the array until the process exits.
}  // extern "C"

namespace {
constexpr int kNoAllocMaxFields = 16;   // fields a call may reduce
constexpr int kNoAllocBlocks = kRedBlocks;
// [field][block] partial sums, then kNoAllocMaxFields final sums
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxFields * kNoAllocBlocks + kNoAllocMaxFields];
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Pass 1 with p and q given at run time: block b sums its fixed chunk of cells
// per field in FP64 (same order as totals_pass1), writing part[s * gridDim.x + b].
template <class T>
__global__ void totals_pass1_rt(const T* __restrict__ f, int p, int q, int nx, int ny, int pitch,
                                double* __restrict__ part) {
  __shared__ double red[32];
  const size_t cells = (size_t)nx * ny, plane = comp_stride(q, pitch, ny);
  const size_t chunk = (cells + gridDim.x - 1) / gridDim.x;
  const size_t lo = blockIdx.x * chunk, hi = min(cells, lo + chunk);
  for (int s = 0; s < p; ++s) {
    double acc = 0.0;
    for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const size_t y = i / nx, x = i - y * nx;
      const size_t o = cell_base(q, p, (int)x, (int)y, pitch);
      for (int k = 0; k < q; ++k) acc += (double)Store<T>::ld(f + (size_t)(k * p + s) * plane + o);
    }
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

template <class T>
int noalloc_launch(const void* f, int p, int q, int nx, int ny, int pitch, double vol, double* scratch, double* out,
                   cudaStream_t st) {
  totals_pass1_rt<T><<<kNoAllocBlocks, 256, 0, st>>>((const T*)f, p, q, nx, ny, pitch, scratch);
  totals_pass2<<<1, 32, 0, st>>>(scratch, kNoAllocBlocks, p, vol, out);
  g_launches += 2;
  return cuda_status(cudaGetLastError());
}
}  // namespace

extern "C" {

int vklb_conservation_totals_noalloc(const void* f_dev, int32_t precision, int32_t q, int32_t p, int64_t nx,
                                     int64_t ny, int64_t pitch, double cell_volume, double* totals,
                                     int32_t totals_on_device, void* cuda_stream) {
  if (!f_dev || !totals) return VKLB_ERR_ARG;
  if (precision < VKLB_FP64 || precision > VKLB_BF16_STORE || (q != 3 && q != 5)) return VKLB_ERR_ARG;
  if (nx < 1 || ny < 1 || pitch < nx || nx > (1 << 30) || ny > (1 << 30) || pitch > (1 << 30)) return VKLB_ERR_ARG;
  if (q == 5 && pitch % 32 != 0) return VKLB_ERR_ARG;   // whole bricks per row
  if (p < 1 || p > kNoAllocMaxFields) return VKLB_ERR_LIMIT;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VKLB_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return VKLB_ERR_LIMIT;
  double* scratch = nullptr;
  {
    // first call on this device: resolve the device address of the array
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return VKLB_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = (double*)ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* out = totals_on_device ? totals : scratch + (size_t)kNoAllocMaxFields * kNoAllocBlocks;
  int rc;
  if (precision == VKLB_FP64)
    rc = noalloc_launch<double>(f_dev, p, q, (int)nx, (int)ny, (int)pitch, cell_volume, scratch, out, st);
  else if (precision == VKLB_FP32)
    rc = noalloc_launch<float>(f_dev, p, q, (int)nx, (int)ny, (int)pitch, cell_volume, scratch, out, st);
  else
    rc = noalloc_launch<__nv_bfloat16>(f_dev, p, q, (int)nx, (int)ny, (int)pitch, cell_volume, scratch, out, st);
  if (rc) return rc;
  if (totals_on_device) return VKLB_OK;
  if ((rc = cuda_status(cudaMemcpyAsync(totals, out, sizeof(double) * p, cudaMemcpyDeviceToHost, st)))) return rc;
  return cuda_status(cudaStreamSynchronize(st));
}

}  // extern "C"
